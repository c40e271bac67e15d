// Fused kernel-row products: squared distances, RBF/Matern epilogue and the
// contraction with W in one kernel, never storing a kernel tile in HBM.
//
// This is Step I of Alg. 2 (K_Bn W, which App. C.1's ColDistMatMat splits by
// columns over GPUs -- here the column split is over CTAs of one GPU with a
// deterministic double-float second-stage reduce) and Step II (the Nystrom sketch
// K_BB Omega, App. C.1 RowDistMatMat), plus the K_BB v products of Alg. 5,
// the posterior mean (Sec. 2) and the hyperparameter adjoint (App. D.1).
//
// Distances use the expansion u = q_i + q_j - 2 x'_i . x'_j on centred,
// pre-scaled data (x' = kappa (x - mean)/ell, q = ||x'||^2): the norm terms and
// the dot product are accumulated together in packed FP32 FMAs
// (fma.rn.f32x2: even and odd feature lanes), then u is clamped at 0.
#include <algorithm>

#include "internal.cuh"

namespace adasap {

int padded_dim(int d) {
  static const int dims[] = {4, 8, 12, 16, 24, 32, 48, 64};
  for (int v : dims)
    if (d <= v) return v;
  return -1;
}

double kernel_kappa(int kern) {
  if (kern == ADASAP_RBF) return 0.8493218002880191;   // sqrt(log2(e) / 2)
  if (kern == ADASAP_MATERN32) return 1.7320508075688772;  // sqrt(3)
  return 2.23606797749979;                               // sqrt(5)
}

// Rows per warp of the narrow kernel: as many as fit a register budget of
// about 96 per thread for row data (DP), accumulators (3 per output: running
// sum, compensation, tile sum) and the row norm.
__host__ __device__ constexpr int narrow_rt(int dp, int na) {
  return (96 / (dp + 3 * na + 2)) < 1 ? 1 : (96 / (dp + 3 * na + 2)) > 8 ? 8 : (96 / (dp + 3 * na + 2));
}

template <int DP, int NA = 1>
struct Narrow {
  static constexpr int RT = narrow_rt(DP, NA);
  static constexpr int TN = DP <= 16 ? 256 : 128;
  // row stride in shared memory: an odd number of float4s keeps a quarter
  // warp's 16-byte loads of consecutive columns on distinct banks
  static constexpr int SP = ((DP / 4) % 2 == 1) ? DP : DP + 4;
  static constexpr int ROWS = 8 * RT;
};

constexpr int kThreads = 256;

// ---------------------------------------------------------------------------
// Narrow kernel: s <= 4 right-hand sides.  Each warp owns RT rows (in
// registers, shared by all lanes); lane l takes columns l, l+32, ... of every
// column tile staged in shared memory.  Per lane and tile the products are
// summed in FP32 and folded into a compensated (Kahan) running sum; lanes are
// combined with shuffles at the end.
// ---------------------------------------------------------------------------
template <int KERN, int DP, int S, bool ADJ>
__global__ void __launch_bounds__(kThreads, 2) k_rows_narrow(RowsArgs a) {
  constexpr int NA = ADJ ? 2 * S : S;
  using C = Narrow<DP, NA>;
  constexpr int RT = C::RT, TN = C::TN, SP = C::SP;
  __shared__ __align__(16) float s_x[TN * SP];
  __shared__ float s_q[TN];
  __shared__ float s_w[TN * S];

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t row0 = (int64_t)blockIdx.x * C::ROWS + warp * RT;
  const int64_t c0 = (int64_t)blockIdx.y * a.cps;
  const int64_t c1 = min(a.ncols, c0 + a.cps);

  float2 rr[RT][DP / 2];
  float rq[RT];
  bool bad[RT];
#pragma unroll
  for (int i = 0; i < RT; ++i) {
    const int64_t ri = row0 + i;
    int64_t src = ri;
    bool valid = ri < a.m;
    bad[i] = false;
    if (valid && a.ridx) {
      const int id = a.ridx[ri];
      bad[i] = id < 0;
      src = id < 0 ? 0 : id;
    }
    valid = valid && !bad[i];
    const float4* p = reinterpret_cast<const float4*>(a.xr + src * DP);
#pragma unroll
    for (int k4 = 0; k4 < DP / 4; ++k4) {
      float4 v = valid ? __ldg(p + k4) : make_float4(0.f, 0.f, 0.f, 0.f);
      rr[i][2 * k4] = make_float2(-2.0f * v.x, -2.0f * v.y);
      rr[i][2 * k4 + 1] = make_float2(-2.0f * v.z, -2.0f * v.w);
    }
    rq[i] = valid ? __ldg(a.qr + src) : 1e30f;
  }

  float acc[RT][NA], cmp[RT][NA];
#pragma unroll
  for (int i = 0; i < RT; ++i)
#pragma unroll
    for (int c = 0; c < NA; ++c) acc[i][c] = cmp[i][c] = 0.0f;

  for (int64_t t0 = c0; t0 < c1; t0 += TN) {
    const int nt = (int)min((int64_t)TN, c1 - t0);
    __syncthreads();
    for (int e = threadIdx.x; e < TN * (DP / 4); e += kThreads) {
      const int j = e / (DP / 4), k4 = e % (DP / 4);
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (j < nt) v = __ldg(reinterpret_cast<const float4*>(a.xc + (t0 + j) * DP) + k4);
      *reinterpret_cast<float4*>(&s_x[j * SP + 4 * k4]) = v;
    }
    for (int j = threadIdx.x; j < TN; j += kThreads) {
      s_q[j] = j < nt ? __ldg(a.qc + t0 + j) : 1e30f;
#pragma unroll
      for (int c = 0; c < S; ++c) s_w[j * S + c] = j < nt ? __ldg(a.w + (t0 + j) * a.ldw + c) : 0.0f;
    }
    __syncthreads();

    float tacc[RT][NA];
#pragma unroll
    for (int i = 0; i < RT; ++i)
#pragma unroll
      for (int c = 0; c < NA; ++c) tacc[i][c] = 0.0f;

#pragma unroll 2
    for (int jj = 0; jj < TN / 32; ++jj) {
      const int j = jj * 32 + lane;
      float2 cx[DP / 2];
      const float4* px = reinterpret_cast<const float4*>(&s_x[j * SP]);
#pragma unroll
      for (int k4 = 0; k4 < DP / 4; ++k4) {
        const float4 v = px[k4];
        cx[2 * k4] = make_float2(v.x, v.y);
        cx[2 * k4 + 1] = make_float2(v.z, v.w);
      }
      const float qj = s_q[j];
      float wj[S];
#pragma unroll
      for (int c = 0; c < S; ++c) wj[c] = s_w[j * S + c];
#pragma unroll
      for (int i = 0; i < RT; ++i) {
        float2 t = make_float2(rq[i], qj);
#pragma unroll
        for (int k = 0; k < DP / 2; ++k) t = ffma2(rr[i][k], cx[k], t);
        const float u = fmaxf(t.x + t.y, 0.0f);
        if (ADJ) {
          float kv, gv;
          kval_grad<KERN>(u, kv, gv);
#pragma unroll
          for (int c = 0; c < S; ++c) {
            tacc[i][c] = fmaf(kv, wj[c], tacc[i][c]);
            tacc[i][S + c] = fmaf(gv, wj[c], tacc[i][S + c]);
          }
        } else {
          const float kv = kval<KERN>(u);
#pragma unroll
          for (int c = 0; c < S; ++c) tacc[i][c] = fmaf(kv, wj[c], tacc[i][c]);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < RT; ++i)
#pragma unroll
      for (int c = 0; c < NA; ++c) {
        const float y = tacc[i][c] - cmp[i][c];
        const float tt = acc[i][c] + y;
        cmp[i][c] = (tt - acc[i][c]) - y;
        acc[i][c] = tt;
      }
  }

#pragma unroll
  for (int i = 0; i < RT; ++i) {
    const int64_t ri = row0 + i;
#pragma unroll
    for (int c = 0; c < NA; ++c) {
      const float v = warp_sum(acc[i][c] - cmp[i][c]);
      if (lane == 0 && ri < a.m)
        a.part[((int64_t)blockIdx.y * a.m + ri) * NA + c] = bad[i] ? __int_as_float(0x7fc00000) : a.sigma2 * v;
    }
  }
}

// ---------------------------------------------------------------------------
// Wide kernel: s up to 128 right-hand sides (Nystrom sketch K_BB Omega,
// multi-RHS Step I).  A CTA owns 64 rows; per 32-column tile it evaluates the
// 64 x 32 kernel tile into shared memory and accumulates the tile times the
// 32 x s slice of W with a register-blocked FP32 product.
// ---------------------------------------------------------------------------
template <int SW>
struct Wide {
  static constexpr int CW = SW >= 32 ? SW / 32 : 1;
  static constexpr int TXN = SW / CW;
  static constexpr int TYN = kThreads / TXN;
  static constexpr int RW = 64 / TYN;
};

template <int KERN, int DP, int SW>
__global__ void __launch_bounds__(kThreads) k_rows_wide(RowsArgs a, int s) {
  constexpr int TM = 64, TJ = 32, SP = Narrow<DP>::SP, KS = TM + 4;
  using Wc = Wide<SW>;
  constexpr int CW = Wc::CW, TXN = Wc::TXN, RW = Wc::RW;
  __shared__ __align__(16) float s_r[TM * SP];
  __shared__ float s_rq[TM];
  __shared__ int s_bad[TM];
  __shared__ __align__(16) float s_c[TJ * SP];
  __shared__ float s_cq[TJ];
  __shared__ __align__(16) float s_k[TJ * KS];
  __shared__ __align__(16) float s_w[TJ * SW];

  const int tid = threadIdx.x;
  const int64_t row0 = (int64_t)blockIdx.x * TM;
  const int64_t c0 = (int64_t)blockIdx.y * a.cps;
  const int64_t c1 = min(a.ncols, c0 + a.cps);

  for (int i = tid; i < TM; i += kThreads) {
    const int64_t ri = row0 + i;
    int64_t src = ri;
    int bad = 0;
    if (ri < a.m && a.ridx) {
      const int id = a.ridx[ri];
      bad = id < 0;
      src = id < 0 ? 0 : id;
    }
    s_bad[i] = bad;
    s_rq[i] = (ri < a.m && !bad) ? __ldg(a.qr + src) : 1e30f;
  }
  for (int e = tid; e < TM * (DP / 4); e += kThreads) {
    const int i = e / (DP / 4), k4 = e % (DP / 4);
    const int64_t ri = row0 + i;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (ri < a.m) {
      int64_t src = ri;
      if (a.ridx) src = max(a.ridx[ri], 0);
      v = __ldg(reinterpret_cast<const float4*>(a.xr + src * DP) + k4);
    }
    *reinterpret_cast<float4*>(&s_r[i * SP + 4 * k4]) =
        make_float4(-2.f * v.x, -2.f * v.y, -2.f * v.z, -2.f * v.w);
  }

  // the row set-up above is read by other threads below even when this split
  // has no columns (the tile loop, and its barriers, then run zero times)
  __syncthreads();
  float acc[RW][CW];
#pragma unroll
  for (int i = 0; i < RW; ++i)
#pragma unroll
    for (int q = 0; q < CW; ++q) acc[i][q] = 0.0f;

  const int kj = tid & 31, krg = tid >> 5;      // kernel-tile phase: column, row group of 8
  const int tx = tid % TXN, ty = tid / TXN;      // product phase

  for (int64_t t0 = c0; t0 < c1; t0 += TJ) {
    const int nt = (int)min((int64_t)TJ, c1 - t0);
    __syncthreads();
    for (int e = tid; e < TJ * (DP / 4); e += kThreads) {
      const int j = e / (DP / 4), k4 = e % (DP / 4);
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (j < nt) v = __ldg(reinterpret_cast<const float4*>(a.xc + (t0 + j) * DP) + k4);
      *reinterpret_cast<float4*>(&s_c[j * SP + 4 * k4]) = v;
    }
    for (int j = tid; j < TJ; j += kThreads) s_cq[j] = j < nt ? __ldg(a.qc + t0 + j) : 1e30f;
    for (int e = tid; e < TJ * SW; e += kThreads) {
      const int j = e / SW, c = e % SW;
      s_w[e] = (j < nt && c < s) ? __ldg(a.w + (t0 + j) * a.ldw + c) : 0.0f;
    }
    __syncthreads();
    {
      float cx[DP];
      const float4* px = reinterpret_cast<const float4*>(&s_c[kj * SP]);
#pragma unroll
      for (int k4 = 0; k4 < DP / 4; ++k4) {
        const float4 v = px[k4];
        cx[4 * k4] = v.x; cx[4 * k4 + 1] = v.y; cx[4 * k4 + 2] = v.z; cx[4 * k4 + 3] = v.w;
      }
      const float qj = s_cq[kj];
#pragma unroll
      for (int ii = 0; ii < 8; ++ii) {
        const int i = krg * 8 + ii;
        float t = s_rq[i] + qj;
#pragma unroll
        for (int k = 0; k < DP; ++k) t = fmaf(s_r[i * SP + k], cx[k], t);
        s_k[kj * KS + i] = kval<KERN>(fmaxf(t, 0.0f));
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int j = 0; j < TJ; ++j) {
      float kv[RW];
#pragma unroll
      for (int i4 = 0; i4 < RW / 4; ++i4) {
        const float4 v = *reinterpret_cast<const float4*>(&s_k[j * KS + ty * RW + 4 * i4]);
        kv[4 * i4] = v.x; kv[4 * i4 + 1] = v.y; kv[4 * i4 + 2] = v.z; kv[4 * i4 + 3] = v.w;
      }
      float wv[CW];
#pragma unroll
      for (int q = 0; q < CW; ++q) wv[q] = s_w[j * SW + tx + TXN * q];
#pragma unroll
      for (int i = 0; i < RW; ++i)
#pragma unroll
        for (int q = 0; q < CW; ++q) acc[i][q] = fmaf(kv[i], wv[q], acc[i][q]);
    }
  }
#pragma unroll
  for (int i = 0; i < RW; ++i) {
    const int li = ty * RW + i;
    const int64_t ri = row0 + li;
    if (ri >= a.m) continue;
#pragma unroll
    for (int q = 0; q < CW; ++q) {
      const int c = tx + TXN * q;
      if (c < s)
        a.part[((int64_t)blockIdx.y * a.m + ri) * s + c] =
            s_bad[li] ? __int_as_float(0x7fc00000) : a.sigma2 * acc[i][q];
    }
  }
}

// ---------------------------------------------------------------------------
int rows_nsplit(int64_t m, int64_t ncols, int s, int dp, bool adjoint) {
  const bool wide = !adjoint && s > 4;
  const int rows_per_cta = wide ? 64 : 8 * narrow_rt(dp, adjoint ? 2 * s : s);
  const int64_t min_cols = wide ? 64 : (dp <= 16 ? 256 : 128);
  const int64_t row_tiles = (m + rows_per_cta - 1) / rows_per_cta;
  // aim at >= 8 waves of 2 CTAs per SM on 148 SMs so the last wave is a small tail
  const int64_t target = 8LL * 148 * 2;
  int64_t ns = (target + row_tiles - 1) / row_tiles;
  const int64_t maxs = std::max<int64_t>(1, (ncols + min_cols - 1) / min_cols);
  ns = std::min(ns, maxs);
  ns = std::max<int64_t>(1, std::min<int64_t>(ns, 65535));
  return (int)ns;
}

template <int KERN, int DP>
static cudaError_t launch_rows_dp(const RowsArgs& a0, int s, int nsplit, bool adjoint, cudaStream_t st) {
  RowsArgs a = a0;
  a.cps = (a.ncols + nsplit - 1) / nsplit;
  if (adjoint || s <= 4) {
    const int rows = 8 * narrow_rt(DP, adjoint ? 2 * s : s);
    const dim3 grid((unsigned)((a.m + rows - 1) / rows), nsplit);
    if (adjoint) {
      switch (s) {
        case 1: k_rows_narrow<KERN, DP, 1, true><<<grid, kThreads, 0, st>>>(a); break;
        case 2: k_rows_narrow<KERN, DP, 2, true><<<grid, kThreads, 0, st>>>(a); break;
        default: return cudaErrorInvalidValue;
      }
    } else {
      switch (s) {
        case 1: k_rows_narrow<KERN, DP, 1, false><<<grid, kThreads, 0, st>>>(a); break;
        case 2: k_rows_narrow<KERN, DP, 2, false><<<grid, kThreads, 0, st>>>(a); break;
        case 3: k_rows_narrow<KERN, DP, 3, false><<<grid, kThreads, 0, st>>>(a); break;
        case 4: k_rows_narrow<KERN, DP, 4, false><<<grid, kThreads, 0, st>>>(a); break;
        default: return cudaErrorInvalidValue;
      }
    }
  } else {
    const dim3 grid((unsigned)((a.m + 63) / 64), nsplit);
    if (s <= 16) k_rows_wide<KERN, DP, 16><<<grid, kThreads, 0, st>>>(a, s);
    else if (s <= 32) k_rows_wide<KERN, DP, 32><<<grid, kThreads, 0, st>>>(a, s);
    else if (s <= 64) k_rows_wide<KERN, DP, 64><<<grid, kThreads, 0, st>>>(a, s);
    else if (s <= 128) k_rows_wide<KERN, DP, 128><<<grid, kThreads, 0, st>>>(a, s);
    else return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int KERN>
static cudaError_t launch_rows_k(int dp, const RowsArgs& a, int s, int nsplit, bool adjoint, cudaStream_t st) {
  switch (dp) {
    case 4: return launch_rows_dp<KERN, 4>(a, s, nsplit, adjoint, st);
    case 8: return launch_rows_dp<KERN, 8>(a, s, nsplit, adjoint, st);
    case 12: return launch_rows_dp<KERN, 12>(a, s, nsplit, adjoint, st);
    case 16: return launch_rows_dp<KERN, 16>(a, s, nsplit, adjoint, st);
    case 24: return launch_rows_dp<KERN, 24>(a, s, nsplit, adjoint, st);
    case 32: return launch_rows_dp<KERN, 32>(a, s, nsplit, adjoint, st);
    case 48: return launch_rows_dp<KERN, 48>(a, s, nsplit, adjoint, st);
    case 64: return launch_rows_dp<KERN, 64>(a, s, nsplit, adjoint, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_rows(int kern, int dp, const RowsArgs& a, int s, int nsplit, bool adjoint,
                        cudaStream_t st) {
  if (a.m <= 0 || a.ncols <= 0) return cudaSuccess;
  switch (kern) {
    case ADASAP_RBF: return launch_rows_k<ADASAP_RBF>(dp, a, s, nsplit, adjoint, st);
    case ADASAP_MATERN32: return launch_rows_k<ADASAP_MATERN32>(dp, a, s, nsplit, adjoint, st);
    case ADASAP_MATERN52: return launch_rows_k<ADASAP_MATERN52>(dp, a, s, nsplit, adjoint, st);
  }
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// out[i][c] = sum_p part[p][i][coff + c] + beta A[aidx i][c] + gamma B[bidx i][c],
// summed in double-float (the products beta A, gamma B split exactly) and
// rounded once to FP32; blocksq (optional) gets each block's sum of out^2.
// body of k_reduce for block bx of gx (the grouped form passes its own indices)
__device__ __forceinline__ void reduce_body(const float* __restrict__ part, int nsplit, int64_t m, int na, int coff,
                                            int s, float* __restrict__ out, int64_t ldo, float beta,
                                            const float* __restrict__ A, const int* __restrict__ aidx, int64_t lda,
                                            float gamma, const float* __restrict__ B, const int* __restrict__ bidx,
                                            int64_t ldb, double* blocksq, int bx, int gx) {
  __shared__ double red[33];
  const int64_t total = m * s;
  double sq = 0.0;
  for (int64_t e = (int64_t)bx * blockDim.x + threadIdx.x; e < total; e += (int64_t)gx * blockDim.x) {
    const int64_t i = s == 1 ? e : e / s;
    const int c = (int)(e - i * s);
    float H = 0.0f, L = 0.0f;
    const float* src = part + i * na + coff + c;
    const int64_t pstride = m * na;
#pragma unroll 4
    for (int p = 0; p < nsplit; ++p) ff_add(H, L, __ldg(src + p * pstride));
    if (beta != 0.0f) {
      const int64_t ai = aidx ? aidx[i] : i;
      const float av = A[ai * lda + c];
      const float pr = beta * av;
      ff_add(H, L, pr);
      L += fmaf(beta, av, -pr);
    }
    if (gamma != 0.0f) {
      const int64_t bi = bidx ? bidx[i] : i;
      const float bv = B[bi * ldb + c];
      const float pr = gamma * bv;
      ff_add(H, L, pr);
      L += fmaf(gamma, bv, -pr);
    }
    const float v = H + L;
    out[i * ldo + c] = v;
    if (blocksq) sq += (double)v * (double)v;
  }
  if (blocksq) {
    const double tot = block_sum(sq, red);
    if (threadIdx.x == 0) blocksq[bx] = tot;
  }
}

__global__ void k_reduce(const float* __restrict__ part, int nsplit, int64_t m, int na, int coff,
                         int s, float* __restrict__ out, int64_t ldo, float beta,
                         const float* __restrict__ A, const int* __restrict__ aidx, int64_t lda,
                         float gamma, const float* __restrict__ B, const int* __restrict__ bidx,
                         int64_t ldb, double* blocksq) {
  reduce_body(part, nsplit, m, na, coff, s, out, ldo, beta, A, aidx, lda, gamma, B, bidx, ldb, blocksq, blockIdx.x,
              gridDim.x);
}

// Grouped plain split sums out = sum_p part[p] (system blockIdx.y of tab), the
// arithmetic of k_reduce with no extra terms.
__global__ void k_split_sum_g(const SplitSumArgs* __restrict__ tab) {
  const SplitSumArgs& a = tab[blockIdx.y];
  reduce_body(a.part, a.nsplit, a.m, a.s, 0, a.s, a.out, a.s, 0.0f, nullptr, nullptr, 0, 0.0f, nullptr, nullptr, 0,
              nullptr, blockIdx.x, gridDim.x);
}

cudaError_t launch_split_sum_grouped(const SplitSumArgs* tab, int nsys, int64_t max_elems, cudaStream_t st) {
  if (nsys <= 0 || max_elems <= 0) return cudaSuccess;
  const dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>((max_elems + 255) / 256, 64)), (unsigned)nsys);
  k_split_sum_g<<<grid, 256, 0, st>>>(tab);
  return cudaGetLastError();
}

cudaError_t launch_reduce(const float* part, int nsplit, int64_t m, int na, int coff, int s,
                          float* out, int64_t ldo, float beta, const float* A, const int* aidx,
                          int64_t lda, float gamma, const float* B, const int* bidx, int64_t ldb,
                          double* blocksq, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  // kReduceBlocks blocks when the per-block sums of squares are wanted (their
  // count is fixed); otherwise about one element per thread, for more loads in
  // flight
  const int blocks = blocksq ? kReduceBlocks
                             : (int)std::max<int64_t>(1, std::min<int64_t>((m * s + 255) / 256, 148 * 16));
  k_reduce<<<blocks, 256, 0, st>>>(part, nsplit, m, na, coff, s, out, ldo, beta, A, aidx, lda, gamma, B, bidx,
                                   ldb, blocksq);
  return cudaGetLastError();
}

__global__ void k_iota32(int* __restrict__ out, int64_t start, int64_t m) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (int)(start + i);
}

cudaError_t launch_iota32(int* out, int64_t start, int64_t m, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((m + 255) / 256, 148 * 8);
  k_iota32<<<blocks, 256, 0, st>>>(out, start, m);
  return cudaGetLastError();
}

__global__ void k_gather(const float* __restrict__ X, const float* __restrict__ q,
                         const int* __restrict__ idx, int64_t m, int dp4, float* __restrict__ out,
                         float* __restrict__ qout) {
  const int64_t total = m * dp4;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / dp4;
    const int k4 = (int)(e - i * dp4);
    const int src = max(idx[i], 0);
    reinterpret_cast<float4*>(out)[i * dp4 + k4] = reinterpret_cast<const float4*>(X)[(int64_t)src * dp4 + k4];
    if (k4 == 0) qout[i] = idx[i] < 0 ? 1e30f : q[src];
  }
}

cudaError_t launch_gather(const float* X, const float* q, const int* idx, int64_t m, int dp,
                          float* out, float* qout, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  const int64_t total = m * (dp / 4);
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 148 * 8);
  k_gather<<<blocks, 256, 0, st>>>(X, q, idx, m, dp / 4, out, qout);
  return cudaGetLastError();
}

__global__ void k_colsum(const float* __restrict__ X, int64_t n, int d, double* partials) {

  __shared__ double red[33];
  for (int k = 0; k < d; ++k) {
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
      acc += (double)X[i * d + k];
    const double tot = block_sum(acc, red);
    if (threadIdx.x == 0) partials[(int64_t)blockIdx.x * d + k] = tot;
  }
}

cudaError_t launch_colsum(const float* X, int64_t n, int d, double* partials, cudaStream_t st) {
  k_colsum<<<kColsumBlocks, 256, 0, st>>>(X, n, d, partials);
  return cudaGetLastError();
}

__global__ void k_transform(const float* __restrict__ X, int64_t n, int d, int dp,
                            const double* __restrict__ mean, double scale, float* __restrict__ out,
                            float* __restrict__ q) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int k = 0; k < dp; ++k) {
      float v = 0.0f;
      if (k < d) v = (float)(((double)X[i * d + k] - mean[k]) * scale);
      out[i * dp + k] = v;
      acc += (double)v * (double)v;
    }
    q[i] = (float)acc;
  }
}

cudaError_t launch_transform(const float* X, int64_t n, int d, int dp, const double* mean_dev,
                             double scale, float* out, float* q, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 148 * 16);
  k_transform<<<blocks, 256, 0, st>>>(X, n, d, dp, mean_dev, scale, out, q);
  return cudaGetLastError();
}

__global__ void k_index32(const int64_t* __restrict__ in, int64_t m, int64_t n, int* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = in[i];
    out[i] = (v >= 0 && v < n) ? (int)v : -1;
  }
}

cudaError_t launch_index32(const int64_t* in, int64_t m, int64_t n, int* out, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((m + 255) / 256, 148 * 8);
  k_index32<<<blocks, 256, 0, st>>>(in, m, n, out);
  return cudaGetLastError();
}

__global__ void k_adj_reduce(const float* __restrict__ part, int nsplit, int64_t m, int s,
                             const float* __restrict__ G, int64_t ldg, int coff, double* blockacc) {
  __shared__ double red[33];
  double ak = 0.0, ag = 0.0;
  const int64_t total = m * s;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / s;
    const int c = (int)(e - i * s);
    double kw = 0.0, gw = 0.0;
    for (int p = 0; p < nsplit; ++p) {
      kw += (double)part[((int64_t)p * m + i) * (2 * s) + c];
      gw += (double)part[((int64_t)p * m + i) * (2 * s) + s + c];
    }
    const double g = (double)G[i * ldg + coff + c];
    ak += g * kw;
    ag += g * gw;
  }
  const double tk = block_sum(ak, red);
  const double tg = block_sum(ag, red);
  if (threadIdx.x == 0) {
    blockacc[2 * blockIdx.x] += tk;
    blockacc[2 * blockIdx.x + 1] += tg;
  }
}

cudaError_t launch_adj_reduce(const float* part, int nsplit, int64_t m, int s, const float* G,
                              int64_t ldg, int coff, double* blockacc, cudaStream_t st) {
  k_adj_reduce<<<kReduceBlocks, 256, 0, st>>>(part, nsplit, m, s, G, ldg, coff, blockacc);
  return cudaGetLastError();
}

}  // namespace adasap
