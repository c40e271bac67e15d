// Step III and IV of Alg. 2 on the GPU:
//   - Gram matrices of b x r panels (FP32 products, or error-free split
//     products for the Gram of M Omega, accumulated in double-float on the
//     FP32 pipes)
//   - the randomized Nystrom factorisation of Alg. 4 on its r x r core
//     (FP64 Cholesky and triangular solves; eigenvectors by FP32 cyclic
//     Jacobi with FP64 Rayleigh-quotient eigenvalues)
//   - the Woodbury applies of App. C.2: (P + rho I)^{-1/2} v
//     (eq. inv_sqrt_nys_woodbury) and the Cholesky-stabilised
//     (P + rho I)^{-1} g
//   - the stepsize of Alg. 5 and the NesterovAcc update of Alg. 6.
//
// The thin SVD of B = Y_nu C^{-1} (Alg. 4) is computed through the r x r
// matrix B^T B = C^{-T} (Y_nu^T Y_nu) C^{-1}: its eigenvectors are B's right
// singular vectors V and its eigenvalues Sigma^2, and U = Y_nu (C^{-1} V Sigma^{-1}).
// Y_nu^T Y_nu comes from the Gram of [Omega | M Omega] without forming Y_nu.

#include <algorithm>
#include <type_traits>

#include "internal.cuh"


namespace adasap {

// ---------------------------------------------------------------------------
// Gram matrix of the row-concatenation [A1 | A2] (m x (c1 + c2), c <= 256),
// accumulated in double-float on the FP32 pipes (FP64 arithmetic runs at a
// small fraction of their rate on this GPU) and returned in FP64.  With
// `exact` every product of two FP32 entries is also kept exactly (p + e).
// Exactness matters for Y_nu^T Y_nu: B^T B = C^{-T} (Y_nu^T Y_nu) C^{-1}
// multiplies its absolute error by cond(C)^2, so FP32 product errors would
// swamp the small Nystrom eigenvalues; everywhere else an FP32 product error
// of eps * |a| |b| is below the data's own rounding.  Only the upper 64 x 64
// tiles whose first row is below `rows` are computed (callers read only the
// entries with min(i, j) < rows; the tiles left out are returned as zero); the
// reduce mirrors them.
// ---------------------------------------------------------------------------
// chunks of at least 32 rows (the launch caps them at about two CTAs per SM over the upper tiles)
int gram_chunks_for(int64_t b) { return (int)std::max<int64_t>(1, std::min<int64_t>(240, (b + 31) / 32)); }

__device__ __forceinline__ float cat_get(const float* A1, int64_t ld1, int c1, const float* A2, int64_t ld2,
                                         int c2, int64_t row, int col) {
  if (col < c1) return A1[row * ld1 + col];
  if (col < c1 + c2) return A2[row * ld2 + (col - c1)];
  return 0.0f;
}

// the p-th computed tile (ti <= tj, 64 ti < rows) of an nt x nt tiling
__device__ __forceinline__ void gram_tile(int p, int nt, int rows, int& ti, int& tj) {
  ti = 0;
  tj = 0;
  for (int i = 0; i < nt && 64 * i < rows; ++i) {
    const int cnt = nt - i;
    if (p < cnt) {
      ti = i;
      tj = i + p;
      return;
    }
    p -= cnt;
  }
}

__host__ __device__ inline int gram_active_tiles(int nt, int rows) {
  int cnt = 0;
  for (int i = 0; i < nt && 64 * i < rows; ++i) cnt += nt - i;
  return cnt;
}

// 64 x 64 output tiles (blockIdx.y = computed tile, blockIdx.x = row chunk),
// 256 threads x (4 x 4) outputs, thread (ty, tx) owning rows 4 ty .. 4 ty + 3 and
// columns 4 tx .. 4 tx + 3 of the tile, so that its operands of one row are two
// 16-byte shared-memory loads (three wavefronts per warp instead of eight); rows
// are staged 32 at a time in shared memory, the next slice prefetched into
// registers while the current one is used.
//   EXACT: every product is split exactly into p + e (p = fl(a b), e = fma(a, b, -p),
//          an error-free transformation), p summed in double-float and e in FP32:
//          the chunk sum carries a relative error of about rows x 2^-48 of sum |a b|
//   else:  FP32 products summed in FP32 over 64 rows, those sums in double-float.
// The chunk's partial of entry (i, j) is written as the pair (hi, lo).
// (body for block (bx, by); the kernels below pass their own block indices)
template <bool EXACT>
__device__ __forceinline__ void gram_part_body(const float* __restrict__ A1, int64_t ld1, int c1,
                                               const float* __restrict__ A2, int64_t ld2, int c2,
                                               int64_t m, int64_t chunk_rows, int rows,
                                               float2* __restrict__ part, int bx, int by) {
  constexpr int TS = 64, KR = 32, PER = KR * TS / 256;  // floats per thread per matrix and slice
  const int c = c1 + c2;
  const int nt = (c + TS - 1) / TS;
  int ti, tj;
  gram_tile(by, nt, rows, ti, tj);
  __shared__ __align__(16) float sa[KR][TS + 4];
  __shared__ __align__(16) float sb[KR][TS + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t r0 = (int64_t)bx * chunk_rows;
  const int64_t r1 = min(m, r0 + chunk_rows);
  float hi[4][4], lo[4][4], H[4][4], L[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      hi[u][v] = 0.0f;
      lo[u][v] = 0.0f;
      H[u][v] = 0.0f;
      L[u][v] = 0.0f;
    }
  float pa[PER], pb[PER];
  auto fetch = [&](int64_t s0) {
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int e = tid + 256 * k;
      const int rr = e / TS, cc = e % TS;
      const int64_t row = s0 + rr;
      const bool ok = row < r1;
      pa[k] = ok ? cat_get(A1, ld1, c1, A2, ld2, c2, row, ti * TS + cc) : 0.0f;
      pb[k] = ok ? cat_get(A1, ld1, c1, A2, ld2, c2, row, tj * TS + cc) : 0.0f;
    }
  };
  if (r0 < r1) fetch(r0);
  int slices = 0;
  for (int64_t s0 = r0; s0 < r1; s0 += KR) {
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int e = tid + 256 * k;
      sa[e / TS][e % TS] = pa[k];
      sb[e / TS][e % TS] = pb[k];
    }
    __syncthreads();
    if (s0 + KR < r1) fetch(s0 + KR);  // in flight during the products below
#pragma unroll 4
    for (int rr = 0; rr < KR; ++rr) {
      const float4 a4 = *reinterpret_cast<const float4*>(&sa[rr][4 * ty]);
      const float4 b4 = *reinterpret_cast<const float4*>(&sb[rr][4 * tx]);
      const float av[4] = {a4.x, a4.y, a4.z, a4.w};
      const float bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          if (EXACT) {
            const float p = av[u] * bv[v];
            const float e = fmaf(av[u], bv[v], -p);
            const float sum = hi[u][v] + p;
            const float z = sum - hi[u][v];
            const float err = (hi[u][v] - (sum - z)) + (p - z);
            hi[u][v] = sum;
            lo[u][v] += err + e;
          } else {
            hi[u][v] = fmaf(av[u], bv[v], hi[u][v]);
          }
        }
    }
    if (!EXACT && ++slices == 2) {
      slices = 0;
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          ff_add(H[u][v], L[u][v], hi[u][v]);
          hi[u][v] = 0.0f;
        }
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int i = ti * TS + 4 * ty + u, j = tj * TS + 4 * tx + v;
      float th, tl;
      if (EXACT) {
        th = hi[u][v];
        tl = lo[u][v];
      } else {
        th = H[u][v];
        tl = L[u][v];
        ff_add(th, tl, hi[u][v]);
      }
      if (i < c && j < c) part[((int64_t)bx * c + i) * c + j] = make_float2(th, tl);
    }
}

template <bool EXACT>
__global__ void __launch_bounds__(256) k_gram_part(const float* __restrict__ A1, int64_t ld1, int c1,
                                                   const float* __restrict__ A2, int64_t ld2, int c2,
                                                   int64_t m, int64_t chunk_rows, int rows,
                                                   float2* __restrict__ part) {
  gram_part_body<EXACT>(A1, ld1, c1, A2, ld2, c2, m, chunk_rows, rows, part, blockIdx.x, blockIdx.y);
}

// G[i][j] = sum over chunks of the (hi, lo) partials, in chunk order within
// each of 8 interleaved subsets and then in subset order (double-float);
// block = 32 entries x 8 subsets.
__device__ __forceinline__ void gram_reduce_body(const float2* __restrict__ part, int chunks, int c, int rows,
                                                 double* __restrict__ G, int bx) {
  __shared__ float2 sh[8][33];
  const int x = threadIdx.x & 31, y = threadIdx.x >> 5;
  const int64_t cc = (int64_t)c * c;
  const int e = bx * 32 + x;
  int i = e / c, j = e % c;
  if ((i >> 6) > (j >> 6)) {
    const int t = i;
    i = j;
    j = t;
  }
  const bool need = e < c * c && 64 * (i >> 6) < rows;
  float H = 0.0f, L = 0.0f;
  if (need) {
    const int64_t o = (int64_t)i * c + j;
#pragma unroll 4
    for (int ch = y; ch < chunks; ch += 8) {
      const float2 v = part[ch * cc + o];
      ff_add(H, L, v.x);
      L += v.y;
    }
  }
  sh[y][x] = make_float2(H, L);
  __syncthreads();
  if (y == 0 && e < c * c) {
    float h = 0.0f, l = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      ff_add(h, l, sh[k][x].x);
      l += sh[k][x].y;
    }
    G[e] = need ? (double)h + (double)l : 0.0;
  }
}

__global__ void __launch_bounds__(256) k_gram_reduce(const float2* __restrict__ part, int chunks, int c, int rows,
                                                     double* __restrict__ G) {
  gram_reduce_body(part, chunks, c, rows, G, blockIdx.x);
}

// Grouped forms (system blockIdx.z / blockIdx.y of tab); blocks past a system's
// own grid return at once.
template <bool EXACT>
__global__ void __launch_bounds__(256) k_gram_part_g(const GramArgs* __restrict__ tab) {
  const GramArgs& a = tab[blockIdx.z];
  if ((int)blockIdx.x >= a.chunks || (int)blockIdx.y >= a.active) return;
  gram_part_body<EXACT>(a.A1, a.ld1, a.c1, a.A2, a.ld2, a.c2, a.m, a.chunk_rows, a.rows, a.part, blockIdx.x,
                        blockIdx.y);
}

__global__ void __launch_bounds__(256) k_gram_reduce_g(const GramArgs* __restrict__ tab) {
  const GramArgs& a = tab[blockIdx.y];
  if ((int)blockIdx.x >= (a.c * a.c + 31) / 32) return;
  gram_reduce_body(a.part, a.chunks, a.c, a.rows, a.G, blockIdx.x);
}

GramArgs gram_fill_args(const float* A1, int64_t ld1, int c1, const float* A2, int64_t ld2, int c2, int64_t m,
                        float2* part, int chunks, double* G, int rows) {
  GramArgs a;
  a.A1 = A1; a.ld1 = ld1; a.c1 = c1; a.A2 = A2; a.ld2 = ld2; a.c2 = c2; a.m = m; a.part = part; a.G = G;
  a.c = c1 + c2;
  const int nt = (a.c + 63) / 64;
  if (rows <= 0 || rows > a.c) rows = a.c;
  a.rows = rows;
  // about two resident CTAs per SM over the computed tiles; fewer partials to reduce
  a.active = gram_active_tiles(nt, rows);
  a.chunks = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)chunks, (int64_t)(296 / a.active), (m + 31) / 32}));
  a.chunk_rows = (m + a.chunks - 1) / a.chunks;
  return a;
}

cudaError_t launch_gram(const float* A1, int64_t ld1, int c1, const float* A2, int64_t ld2, int c2,
                        int64_t m, float2* part, int chunks, double* G, bool exact, cudaStream_t st, int rows) {
  const GramArgs a = gram_fill_args(A1, ld1, c1, A2, ld2, c2, m, part, chunks, G, rows);
  if (exact)
    k_gram_part<true><<<dim3(a.chunks, a.active), 256, 0, st>>>(A1, ld1, c1, A2, ld2, c2, m, a.chunk_rows, a.rows,
                                                                 part);
  else
    k_gram_part<false><<<dim3(a.chunks, a.active), 256, 0, st>>>(A1, ld1, c1, A2, ld2, c2, m, a.chunk_rows, a.rows,
                                                                  part);
  k_gram_reduce<<<(a.c * a.c + 31) / 32, 256, 0, st>>>(part, a.chunks, a.c, a.rows, G);
  return cudaGetLastError();
}

cudaError_t launch_gram_grouped(const GramArgs* tab, int nsys, int max_chunks, int max_active, int max_c, bool exact,
                                cudaStream_t st) {
  if (nsys <= 0) return cudaSuccess;
  if (exact) k_gram_part_g<true><<<dim3(max_chunks, max_active, nsys), 256, 0, st>>>(tab);
  else k_gram_part_g<false><<<dim3(max_chunks, max_active, nsys), 256, 0, st>>>(tab);
  k_gram_reduce_g<<<dim3((max_c * max_c + 31) / 32, nsys), 256, 0, st>>>(tab);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// One-CTA Cholesky (lower, in place) of an r x r matrix in shared memory with
// leading dimension ld (r + 1 keeps column reads conflict free).  Right-looking
// with deferred scaling, so a column costs one barrier: step k subtracts
// A[i][k] A[j][k] / d_k from the trailing entries (d_k the pivot, column k
// still unscaled), and the factor L[i][k] = A[i][k] / sqrt(d_k) is formed
// once at the end.  Returns false, uniformly over the block, if a pivot is
// not positive.  `piv` is caller shared scratch of r entries.
// FP64 issue is scarce on this GPU (an FP64 warp instruction holds a
// sub-partition's pipe for 64 cycles however many lanes are active), so in
// the FP64 instance the trailing entries are dealt to the threads densely:
// they are numbered column by column from the right (column r - 1 first), so
// that the entries still to update at step k (column > k) are the first
// (r - 1 - k)(r - k) / 2 of the numbering and every warp but the last runs
// full.  The pivot's reciprocal is taken once, by the thread that owns
// the next pivot: it updates that entry first and starts the FP64 division
// (about 430 cycles here) while the other warps update the rest of the step
// (piv[k] holds 1 / d_k until the end).  Launch with kCholThreads threads.
// ---------------------------------------------------------------------------
constexpr int kCholThreads = 512;
constexpr int kCholItems = (kMaxRank * (kMaxRank - 1) / 2 + kCholThreads - 1) / kCholThreads;

template <typename T>
__device__ bool chol_lower_smem(T* A, int r, int ld, T* piv) {
  if constexpr (sizeof(T) == 4) {
    // FP32: row loops (a warp per row, lanes along it), which measured faster
    // than the dense dealing below, the FP32 pipe being plentiful
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = 0; k < r; ++k) {
      __syncthreads();
      const T d = A[k * ld + k];
      if (!(d > T(0) && isfinite(d))) return false;
      const T rd = T(1) / d;
      for (int i = k + 1 + warp; i < r; i += nw) {
        const T aik = A[i * ld + k] * rd;
        for (int j = k + 1 + lane; j <= i; j += 32) A[i * ld + j] -= aik * A[j * ld + k];
      }
    }
  } else {
    // this thread's trailing entries (i, j), j >= 1, packed as (i << 8) | j
    int ij[kCholItems];
    const int ntrail = (r - 1) * r / 2;
#pragma unroll
    for (int u = 0; u < kCholItems; ++u) {
      const int e = threadIdx.x + kCholThreads * u;
      int packed = 0;
      if (e < ntrail) {
        // the block of column r - 1 - c holds c + 1 entries and starts at c (c + 1) / 2
        int c = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
        if (c * (c + 1) / 2 > e) --c;
        if ((c + 1) * (c + 2) / 2 <= e) ++c;
        const int j = r - 1 - c;
        packed = ((j + e - c * (c + 1) / 2) << 8) | j;
      }
      ij[u] = packed;
    }
    if (threadIdx.x == 0) piv[0] = T(1) / A[0];
    for (int k = 0; k < r; ++k) {
      __syncthreads();
      const T d = A[k * ld + k];
      if (!(d > T(0) && isfinite(d))) return false;
      const T rd = piv[k];
      const int m = r - 1 - k, active = m * (m + 1) / 2;
      // entry (k + 1, k + 1) opens the block of column k + 1: number (m - 1) m / 2
      const int ed = m >= 1 ? (m - 1) * m / 2 : -1;
      if (ed >= 0 && (int)threadIdx.x == ed % kCholThreads) {
        const int i = k + 1;
        const T aik = A[i * ld + k] * rd;
        A[i * ld + i] -= aik * A[i * ld + k];
        piv[i] = T(1) / A[i * ld + i];
      }
#pragma unroll
      for (int u = 0; u < kCholItems; ++u) {
        const int e = (int)threadIdx.x + kCholThreads * u;
        if (e < active && e != ed) {
          const int i = ij[u] >> 8, j = ij[u] & 255;
          const T aik = A[i * ld + k] * rd;
          A[i * ld + j] -= aik * A[j * ld + k];
        }
      }
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < r; k += blockDim.x) piv[k] = T(1) / sqrt(A[k * ld + k]);
  __syncthreads();
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e / r, j = e % r;
    if (j < i) A[i * ld + j] *= piv[j];
  }
  __syncthreads();
  for (int k = threadIdx.x; k < r; k += blockDim.x) A[k * ld + k] = T(1) / piv[k];
  __syncthreads();
  return true;
}

// Alg. 4, first half: Delta, C = chol(Omega^T M Omega + Delta Omega^T Omega)
// (stored as the lower factor L = C^T), and Y_nu^T Y_nu.
__global__ void __launch_bounds__(kCholThreads) k_nys_chol(const double* __restrict__ G, const double* __restrict__ Gyy,
                                                  int r, double eps,
                                                  double* __restrict__ Lout, double* __restrict__ Gnu,
                                                  DevScalars* sc) {
  extern __shared__ double sh[];
  __shared__ double red[33];
  __shared__ double piv[kMaxRank];
  const int ld = r + 1, c = 2 * r;
  double tr = 0.0;
  for (int i = threadIdx.x; i < r; i += blockDim.x) tr += G[(int64_t)i * c + r + i];
  tr = block_sum(tr, red);
  double delta = eps * tr;
  bool ok = false;
  int attempt = 0;
  for (; attempt < 4; ++attempt) {
#pragma unroll 2
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
      const int i = e / r, j = e % r;
      const double oty = 0.5 * (G[(int64_t)i * c + r + j] + G[(int64_t)j * c + r + i]);
      sh[i * ld + j] = oty + delta * G[(int64_t)i * c + j];
    }
    __syncthreads();
    ok = chol_lower_smem<double>(sh, r, ld, piv);
    __syncthreads();
    if (ok) break;
    delta *= 10.0;
  }
  if (!ok) {
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) sh[(e / r) * ld + e % r] = (e / r == e % r) ? 1.0 : 0.0;
    if (threadIdx.x == 0) set_status(sc, ADASAP_ENUMERIC, 1);
    __syncthreads();
  }
#pragma unroll 4
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e / r, j = e % r;
    Lout[e] = (j <= i) ? sh[i * ld + j] : 0.0;
    const double yty = Gyy[(int64_t)i * r + j];
    const double cross = G[(int64_t)i * c + r + j] + G[(int64_t)j * c + r + i];
    Gnu[e] = yty + delta * cross + delta * delta * G[(int64_t)i * c + j];
  }
  if (threadIdx.x == 0) {
    sc->delta = delta;
    sc->chol_retries = attempt;
  }
}

// Column-wise triangular solves with the lower factor L (r x r, row-major):
//   upper == 0:  L X = R'     upper == 1:  L^T X = R'
// where R' = trans ? R^T : R.  L and the reciprocals of its diagonal are
// staged in shared memory; one warp per right-hand side column solves in column
// (axpy) form -- lane l holds rows l, l + 32, ...; at step i the owner of row i
// finishes x_i, broadcasts it, and every lane subtracts L[k][i] x_i (lower) or
// L[i][k] x_i (upper) from its rows still to come, so a step needs no
// reduction (half the FP64 instructions of the dot-product form).  A lane
// holds KJ = ceil(r / 32) rows, so a step issues no FP64 instruction for a
// group of 32 rows that lies wholly past r.
constexpr int kTrsmWarps = 4;
template <typename T, int KJ>
__global__ void __launch_bounds__(32 * kTrsmWarps) k_trsm(const double* __restrict__ L, int r,
                                                          const double* __restrict__ R, int trans, int upper,
                                                          double* __restrict__ X, float* __restrict__ X32, int t32) {
  extern __shared__ double shd_trsm[];
  const int ld = r + 1;
  T* sL = reinterpret_cast<T*>(shd_trsm);  // r x (r + 1)
  T* rinv = sL + r * ld;                  // r
  // L (FP64, 16-byte aligned) in batches of 16 double2 loads a thread, all issued
  // before any is stored: a handful of round trips to L2 instead of one per entry
  {
    const int n2 = r * r / 2;
    const double2* L2 = reinterpret_cast<const double2*>(L);
    for (int base = threadIdx.x; base < n2; base += 16 * blockDim.x) {
      double2 v[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int e2 = base + u * blockDim.x;
        v[u] = e2 < n2 ? __ldg(L2 + e2) : make_double2(0.0, 0.0);
      }
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int e = 2 * (base + u * blockDim.x);
        if (e < 2 * n2) {
          sL[(e / r) * ld + e % r] = (T)v[u].x;
          sL[((e + 1) / r) * ld + (e + 1) % r] = (T)v[u].y;
        }
      }
    }
    if ((r * r) & 1) {
      const int e = r * r - 1;
      if (threadIdx.x == 0) sL[(e / r) * ld + e % r] = (T)L[e];
    }
  }
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int col = blockIdx.x * kTrsmWarps + warp;
  T x[KJ];
#pragma unroll
  for (int j = 0; j < KJ; ++j) {
    const int k = lane + 32 * j;
    x[j] = (col < r && k < r) ? (T)(trans ? R[(int64_t)col * r + k] : R[(int64_t)k * r + col]) : T(0);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < r; i += blockDim.x) rinv[i] = T(1) / sL[i * ld + i];
  __syncthreads();
  if (col >= r) return;
  for (int step = 0; step < r; ++step) {
    const int i = upper ? r - 1 - step : step;
    const int jo = i >> 5, lo = i & 31;
    T xi = x[0];
#pragma unroll
    for (int j = 1; j < KJ; ++j)
      if (jo == j) xi = x[j];
    xi = __shfl_sync(full, xi * rinv[i], lo);
#pragma unroll
    for (int j = 0; j < KJ; ++j) {
      const int k = lane + 32 * j;
      // a group of 32 rows with none left to update issues no FP64 instruction
      // (a predicated-off one would still hold the sub-partition's FP64 pipe)
      if (!upper ? (32 * j + 31 > i) : (32 * j < i)) {
        if (k == i) x[j] = xi;
        else if (!upper ? (k > i && k < r) : (k < i)) x[j] -= (upper ? sL[i * ld + k] : sL[k * ld + i]) * xi;
      } else if (j == jo && k == i) {
        x[j] = xi;
      }
    }
  }
#pragma unroll
  for (int j = 0; j < KJ; ++j) {
    const int k = lane + 32 * j;
    if (k < r) {
      X[(int64_t)k * r + col] = (double)x[j];
      if (X32) X32[t32 ? (int64_t)col * r + k : (int64_t)k * r + col] = (float)x[j];
    }
  }
}

// X32 (optional): an FP32 copy of X, transposed when t32 (the form k_make_u reads)
template <typename T = double>
static cudaError_t trsm(const double* L, int r, const double* R, int trans, int upper, double* X, cudaStream_t st,
                        float* X32 = nullptr, int t32 = 0) {
  if (reinterpret_cast<uintptr_t>(L) & 15u) return cudaErrorMisalignedAddress;   // staged by double2 loads
  const size_t smem = ((size_t)r * (r + 1) + r) * sizeof(T);
  const dim3 grid((r + kTrsmWarps - 1) / kTrsmWarps), block(32 * kTrsmWarps);
  switch ((r + 31) / 32) {
    case 1: k_trsm<T, 1><<<grid, block, smem, st>>>(L, r, R, trans, upper, X, X32, t32); break;
    case 2: k_trsm<T, 2><<<grid, block, smem, st>>>(L, r, R, trans, upper, X, X32, t32); break;
    case 3: k_trsm<T, 3><<<grid, block, smem, st>>>(L, r, R, trans, upper, X, X32, t32); break;
    default: k_trsm<T, 4><<<grid, block, smem, st>>>(L, r, R, trans, upper, X, X32, t32); break;
  }
  return cudaGetLastError();
}

// Eigenvectors of the symmetric PSD r x r matrix A by one-sided (Hestenes)
// Jacobi in FP32: W = A V is rotated column pair by column pair until its
// columns are orthogonal; then A V = W and, A being PSD, V holds A's
// eigenvectors (the eigenvalues are refined in FP64 by k_rayleigh).
// Parallel round-robin ordering: in each of the r2 - 1 rounds of a sweep the
// r2/2 disjoint pairs are rotated concurrently, one half-warp per pair, so a
// round needs one barrier.  W and V are column-major in shared memory; the
// squared column norms are carried along (updated exactly for each rotation and
// recomputed every sweep), so a pair needs one dot product.  A pair is skipped
// when |w_p . w_q| <= 1e-6 |w_p| |w_q| or when it is below what the columns'
// absolute FP32 noise can produce; sweeps stop when one rotates nothing (at
// most kJacobiSweeps; Jacobi converges quadratically).
// The rounds are bound by instruction issue on the one SM, so a pair is
// handled by 16 lanes with eight rows each (float4 slots l and l + 16 of the
// column, so that a half-warp touches one contiguous 256-byte span; packed
// f32x2 arithmetic), the two pairs of a warp share every shuffle, and every lane
// of a pair computes the rotation itself (no broadcast: 0.70 -> 0.60 us a round
// at r = 50, 1.33 -> 1.22 us at r = 100).  A two-sided form on the r x r matrix
// (angles from three entries, no dot products, 2 x 2 block updates) converged in
// fewer sweeps but took longer a round (0.84 us at r = 50) and was not taken.
constexpr int kJacobiSweeps = 12;
static_assert(kMaxRank == 128, "Jacobi column slices assume 16 lanes x 8 rows");

__device__ __forceinline__ float2 f2lo(float4 x) { return make_float2(x.x, x.y); }
__device__ __forceinline__ float2 f2hi(float4 x) { return make_float2(x.z, x.w); }
__device__ __forceinline__ float4 f4(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }
// (c a - s b, s a + c b) on four rows
__device__ __forceinline__ void rotate4(float4& a, float4& b, float2 c2, float2 s2, float2 ns2) {
  const float2 alo = f2lo(a), ahi = f2hi(a), blo = f2lo(b), bhi = f2hi(b);
  a = f4(ffma2(c2, alo, fmul2(ns2, blo)), ffma2(c2, ahi, fmul2(ns2, bhi)));
  b = f4(ffma2(s2, alo, fmul2(c2, blo)), ffma2(s2, ahi, fmul2(c2, bhi)));
}

__global__ void __launch_bounds__(1024) k_jacobi(const double* __restrict__ A, int r, float* __restrict__ Vout,
                                                 DevScalars* sc) {
  extern __shared__ float4 shj[];
  const int r2 = r + (r & 1);
  const int cs = (r2 + 3) / 4;   // float4 per column (<= 32)
  const int ld = 4 * cs;         // floats per column
  float4* w = shj;               // r2 columns x cs float4
  float4* v = shj + r2 * cs;
  __shared__ float nrm[kMaxRank];
  __shared__ float mxs[32];
  __shared__ int rot_flag;   // set by any pair rotated in the current sweep
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int hl = lane & 15, hsel = lane >> 4;
  const unsigned full = 0xffffffffu;
  const int s0 = hl, s1 = hl + 16;  // this lane's two float4 slots of a column
  const bool has0 = s0 < cs, has1 = s1 < cs;
  double mx = 0.0;
  for (int i = threadIdx.x; i < r; i += blockDim.x) mx = fmax(mx, fabs(A[(int64_t)i * r + i]));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(full, mx, o));
  if (lane == 0) mxs[warp] = (float)mx;
  if (threadIdx.x == 0) rot_flag = 0;
  __syncthreads();
  float amax = 0.f;
  for (int k = 0; k < nw; ++k) amax = fmaxf(amax, mxs[k]);
  const double scale = amax > 0.f ? 1.0 / (double)amax : 1.0;
  float* wf = reinterpret_cast<float*>(w);
  float* vf = reinterpret_cast<float*>(v);
#pragma unroll 4
  for (int e = threadIdx.x; e < r2 * ld; e += blockDim.x) {
    const int col = e / ld, row = e % ld;
    wf[e] = (row < r && col < r) ? (float)(A[(int64_t)row * r + col] * scale) : 0.0f;
    vf[e] = (row == col) ? 1.0f : 0.0f;
  }
  __syncthreads();
  const int half = r2 / 2;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  float noise2 = 0.f;
  int sweep = 0;
  for (; sweep < kJacobiSweeps; ++sweep) {
    // exact squared column norms at the start of every sweep, one half-warp per column
    for (int c0 = 2 * warp; c0 < r2; c0 += 2 * nw) {  // warp-uniform trip count (shuffles below)
      const int col = c0 + hsel;
      const bool ok = col < r2;
      const float4 x0 = (ok && has0) ? w[col * cs + s0] : z4;
      const float4 x1 = (ok && has1) ? w[col * cs + s1] : z4;
      float t = fmaf(x0.x, x0.x, fmaf(x0.y, x0.y, fmaf(x0.z, x0.z, x0.w * x0.w)));
      t = fmaf(x1.x, x1.x, fmaf(x1.y, x1.y, fmaf(x1.z, x1.z, fmaf(x1.w, x1.w, t))));
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) t += __shfl_xor_sync(full, t, o);
      if (ok && hl == 0) nrm[col] = t;
    }
    __syncthreads();
    if (sweep == 0) {
      float nmax = 0.f;
      for (int k = 0; k < r2; ++k) nmax = fmaxf(nmax, nrm[k]);
      // absolute FP32 noise carried by every column after rotations against the largest
      const float noise = 4.0f * 1.1920929e-7f * sqrtf(nmax);
      noise2 = noise * noise;
    }
    for (int round = 0; round < r2 - 1; ++round) {
      const int m = 2 * warp + hsel;  // this half-warp's pair
      const bool act = m < half;
      int p = 0, q = 0;
      if (m == 0) {
        p = round;
        q = r2 - 1;
      } else {
        p = round + m;
        if (p >= r2 - 1) p -= r2 - 1;
        q = round - m;
        if (q < 0) q += r2 - 1;
      }
      if (p > q) {
        const int t = p;
        p = q;
        q = t;
      }
      float4 a0 = z4, a1 = z4, b0 = z4, b1 = z4;
      float al = 0.f, be = 0.f;
      if (act) {
        if (has0) {
          a0 = w[p * cs + s0];
          b0 = w[q * cs + s0];
        }
        if (has1) {
          a1 = w[p * cs + s1];
          b1 = w[q * cs + s1];
        }
        al = nrm[p];
        be = nrm[q];
      }
      float2 g2 = fmul2(f2lo(a0), f2lo(b0));
      g2 = ffma2(f2hi(a0), f2hi(b0), g2);
      g2 = ffma2(f2lo(a1), f2lo(b1), g2);
      g2 = ffma2(f2hi(a1), f2hi(b1), g2);
      float g = g2.x + g2.y;
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) g += __shfl_xor_sync(full, g, o);
      // rotation parameters, on every lane of the half-warp: the butterfly above leaves
      // the same sum in each lane (each level adds the same two values, in either order),
      // so all of them take the same decision and rotation without a broadcast
      // |g| > 1e-6 |w_p| |w_q|  and  |g| > noise sqrt(|w_p|^2 + |w_q|^2)
      const float gg = g * g;
      const bool doit = act && gg > 1e-12f * al * be && gg > noise2 * (al + be);
      if (doit) {
        const float zeta = __fdividef(be - al, 2.0f * g);
        const float z2 = fmaf(zeta, zeta, 1.0f);
        const float t = copysignf(1.0f, zeta) * __fdividef(1.0f, fabsf(zeta) + z2 * rsqrtf(z2));
        const float c = rsqrtf(fmaf(t, t, 1.0f));
        const float sn = c * t;
        // norms after a rotation that zeroes the pair's inner product (every lane has
        // read nrm[p] and nrm[q] above, before this warp-synchronous write)
        __syncwarp(hsel ? 0xffff0000u : 0x0000ffffu);
        if (hl == 0) {
          nrm[p] = c * c * al - 2.0f * c * sn * g + sn * sn * be;
          nrm[q] = sn * sn * al + 2.0f * c * sn * g + c * c * be;
        }
        const float2 c2 = make_float2(c, c), s2 = make_float2(sn, sn), ns2 = make_float2(-sn, -sn);
        if (has0) {
          rotate4(a0, b0, c2, s2, ns2);
          w[p * cs + s0] = a0;
          w[q * cs + s0] = b0;
          float4 x = v[p * cs + s0], y = v[q * cs + s0];
          rotate4(x, y, c2, s2, ns2);
          v[p * cs + s0] = x;
          v[q * cs + s0] = y;
        }
        if (has1) {
          rotate4(a1, b1, c2, s2, ns2);
          w[p * cs + s1] = a1;
          w[q * cs + s1] = b1;
          float4 x = v[p * cs + s1], y = v[q * cs + s1];
          rotate4(x, y, c2, s2, ns2);
          v[p * cs + s1] = x;
          v[q * cs + s1] = y;
        }
      }
      if (doit) rot_flag = 1;
      __syncthreads();
    }
    const int rotated = rot_flag;
    __syncthreads();
    if (threadIdx.x == 0) rot_flag = 0;
    if (!rotated) break;
  }
  if (threadIdx.x == 0) sc->jacobi_sweeps = sweep;
  // Vout row-major: Vout[k * r + i] = component k of eigenvector i
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int k = e / r, i = e % r;
    Vout[e] = vf[i * ld + k];
  }
}

// lambda_i = v_i^T A v_i / v_i^T v_i in FP64 (one block per eigenvector).  Few
// instructions by design: the blocks run beside the block-row product on its SMs,
// and a heavier form (every lane busy on FP64 work) measured slower there.
__global__ void k_rayleigh(const double* __restrict__ A, const float* __restrict__ V, int r, double* __restrict__ lam) {
  __shared__ double red[33];
  const int i = blockIdx.x;
  double num = 0.0, den = 0.0;
  for (int k = threadIdx.x; k < r; k += blockDim.x) {
    double w = 0.0;
#pragma unroll 8
    for (int j = 0; j < r; ++j) w += A[(int64_t)k * r + j] * (double)V[(int64_t)j * r + i];
    const double vk = (double)V[(int64_t)k * r + i];
    num += vk * w;
    den += vk * vk;
  }
  num = block_sum(num, red);
  den = block_sum(den, red);
  if (threadIdx.x == 0) lam[i] = num / den;
}

// Key of a double whose unsigned order is the order of the values (sign bit
// set for non-negatives, all bits flipped for negatives), so that ranks are
// taken with integer compares rather than on the FP64 pipe.
__device__ __forceinline__ unsigned long long order_key(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

// Sort eigenpairs (descending), S = max(0, Sigma^2 - Delta), rho = S_r + lambda,
// and T' = V Sigma^{-1} (columns normalised) for U = Y_nu L^{-T} T'.  V is staged
// in shared memory; each column norm is summed in four parts by four groups of
// 64 threads, and each column of T' takes one reciprocal (FP64 division and
// square root cost about 430 and 675 cycles on this GPU).
constexpr int kFinThreads = 256;
__global__ void __launch_bounds__(kFinThreads) k_nys_finalize(const double* __restrict__ lam,
                                                               const float* __restrict__ V, int r, double lam_reg,
                                                               DevScalars* sc, double* __restrict__ S,
                                                               double* __restrict__ keep, double* __restrict__ Tp) {
  extern __shared__ float sV[];   // r x r
  __shared__ int perm[kMaxRank];
  __shared__ unsigned long long key[kMaxRank];
  __shared__ double n2p[4][kMaxRank];
  __shared__ double rcp[kMaxRank];
  const int tid = threadIdx.x;
  const double delta = sc->delta;
#pragma unroll 8
  for (int e = tid; e < r * r; e += kFinThreads) sV[e] = V[e];
  for (int i = tid; i < r; i += kFinThreads) {
    key[i] = order_key(lam[i]);
    perm[i] = i;   // stays a valid index even if a NaN leaves a rank unfilled
  }
  __syncthreads();
  for (int i = tid; i < r; i += kFinThreads) {
    const unsigned long long ki = key[i];
    int rank = 0;
    for (int j = 0; j < r; ++j) {
      const unsigned long long kj = key[j];
      rank += (kj > ki) || (kj == ki && j < i);
    }
    perm[rank] = i;
  }
  {
    const int part = tid >> 6, kq = (r + 3) / 4, k0 = part * kq, k1 = min(r, k0 + kq);
    for (int i = tid & 63; i < r; i += 64) {
      double n2 = 0.0;
      for (int k = k0; k < k1; ++k) {
        const double v = (double)sV[k * r + i];
        n2 = fma(v, v, n2);
      }
      n2p[part][i] = n2;
    }
  }
  __syncthreads();
  for (int q = tid; q < r; q += kFinThreads) {
    const int i = perm[q];
    const double li = lam[i];
    const double sq = fmax(0.0, li - delta);
    S[q] = sq;
    keep[q] = sq > 0.0 ? 1.0 : 0.0;
    const double sg = li > 0.0 ? sqrt(li) : 0.0;
    const double nr = sqrt((n2p[0][i] + n2p[1][i]) + (n2p[2][i] + n2p[3][i]));
    // a dropped eigenpair (S_q = 0) contributes exactly nothing to either Woodbury form
    // (eqs. inv_nys_woodbury and inv_sqrt_nys_woodbury), so its U column is set to 0
    // instead of V / sigma with sigma ~ 0
    rcp[q] = (sq > 0.0 && sg > 0.0) ? 1.0 / (nr * sg) : 0.0;
    if (!isfinite(li)) set_status(sc, ADASAP_ENUMERIC, 2);
    if (q == r - 1) sc->rho = sq + lam_reg;
  }
  __syncthreads();
  for (int e = tid; e < r * r; e += kFinThreads) {
    const int k = e / r, q = e % r;
    Tp[e] = (double)sV[k * r + perm[q]] * rcp[q];
  }
}

// U = (A1 + delta A2) T'  (b x r), T' (r x r) given in FP32 by the triangular
// solve that forms it (converted once, not in every block), delta = sc->delta or
// 0 when A2 is NULL.
//   Nystrom: A1 = M Omega, A2 = Omega, T' = T      (U = Y_nu T)
//   QR:      A1 = Omega,   A2 = NULL,  T' = L^{-T} (Omega R^{-1}, R = L^T)
// A block takes kMuRows rows of U; warp w of its 8 rows 8w .. 8w + 7 and lane l of
// the columns l + 32 q (q < CQ = ceil(r / 32)), so that each k costs two broadcast
// float4 loads of the (transposed) rows and CQ loads of T' for 8 CQ FMAs.
constexpr int kMuRows = 64;
constexpr int kMuLd = kMuRows + 4;   // transposed rows: 4-way conflicts on the staging stores
template <int CQ>
__global__ void __launch_bounds__(256) k_make_u(const float* __restrict__ A1, const float* __restrict__ A2, int64_t b,
                                                int r, const float* __restrict__ T32, const DevScalars* sc,
                                                float* __restrict__ U) {
  extern __shared__ __align__(16) float shm[];
  float* sT = shm;                          // r x r
  float* sY = shm + ((r * r + 3) & ~3);     // [k][row], leading dimension kMuLd
  const float fdelta = A2 ? (float)sc->delta : 0.0f;
  // T' and the block's rows (both 16-byte aligned: row0 r is a multiple of 4) by
  // float4 loads, each batch issued before any is stored
  {
    const int n4 = r * r / 4;
    const float4* T4 = reinterpret_cast<const float4*>(T32);
    for (int base = threadIdx.x; base < n4; base += 8 * blockDim.x) {
      float4 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e4 = base + u * blockDim.x;
        v[u] = e4 < n4 ? __ldg(T4 + e4) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e4 = base + u * blockDim.x;
        if (e4 < n4) reinterpret_cast<float4*>(sT)[e4] = v[u];
      }
    }
    for (int e = 4 * n4 + threadIdx.x; e < r * r; e += blockDim.x) sT[e] = T32[e];
  }
  const int64_t row0 = (int64_t)blockIdx.x * kMuRows;
  {
    // rows row0 .. row0 + kMuRows - 1 are kMuRows r contiguous floats of A1 (and A2)
    const int64_t nval = min((int64_t)kMuRows, b - row0) * r;   // valid floats
    const int n4 = kMuRows * r / 4;
    const float4* Y1 = reinterpret_cast<const float4*>(A1 + row0 * r);
    const float4* Y2 = A2 ? reinterpret_cast<const float4*>(A2 + row0 * r) : nullptr;
    for (int base = threadIdx.x; base < n4; base += 4 * blockDim.x) {
      float4 v1[4], v2[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e4 = base + u * blockDim.x;
        const int64_t f = 4 * (int64_t)e4;
        v1[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        v2[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (e4 < n4 && f + 3 < nval) {
          v1[u] = __ldg(Y1 + e4);
          if (Y2) v2[u] = __ldg(Y2 + e4);
        } else if (e4 < n4 && f < nval) {   // the float4 that holds the last valid rows' end
          const float* y1 = A1 + row0 * r + f;
          const float* y2 = A2 ? A2 + row0 * r + f : nullptr;
          v1[u].x = y1[0];
          if (y2) v2[u].x = y2[0];
          if (f + 1 < nval) { v1[u].y = y1[1]; if (y2) v2[u].y = y2[1]; }
          if (f + 2 < nval) { v1[u].z = y1[2]; if (y2) v2[u].z = y2[2]; }
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e4 = base + u * blockDim.x;
        if (e4 >= n4) continue;
        const float a1[4] = {v1[u].x, v1[u].y, v1[u].z, v1[u].w};
        const float a2[4] = {v2[u].x, v2[u].y, v2[u].z, v2[u].w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int e = 4 * e4 + t;
          const int rr = e / r, k = e % r;
          float v = 0.0f;
          if ((int64_t)e < nval) v = A2 ? fmaf(fdelta, a2[t], a1[t]) : a1[t];
          sY[k * kMuLd + rr] = v;
        }
      }
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float acc[8][CQ];
#pragma unroll
  for (int u = 0; u < 8; ++u)
#pragma unroll
    for (int q = 0; q < CQ; ++q) acc[u][q] = 0.0f;
  for (int k = 0; k < r; ++k) {
    const float4 y0 = *reinterpret_cast<const float4*>(&sY[k * kMuLd + warp * 8]);
    const float4 y1 = *reinterpret_cast<const float4*>(&sY[k * kMuLd + warp * 8 + 4]);
    const float yv[8] = {y0.x, y0.y, y0.z, y0.w, y1.x, y1.y, y1.z, y1.w};
#pragma unroll
    for (int q = 0; q < CQ; ++q) {
      const int c = lane + 32 * q;
      const float tv = c < r ? sT[k * r + c] : 0.0f;
#pragma unroll
      for (int u = 0; u < 8; ++u) acc[u][q] = fmaf(yv[u], tv, acc[u][q]);
    }
  }
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int64_t row = row0 + warp * 8 + u;
    if (row >= b) continue;
#pragma unroll
    for (int q = 0; q < CQ; ++q) {
      const int c = lane + 32 * q;
      if (c < r) U[row * r + c] = acc[u][q];
    }
  }
}

static size_t make_u_smem(int r) { return ((size_t)((r * r + 3) & ~3) + (size_t)kMuLd * r) * sizeof(float); }

static cudaError_t make_u(const float* A1, const float* A2, int64_t b, int r, const float* T32, const DevScalars* sc,
                          float* U, cudaStream_t st) {
  // the kernel stages by float4 loads (its operands are allocation bases)
  if ((reinterpret_cast<uintptr_t>(A1) | reinterpret_cast<uintptr_t>(A2) | reinterpret_cast<uintptr_t>(T32)) & 15u)
    return cudaErrorMisalignedAddress;
  const unsigned grid = (unsigned)((b + kMuRows - 1) / kMuRows);
  const size_t smem = make_u_smem(r);
  switch ((r + 31) / 32) {
    case 1: k_make_u<1><<<grid, 256, smem, st>>>(A1, A2, b, r, T32, sc, U); break;
    case 2: k_make_u<2><<<grid, 256, smem, st>>>(A1, A2, b, r, T32, sc, U); break;
    case 3: k_make_u<3><<<grid, 256, smem, st>>>(A1, A2, b, r, T32, sc, U); break;
    default: k_make_u<4><<<grid, 256, smem, st>>>(A1, A2, b, r, T32, sc, U); break;
  }
  return cudaGetLastError();
}

// FP64 Cholesky of an r x r SPD matrix into a lower factor (identity and a
// status on failure), one CTA.
template <typename T>
__global__ void __launch_bounds__(kCholThreads) k_chol_plain(const double* __restrict__ G, int r, double* __restrict__ L,
                                                    DevScalars* sc, int detail) {
  extern __shared__ double shd_chol[];
  T* sh = reinterpret_cast<T*>(shd_chol);
  __shared__ T piv[kMaxRank];
  const int ld = r + 1;
#pragma unroll 8
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) sh[(e / r) * ld + e % r] = (T)G[e];
  __syncthreads();
  const bool ok = chol_lower_smem<T>(sh, r, ld, piv);
  __syncthreads();
  if (!ok && threadIdx.x == 0) set_status(sc, ADASAP_ENUMERIC, detail);
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e / r, j = e % r;
    L[e] = ok ? ((j <= i) ? (double)sh[i * ld + j] : 0.0) : (i == j ? 1.0 : 0.0);
  }
}

// Thin QR of the Gaussian test matrix by CholeskyQR2 (Omega <- Omega R^{-1}
// twice, Omega^T Omega = R^T R in FP64), in place; tmp is b x r scratch.
cudaError_t launch_orthonormalize(CoreBufs& cb, float* Om, float* tmp, DevScalars* sc, cudaStream_t st) {
  const int r = cb.r;
  cudaError_t e;
  for (int pass = 0; pass < 2; ++pass) {
    const float* src = pass == 0 ? Om : tmp;
    float* dst = pass == 0 ? tmp : Om;
    // pass 1 exact when Omega is near square (cond(Omega)^2 can exceed FP32's reach);
    // for b >= 4r a Gaussian Omega has cond ~ (1 + sqrt(r/b)) / (1 - sqrt(r/b)) <= 3.
    // Pass 2 sees cond ~ 1.
    // For b >= 4r the factorisations need only FP32 arithmetic (the target is FP32
    // orthogonality and cond(Omega) <= 3), which avoids B300's slow FP64 latency chains.
    const bool exact = pass == 0 && cb.b < 4 * (int64_t)r;
    const bool wide64 = cb.b < 4 * (int64_t)r;
    if ((e = launch_gram(src, r, r, nullptr, 0, 0, cb.b, cb.gram_part, cb.gram_chunks, cb.X1, exact, st))) return e;
    if (wide64) {
      k_chol_plain<double><<<1, kCholThreads, (size_t)r * (r + 1) * sizeof(double), st>>>(cb.X1, r, cb.Lc, sc, 6);
      if ((e = trsm<double>(cb.Lc, r, cb.Ident, 0, 0, cb.A, st, cb.T32, 1))) return e;   // A = L^{-1}
    } else {
      k_chol_plain<float><<<1, kCholThreads, (size_t)r * (r + 1) * sizeof(double), st>>>(cb.X1, r, cb.Lc, sc, 6);
      if ((e = trsm<float>(cb.Lc, r, cb.Ident, 0, 0, cb.A, st, cb.T32, 1))) return e;
    }
    if ((e = make_u(src, nullptr, cb.b, r, cb.T32, sc, dst, st))) return e;   // T32 = (L^{-1})^T
  }
  return cudaGetLastError();
}

cudaError_t launch_nystrom_grams(CoreBufs& cb, const float* Om, const float* Ysk, cudaStream_t st) {
  const int r = cb.r;
  cudaError_t e;
  // Gram of [Omega | M Omega] -> (Omega^T Omega, Omega^T Y, Y^T Y)
  // (the Y^T Y block of this one is not used: the exact Gram below supplies it)
  if ((e = launch_gram(Om, r, r, Ysk, r, r, cb.b, cb.gram_part, cb.gram_chunks, cb.G, false, st, r))) return e;
  return launch_gram(Ysk, r, r, nullptr, 0, 0, cb.b, cb.gram_part, cb.gram_chunks, cb.Gyy, true, st);
}

cudaError_t launch_nystrom_core(CoreBufs& cb, double eps, double lam, DevScalars* sc, const float* Om,
                                const float* Ysk, cudaStream_t st) {
  const int r = cb.r;
  cudaError_t e;
  const size_t sm_chol = (size_t)r * (r + 1) * sizeof(double);
  k_nys_chol<<<1, kCholThreads, sm_chol, st>>>(cb.G, cb.Gyy, r, eps, cb.Lc, cb.Gnu, sc);
  // A = L^{-1} Gnu L^{-T}  (= C^{-T} Y_nu^T Y_nu C^{-1} = B^T B)
  if ((e = trsm(cb.Lc, r, cb.Gnu, 0, 0, cb.X1, st))) return e;
  if ((e = trsm(cb.Lc, r, cb.X1, 1, 0, cb.A, st))) return e;
  const int r2 = r + (r & 1);
  k_jacobi<<<1, 32 * ((r2 / 2 + 1) / 2), (size_t)2 * r2 * (4 * ((r2 + 3) / 4)) * sizeof(float), st>>>(
      cb.A, r, cb.V32, sc);
  k_rayleigh<<<r, 128, 0, st>>>(cb.A, cb.V32, r, cb.lam);
  k_nys_finalize<<<1, kFinThreads, (size_t)r * r * sizeof(float), st>>>(cb.lam, cb.V32, r, lam, sc, cb.S, cb.keep,
                                                                        cb.X1);
  // T = L^{-T} T'
  if ((e = trsm(cb.Lc, r, cb.X1, 0, 1, cb.T, st, cb.T32, 0))) return e;
  return make_u(Ysk, Om, cb.b, r, cb.T32, sc, cb.U, st);
}

// M = (rho S^{-1} + U^T U)^{-1} on the kept eigenpairs (App. C.2, stabilised
// form; a dropped pair keeps a unit diagonal and zero coupling).  With U close
// to orthonormal the matrix is D + E with D = diag(1 + rho / S_k) in [1, inf)
// and E small, i.e. well conditioned after diagonal scaling, so the inverse is
// taken in FP32 by Gauss-Jordan elimination without pivoting (its pivots are
// those of the Cholesky factorisation; a non-positive one is reported).  The
// elimination ping-pongs between two copies, one barrier per column.
constexpr int kWfThreads = 512;
__device__ __forceinline__ void set4(float4& x, int c, float v) {
  if (c == 0) x.x = v;
  else if (c == 1) x.y = v;
  else if (c == 2) x.z = v;
  else x.w = v;
}
// KI items (a float4 of a row each) per thread, fixed over the elimination; the
// pivot's reciprocal is taken once per column, by the thread that finishes the
// next pivot, and staged in shared memory.
template <int KI>
__global__ void __launch_bounds__(kWfThreads) k_wfactor(const double* __restrict__ UtU, int r,
                                                        const double* __restrict__ S, const double* __restrict__ keep,
                                                        DevScalars* sc, float* __restrict__ Minv,
                                                        float* __restrict__ Gu) {
  extern __shared__ float4 shw4[];
  __shared__ double sdiag[kMaxRank];
  __shared__ float skeep[kMaxRank];
  __shared__ float prcp[kMaxRank];
  const int nb = (r + 3) / 4;    // float4 per row
  const int ld = 4 * nb;         // rows padded with zeros to a multiple of 4
  float4* buf0 = shw4;
  float4* buf1 = shw4 + r * nb;
  const double rho = sc->rho;
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    const double kp = keep[i];
    skeep[i] = (float)kp;
    sdiag[i] = kp > 0.0 ? rho / S[i] : 1.0;
  }
  __syncthreads();
#pragma unroll 4
  for (int e = threadIdx.x; e < r * ld; e += blockDim.x) {
    const int i = e / ld, j = e % ld;
    float val = 0.0f;
    if (j < r) {
      const double g = UtU[i * r + j];
      const float gf = (float)g;
      Gu[i * r + j] = gf;
      // keep is 0 or 1, so keep_i keep_j g is g or a zero of g's sign
      val = (i == j) ? (float)((double)(skeep[i] * skeep[j]) * g + sdiag[i]) : gf * (skeep[i] * skeep[j]);
    }
    reinterpret_cast<float*>(buf0)[e] = val;
  }
  int it_i[KI], it_j[KI];
#pragma unroll
  for (int m = 0; m < KI; ++m) {
    const int e = threadIdx.x + m * kWfThreads;
    it_i[m] = e < r * nb ? e / nb : -1;
    it_j[m] = e < r * nb ? e % nb : 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) prcp[0] = 1.0f / reinterpret_cast<const float*>(buf0)[0];
  bool ok = true;
  int cur = 0;
  for (int k = 0; k < r; ++k) {
    __syncthreads();
    const float4* A4 = cur ? buf1 : buf0;
    float4* B4 = cur ? buf0 : buf1;
    const float* Af = reinterpret_cast<const float*>(A4);
    const float pv = Af[k * ld + k];
    if (!(pv > 0.0f && isfinite(pv))) {
      ok = false;
      break;
    }
    const float rp = prcp[k];
    const int kb = k >> 2, kc = k & 3;
    float4 ov[KI];
#pragma unroll
    for (int m = 0; m < KI; ++m) {
      const int i = it_i[m], jb = it_j[m];
      if (i < 0) continue;
      const float4 akj = A4[k * nb + jb];
      float4 o;
      if (i == k) {
        o = make_float4(akj.x * rp, akj.y * rp, akj.z * rp, akj.w * rp);
        if (jb == kb) set4(o, kc, rp);
      } else {
        const float fi = Af[i * ld + k] * rp;
        const float4 aij = A4[i * nb + jb];
        o = make_float4(fmaf(-fi, akj.x, aij.x), fmaf(-fi, akj.y, aij.y), fmaf(-fi, akj.z, aij.z),
                        fmaf(-fi, akj.w, aij.w));
        if (jb == kb) set4(o, kc, -fi);
      }
      ov[m] = o;
    }
#pragma unroll
    for (int m = 0; m < KI; ++m) {
      const int i = it_i[m], jb = it_j[m];
      if (i < 0) continue;
      B4[i * nb + jb] = ov[m];
      if (i == k + 1 && jb == ((k + 1) >> 2)) {
        const int c = (k + 1) & 3;
        prcp[k + 1] = 1.0f / (c == 0 ? ov[m].x : c == 1 ? ov[m].y : c == 2 ? ov[m].z : ov[m].w);
      }
    }
    cur ^= 1;
  }
  __syncthreads();
  if (!ok && threadIdx.x == 0) set_status(sc, ADASAP_ENUMERIC, 3);
  const float* Mf = reinterpret_cast<const float*>(cur ? buf1 : buf0);
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e / r, j = e % r;
    Minv[e] = ok ? Mf[i * ld + j] : (i == j ? 1.0f : 0.0f);
  }
}

// Per-iteration constants of the inverse square root (eq. inv_sqrt_nys_woodbury):
// cis_k = (S_k + rho)^{-1/2} - rho^{-1/2}.
__global__ void k_invsqrt_coef(const double* __restrict__ S, int r, const DevScalars* sc, double* __restrict__ cis) {
  const double rho = sc->rho;
  const double irs = 1.0 / sqrt(rho);
  for (int k = threadIdx.x; k < r; k += blockDim.x) cis[k] = 1.0 / sqrt(S[k] + rho) - irs;
}

cudaError_t launch_woodbury_factor(CoreBufs& cb, double lam, DevScalars* sc, cudaStream_t st) {
  (void)lam;
  const int r = cb.r;
  cudaError_t e;
  if ((e = launch_gram(cb.U, r, r, nullptr, 0, 0, cb.b, cb.gram_part, cb.gram_chunks, cb.X1, false, st))) return e;
  const size_t smw = (size_t)2 * r * (4 * ((r + 3) / 4)) * sizeof(float);
  const int items = r * ((r + 3) / 4);   // float4 of the r rows
  if (items <= 2 * kWfThreads) k_wfactor<2><<<1, kWfThreads, smw, st>>>(cb.X1, r, cb.S, cb.keep, sc, cb.Minv, cb.Gu);
  else if (items <= 5 * kWfThreads) k_wfactor<5><<<1, kWfThreads, smw, st>>>(cb.X1, r, cb.S, cb.keep, sc, cb.Minv, cb.Gu);
  else k_wfactor<8><<<1, kWfThreads, smw, st>>>(cb.X1, r, cb.S, cb.keep, sc, cb.Minv, cb.Gu);
  k_invsqrt_coef<<<1, 128, 0, st>>>(cb.S, r, sc, cb.cis);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Woodbury applies.
// ---------------------------------------------------------------------------
int utv_chunks_for(int64_t b) { return (int)std::max<int64_t>(1, std::min<int64_t>(148, (b + 127) / 128)); }

// part[ch][o], o = k*s + c: sum over the rows i of chunk ch of U[i][k] v[i][c].
// blockIdx.y selects a group of 2048 outputs (8 per thread).
constexpr int kUtvOut = 8;
__global__ void __launch_bounds__(256) k_utv(const float* __restrict__ U, int64_t b, int r, const float* __restrict__ v,
                                             int s, int64_t ldv, int64_t chunk_rows, double* __restrict__ part) {
  extern __shared__ float shm[];
  float* su = shm;           // 32 x r
  float* sv = shm + 32 * r;  // 32 x s
  const int64_t r0 = (int64_t)blockIdx.x * chunk_rows;
  const int64_t r1 = min(b, r0 + chunk_rows);
  const int nout = r * s;
  const int obase = blockIdx.y * 256 * kUtvOut;
  double acc[kUtvOut];
#pragma unroll
  for (int q = 0; q < kUtvOut; ++q) acc[q] = 0.0;
  for (int64_t s0 = r0; s0 < r1; s0 += 32) {
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * r; e += blockDim.x) {
      const int64_t row = s0 + e / r;
      su[e] = row < r1 ? U[row * r + e % r] : 0.0f;
    }
    for (int e = threadIdx.x; e < 32 * s; e += blockDim.x) {
      const int64_t row = s0 + e / s;
      sv[e] = row < r1 ? v[row * ldv + e % s] : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kUtvOut; ++q) {
      const int o = obase + threadIdx.x + 256 * q;
      if (o < nout) {
        const int k = o / s, c = o % s;
        float f = 0.0f;
        for (int rr = 0; rr < 32; ++rr) f = fmaf(su[rr * r + k], sv[rr * s + c], f);
        acc[q] += (double)f;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < kUtvOut; ++q) {
    const int o = obase + threadIdx.x + 256 * q;
    if (o < nout) part[(int64_t)blockIdx.x * nout + o] = acc[q];
  }
}

// Small FP64 step between U^T v and the apply.  alpha[0] = coefficient of v,
// alpha[1] = 1/||v|| of the input (normalised mode).
// Coefficients of the multi-RHS applies from the k_utv partials, spread over many
// blocks (the FP64 sums of the chunk partials were the bottleneck of a one-block
// form on this GPU's FP64 pipe): thread o sums the chunks of output o = k*s + c.
//   kInv:  qk[o] = keep_k q[o] (FP32), finished by k_wcoef_inv
//   else:  coef[o] = scale q[o] ((S_k + rho)^{-1/2} - rho^{-1/2}), alpha = scale rho^{-1/2}
constexpr int kWcoefThreads = 128;
__global__ void __launch_bounds__(kWcoefThreads) k_wcoef(int mode, const double* __restrict__ part, int chunks, int r,
                                                         int s, const double* __restrict__ S,
                                                         const double* __restrict__ keep,
                                                         const double* __restrict__ sq_part, DevScalars* sc,
                                                         float* __restrict__ coef, float* __restrict__ qk,
                                                         double* __restrict__ alpha) {
  __shared__ double red[33];
  const double rho = sc->rho;
  double scale = 1.0;
  if (mode == kInvSqrtNormalised) {
    double t = 0.0;
    for (int i = threadIdx.x; i < kReduceBlocks; i += blockDim.x) t += sq_part[i];
    t = block_sum(t, red);
    scale = t > 0.0 ? 1.0 / sqrt(t) : 0.0;
  }
  const int nout = r * s;
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o < nout) {
    double q = 0.0;
    for (int ch = 0; ch < chunks; ++ch) q += part[(int64_t)ch * nout + o];
    const int k = o / s;
    if (mode == kInv) qk[o] = (float)(keep[k] * q);
    else coef[o] = (float)(scale * q * (1.0 / sqrt(S[k] + rho) - 1.0 / sqrt(rho)));
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (mode == kInv) {
      alpha[0] = 1.0 / rho;
    } else {
      alpha[0] = scale / sqrt(rho);
      if (mode == kInvSqrtNormalised) alpha[1] = scale;
    }
  }
}

// kInv: coef = -keep . M qk / rho with M = (rho S^{-1} + U^T U)^{-1} (FP32: M is well
// conditioned); block k, thread c.
__global__ void k_wcoef_inv(int r, int s, const double* __restrict__ keep, const float* __restrict__ Minv,
                            const float* __restrict__ qk, DevScalars* sc, float* __restrict__ coef) {
  const int k = blockIdx.x;
  const double rho = sc->rho;
  for (int c = threadIdx.x; c < s; c += blockDim.x) {
    float acc = 0.0f;
    for (int j = 0; j < r; ++j) acc = fmaf(Minv[k * r + j], qk[j * s + c], acc);
    coef[k * s + c] = (float)(-keep[k] * (double)acc / rho);
  }
}

// out[i][c] = alpha v[i][c] + sum_k U[i][k] coef[k][c]; optional per-block
// partials of sum(out^2) and sum(out * dotv) (s == 1).
__global__ void __launch_bounds__(256) k_wapply(const float* __restrict__ U, int64_t b, int r, const float* __restrict__ v,
                                                int s, const float* __restrict__ coef, const double* __restrict__ alpha,
                                                float* __restrict__ out, double* sq_part, double* dot_part,
                                                const float* __restrict__ dotv) {
  extern __shared__ float scoef[];  // r x s
  __shared__ double red[33];
  for (int e = threadIdx.x; e < r * s; e += blockDim.x) scoef[e] = coef[e];
  __syncthreads();
  const float al = (float)alpha[0];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t wstride = (int64_t)gridDim.x * (blockDim.x >> 5);
  double sq = 0.0, dt = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; i < b; i += wstride) {
    if (s == 1) {
      float acc = 0.0f;
      for (int k = lane; k < r; k += 32) acc = fmaf(U[i * r + k], scoef[k], acc);
      acc = warp_sum(acc);
      const float o = fmaf(al, v[i], acc);
      if (lane == 0) {
        out[i] = o;
        sq += (double)o * (double)o;
        if (dotv) dt += (double)o * (double)dotv[i];
      }
    } else {
      for (int c = lane; c < s; c += 32) {
        float acc = 0.0f;
        for (int k = 0; k < r; ++k) acc = fmaf(U[i * r + k], scoef[k * s + c], acc);
        out[i * s + c] = fmaf(al, v[i * s + c], acc);
      }
    }
  }
  if (sq_part) {
    const double t = block_sum(sq, red);
    if (threadIdx.x == 0) sq_part[blockIdx.x] = t;
  }
  if (dot_part) {
    const double t = block_sum(dt, red);
    if (threadIdx.x == 0) dot_part[blockIdx.x] = t;
  }
}

// identity preconditioner (ADASAP-I): out = alpha v with alpha = 1 or 1/||v||
__global__ void k_iapply(int normalised, const float* __restrict__ v, int64_t count, const double* __restrict__ sq_in,
                         float* __restrict__ out, double* __restrict__ alpha, double* sq_part, double* dot_part,
                         const float* __restrict__ dotv) {
  __shared__ double red[33];
  __shared__ double sscale;
  if (threadIdx.x == 0) sscale = 1.0;
  __syncthreads();
  if (normalised) {
    double t = 0.0;
    for (int i = threadIdx.x; i < kReduceBlocks; i += blockDim.x) t += sq_in[i];
    t = block_sum(t, red);
    if (threadIdx.x == 0) sscale = t > 0.0 ? 1.0 / sqrt(t) : 0.0;
    __syncthreads();
  }
  const double scale = sscale;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    alpha[0] = scale;
    if (normalised) alpha[1] = scale;
  }
  double sq = 0.0, dt = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const float o = (float)(scale * (double)v[i]);
    out[i] = o;
    sq += (double)o * (double)o;
    if (dotv) dt += (double)o * (double)dotv[i];
  }
  if (sq_part) {
    const double t = block_sum(sq, red);
    if (threadIdx.x == 0) sq_part[blockIdx.x] = t;
  }
  if (dot_part) {
    const double t = block_sum(dt, red);
    if (threadIdx.x == 0) dot_part[blockIdx.x] = t;
  }
}

cudaError_t launch_woodbury_apply(CoreBufs& cb, int mode, const float* v, int s, float* out, bool want_sq,
                                  bool want_dot, const float* dotv, DevScalars* sc, cudaStream_t st) {
  double* sqp = want_sq ? cb.sq_part : nullptr;
  double* dtp = want_dot ? cb.dot_part : nullptr;
  if (cb.r == 0) {  // identity preconditioner
    k_iapply<<<kReduceBlocks, 256, 0, st>>>(mode == kInvSqrtNormalised, v, cb.b * s, cb.sq_part, out, cb.alpha, sqp,
                                            dtp, dotv);
    return cudaGetLastError();
  }
  const int r = cb.r;
  const int64_t chunk_rows = (cb.b + cb.utv_chunks - 1) / cb.utv_chunks;
  const int ogroups = (r * s + 256 * kUtvOut - 1) / (256 * kUtvOut);
  k_utv<<<dim3(cb.utv_chunks, ogroups), 256, (size_t)(32 * r + 32 * s) * sizeof(float), st>>>(cb.U, cb.b, r, v, s, s,
                                                                                               chunk_rows, cb.utv_part);
  k_wcoef<<<(r * s + kWcoefThreads - 1) / kWcoefThreads, kWcoefThreads, 0, st>>>(
      mode, cb.utv_part, cb.utv_chunks, r, s, cb.S, cb.keep, cb.sq_part, sc, cb.coef, cb.qk, cb.alpha);
  if (mode == kInv) k_wcoef_inv<<<r, 64, 0, st>>>(r, s, cb.keep, cb.Minv, cb.qk, sc, cb.coef);
  k_wapply<<<kReduceBlocks, 256, (size_t)r * s * sizeof(float), st>>>(cb.U, cb.b, r, v, s, cb.coef, cb.alpha, out,
                                                                       sqp, dtp, dotv);
  return cudaGetLastError();
}

// eta = 1 / lambda_hat, lambda_hat = (1/||v_{N-1}||) * sum(w_N . v_{N-1}) (Alg. 5,
// Rayleigh-quotient reading).  A failed factorisation (status != 0) gives eta = 0.
__global__ void k_set_eta(const double* __restrict__ dot_part, int nparts, const double* __restrict__ alpha,
                          DevScalars* sc) {
  __shared__ double red[33];
  double t = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) t += dot_part[i];
  t = block_sum(t, red);
  if (threadIdx.x == 0) {
    const double lam_hat = alpha[1] * t;
    sc->lam_hat = lam_hat;
    double eta = (lam_hat > 0.0 && isfinite(lam_hat)) ? 1.0 / lam_hat : 0.0;
    if (!(lam_hat > 0.0 && isfinite(lam_hat))) set_status(sc, ADASAP_ENUMERIC, 4);
    if (sc->status != 0) eta = 0.0;
    sc->eta = eta;
  }
}

cudaError_t launch_set_eta(CoreBufs& cb, DevScalars* sc, int identity, cudaStream_t st) {
  // (identity preconditioner only: per-block partials of the k_iapply dot product)
  k_set_eta<<<1, 256, 0, st>>>(cb.dot_part, identity ? kReduceBlocks : 1, cb.alpha, sc);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// NesterovAcc (Alg. 6) as a dense pass over all n x s entries followed by the
// correction of the b rows of the block (the direction is zero elsewhere):
//   dense:   W' = Z;  V' = beta V + (1 - beta) Z;  Z' = alpha V'' + (1 - alpha) W'
//            with V'' = V' (standard) or V (literal)
//   scatter: W' -= eta D;  V' -= gamma eta D;
//            Z' -= (alpha gamma eta + (1 - alpha) eta) D   (standard)
//            Z' -= (1 - alpha) eta D                       (literal)
// ---------------------------------------------------------------------------
__global__ void k_nesterov(float* __restrict__ W, float* __restrict__ V, float* __restrict__ Z, int64_t count,
                           float beta, float alpha, int literal) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    const float z = Z[e], v = V[e];
    const float v1 = fmaf(beta, v, (1.0f - beta) * z);
    const float vz = literal ? v : v1;
    W[e] = z;
    V[e] = v1;
    Z[e] = fmaf(alpha, vz, (1.0f - alpha) * z);
  }
}

// Tail averaging (Alg. 1 / 2): Wbar += W after each averaged iteration; at the
// end W = Wbar / count.
__global__ void k_tail_add(const float* __restrict__ W, float* __restrict__ Wbar, int64_t count) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
    Wbar[e] += W[e];
}
__global__ void k_tail_finish(const float* __restrict__ Wbar, float* __restrict__ W, int64_t count, float inv) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
    W[e] = Wbar[e] * inv;
}
cudaError_t launch_tail_add(const float* W, float* Wbar, int64_t count, cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>((count + 255) / 256, 148 * 8);
  k_tail_add<<<blocks, 256, 0, st>>>(W, Wbar, count);
  return cudaGetLastError();
}
cudaError_t launch_tail_finish(const float* Wbar, float* W, int64_t count, float inv, cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>((count + 255) / 256, 148 * 8);
  k_tail_finish<<<blocks, 256, 0, st>>>(Wbar, W, count, inv);
  return cudaGetLastError();
}

cudaError_t launch_nesterov(float* W, float* V, float* Z, int64_t count, float beta, float alpha, int literal,
                            cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>((count + 255) / 256, 148 * 16);
  k_nesterov<<<blocks, 256, 0, st>>>(W, V, Z, count, beta, alpha, literal);
  return cudaGetLastError();
}

__global__ void k_scatter(float* __restrict__ W, float* __restrict__ V, float* __restrict__ Z, const int* __restrict__ B,
                          int64_t b, int s, const float* __restrict__ D, float gamma, float alpha, int literal,
                          const DevScalars* sc) {
  const double eta = sc->eta;
  const float fw = (float)eta;
  const float fv = (float)(gamma * eta);
  const float fz = literal ? (float)((1.0 - alpha) * eta) : (float)(alpha * gamma * eta + (1.0 - alpha) * eta);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < b * s; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / s;
    const int c = (int)(e - i * s);
    const int64_t j = (int64_t)B[i] * s + c;
    const float d = D[e];
    W[j] = fmaf(-fw, d, W[j]);
    V[j] = fmaf(-fv, d, V[j]);
    Z[j] = fmaf(-fz, d, Z[j]);
  }
}

cudaError_t launch_scatter(float* W, float* V, float* Z, const int* B, int64_t b, int s, const float* D, float gamma,
                           float alpha, int literal, DevScalars* sc, cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>((b * s + 255) / 256, 148 * 8);
  k_scatter<<<std::max(blocks, 1), 256, 0, st>>>(W, V, Z, B, b, s, D, gamma, alpha, literal, sc);
  return cudaGetLastError();
}

__global__ void k_sum_blocks(const double* __restrict__ parts, int count, double* dst, int add) {
  __shared__ double red[33];
  double t = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) t += parts[i];
  t = block_sum(t, red);
  if (threadIdx.x == 0) *dst = add ? *dst + t : t;
}

cudaError_t launch_sum_blocks(const double* parts, int count, double* dst, cudaStream_t st) {
  k_sum_blocks<<<1, 256, 0, st>>>(parts, count, dst, 0);
  return cudaGetLastError();
}

cudaError_t launch_sum_blocks_add(const double* parts, int count, double* dst, cudaStream_t st) {
  k_sum_blocks<<<1, 256, 0, st>>>(parts, count, dst, 1);
  return cudaGetLastError();
}

__global__ void k_trace(DevScalars* sc, double* trace) {
  const long long t = sc->t;
  trace[2 * t] = sc->eta;
  trace[2 * t + 1] = sc->rho;
}
cudaError_t launch_trace(DevScalars* sc, double* trace, cudaStream_t st) {
  k_trace<<<1, 1, 0, st>>>(sc, trace);
  return cudaGetLastError();
}

__global__ void k_tick(DevScalars* sc) { sc->t += 1; }
cudaError_t launch_tick(DevScalars* sc, cudaStream_t st) {
  k_tick<<<1, 1, 0, st>>>(sc);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Single-RHS Woodbury applies (App. C.2) and the randomized-powering steps of
// Alg. 5 as two whole-GPU launches over contiguous row chunks (one chunk per
// block, at most 64 rows, so that each warp takes one group of eight rows):
//   A  the chunk's rows of h (the input v, or h = sum_p part[p] + lambda a for a
//      powering step), and its FP32 partials of U^T h, ||h||^2 and a . h: a warp
//      takes eight rows at a time, lanes split the r columns.  The last block to
//      finish sums the partials of all chunks in a fixed order (so the result does
//      not depend on which block is last) in double-float, and forms the r
//      coefficients of out = alpha h + U coef.  Its operands (the r x r matrix,
//      cis or keep, rho) are fetched into registers together with the partials,
//      so that the tail of the launch is one round trip to L2 and a few barriers.
//   B  out = alpha h + U coef over the chunk's rows, eight rows per warp
//      with the row sums reduced across lanes by a transposing butterfly
// Modes (see ApplyMode):
//   kInvSqrtNormalised  out = P^{-1/2} v / ||v||
//   kInv                out = P^{-1} v (stabilised form, through M)
//   kInvUnit            out = P^{-1/2} P^{-1/2} h / ||P^{-1/2} h||: with a_i =
//                       P^{-1/2} v_i and v_i of unit norm, a_{i+1} = P^{-1/2}
//                       v_{i+1} for v_{i+1} = P^{-1/2} H a_i / ||.|| (Alg. 5)
//   kRayleighEta        lambda_hat = a . h = v^T P^{-1/2} H P^{-1/2} v, eta =
//                       1 / lambda_hat (no output rows)
// ---------------------------------------------------------------------------
constexpr int kWbThreads = 256, kWbWarps = kWbThreads / 32, kWbRows = 8;
constexpr int kWbSlots = kMaxRank + 2;     // per-chunk partials: U^T h, ||h||^2, a . h
constexpr int kWbSlotsP = (kWbSlots + 3) & ~3;   // float4-aligned stride of one chunk's partials
constexpr int kWbG4 = kWbSlotsP / 4;             // float4 groups of one chunk
constexpr int kWbSub = kWbThreads / kWbG4;       // chunk subsets summed side by side by the last block
constexpr int kWbMaxChunks = 296;
static_assert(kWbThreads >= kMaxRank, "one thread per coefficient");

// Sum over the 32 lanes of eight per-lane values x[0..7]; on return lane l
// holds in x[0] the total of value l >> 2.
__device__ __forceinline__ void transpose_sum8(float x[8], int lane) {
  const unsigned full = 0xffffffffu;
  {
    const bool hi = lane & 16;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const float send = hi ? x[t] : x[t + 4];
      const float keepv = hi ? x[t + 4] : x[t];
      x[t] = keepv + __shfl_xor_sync(full, send, 16);
    }
  }
  {
    const bool hi = lane & 8;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const float send = hi ? x[t] : x[t + 2];
      const float keepv = hi ? x[t + 2] : x[t];
      x[t] = keepv + __shfl_xor_sync(full, send, 8);
    }
  }
  {
    const bool hi = lane & 4;
    const float send = hi ? x[0] : x[1];
    const float keepv = hi ? x[1] : x[0];
    x[0] = keepv + __shfl_xor_sync(full, send, 4);
  }
  x[0] += __shfl_xor_sync(full, x[0], 2);
  x[0] += __shfl_xor_sync(full, x[0], 1);
}

// The r x r matrix of the coefficient step (U^T U or M), fetched into registers
// by the last block before its partial sums arrive: warps take four rows at a
// time (rows 4 w + 32 p + u), lanes split the columns.
constexpr int kMvPass = kMaxRank / (4 * kWbWarps);
struct MvRegs {
  float m[kMvPass][4][kMaxRank / 32];
};
__device__ __forceinline__ void mv_fetch(const float* __restrict__ M, int r, MvRegs& R) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int p = 0; p < kMvPass; ++p)
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int jj = 0; jj < kMaxRank / 32; ++jj) {
        const int k = 4 * warp + 32 * p + u, j = lane + 32 * jj;
        R.m[p][u][jj] = (k < r && j < r) ? __ldg(M + k * r + j) : 0.0f;
      }
}

// y[k] = sum_j M[k][j] x[j] from the fetched rows (x in shared memory)
__device__ __forceinline__ void mv_apply(const MvRegs& R, const float* x, int r, double* y) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float xv[kMaxRank / 32];
#pragma unroll
  for (int jj = 0; jj < kMaxRank / 32; ++jj) xv[jj] = (lane + 32 * jj < r) ? x[lane + 32 * jj] : 0.0f;
#pragma unroll
  for (int p = 0; p < kMvPass; ++p)
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      float t = 0.0f;
#pragma unroll
      for (int jj = 0; jj < kMaxRank / 32; ++jj) t = fmaf(R.m[p][u][jj], xv[jj], t);
      t = warp_sum(t);
      const int k = 4 * warp + 32 * p + u;
      if (lane == 0 && k < r) y[k] = (double)t;
    }
}

// Scalars of the coefficient step, formed once by thread 0 while the partials load.
struct WbScalars {
  double rho, irho, irs;
};

// Coefficients of out = alpha h + U coef from the totals q (U^T h, ||h||^2,
// a . h), by one block: written to a.wcoef[0..r) and a.wcoef[kMaxRank] = alpha.
// Thread k < r holds cis_k (kInvUnit, kInvSqrtNormalised) or keep_k (kInv).
__device__ void wb_coefficients(const WbArgs& a, const double* q, double* ys, double* zs, double* red,
                                const MvRegs& R, const WbScalars& w, double cis_k, double keep_k) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, tid = threadIdx.x;
  const int r = a.r;
  const int mode = a.mode;
  float* coef = a.wcoef;
  if (mode == kRayleighEta) {
    if (tid == 0) {
      // lambda_hat = a . h -> eta (Alg. 5)
      DevScalars* sc = a.sc;
      const double lam_hat = q[kMaxRank + 1];
      sc->lam_hat = lam_hat;
      double eta = (lam_hat > 0.0 && isfinite(lam_hat)) ? 1.0 / lam_hat : 0.0;
      if (!(lam_hat > 0.0 && isfinite(lam_hat))) set_status(sc, ADASAP_ENUMERIC, 4);
      if (sc->status != 0) eta = 0.0;
      sc->eta = eta;
    }
    return;
  }
  __shared__ float xs[kMaxRank];
  if (mode == kInv) {
    // coef = -keep . M (keep . q) / rho
    if (tid < r) xs[tid] = (float)(keep_k * q[tid]);
    __syncthreads();
    mv_apply(R, xs, r, zs);
    __syncthreads();
    if (tid < r) coef[tid] = (float)(-keep_k * zs[tid] * w.irho);
    if (tid == 0) coef[kMaxRank] = (float)w.irho;
  } else if (mode == kInvUnit) {
    // The two inverse-square-root applies of Alg. 5 in closed form, exact for any U
    // (P^{-1/2} = rho^{-1/2} I + U diag(cis) U^T, G = U^T U, t = U^T h, y = cis . t, z = G y):
    //   w = P^{-1/2} h = rho^{-1/2} h + U y,  ||w||^2 = ||h||^2 / rho + 2 rho^{-1/2} t.y + y.z
    //   P^{-1/2} w = rho^{-1} h + U (rho^{-1/2} y + cis . (rho^{-1/2} t + z))
    if (tid < r) {
      ys[tid] = cis_k * q[tid];
      xs[tid] = (float)ys[tid];
    }
    __syncthreads();
    mv_apply(R, xs, r, zs);
    __syncthreads();
    if (warp == 0) {
      double acc2 = 0.0;
      for (int k = lane; k < r; k += 32) acc2 += 2.0 * w.irs * q[k] * ys[k] + ys[k] * zs[k];
      acc2 = warp_sum(acc2);
      if (lane == 0) {
        const double w2 = q[kMaxRank] * w.irho + acc2;
        red[32] = w2 > 0.0 ? 1.0 / sqrt(w2) : 0.0;
      }
    }
    __syncthreads();
    const double scale = red[32];
    if (tid < r) coef[tid] = (float)(scale * (w.irs * ys[tid] + cis_k * (w.irs * q[tid] + zs[tid])));
    if (tid == 0) coef[kMaxRank] = (float)(scale * w.irho);
  } else {
    const double scale = q[kMaxRank] > 0.0 ? 1.0 / sqrt(q[kMaxRank]) : 0.0;
    if (tid < r) coef[tid] = (float)(scale * q[tid] * cis_k);
    if (tid == 0) coef[kMaxRank] = (float)(scale * w.irs);
  }
}

// Chunk `chunk` of launch A (partials; the last chunk to finish reduces them).
__device__ __forceinline__ void wb_partials_body(const WbArgs& a, int chunk) {
  __shared__ float wtmp[kWbWarps][kMaxRank];
  __shared__ float wred[2][kWbWarps];
  __shared__ float sh_hi[kWbSub][kWbSlotsP];
  __shared__ float sh_lo[kWbSub][kWbSlotsP];
  __shared__ double red[33];
  __shared__ double q[kWbSlots];
  __shared__ double ys[kMaxRank];
  __shared__ double zs[kMaxRank];
  __shared__ WbScalars wsc;
  __shared__ int s_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, tid = threadIdx.x;
  const int r = a.r;
  const int mode = a.mode;
  const bool from_part = mode == kInvUnit || mode == kRayleighEta;
  const bool need_u = mode != kRayleighEta;
  constexpr int KJ = kMaxRank / 32;
  const int64_t r0 = (int64_t)chunk * a.per, r1 = min(a.b, r0 + a.per);
  float acc[KJ];
#pragma unroll
  for (int j = 0; j < KJ; ++j) acc[j] = 0.0f;
  // ||h||^2 and a . h: lane t < kWbRows sums row t of every group in FP32
  float hsq = 0.0f, ah = 0.0f;
  for (int64_t i0 = r0 + (int64_t)warp * kWbRows; i0 < r1; i0 += (int64_t)kWbWarps * kWbRows) {
    float hv[kWbRows];
    if (from_part) {
      float pv[kWbRows];
#pragma unroll
      for (int t = 0; t < kWbRows; ++t) pv[t] = 0.0f;
      for (int p0 = 0; p0 < a.nsplit; p0 += 32) {
        const int p = p0 + lane;
#pragma unroll
        for (int t = 0; t < kWbRows; ++t) {
          const int64_t i = i0 + t;
          if (p < a.nsplit && i < r1) pv[t] += a.part[(int64_t)p * a.b + i];
        }
      }
      transpose_sum8(pv, lane);
#pragma unroll
      for (int t = 0; t < kWbRows; ++t) {
        const int64_t i = i0 + t;
        const float ai = i < r1 ? a.a[i] : 0.0f;
        hv[t] = i < r1 ? fmaf(a.lam, ai, __shfl_sync(0xffffffffu, pv[0], 4 * t)) : 0.0f;
        if (lane == t) ah = fmaf(ai, hv[t], ah);
      }
      if (mode == kInvUnit && lane < kWbRows && i0 + lane < r1) {
        float mine = hv[0];
#pragma unroll
        for (int t = 1; t < kWbRows; ++t) mine = (lane == t) ? hv[t] : mine;
        a.hbuf[i0 + lane] = mine;
      }
    } else {
#pragma unroll
      for (int t = 0; t < kWbRows; ++t) hv[t] = (i0 + t < r1) ? a.v[i0 + t] : 0.0f;
    }
    if (need_u) {
      float u[kWbRows][KJ];
#pragma unroll
      for (int t = 0; t < kWbRows; ++t) {
        const int64_t i = i0 + t;
#pragma unroll
        for (int j = 0; j < KJ; ++j) {
          const int k = lane + 32 * j;
          u[t][j] = (i < r1 && k < r) ? a.U[i * r + k] : 0.0f;
        }
      }
#pragma unroll
      for (int t = 0; t < kWbRows; ++t) {
#pragma unroll
        for (int j = 0; j < KJ; ++j) acc[j] = fmaf(u[t][j], hv[t], acc[j]);
        if (lane == t) hsq = fmaf(hv[t], hv[t], hsq);
      }
    }
  }
  // the chunk's partials in FP32, warps added in warp order
#pragma unroll
  for (int j = 0; j < KJ; ++j) wtmp[warp][lane + 32 * j] = acc[j];
  hsq = warp_sum(hsq);
  ah = warp_sum(ah);
  if (lane == 0) {
    wred[0][warp] = hsq;
    wred[1][warp] = ah;
  }
  __syncthreads();
  float* dst = a.wpart + (int64_t)chunk * kWbSlotsP;
  for (int k = tid; k < kWbSlotsP; k += kWbThreads) {
    float t = 0.0f;
    if (k < r && need_u) {
#pragma unroll
      for (int w = 0; w < kWbWarps; ++w) t += wtmp[w][k];
    } else if (k == kMaxRank || k == kMaxRank + 1) {
#pragma unroll
      for (int w = 0; w < kWbWarps; ++w) t += wred[k - kMaxRank][w];
    }
    dst[k] = t;
  }
  // The last block to finish sums the partials of all chunks; no block waits
  // for another.
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = atomicAdd(a.count, 1u) == (unsigned)a.nchunk - 1u;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // operands of the coefficient step, in flight with the partials below
  MvRegs R;
  const float* M = mode == kInv ? a.Minv : (mode == kInvUnit ? a.Gu : nullptr);
  if (M) mv_fetch(M, r, R);
  double cis_k = 0.0, keep_k = 0.0;
  if (tid < r) {
    if (mode == kInv) keep_k = a.keep[tid];
    else if (mode != kRayleighEta) cis_k = a.cis[tid];
  }
  if (tid == 0 && mode != kRayleighEta) {
    const double rho = a.sc->rho;
    wsc.rho = rho;
    wsc.irho = 1.0 / rho;
    wsc.irs = 1.0 / sqrt(rho);
  }
  // thread (g, j) adds float4 group g of chunks j, j + kWbSub, ... in double-float;
  // the kWbSub subsets are then added in subset order
  {
    const int g = tid % kWbG4, j = tid / kWbG4;
    float H[4] = {0.0f, 0.0f, 0.0f, 0.0f}, L[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (j < kWbSub) {
      const float4* src = reinterpret_cast<const float4*>(a.wpart) + g;
#pragma unroll 8
      for (int c = j; c < a.nchunk; c += kWbSub) {
        const float4 v = __ldcg(src + (int64_t)c * kWbG4);
        ff_add(H[0], L[0], v.x);
        ff_add(H[1], L[1], v.y);
        ff_add(H[2], L[2], v.z);
        ff_add(H[3], L[3], v.w);
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        sh_hi[j][4 * g + e] = H[e];
        sh_lo[j][4 * g + e] = L[e];
      }
    }
  }
  __syncthreads();
  for (int k = tid; k < kWbSlots; k += kWbThreads) {
    float H = 0.0f, L = 0.0f;
#pragma unroll
    for (int j = 0; j < kWbSub; ++j) {
      ff_add(H, L, sh_hi[j][k]);
      L += sh_lo[j][k];
    }
    q[k] = (double)H + (double)L;
  }
  if (tid == 0) *a.count = 0u;
  __syncthreads();
  wb_coefficients(a, q, ys, zs, red, R, wsc, cis_k, keep_k);
}

__global__ void __launch_bounds__(kWbThreads) k_wb_partials(WbArgs a) { wb_partials_body(a, blockIdx.x); }

// Launch B: out = U coef + alpha h, chunk `chunk` of the rows.
__device__ __forceinline__ void wb_apply_body(const WbArgs& a, int chunk) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = a.r;
  constexpr int KJ = kMaxRank / 32;
  const float al = a.wcoef[kMaxRank];
  float cf[KJ];
#pragma unroll
  for (int j = 0; j < KJ; ++j) cf[j] = (lane + 32 * j < r) ? a.wcoef[lane + 32 * j] : 0.0f;
  const float* hsrc = a.mode == kInvUnit ? a.hbuf : a.v;
  const int64_t r0 = (int64_t)chunk * a.per, r1 = min(a.b, r0 + a.per);
  for (int64_t i0 = r0 + (int64_t)warp * kWbRows; i0 < r1; i0 += (int64_t)kWbWarps * kWbRows) {
    float x[kWbRows];
#pragma unroll
    for (int t = 0; t < kWbRows; ++t) {
      const int64_t i = i0 + t;
      float sacc = 0.0f;
#pragma unroll
      for (int j = 0; j < KJ; ++j) {
        const int k = lane + 32 * j;
        sacc = fmaf((i < r1 && k < r) ? a.U[i * r + k] : 0.0f, cf[j], sacc);
      }
      x[t] = sacc;
    }
    transpose_sum8(x, lane);
    const int64_t i = i0 + (lane >> 2);
    if ((lane & 3) == 0 && i < r1) a.out[i] = fmaf(al, hsrc[i], x[0]);
  }
}

__global__ void __launch_bounds__(kWbThreads) k_wb_apply(WbArgs a) { wb_apply_body(a, blockIdx.x); }

// Grouped forms over a flat grid of the (system, chunk) pairs: block x works on
// chunk x - start[s] of the system s with start[s] <= x < start[s + 1] (start: the
// prefix sums of the systems' chunk counts), so no block is idle.  Three CTAs of
// the partials fit an SM, so that the usual few hundred blocks run as one wave.
__device__ __forceinline__ int wb_system_of(const int* __restrict__ start, int ngrp, int x) {
  int lo = 0, hi = ngrp - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (start[mid] <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(kWbThreads, 3) k_wb_partials_g(const WbArgs* __restrict__ g,
                                                                  const int* __restrict__ start, int ngrp) {
  const int sys = wb_system_of(start, ngrp, (int)blockIdx.x);
  wb_partials_body(g[sys], (int)blockIdx.x - start[sys]);
}

__global__ void __launch_bounds__(kWbThreads) k_wb_apply_g(const WbArgs* __restrict__ g, const int* __restrict__ start,
                                                           int ngrp) {
  const int sys = wb_system_of(start, ngrp, (int)blockIdx.x);
  wb_apply_body(g[sys], (int)blockIdx.x - start[sys]);
}

static void fill_wb(WbArgs& a, CoreBufs& cb) {
  a.U = cb.U; a.b = cb.b; a.r = cb.r; a.keep = cb.keep; a.Minv = cb.Minv; a.Gu = cb.Gu; a.S = cb.S; a.cis = cb.cis;
  a.wpart = cb.wb_part;
  a.wcoef = cb.wb_coef;
  a.count = cb.wb_count;
  a.nchunk = wb_chunks_for(cb.b);
  a.per = (cb.b + a.nchunk - 1) / a.nchunk;
}

static cudaError_t launch_wb(WbArgs& a, CoreBufs& cb, cudaStream_t st) {
  fill_wb(a, cb);
  k_wb_partials<<<a.nchunk, kWbThreads, 0, st>>>(a);
  if (a.mode != kRayleighEta) k_wb_apply<<<a.nchunk, kWbThreads, 0, st>>>(a);
  return cudaGetLastError();
}

WbArgs wb_args_single(CoreBufs& cb, int mode, const float* v, float* out, DevScalars* sc) {
  WbArgs a{};
  a.mode = mode; a.v = v; a.sc = sc; a.out = out;
  fill_wb(a, cb);
  return a;
}

WbArgs wb_args_power(CoreBufs& cb, int mode, const float* part, int nsplit, float lam, const float* acur,
                     float* hbuf, float* anext, DevScalars* sc) {
  WbArgs a{};
  a.mode = mode; a.part = part; a.nsplit = nsplit; a.a = acur; a.lam = lam; a.hbuf = hbuf; a.sc = sc; a.out = anext;
  fill_wb(a, cb);
  return a;
}

cudaError_t launch_wb_grouped(const WbArgs* g, const int* start, int ngrp, int nblocks, int mode, cudaStream_t st) {
  if (ngrp < 1 || nblocks < 1) return cudaSuccess;
  k_wb_partials_g<<<nblocks, kWbThreads, 0, st>>>(g, start, ngrp);
  if (mode != kRayleighEta) k_wb_apply_g<<<nblocks, kWbThreads, 0, st>>>(g, start, ngrp);
  return cudaGetLastError();
}

// chunks of at most 64 rows (one group of eight rows per warp) while that keeps
// the last block's sum short
int wb_chunks_for(int64_t b) { return (int)std::max<int64_t>(1, std::min<int64_t>(kWbMaxChunks, (b + 63) / 64)); }
size_t wb_part_floats(int64_t b) { return (size_t)wb_chunks_for(b) * kWbSlotsP; }

cudaError_t launch_wb_single(CoreBufs& cb, int mode, const float* v, float* out, DevScalars* sc, cudaStream_t st) {
  WbArgs a{};
  a.mode = mode; a.v = v; a.sc = sc; a.out = out;
  return launch_wb(a, cb, st);
}

cudaError_t launch_power_step(CoreBufs& cb, int mode, const float* part, int nsplit, float lam, const float* acur,
                              float* hbuf, float* anext, DevScalars* sc, cudaStream_t st) {
  WbArgs a{};
  a.mode = mode; a.part = part; a.nsplit = nsplit; a.a = acur; a.lam = lam; a.hbuf = hbuf; a.sc = sc; a.out = anext;
  return launch_wb(a, cb, st);
}

template <typename T>
static cudaError_t trsm_init(int smem) {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_trsm<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))) return e;
  if ((e = cudaFuncSetAttribute(k_trsm<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))) return e;
  if ((e = cudaFuncSetAttribute(k_trsm<T, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))) return e;
  return cudaFuncSetAttribute(k_trsm<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

cudaError_t core_init() {
  const int big = 200 * 1024;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_nys_chol, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = cudaFuncSetAttribute(k_make_u<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = cudaFuncSetAttribute(k_make_u<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = cudaFuncSetAttribute(k_make_u<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = cudaFuncSetAttribute(k_make_u<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = cudaFuncSetAttribute(k_chol_plain<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = cudaFuncSetAttribute(k_chol_plain<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = trsm_init<double>(big)) || (e = trsm_init<float>(big))) return e;
  if ((e = cudaFuncSetAttribute(k_wfactor<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = cudaFuncSetAttribute(k_wfactor<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = cudaFuncSetAttribute(k_wfactor<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = cudaFuncSetAttribute(k_nys_finalize, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = cudaFuncSetAttribute(k_wapply, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  return cudaSuccess;
}

}  // namespace adasap
