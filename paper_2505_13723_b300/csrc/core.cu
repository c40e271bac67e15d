// Step III and IV of Alg. 2 on the GPU:
//   - Gram matrices of b x r panels (FP32 products, FP64 accumulation)
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
#include <cooperative_groups.h>

#include <algorithm>
#include <type_traits>

#include "internal.cuh"

namespace cg = cooperative_groups;

namespace adasap {

// ---------------------------------------------------------------------------
// Gram matrix of the row-concatenation [A1 | A2] (m x (c1 + c2), c <= 256),
// accumulated in FP64.  With `exact` the products of the FP32 entries are
// formed in FP64 (exact: 24 + 24 bits).  Exactness matters for Y_nu^T Y_nu:
// B^T B = C^{-T} (Y_nu^T Y_nu) C^{-1} multiplies its absolute error by cond(C)^2,
// so FP32 products would swamp the small Nystrom eigenvalues; everywhere else
// an FP32 product error of eps * |a| |b| is below the data's own rounding.
// Only upper 64 x 64 tiles are computed; the reduce mirrors them.
// ---------------------------------------------------------------------------
// chunks of at least 32 rows, enough CTAs (chunks x upper tiles) for ~4 per SM at c = 2r <= 256
int gram_chunks_for(int64_t b) { return (int)std::max<int64_t>(1, std::min<int64_t>(240, (b + 31) / 32)); }

__device__ __forceinline__ float cat_get(const float* A1, int64_t ld1, int c1, const float* A2, int64_t ld2,
                                         int c2, int64_t row, int col) {
  if (col < c1) return A1[row * ld1 + col];
  if (col < c1 + c2) return A2[row * ld2 + (col - c1)];
  return 0.0f;
}

// 64 x 64 output tiles, 256 threads x (4 x 4) outputs, 16-row slices.
// EXACT: products and sums in FP64 (exact products of FP32 entries);
// otherwise FP32 products summed in FP32 over a 16-row slice, then in FP64.
template <bool EXACT>
__global__ void __launch_bounds__(256) k_gram_part(const float* __restrict__ A1, int64_t ld1, int c1,
                                                   const float* __restrict__ A2, int64_t ld2, int c2,
                                                   int64_t m, int64_t chunk_rows, double* __restrict__ part) {
  constexpr int TS = 64, KR = 16;
  using T = typename std::conditional<EXACT, double, float>::type;
  const int ti = blockIdx.y, tj = blockIdx.z;
  if (ti > tj) return;
  const int c = c1 + c2;
  __shared__ T sa[KR][TS + 1];
  __shared__ T sb[KR][TS + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t r0 = (int64_t)blockIdx.x * chunk_rows;
  const int64_t r1 = min(m, r0 + chunk_rows);
  double acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0.0;
  for (int64_t s0 = r0; s0 < r1; s0 += KR) {
    __syncthreads();
    for (int e = tid; e < KR * TS; e += 256) {
      const int rr = e / TS, cc = e % TS;
      const int64_t row = s0 + rr;
      const bool ok = row < r1;
      sa[rr][cc] = ok ? (T)cat_get(A1, ld1, c1, A2, ld2, c2, row, ti * TS + cc) : (T)0;
      sb[rr][cc] = ok ? (T)cat_get(A1, ld1, c1, A2, ld2, c2, row, tj * TS + cc) : (T)0;
    }
    __syncthreads();
    T f[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) f[u][v] = (T)0;
#pragma unroll 4
    for (int rr = 0; rr < KR; ++rr) {
      T a[4], bb[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = sa[rr][ty + 16 * u];
        bb[u] = sb[rr][tx + 16 * u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) f[u][v] = fma(a[u], bb[v], f[u][v]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] += (double)f[u][v];
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int i = ti * TS + ty + 16 * u, j = tj * TS + tx + 16 * v;
      if (i < c && j < c) part[((int64_t)blockIdx.x * c + i) * c + j] = acc[u][v];
    }
}

__global__ void k_gram_reduce(const double* __restrict__ part, int chunks, int c, double* __restrict__ G) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < c * c; e += gridDim.x * blockDim.x) {
    int i = e / c, j = e % c;
    if ((i >> 6) > (j >> 6)) { const int t = i; i = j; j = t; }
    double acc = 0.0;
    for (int ch = 0; ch < chunks; ++ch) acc += part[((int64_t)ch * c + i) * c + j];
    G[e] = acc;
  }
}

cudaError_t launch_gram(const float* A1, int64_t ld1, int c1, const float* A2, int64_t ld2, int c2,
                        int64_t m, double* part, int chunks, double* G, bool exact, cudaStream_t st) {
  const int c = c1 + c2;
  const int nt = (c + 63) / 64;
  const int64_t chunk_rows = (m + chunks - 1) / chunks;
  if (exact)
    k_gram_part<true><<<dim3(chunks, nt, nt), 256, 0, st>>>(A1, ld1, c1, A2, ld2, c2, m, chunk_rows, part);
  else
    k_gram_part<false><<<dim3(chunks, nt, nt), 256, 0, st>>>(A1, ld1, c1, A2, ld2, c2, m, chunk_rows, part);
  k_gram_reduce<<<std::min(148, (c * c + 255) / 256), 256, 0, st>>>(part, chunks, c, G);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// One-CTA FP64 Cholesky (lower, in place) of an r x r matrix in shared memory
// with leading dimension ld (r + 1 keeps column reads conflict free).
// Returns false, uniformly over the block, if a pivot is not positive.
// ---------------------------------------------------------------------------
template <typename T>
__device__ bool chol_lower_smem(T* A, int r, int ld, int* flag) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __shared__ T s_rdk;
  for (int k = 0; k < r; ++k) {
    if (threadIdx.x == 0) {
      const T d = A[k * ld + k];
      *flag = (d > T(0) && isfinite(d)) ? 0 : 1;
      if (!*flag) {
        const T sd = sqrt(d);
        A[k * ld + k] = sd;
        s_rdk = T(1) / sd;
      }
    }
    __syncthreads();
    if (*flag) return false;
    const T rdk = s_rdk;
    for (int i = k + 1 + threadIdx.x; i < r; i += blockDim.x) A[i * ld + k] *= rdk;
    __syncthreads();
    for (int i = k + 1 + warp; i < r; i += nw) {
      const T lik = A[i * ld + k];
      for (int j = k + 1 + lane; j <= i; j += 32) A[i * ld + j] -= lik * A[j * ld + k];
    }
    __syncthreads();
  }
  return true;
}

// Alg. 4, first half: Delta, C = chol(Omega^T M Omega + Delta Omega^T Omega)
// (stored as the lower factor L = C^T), and Y_nu^T Y_nu.
__global__ void __launch_bounds__(512) k_nys_chol(const double* __restrict__ G, const double* __restrict__ Gyy,
                                                  int r, double eps,
                                                  double* __restrict__ Lout, double* __restrict__ Gnu,
                                                  DevScalars* sc) {
  extern __shared__ double sh[];
  __shared__ double red[33];
  __shared__ int flag;
  const int ld = r + 1, c = 2 * r;
  double tr = 0.0;
  for (int i = threadIdx.x; i < r; i += blockDim.x) tr += G[(int64_t)i * c + r + i];
  tr = block_sum(tr, red);
  double delta = eps * tr;
  bool ok = false;
  int attempt = 0;
  for (; attempt < 4; ++attempt) {
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
      const int i = e / r, j = e % r;
      const double oty = 0.5 * (G[(int64_t)i * c + r + j] + G[(int64_t)j * c + r + i]);
      sh[i * ld + j] = oty + delta * G[(int64_t)i * c + j];
    }
    __syncthreads();
    ok = chol_lower_smem(sh, r, ld, &flag);
    __syncthreads();
    if (ok) break;
    delta *= 10.0;
  }
  if (!ok) {
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) sh[(e / r) * ld + e % r] = (e / r == e % r) ? 1.0 : 0.0;
    if (threadIdx.x == 0) set_status(sc, ADASAP_ENUMERIC, 1);
    __syncthreads();
  }
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
// staged in shared memory; one warp per right-hand side column.
constexpr int kTrsmWarps = 4;
template <typename T>
__global__ void __launch_bounds__(32 * kTrsmWarps) k_trsm(const double* __restrict__ L, int r,
                                                          const double* __restrict__ R, int trans, int upper,
                                                          double* __restrict__ X) {
  extern __shared__ double shd_trsm[];
  const int ld = r + 1;
  T* sL = reinterpret_cast<T*>(shd_trsm);  // r x (r + 1)
  T* rinv = sL + r * ld;                  // r
  T* xs = rinv + r;                       // kTrsmWarps x r
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) sL[(e / r) * ld + e % r] = (T)L[e];
  __syncthreads();
  for (int i = threadIdx.x; i < r; i += blockDim.x) rinv[i] = T(1) / sL[i * ld + i];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int col = blockIdx.x * kTrsmWarps + warp;
  if (col >= r) return;
  T* x = xs + warp * r;
  for (int step = 0; step < r; ++step) {
    const int i = upper ? r - 1 - step : step;
    T part = T(0);
    if (!upper) {
      for (int k = lane; k < i; k += 32) part += sL[i * ld + k] * x[k];
    } else {
      for (int k = i + 1 + lane; k < r; k += 32) part += sL[k * ld + i] * x[k];
    }
    part = warp_sum(part);
    if (lane == 0) {
      const T rhs = (T)(trans ? R[(int64_t)col * r + i] : R[(int64_t)i * r + col]);
      x[i] = (rhs - part) * rinv[i];
    }
    __syncwarp();
  }
  for (int i = lane; i < r; i += 32) X[(int64_t)i * r + col] = (double)x[i];
}

template <typename T = double>
static cudaError_t trsm(const double* L, int r, const double* R, int trans, int upper, double* X, cudaStream_t st) {
  const size_t smem = ((size_t)r * (r + 1) + r + (size_t)kTrsmWarps * r) * sizeof(T);
  k_trsm<T><<<(r + kTrsmWarps - 1) / kTrsmWarps, 32 * kTrsmWarps, smem, st>>>(L, r, R, trans, upper, X);
  return cudaGetLastError();
}

// Eigenvectors of the symmetric PSD r x r matrix A by one-sided (Hestenes)
// Jacobi in FP32: W = A V is rotated column pair by column pair until its
// columns are orthogonal; then A V = W and, A being PSD, V holds A's
// eigenvectors (the eigenvalues are refined in FP64 by k_rayleigh).
// Parallel round-robin ordering: in each of the r2 - 1 rounds of a sweep the
// r2/2 disjoint pairs are rotated concurrently, one warp per pair, so a round
// needs one barrier.  W and V are column-major in shared memory; the squared
// column norms are carried along (updated exactly for each rotation and
// recomputed every sweep), so a pair needs one dot product.  A pair is skipped
// when |w_p . w_q| <= 1e-6 |w_p| |w_q| or when it is below what the columns'
// absolute FP32 noise can produce; sweeps stop when one rotates nothing (at
// most kJacobiSweeps; Jacobi converges quadratically).
constexpr int kJacobiSweeps = 12;
__global__ void __launch_bounds__(1024) k_jacobi(const double* __restrict__ A, int r, float* __restrict__ Vout,
                                                 DevScalars* sc) {
  extern __shared__ float shf[];
  const int r2 = r + (r & 1);
  float* w = shf;               // r2 columns x r2 rows (column-major)
  float* v = shf + r2 * r2;
  __shared__ float nrm[kMaxRank];
  __shared__ float mxs[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double mx = 0.0;
  for (int i = threadIdx.x; i < r; i += blockDim.x) mx = fmax(mx, fabs(A[(int64_t)i * r + i]));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) mxs[warp] = (float)mx;
  __syncthreads();
  float amax = 0.f;
  for (int k = 0; k < nw; ++k) amax = fmaxf(amax, mxs[k]);
  const double scale = amax > 0.f ? 1.0 / (double)amax : 1.0;
  for (int e = threadIdx.x; e < r2 * r2; e += blockDim.x) {
    const int col = e / r2, row = e % r2;
    w[e] = (row < r && col < r) ? (float)(A[(int64_t)row * r + col] * scale) : 0.0f;
    v[e] = (row == col) ? 1.0f : 0.0f;
  }
  __syncthreads();
  const int half = r2 / 2;
  float noise = 0.f;
  int sweep = 0;
  for (; sweep < kJacobiSweeps; ++sweep) {
    // exact squared column norms at the start of every sweep
    for (int col = warp; col < r2; col += nw) {
      float t = 0.f;
      for (int k = lane; k < r2; k += 32) t = fmaf(w[col * r2 + k], w[col * r2 + k], t);
      t = warp_sum(t);
      if (lane == 0) nrm[col] = t;
    }
    __syncthreads();
    if (sweep == 0) {
      float nmax = 0.f;
      for (int k = 0; k < r2; ++k) nmax = fmaxf(nmax, nrm[k]);
      // absolute FP32 noise carried by every column after rotations against the largest
      noise = 4.0f * 1.1920929e-7f * sqrtf(nmax);
    }
    int rotated = 0;
    for (int round = 0; round < r2 - 1; ++round) {
      // a warp owns pairs m = warp and m = warp + nw (r2 <= 128, nw = 32): both are
      // processed together so their latency chains overlap
      int pp[2], qq[2];
      bool act[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int m = warp + h * nw;
        act[h] = m < half;
        int p = 0, q = 0;
        if (m == 0) { p = round; q = r2 - 1; }
        else {
          p = round + m;
          if (p >= r2 - 1) p -= r2 - 1;
          q = round - m;
          if (q < 0) q += r2 - 1;
        }
        pp[h] = p < q ? p : q;
        qq[h] = p < q ? q : p;
      }
      float ga[2] = {0.f, 0.f};
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (!act[h]) continue;
        const float* wp = w + pp[h] * r2;
        const float* wq = w + qq[h] * r2;
        for (int k = lane; k < r2; k += 32) ga[h] = fmaf(wp[k], wq[k], ga[h]);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        ga[0] += __shfl_xor_sync(0xffffffffu, ga[0], o);
        ga[1] += __shfl_xor_sync(0xffffffffu, ga[1], o);
      }
      int mine = 0;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (!act[h]) continue;
        const int p = pp[h], q = qq[h];
        const float al = nrm[p], be = nrm[q], g = ga[h];
        const float ab = al * be;
        const float sab = ab * rsqrtf(fmaxf(ab, 1e-37f));
        const float sa = al * rsqrtf(fmaxf(al, 1e-37f)), sb = be * rsqrtf(fmaxf(be, 1e-37f));
        if (fabsf(g) > 1e-6f * sab && fabsf(g) > noise * (sa + sb)) {
          const float zeta = __fdividef(be - al, 2.0f * g);
          const float z2 = fmaf(zeta, zeta, 1.0f);
          const float t = copysignf(1.0f, zeta) * __fdividef(1.0f, fabsf(zeta) + z2 * rsqrtf(z2));
          const float c = rsqrtf(fmaf(t, t, 1.0f));
          const float sn = c * t;
          float* wp = w + p * r2;
          float* wq = w + q * r2;
          float* vp = v + p * r2;
          float* vq = v + q * r2;
          for (int k = lane; k < r2; k += 32) {
            const float a = wp[k], bq = wq[k];
            wp[k] = c * a - sn * bq;
            wq[k] = sn * a + c * bq;
            const float x = vp[k], y = vq[k];
            vp[k] = c * x - sn * y;
            vq[k] = sn * x + c * y;
          }
          if (lane == 0) {
            // norms after a rotation that zeroes the pair's inner product
            nrm[p] = c * c * al - 2.0f * c * sn * g + sn * sn * be;
            nrm[q] = sn * sn * al + 2.0f * c * sn * g + c * c * be;
          }
          mine = 1;
        }
      }
      rotated |= __syncthreads_or(mine);
    }
    if (!rotated) break;
  }
  if (threadIdx.x == 0) sc->jacobi_sweeps = sweep;
  // Vout row-major: Vout[k * r + i] = component k of eigenvector i
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int k = e / r, i = e % r;
    Vout[e] = v[i * r2 + k];
  }
}

// lambda_i = v_i^T A v_i / v_i^T v_i in FP64 (one block per eigenvector)
__global__ void k_rayleigh(const double* __restrict__ A, const float* __restrict__ V, int r, double* __restrict__ lam) {
  __shared__ double red[33];
  const int i = blockIdx.x;
  double num = 0.0, den = 0.0;
  for (int k = threadIdx.x; k < r; k += blockDim.x) {
    double w = 0.0;
    for (int j = 0; j < r; ++j) w += A[(int64_t)k * r + j] * (double)V[(int64_t)j * r + i];
    const double vk = (double)V[(int64_t)k * r + i];
    num += vk * w;
    den += vk * vk;
  }
  num = block_sum(num, red);
  den = block_sum(den, red);
  if (threadIdx.x == 0) lam[i] = num / den;
}

// Sort eigenpairs (descending), S = max(0, Sigma^2 - Delta), rho = S_r + lambda,
// and T' = V Sigma^{-1} (columns normalised) for U = Y_nu L^{-T} T'.
__global__ void k_nys_finalize(const double* __restrict__ lam, const float* __restrict__ V, int r, double lam_reg,
                               DevScalars* sc, double* __restrict__ S, double* __restrict__ keep,
                               double* __restrict__ Tp) {
  __shared__ int perm[kMaxRank];
  __shared__ double sig[kMaxRank];
  __shared__ double nrm[kMaxRank];
  const double delta = sc->delta;
  for (int i = threadIdx.x; i < r; i += blockDim.x) perm[i] = i;  // stays a valid index even if ranks collide (NaN)
  __syncthreads();
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    const double li = lam[i];
    int rank = 0;
    for (int j = 0; j < r; ++j) {
      const double lj = lam[j];
      rank += (lj > li) || (lj == li && j < i);
    }
    if (rank < r) perm[rank] = i;
    double n2 = 0.0;
    for (int k = 0; k < r; ++k) n2 += (double)V[(int64_t)k * r + i] * (double)V[(int64_t)k * r + i];
    nrm[i] = sqrt(n2);
  }
  __syncthreads();
  for (int q = threadIdx.x; q < r; q += blockDim.x) {
    const double li = lam[perm[q]];
    const double sq = fmax(0.0, li - delta);
    S[q] = sq;
    keep[q] = sq > 0.0 ? 1.0 : 0.0;
    sig[q] = li > 0.0 ? sqrt(li) : 0.0;
    if (!isfinite(li)) set_status(sc, ADASAP_ENUMERIC, 2);
  }
  __syncthreads();
  if (threadIdx.x == 0) sc->rho = S[r - 1] + lam_reg;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int k = e / r, q = e % r;
    const int i = perm[q];
    // a dropped eigenpair (S_q = 0) contributes exactly nothing to either Woodbury form
    // (eqs. inv_nys_woodbury and inv_sqrt_nys_woodbury), so its U column is set to 0
    // instead of V / sigma with sigma ~ 0
    Tp[e] = (S[q] > 0.0 && sig[q] > 0.0) ? (double)V[(int64_t)k * r + i] / (nrm[i] * sig[q]) : 0.0;
  }
}

// U = (A1 + delta A2) T'  (b x r), T' = T or T^T (r x r FP64, staged as FP32 in
// shared memory), delta = sc->delta or 0 when A2 is NULL.  Rows in blocks of 32.
//   Nystrom: A1 = M Omega, A2 = Omega, T' = T      (U = Y_nu T)
//   QR:      A1 = Omega,   A2 = NULL,  T' = L^{-T} (Omega R^{-1}, R = L^T)
__global__ void __launch_bounds__(256) k_make_u(const float* __restrict__ A1, const float* __restrict__ A2, int64_t b,
                                                int r, const double* __restrict__ T, int transT, const DevScalars* sc,
                                                float* __restrict__ U) {
  extern __shared__ float shm[];
  float* sT = shm;                  // r x r
  float* sY = shm + r * r;          // 32 x r
  const double delta = A2 ? sc->delta : 0.0;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x)
    sT[e] = (float)(transT ? T[(e % r) * r + e / r] : T[e]);
  const int64_t row0 = (int64_t)blockIdx.x * 32;
  for (int e = threadIdx.x; e < 32 * r; e += blockDim.x) {
    const int rr = e / r, k = e % r;
    const int64_t row = row0 + rr;
    float v = 0.0f;
    if (row < b) v = A2 ? (float)((double)A1[row * r + k] + delta * (double)A2[row * r + k]) : A1[row * r + k];
    sY[e] = v;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int CQ = kMaxRank / 32;
  float acc[4][CQ];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int q = 0; q < CQ; ++q) acc[u][q] = 0.0f;
  for (int k = 0; k < r; ++k) {
    float yv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) yv[u] = sY[(warp * 4 + u) * r + k];
#pragma unroll
    for (int q = 0; q < CQ; ++q) {
      const int c = lane + 32 * q;
      const float tv = c < r ? sT[k * r + c] : 0.0f;
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u][q] = fmaf(yv[u], tv, acc[u][q]);
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int64_t row = row0 + warp * 4 + u;
    if (row >= b) continue;
#pragma unroll
    for (int q = 0; q < CQ; ++q) {
      const int c = lane + 32 * q;
      if (c < r) U[row * r + c] = acc[u][q];
    }
  }
}

static cudaError_t make_u(const float* A1, const float* A2, int64_t b, int r, const double* T, int transT,
                          const DevScalars* sc, float* U, cudaStream_t st) {
  k_make_u<<<(unsigned)((b + 31) / 32), 256, (size_t)(r * r + 32 * r) * sizeof(float), st>>>(A1, A2, b, r, T, transT,
                                                                                            sc, U);
  return cudaGetLastError();
}

// FP64 Cholesky of an r x r SPD matrix into a lower factor (identity and a
// status on failure), one CTA.
template <typename T>
__global__ void __launch_bounds__(512) k_chol_plain(const double* __restrict__ G, int r, double* __restrict__ L,
                                                    DevScalars* sc, int detail) {
  extern __shared__ double shd_chol[];
  T* sh = reinterpret_cast<T*>(shd_chol);
  __shared__ int flag;
  const int ld = r + 1;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) sh[(e / r) * ld + e % r] = (T)G[e];
  __syncthreads();
  const bool ok = chol_lower_smem<T>(sh, r, ld, &flag);
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
      k_chol_plain<double><<<1, 512, (size_t)r * (r + 1) * sizeof(double), st>>>(cb.X1, r, cb.Lc, sc, 6);
      if ((e = trsm<double>(cb.Lc, r, cb.Ident, 0, 0, cb.A, st))) return e;      // A = L^{-1}
    } else {
      k_chol_plain<float><<<1, 512, (size_t)r * (r + 1) * sizeof(double), st>>>(cb.X1, r, cb.Lc, sc, 6);
      if ((e = trsm<float>(cb.Lc, r, cb.Ident, 0, 0, cb.A, st))) return e;
    }
    if ((e = make_u(src, nullptr, cb.b, r, cb.A, 1, sc, dst, st))) return e;
  }
  return cudaGetLastError();
}

cudaError_t launch_nystrom_core(CoreBufs& cb, double eps, double lam, DevScalars* sc, const float* Om,
                                const float* Ysk, cudaStream_t st) {
  const int r = cb.r;
  cudaError_t e;
  // Gram of [Omega | M Omega] -> (Omega^T Omega, Omega^T Y, Y^T Y)
  if ((e = launch_gram(Om, r, r, Ysk, r, r, cb.b, cb.gram_part, cb.gram_chunks, cb.G, false, st))) return e;
  if ((e = launch_gram(Ysk, r, r, nullptr, 0, 0, cb.b, cb.gram_part, cb.gram_chunks, cb.Gyy, true, st))) return e;
  const size_t sm_chol = (size_t)r * (r + 1) * sizeof(double);
  k_nys_chol<<<1, 512, sm_chol, st>>>(cb.G, cb.Gyy, r, eps, cb.Lc, cb.Gnu, sc);
  // A = L^{-1} Gnu L^{-T}  (= C^{-T} Y_nu^T Y_nu C^{-1} = B^T B)
  if ((e = trsm(cb.Lc, r, cb.Gnu, 0, 0, cb.X1, st))) return e;
  if ((e = trsm(cb.Lc, r, cb.X1, 1, 0, cb.A, st))) return e;
  const int r2 = r + (r & 1);
  k_jacobi<<<1, 1024, (size_t)2 * r2 * r2 * sizeof(float), st>>>(cb.A, r, cb.V32, sc);
  k_rayleigh<<<r, 128, 0, st>>>(cb.A, cb.V32, r, cb.lam);
  k_nys_finalize<<<1, 256, 0, st>>>(cb.lam, cb.V32, r, lam, sc, cb.S, cb.keep, cb.X1);
  // T = L^{-T} T'
  if ((e = trsm(cb.Lc, r, cb.X1, 0, 1, cb.T, st))) return e;
  return make_u(Ysk, Om, cb.b, r, cb.T, 0, sc, cb.U, st);
}

// L_w L_w^T = rho S^{-1} + U^T U on the kept eigenpairs (App. C.2, stabilised form)
__global__ void __launch_bounds__(512) k_wchol(const double* __restrict__ UtU, int r, const double* __restrict__ S,
                                               const double* __restrict__ keep, DevScalars* sc,
                                               double* __restrict__ Lw) {
  extern __shared__ double sh[];
  __shared__ int flag;
  const int ld = r + 1;
  const double rho = sc->rho;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e / r, j = e % r;
    double v = keep[i] * keep[j] * UtU[e];
    if (i == j) v += keep[i] > 0.0 ? rho / S[i] : 1.0;
    sh[i * ld + j] = v;
  }
  __syncthreads();
  const bool ok = chol_lower_smem(sh, r, ld, &flag);
  __syncthreads();
  if (!ok && threadIdx.x == 0) set_status(sc, ADASAP_ENUMERIC, 3);
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e / r, j = e % r;
    Lw[e] = ok ? ((j <= i) ? sh[i * ld + j] : 0.0) : (i == j ? 1.0 : 0.0);
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
  k_wchol<<<1, 512, (size_t)r * (r + 1) * sizeof(double), st>>>(cb.X1, r, cb.S, cb.keep, sc, cb.Lw);
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
__global__ void __launch_bounds__(256) k_wcoef(int mode, const double* __restrict__ part, int chunks, int r, int s,
                                               const double* __restrict__ S, const double* __restrict__ keep,
                                               const double* __restrict__ Lw, const double* __restrict__ sq_part,
                                               DevScalars* sc, float* __restrict__ coef, double* __restrict__ alpha) {
  extern __shared__ double q[];  // r x s
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
  for (int o = threadIdx.x; o < nout; o += blockDim.x) {
    double acc = 0.0;
    for (int ch = 0; ch < chunks; ++ch) acc += part[(int64_t)ch * nout + o];
    q[o] = acc;
  }
  __syncthreads();
  if (mode == kInv) {
    // y = L^{-T} L^{-1} (keep . q): one warp per column, lanes split each dot product
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c = warp; c < s; c += nw) {
      for (int i = 0; i < r; ++i) {
        double part = 0.0;
        for (int k = lane; k < i; k += 32) part += Lw[i * r + k] * q[k * s + c];
        part = warp_sum(part);
        if (lane == 0) q[i * s + c] = (keep[i] * q[i * s + c] - part) / Lw[i * r + i];
        __syncwarp();
      }
      for (int i = r - 1; i >= 0; --i) {
        double part = 0.0;
        for (int k = i + 1 + lane; k < r; k += 32) part += Lw[k * r + i] * q[k * s + c];
        part = warp_sum(part);
        if (lane == 0) q[i * s + c] = (q[i * s + c] - part) / Lw[i * r + i];
        __syncwarp();
      }
    }
    __syncthreads();
    for (int o = threadIdx.x; o < nout; o += blockDim.x) coef[o] = (float)(-keep[o / s] * q[o] / rho);
    if (threadIdx.x == 0) alpha[0] = 1.0 / rho;
  } else {
    const double irs = 1.0 / sqrt(rho);
    for (int o = threadIdx.x; o < nout; o += blockDim.x) {
      const int k = o / s;
      coef[o] = (float)(scale * q[o] * (1.0 / sqrt(S[k] + rho) - irs));
    }
    if (threadIdx.x == 0) {
      alpha[0] = scale * irs;
      if (mode == kInvSqrtNormalised) alpha[1] = scale;
    }
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
  k_wcoef<<<1, 256, (size_t)r * s * sizeof(double), st>>>(mode, cb.utv_part, cb.utv_chunks, r, s, cb.S, cb.keep,
                                                          cb.Lw, cb.sq_part, sc, cb.coef, cb.alpha);
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
  // the identity path leaves per-block partials; the cluster apply leaves one sum
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

__global__ void k_sum_blocks(const double* __restrict__ parts, int count, double* dst) {
  __shared__ double red[33];
  double t = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) t += parts[i];
  t = block_sum(t, red);
  if (threadIdx.x == 0) *dst = t;
}

cudaError_t launch_sum_blocks(const double* parts, int count, double* dst, cudaStream_t st) {
  k_sum_blocks<<<1, 256, 0, st>>>(parts, count, dst);
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
// One single-RHS Woodbury apply (App. C.2) in one launch of an 8-CTA cluster:
//   mode kInvSqrtNormalised:  out = (P + rho I)^{-1/2} (v / ||v||)
//   mode kInvSqrt:            out = (P + rho I)^{-1/2} v
//   mode kInv:                out = (P + rho I)^{-1} v  (Cholesky-stabilised form)
// Phase 1: each CTA reduces U^T v and ||v||^2 over its rows (a warp takes
// eight rows at a time, lanes split k; FP32 per warp, FP64 across warps); the
// partials meet through distributed shared memory; every CTA forms the
// coefficients; phase 3 writes its rows of out = alpha v + U coef (one thread
// per row) and, optionally, partial sums of out . dotv that CTA 0 collects
// into *dot_out.
// ---------------------------------------------------------------------------
constexpr int kWbCluster = 8, kWbThreads = 256, kWbWarps = kWbThreads / 32, kWbRows = 8;

struct WbArgs {
  const float* U;
  int64_t b;
  int r;
  const float* v;
  int mode;
  const double* keep;
  const double* Lw;
  const double* cis;
  const DevScalars* sc;
  float* out;
  const float* dotv;
  double* alpha;    // [0] alpha used, [1] 1/||v|| in normalised mode
  double* dot_out;  // sum(out . dotv) when dotv != NULL
};

__global__ void __cluster_dims__(kWbCluster, 1, 1) __launch_bounds__(kWbThreads) k_wb_cluster(WbArgs a) {
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  __shared__ double part[kMaxRank + 2];        // this CTA's U^T v, ||v||^2, out . dotv
  __shared__ double q[kMaxRank + 1];
  __shared__ float coef[kMaxRank];
  __shared__ float wtmp[kWbWarps][kMaxRank];
  __shared__ double red[33];
  __shared__ double s_alpha;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = a.r;
  constexpr int KJ = kMaxRank / 32;
  const int64_t per = (a.b + kWbCluster - 1) / kWbCluster;
  const int64_t r0 = (int64_t)rank * per, r1 = min(a.b, r0 + per);
  // ---- phase 1
  float acc[KJ];
#pragma unroll
  for (int j = 0; j < KJ; ++j) acc[j] = 0.0f;
  double vsq = 0.0;
  for (int64_t i0 = r0 + (int64_t)warp * kWbRows; i0 < r1; i0 += (int64_t)kWbWarps * kWbRows) {
    float vi[kWbRows], u[kWbRows][KJ];
#pragma unroll
    for (int t = 0; t < kWbRows; ++t) {
      const int64_t i = i0 + t;
      const bool ok = i < r1;
      vi[t] = ok ? a.v[i] : 0.0f;
#pragma unroll
      for (int j = 0; j < KJ; ++j) {
        const int k = lane + 32 * j;
        u[t][j] = (ok && k < r) ? a.U[i * r + k] : 0.0f;
      }
    }
#pragma unroll
    for (int t = 0; t < kWbRows; ++t) {
#pragma unroll
      for (int j = 0; j < KJ; ++j) acc[j] = fmaf(u[t][j], vi[t], acc[j]);
      if (lane == 0) vsq += (double)vi[t] * (double)vi[t];
    }
  }
#pragma unroll
  for (int j = 0; j < KJ; ++j) {
    const int k = lane + 32 * j;
    if (k < r) wtmp[warp][k] = acc[j];
  }
  const double vsq_t = block_sum(vsq, red);   // contains __syncthreads
  for (int k = threadIdx.x; k < r; k += kWbThreads) {
    double t = 0.0;
    for (int w = 0; w < kWbWarps; ++w) t += (double)wtmp[w][k];
    part[k] = t;
  }
  if (threadIdx.x == 0) part[r] = vsq_t;
  cl.sync();
  // ---- phase 2: gather partials from every CTA of the cluster
  for (int k = threadIdx.x; k <= r; k += kWbThreads) {
    double t = 0.0;
#pragma unroll
    for (int c = 0; c < kWbCluster; ++c) t += cl.map_shared_rank(part, c)[k];
    q[k] = t;
  }
  __syncthreads();
  const double rho = a.sc->rho;
  if (a.mode == kInv) {
    // y = Lw^{-T} Lw^{-1} (keep . q) by warp 0, lanes splitting the dot products
    if (warp == 0) {
      for (int i = 0; i < r; ++i) {
        double pt = 0.0;
        for (int k = lane; k < i; k += 32) pt += a.Lw[i * r + k] * q[k];
        pt = warp_sum(pt);
        if (lane == 0) q[i] = (a.keep[i] * q[i] - pt) / a.Lw[i * r + i];
        __syncwarp();
      }
      for (int i = r - 1; i >= 0; --i) {
        double pt = 0.0;
        for (int k = i + 1 + lane; k < r; k += 32) pt += a.Lw[k * r + i] * q[k];
        pt = warp_sum(pt);
        if (lane == 0) q[i] = (q[i] - pt) / a.Lw[i * r + i];
        __syncwarp();
      }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < r; k += kWbThreads) coef[k] = (float)(-a.keep[k] * q[k] / rho);
    if (threadIdx.x == 0) s_alpha = 1.0 / rho;
  } else {
    const double scale = (a.mode == kInvSqrtNormalised) ? (q[r] > 0.0 ? 1.0 / sqrt(q[r]) : 0.0) : 1.0;
    for (int k = threadIdx.x; k < r; k += kWbThreads) coef[k] = (float)(scale * q[k] * a.cis[k]);
    if (threadIdx.x == 0) {
      s_alpha = scale / sqrt(rho);
      if (rank == 0) {
        a.alpha[0] = s_alpha;
        if (a.mode == kInvSqrtNormalised) a.alpha[1] = scale;
      }
    }
  }
  __syncthreads();
  const float al = (float)s_alpha;
  // ---- phase 3: out rows, one thread per row (independent loads)
  double dt = 0.0;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += kWbThreads) {
    const float* ui = a.U + i * r;
    float t0 = 0.0f, t1 = 0.0f, t2 = 0.0f, t3 = 0.0f;
    int k = 0;
    for (; k + 4 <= r; k += 4) {
      t0 = fmaf(ui[k], coef[k], t0);
      t1 = fmaf(ui[k + 1], coef[k + 1], t1);
      t2 = fmaf(ui[k + 2], coef[k + 2], t2);
      t3 = fmaf(ui[k + 3], coef[k + 3], t3);
    }
    for (; k < r; ++k) t0 = fmaf(ui[k], coef[k], t0);
    const float o = fmaf(al, a.v[i], (t0 + t1) + (t2 + t3));
    a.out[i] = o;
    if (a.dotv) dt += (double)o * (double)a.dotv[i];
  }
  if (a.dotv) {
    const double dtt = block_sum(dt, red);
    if (threadIdx.x == 0) part[kMaxRank + 1] = dtt;
  }
  cl.sync();
  if (a.dotv && rank == 0 && threadIdx.x == 0) {
    double t = 0.0;
    for (int c = 0; c < kWbCluster; ++c) t += cl.map_shared_rank(part, c)[kMaxRank + 1];
    *a.dot_out = t;
  }
  cl.sync();  // no CTA leaves while rank 0 may still read its shared memory
}

cudaError_t launch_wb_cluster(CoreBufs& cb, int mode, const float* v, float* out, const float* dotv, DevScalars* sc,
                              cudaStream_t st) {
  WbArgs a;
  a.U = cb.U; a.b = cb.b; a.r = cb.r; a.v = v; a.mode = mode; a.keep = cb.keep; a.Lw = cb.Lw; a.cis = cb.cis;
  a.sc = sc; a.out = out; a.dotv = dotv; a.alpha = cb.alpha; a.dot_out = cb.dot_part;
  k_wb_cluster<<<kWbCluster, kWbThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t core_init() {
  const int big = 200 * 1024;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_nys_chol, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = cudaFuncSetAttribute(k_make_u, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = cudaFuncSetAttribute(k_chol_plain<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = cudaFuncSetAttribute(k_chol_plain<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = cudaFuncSetAttribute(k_trsm<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = cudaFuncSetAttribute(k_trsm<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = cudaFuncSetAttribute(k_wchol, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = cudaFuncSetAttribute(k_wcoef, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = cudaFuncSetAttribute(k_wapply, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  return cudaSuccess;
}

}  // namespace adasap
