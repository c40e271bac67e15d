// Random-feature prior draws and the pieces of pathwise conditioning (Sec. 2.1):
//
//   f(x)_j = sqrt(2 sigma2 / q) * sum_l theta[l][j] cos(omega_l . x + phase_l)
//
// with omega_l = s_l z_l / ell, s_l = 1 (RBF) or sqrt(2 nu / u_l) (Matern-nu;
// u_l ~ chi^2(2 nu) makes omega_l a multivariate Student t draw, the Matern
// spectral density).  Points arrive in the context's centred, scaled form
// x' = kappa (x - mean) / ell, so the kernel uses
//   omega_l . x = (s_l z_l / kappa) . x' + s_l (z_l . mean) / ell.
//
// The feature sum is a contraction over q (2048 in the paper's runs) with s
// right-hand sides; both forms here run on the FP32 pipe:
//   k_rf_rows   (s <= 8): one thread per point, the s sums in registers;
//   k_rf_tiled  (s > 8):  64 points x all s columns per block, the 64 x 64
//               cosine tile staged in shared memory and contracted with the
//               64 x s coefficient chunk by 4 x ceil(s / 16) register tiles.
// Epilogue (both): out[i][j] = sign * f + (y ? y[i] : 0) + gz * Z[i][j], which
// forms the pathwise right-hand sides y - f(X) - zeta (sign = -1, gz = -1) or
// adds f(X*) to the posterior product k(X*, X) W in place (sign = 1, gz = 1,
// Z = out).
#include <algorithm>
#include <cmath>

#include "internal.cuh"

namespace adasap {

constexpr int kRfThreads = 256;
constexpr int kRfChunk = 64;   // features per shared-memory chunk
constexpr int kRfRows = 64;    // points per block of the tiled form

__global__ void k_rf_prep(const float* __restrict__ z, const float* __restrict__ u, const float* __restrict__ phase,
                          int q, int d, int dp, int kern, const double* __restrict__ mean, double ell, double kappa,
                          float* __restrict__ omega, float* __restrict__ cphase) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= q) return;
  double sc = 1.0;
  if (kern != ADASAP_RBF) {
    const double nu = kern == ADASAP_MATERN32 ? 1.5 : 2.5;
    sc = sqrt(2.0 * nu / (double)u[l]);
  }
  double zm = 0.0;
  for (int k = 0; k < dp; ++k) {
    const double zk = k < d ? (double)z[(int64_t)l * d + k] : 0.0;
    omega[(int64_t)l * dp + k] = (float)(sc * zk / kappa);
    if (k < d) zm += zk * mean[k];
  }
  cphase[l] = (float)((double)phase[l] + sc * zm / ell);
}

struct RfArgs {
  const float* x;       // m x dp points (x' form)
  int64_t m;
  int dp;
  const float* omega;   // q x dp
  const float* cph;     // q
  const float* theta;   // q x s
  int q, s;
  float scale;          // sqrt(2 sigma2 / q) * sign
  const float* y;       // optional, m
  const float* zin;     // optional, m x ldz from column zoff (read before out is written)
  int64_t ldz;
  int zoff;
  float gz;
  float* out;           // m x ldo, columns coff .. coff + s - 1
  int64_t ldo;
  int coff;
};

__device__ __forceinline__ float rf_out(const RfArgs& a, int64_t i, int j, float f) {
  float v = a.scale * f;
  if (a.y) v += a.y[i];
  if (a.zin) v = fmaf(a.gz, a.zin[i * a.ldz + a.zoff + j], v);
  return v;
}

template <int NS, int DPM>
__global__ void __launch_bounds__(kRfThreads) k_rf_rows(RfArgs a) {
  extern __shared__ float sm[];
  float* so = sm;                          // [kRfChunk][dp]
  float* sc = so + kRfChunk * a.dp;        // [kRfChunk]
  float* st = sc + kRfChunk;               // [kRfChunk][s]
  const int64_t i = (int64_t)blockIdx.x * kRfThreads + threadIdx.x;
  const bool live = i < a.m;
  float x[DPM];
#pragma unroll
  for (int k = 0; k < DPM; ++k) x[k] = (live && k < a.dp) ? a.x[i * a.dp + k] : 0.0f;
  float acc[NS];
#pragma unroll
  for (int j = 0; j < NS; ++j) acc[j] = 0.0f;
  for (int l0 = 0; l0 < a.q; l0 += kRfChunk) {
    const int nl = min(kRfChunk, a.q - l0);
    __syncthreads();
    for (int e = threadIdx.x; e < nl * a.dp; e += kRfThreads) so[e] = a.omega[(int64_t)l0 * a.dp + e];
    for (int e = threadIdx.x; e < nl; e += kRfThreads) sc[e] = a.cph[l0 + e];
    for (int e = threadIdx.x; e < nl * a.s; e += kRfThreads) st[e] = a.theta[(int64_t)l0 * a.s + e];
    __syncthreads();
    for (int l = 0; l < nl; ++l) {
      float arg = sc[l];
#pragma unroll
      for (int k = 0; k < DPM; ++k)
        if (k < a.dp) arg = fmaf(so[l * a.dp + k], x[k], arg);
      const float c = cosf(arg);
#pragma unroll
      for (int j = 0; j < NS; ++j)
        if (j < a.s) acc[j] = fmaf(c, st[l * a.s + j], acc[j]);
    }
  }
  if (!live) return;
#pragma unroll
  for (int j = 0; j < NS; ++j)
    if (j < a.s) a.out[i * a.ldo + a.coff + j] = rf_out(a, i, j, acc[j]);
}

// 64 points x all s columns per block: thread (tr, tc) owns points 4 tr .. 4 tr + 3
// and columns tc + 16 c (c < CPT).
template <int CPT>
__global__ void __launch_bounds__(kRfThreads) k_rf_tiled(RfArgs a) {
  extern __shared__ float sm[];
  const int ldx = a.dp + 1;                         // odd stride: conflict-free point reads
  float* sx = sm;                                   // [kRfRows][dp + 1]
  float* so = sx + kRfRows * ldx;                   // [kRfChunk][dp]
  float* sc = so + kRfChunk * a.dp;                 // [kRfChunk]
  float* st = sc + kRfChunk;                        // [kRfChunk][16 CPT]
  float* sphi = st + kRfChunk * 16 * CPT;           // [kRfChunk][kRfRows + 1]
  const int tr = threadIdx.x >> 4, tc = threadIdx.x & 15;
  const int64_t i0 = (int64_t)blockIdx.x * kRfRows;
  const int spad = 16 * CPT;
  for (int e = threadIdx.x; e < kRfRows * a.dp; e += kRfThreads) {
    const int p = e / a.dp, k = e - p * a.dp;
    sx[p * ldx + k] = i0 + p < a.m ? a.x[i0 * a.dp + e] : 0.0f;
  }
  float acc[4][CPT];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < CPT; ++c) acc[r][c] = 0.0f;
  for (int l0 = 0; l0 < a.q; l0 += kRfChunk) {
    const int nl = min(kRfChunk, a.q - l0);
    __syncthreads();
    for (int e = threadIdx.x; e < kRfChunk * a.dp; e += kRfThreads)
      so[e] = e < nl * a.dp ? a.omega[(int64_t)l0 * a.dp + e] : 0.0f;
    for (int e = threadIdx.x; e < kRfChunk; e += kRfThreads) sc[e] = e < nl ? a.cph[l0 + e] : 0.0f;
    for (int e = threadIdx.x; e < kRfChunk * spad; e += kRfThreads) {
      const int l = e / spad, j = e - l * spad;
      st[e] = (l < nl && j < a.s) ? a.theta[(int64_t)(l0 + l) * a.s + j] : 0.0f;
    }
    __syncthreads();
    // cosine tile: entry (point p, feature l), 16 per thread
    for (int e = threadIdx.x; e < kRfRows * kRfChunk; e += kRfThreads) {
      const int l = e / kRfRows, p = e - l * kRfRows;
      float arg = sc[l];
      for (int k = 0; k < a.dp; ++k) arg = fmaf(so[l * a.dp + k], sx[p * ldx + k], arg);
      sphi[l * (kRfRows + 1) + p] = cosf(arg);
    }
    __syncthreads();
    for (int l = 0; l < nl; ++l) {
      float ph[4], th[CPT];
#pragma unroll
      for (int r = 0; r < 4; ++r) ph[r] = sphi[l * (kRfRows + 1) + 4 * tr + r];
#pragma unroll
      for (int c = 0; c < CPT; ++c) th[c] = st[l * spad + tc + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < CPT; ++c) acc[r][c] = fmaf(ph[r], th[c], acc[r][c]);
    }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int64_t i = i0 + 4 * tr + r;
    if (i >= a.m) continue;
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      const int j = tc + 16 * c;
      if (j < a.s) a.out[i * a.ldo + a.coff + j] = rf_out(a, i, j, acc[r][c]);
    }
  }
}

cudaError_t launch_rf_prep(const float* z, const float* u, const float* phase, int q, int d, int dp, int kern,
                           const double* mean, double ell, double kappa, float* omega, float* cphase,
                           cudaStream_t st) {
  if (q <= 0) return cudaSuccess;
  k_rf_prep<<<(q + 127) / 128, 128, 0, st>>>(z, u, phase, q, d, dp, kern, mean, ell, kappa, omega, cphase);
  return cudaGetLastError();
}

template <int NS>
static cudaError_t rf_rows(const RfArgs& a, cudaStream_t st) {
  const size_t smem = (size_t)(kRfChunk * a.dp + kRfChunk + kRfChunk * a.s) * sizeof(float);
  const int64_t blocks = (a.m + kRfThreads - 1) / kRfThreads;
  if (a.dp <= 16) k_rf_rows<NS, 16><<<(unsigned)blocks, kRfThreads, smem, st>>>(a);
  else k_rf_rows<NS, kMaxDim><<<(unsigned)blocks, kRfThreads, smem, st>>>(a);
  return cudaGetLastError();
}

template <int CPT>
static cudaError_t rf_tiled(const RfArgs& a, cudaStream_t st) {
  const size_t smem = (size_t)(kRfRows * (a.dp + 1) + kRfChunk * a.dp + kRfChunk + kRfChunk * 16 * CPT +
                               kRfChunk * (kRfRows + 1)) * sizeof(float);
  const int64_t blocks = (a.m + kRfRows - 1) / kRfRows;
  k_rf_tiled<CPT><<<(unsigned)blocks, kRfThreads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t rf_init() {
  // the tiled form at s = 128 needs 64 x 128 coefficients plus the tiles (> 48 KB)
  const int big = 160 * 1024;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_rf_tiled<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big)) ||
      (e = cudaFuncSetAttribute(k_rf_tiled<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, big)) ||
      (e = cudaFuncSetAttribute(k_rf_tiled<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, big)))
    return e;
  return cudaSuccess;
}

cudaError_t launch_rf_apply(const float* x, int64_t m, int dp, const float* omega, const float* cphase,
                            const float* theta, int q, int s, float scale, const float* y, const float* zin,
                            int64_t ldz, int zoff, float gz, float* out, int64_t ldo, int coff, cudaStream_t st) {
  if (m <= 0 || s <= 0) return cudaSuccess;
  if (s > kMaxRhs || dp > kMaxDim || q <= 0) return cudaErrorInvalidValue;
  RfArgs a;
  a.x = x; a.m = m; a.dp = dp; a.omega = omega; a.cph = cphase; a.theta = theta; a.q = q; a.s = s;
  a.scale = scale; a.y = y; a.zin = zin; a.ldz = ldz; a.zoff = zoff; a.gz = gz; a.out = out; a.ldo = ldo;
  a.coff = coff;
  if (s == 1) return rf_rows<1>(a, st);
  if (s <= 4) return rf_rows<4>(a, st);
  if (s <= 8) return rf_rows<8>(a, st);
  if (s <= 32) return rf_tiled<2>(a, st);
  if (s <= 64) return rf_tiled<4>(a, st);
  return rf_tiled<8>(a, st);
}

// Test RMSE of the posterior mean and the mean NLL under N(mean, sample variance
// (divisor s - 1) + noise): per-block FP64 partial sums [err^2, nll] in parts.
__global__ void k_rmse_nll(const float* __restrict__ mean, int64_t ldm, const float* __restrict__ smp, int64_t lds,
                           int s, const float* __restrict__ yt, int64_t m, double noise, double* parts) {
  __shared__ double red[33];
  double se = 0.0, nl = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    double mu = 0.0;
    for (int j = 0; j < s; ++j) mu += (double)smp[i * lds + j];
    mu /= s;
    double ss = 0.0;
    for (int j = 0; j < s; ++j) {
      const double dv = (double)smp[i * lds + j] - mu;
      ss += dv * dv;
    }
    const double var = ss / (s - 1) + noise;
    const double e = (double)yt[i] - (double)mean[i * ldm];
    se += e * e;
    nl += 0.5 * log(2.0 * 3.141592653589793 * var) + e * e / (2.0 * var);
  }
  se = block_sum(se, red);
  nl = block_sum(nl, red);
  if (threadIdx.x == 0) {
    parts[2 * blockIdx.x] = se;
    parts[2 * blockIdx.x + 1] = nl;
  }
}

cudaError_t launch_rmse_nll(const float* mean, int64_t ldm, const float* smp, int64_t lds, int s, const float* yt,
                            int64_t m, double noise, double* parts, int blocks, cudaStream_t st) {
  k_rmse_nll<<<blocks, 256, 0, st>>>(mean, ldm, smp, lds, s, yt, m, noise, parts);
  return cudaGetLastError();
}

}  // namespace adasap
