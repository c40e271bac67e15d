// Shared device helpers of the ADASAP CUDA path (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "adasap.h"

namespace adasap {

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;

// ---- PTX one-instruction approximations (MUFU) and packed FP32 -------------
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// sqrt(v) for finite v >= 0 on the FMA pipe (no special-function unit): a seed for
// 1/sqrt(v) from the IEEE bit pattern (the exponent halved and negated by one
// integer subtraction: the magic-constant method, analysed by C. Lomont, "Fast
// inverse square root", 2003), two Newton steps r <- r (3/2 - v r^2 / 2) (relative
// error 3.4e-2 -> 1.7e-3 -> 4.6e-6), then one coupled correction of s = v r,
// s <- s + (r / 2)(v - s^2), which squares the error again.  v is first clamped to
// at least 1e-30 (at v = 0 the seed's square would overflow; sqrt(1e-30) = 1e-15
// is zero for every kernel epilogue here), and over [1e-30, 1e21] the result is
// within 0.5 ulp of the correctly rounded square root.  Eleven FMA-pipe
// operations, two integer ones and the clamp, used for a share of the entries of
// the Matern epilogues, whose sqrt.approx would otherwise take half of the
// special-function unit's time.
__device__ __forceinline__ float sqrt_fma(float v) {
  v = fmaxf(v, 1e-30f);
  float r = __int_as_float(0x5f3759df - (__float_as_int(v) >> 1));
  const float h = 0.5f * v;
  r = r * fmaf(-h, r * r, 1.5f);
  r = r * fmaf(-h, r * r, 1.5f);
  const float s = v * r;
  return fmaf(0.5f * r, fmaf(-s, s, v), s);
}

// d = a * b + c on two lanes at once (sm_100+ packed FP32 FMA)
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  unsigned long long ra = *reinterpret_cast<unsigned long long*>(&a);
  unsigned long long rb = *reinterpret_cast<unsigned long long*>(&b);
  unsigned long long rc = *reinterpret_cast<unsigned long long*>(&c);
  unsigned long long rd;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(rd) : "l"(ra), "l"(rb), "l"(rc));
  return *reinterpret_cast<float2*>(&rd);
}

__device__ __forceinline__ float2 fmul2(float2 a, float2 b) {
  unsigned long long ra = *reinterpret_cast<unsigned long long*>(&a);
  unsigned long long rb = *reinterpret_cast<unsigned long long*>(&b);
  unsigned long long rd;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
  return *reinterpret_cast<float2*>(&rd);
}

// ---- kernel epilogues --------------------------------------------------------
// Columns and rows are stored pre-scaled: x' = kappa (x - mean) / ell with
//   RBF  kappa^2 = log2(e)/2   -> u = kappa^2 r~^2,  k = sigma2 * 2^(-u)
//   M32  kappa^2 = 3           -> u = a^2,           k = sigma2 (1 + a) e^(-a)
//   M52  kappa^2 = 5           -> u = a^2,           k = sigma2 (1 + a + a^2/3) e^(-a)
// where r~ = r / ell and u = ||x'_i - x'_j||^2 >= 0.  kval returns k / sigma2.
template <int KERN>
__device__ __forceinline__ float kval(float u) {
  if (KERN == ADASAP_RBF) return ex2_approx(-u);
  float a = sqrt_approx(fmaxf(u, 0.0f));
  float e = ex2_approx(-kLog2e * a);
  if (KERN == ADASAP_MATERN32) return fmaf(a, e, e);
  float p = fmaf(a, fmaf(a, 1.0f / 3.0f, 1.0f), 1.0f);
  return p * e;
}
// k / sigma2 and g = ell * (dk/dell) / sigma2 together (adjoint):
//   RBF  g = r~^2 e^(-r~^2/2) = 2 ln2 u 2^(-u)
//   M32  g = a^2 e^(-a)
//   M52  g = a^2 (1 + a) e^(-a) / 3
template <int KERN>
__device__ __forceinline__ void kval_grad(float u, float& kv, float& gv) {
  if (KERN == ADASAP_RBF) {
    float e = ex2_approx(-u);
    kv = e;
    gv = (2.0f * kLn2) * u * e;
    return;
  }
  float a = sqrt_approx(fmaxf(u, 0.0f));
  float e = ex2_approx(-kLog2e * a);
  if (KERN == ADASAP_MATERN32) {
    kv = fmaf(a, e, e);
    gv = u * e;
  } else {
    kv = fmaf(a, fmaf(a, 1.0f / 3.0f, 1.0f), 1.0f) * e;
    gv = u * fmaf(a, e, e) * (1.0f / 3.0f);
  }
}

// ---- reductions ------------------------------------------------------------
// (H, L) += x in double-float arithmetic (Knuth's TwoSum: H + x is split exactly
// into its rounded sum and rounding error, the error accumulated in L).  Sums of
// FP32 terms carried this way keep about 48 bits on the FP32 pipes; FP64
// arithmetic runs at a small fraction of their rate on this GPU.
__device__ __forceinline__ void ff_add(float& H, float& L, float x) {
  const float s = H + x;
  const float z = s - H;
  L += (H - (s - z)) + (x - z);
  H = s;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// Block-wide double sum; every thread gets the result.  blockDim.x <= 1024.
__device__ __forceinline__ double block_sum(double v, double* red /* >= 33 doubles */) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double w = (lane < (int)((blockDim.x + 31) >> 5)) ? red[lane] : 0.0;
    w = warp_sum(w);
    if (lane == 0) red[32] = w;
  }
  __syncthreads();
  return red[32];
}

// ---- device status -----------------------------------------------------------
// Scalars shared by the kernels of one solve (device memory).
struct DevScalars {
  double delta;      // Nystrom shift Delta (Alg. 4)
  double rho;        // damping rho = S_rr + lambda
  double eta;        // stepsize eta_B (Alg. 5)
  double lam_hat;    // Rayleigh quotient of the power iteration
  double ysq;        // ||Y||_F^2
  double resid_sq;   // sum of squares of the sampled residual
  double dot;        // scratch dot product (power iteration)
  int status;        // first error (adasap_status), 0 if none
  int detail;        // stage of the first error: 1 Nystrom core Cholesky, 2 non-finite
                     // eigenvalue, 3 Woodbury Cholesky, 4 non-positive stepsize estimate,
                     // 5 schedule row out of range, 6 test-matrix QR Cholesky,
                     // 7 exact block Cholesky (SAP)
  int chol_retries;  // number of Delta increases in the last iteration
  int jacobi_sweeps; // sweeps of the last eigen-solve
  long long t;       // iteration counter
};

__device__ __forceinline__ void set_status(DevScalars* sc, int code, int detail = 0) {
  if (atomicCAS(&sc->status, 0, code) == 0) sc->detail = detail;
}

}  // namespace adasap
