// Device randomness of Alg. 2: the block B (b distinct rows, uniform; Sec. 4.3),
// the Gaussian Nystrom test matrix Omega (Alg. 2 Step II) and the start vector
// v0 of the randomized powering (Alg. 5).
//
// Generator: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
//   (hi0, lo0) = 0xD2511F53 * c0, (hi1, lo1) = 0xCD9E8D57 * c2,
//   c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0),
// with the key bumped by (0x9E3779B9, 0xBB67AE85) between rounds.
// Key = (seed mod 2^32, seed >> 32).  Stream tags: FEISTEL 1, OMEGA 2, V0 3, CHECK 4.
//
// Block B[i] = pi_t(i): pi_t is a permutation of [n] built from a balanced
// 4-round Feistel network on 2h bits (2^(2h) >= n) whose round j maps
// (L, R) -> (R, L ^ (word0(Philox(R, t, j, FEISTEL)) & mask)), applied
// repeatedly until the value falls below n (cycle walking, Black & Rogaway,
// CT-RSA 2002).  The walk ends because pi_t's cycle through i contains i < n.
//
// Normals: element e of a stream at iteration t uses Philox counter
// (e / 4, t, 0, tag); word pairs (0,1) and (2,3) give two normals each by
// Box-Muller with u(w) = (w + 0.5) 2^-32: rad = sqrt(-2 ln u(w_even)),
// (rad cos 2 pi u(w_odd), rad sin 2 pi u(w_odd)).
#include <algorithm>

#include "internal.cuh"
#include "prep.cuh"

namespace adasap {

__global__ void k_sample_block(uint64_t seed, const long long* __restrict__ t_dev, int64_t t_host, int64_t n,
                               int64_t b, int h, int tag, int* __restrict__ B32, int64_t* __restrict__ B64) {
  const uint32_t t = (uint32_t)(t_dev ? *t_dev : t_host);
  const uint2 key = seed_key(seed);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < b; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = feistel_index(i, n, h, t, tag, key);
    if (B32) B32[i] = (int)x;
    if (B64) B64[i] = x;
  }
}

cudaError_t launch_sample_block(uint64_t seed, const long long* t_dev, int64_t t_host, int64_t n, int64_t b,
                                int stream_tag, int* B32, int64_t* B64, cudaStream_t st) {
  if (b <= 0) return cudaSuccess;
  const int h = feistel_half_bits(n);
  const int blocks = (int)std::min<int64_t>((b + 255) / 256, 148 * 8);
  k_sample_block<<<blocks, 256, 0, st>>>(seed, t_dev, t_host, n, b, h, stream_tag, B32, B64);
  return cudaGetLastError();
}

__global__ void k_normals(uint64_t seed, const long long* __restrict__ t_dev, int64_t t_host, int64_t count, int tag,
                          float scale, float* __restrict__ out) {
  // iteration counter: the device counter (when given) plus the host offset
  const uint32_t t = (uint32_t)((t_dev ? *t_dev : 0) + t_host);
  const uint2 key = seed_key(seed);
  const int64_t nblk = (count + 3) / 4;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nblk; j += (int64_t)gridDim.x * blockDim.x)
    normals4(j, t, tag, key, scale, count, out);
}

cudaError_t launch_normals(uint64_t seed, const long long* t_dev, int64_t t_host, int64_t count, int stream_tag,
                           float scale, float* out, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>(((count + 3) / 4 + 255) / 256, 148 * 8);
  k_normals<<<blocks, 256, 0, st>>>(seed, t_dev, t_host, count, stream_tag, scale, out);
  return cudaGetLastError();
}

// Omega of iteration t + offset of a caller-supplied schedule (nothing when
// t + offset >= T, past the schedule's last iteration).
__global__ void k_copy_omega(const float* __restrict__ Om_s, const long long* __restrict__ t_dev, int offset,
                             int64_t T, int64_t total, float* __restrict__ Om) {
  const long long t = *t_dev + offset;
  if (t >= T) return;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    Om[e] = Om_s[t * total + e];
}

cudaError_t launch_copy_omega(const float* Om_s, const long long* t_dev, int offset, int64_t T, int64_t b, int r,
                              float* Om, cudaStream_t st) {
  const int64_t total = b * (int64_t)r;
  if (total <= 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 148 * 8);
  k_copy_omega<<<blocks, 256, 0, st>>>(Om_s, t_dev, offset, T, total, Om);
  return cudaGetLastError();
}

// Iteration t of a caller-supplied schedule; rows outside [0, n) are an error
// (status EINVAL) and are replaced by row 0 so nothing reads out of bounds.
__global__ void k_copy_schedule(const int64_t* __restrict__ Bs, const float* __restrict__ Om_s,
                                const float* __restrict__ v0s, const long long* __restrict__ t_dev, int64_t n,
                                int64_t b, int r, int* __restrict__ B32, float* __restrict__ Om, float* __restrict__ v0,
                                DevScalars* sc) {
  const long long t = *t_dev;
  const int64_t total = b * (int64_t)r;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    if (Om_s) Om[e] = Om_s[t * total + e];
    if (e < b) {
      const int64_t v = Bs[t * b + e];
      const bool ok = v >= 0 && v < n;
      if (!ok) set_status(sc, ADASAP_EINVAL, 5);
      B32[e] = ok ? (int)v : 0;
      v0[e] = v0s[t * b + e];
    }
  }
}

cudaError_t launch_copy_schedule(const int64_t* Bs, const float* Om_s, const float* v0s, const long long* t_dev,
                                 int64_t n, int64_t b, int r, int* B32, float* Om, float* v0, DevScalars* sc,
                                 cudaStream_t st) {
  const int64_t total = std::max<int64_t>(b * (int64_t)std::max(r, 1), b);
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 148 * 8);
  k_copy_schedule<<<blocks, 256, 0, st>>>(Bs, r > 0 ? Om_s : nullptr, v0s, t_dev, n, b, std::max(r, 1), B32, Om, v0,
                                          sc);
  return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// k_head_prep: one launch for the inputs of an iteration (see HeadPrepArgs).
// Work items of system y: rows j < npad (sample, gather and split operand of
// row j; padding rows past b), then the (b + 3) / 4 normal quadruples of v0,
// then the npad x sp elements of Omega_t's operand (and its copy).  The row
// items read nothing another item writes, so no item waits for another.
// ---------------------------------------------------------------------------
int64_t head_prep_work(const HeadPrepArgs& a) { return a.npad + (a.b + 3) / 4 + a.npad * a.sp; }

int feistel_half_width(int64_t n) { return feistel_half_bits(n); }

template <int KP>
__global__ void k_head_prep(const HeadPrepArgs* __restrict__ tab) {
  const HeadPrepArgs a = tab[blockIdx.y];
  const uint32_t t = (uint32_t)*a.t_dev;
  const uint2 key = seed_key(a.seed);
  const int64_t nrow = a.npad, nnorm = (a.b + 3) / 4;
  const int64_t total = nrow + nnorm + a.npad * a.sp;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    if (e < nrow) {
      int64_t src = -1;
      if (e < a.b) {
        src = feistel_index(e, a.n, a.h, t, 1, key);
        a.B32[e] = (int)src;
        const float4* xs = reinterpret_cast<const float4*>(a.Xc + src * a.dp);
        float4* xd = reinterpret_cast<float4*>(a.XB + e * a.dp);
        for (int k4 = 0; k4 < a.dp / 4; ++k4) xd[k4] = xs[k4];
        a.qB[e] = a.qc[src];
      }
      build_tc_row<KP>(a.Xc, a.qc, src, a.d, a.dp, e, a.XBhi, a.XBlo);
    } else if (e < nrow + nnorm) {
      normals4(e - nrow, t, 3, key, 1.0f, a.b, a.v0);
    } else {
      const int64_t f = e - nrow - nnorm;
      const int64_t j = f / a.sp;
      const int c = (int)(f - j * a.sp);
      const bool in = j < a.b && c < a.r;
      const float v = in ? a.OmN[j * a.r + c] : 0.0f;
      if (in) a.Om[j * a.r + c] = v;
      build_w_elem(v, j, c, a.sp, 3, a.whi, a.wlo);
    }
  }
}

cudaError_t launch_head_prep(const HeadPrepArgs* tab, int nsys, int kp, int64_t max_work, cudaStream_t st) {
  if (nsys <= 0 || max_work <= 0) return cudaSuccess;
  const dim3 grid((unsigned)std::min<int64_t>((max_work + 255) / 256, nsys > 1 ? 64 : 148 * 8), (unsigned)nsys);
  if (kp == 16) k_head_prep<16><<<grid, 256, 0, st>>>(tab);
  else if (kp == 32) k_head_prep<32><<<grid, 256, 0, st>>>(tab);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace adasap
