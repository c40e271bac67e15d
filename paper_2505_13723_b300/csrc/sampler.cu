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

namespace adasap {

__host__ __device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
#pragma unroll
  for (int rnd = 0; rnd < 10; ++rnd) {
    if (rnd > 0) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint64_t p0 = (uint64_t)M0 * c.x;
    const uint64_t p1 = (uint64_t)M1 * c.z;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

__device__ __forceinline__ uint2 seed_key(uint64_t seed) {
  return make_uint2((uint32_t)(seed & 0xFFFFFFFFull), (uint32_t)(seed >> 32));
}

static int feistel_half_bits(int64_t n) {
  int k = 2;
  while (k < 62 && (1LL << k) < n) ++k;
  return (k + 1) / 2;
}

__global__ void k_sample_block(uint64_t seed, const long long* __restrict__ t_dev, int64_t t_host, int64_t n,
                               int64_t b, int h, int tag, int* __restrict__ B32, int64_t* __restrict__ B64) {
  const uint32_t t = (uint32_t)(t_dev ? *t_dev : t_host);
  const uint2 key = seed_key(seed);
  const uint32_t mask = (h >= 32) ? 0xFFFFFFFFu : ((1u << h) - 1u);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < b; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t x = (uint64_t)i;
    // every step applies the bijection of [0, 2^(2h)); the walk returns below n
    // within the cycle of i, so it terminates
    do {
      uint32_t L = (uint32_t)(x >> h) & mask, R = (uint32_t)x & mask;
      for (uint32_t j = 0; j < 4; ++j) {
        const uint32_t F = philox4x32_10(make_uint4(R, t, j, (uint32_t)tag), key).x & mask;
        const uint32_t nl = R;
        R = L ^ F;
        L = nl;
      }
      x = ((uint64_t)L << h) | R;
    } while (x >= (uint64_t)n);
    if (B32) B32[i] = (int)x;
    if (B64) B64[i] = (int64_t)x;
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
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nblk; j += (int64_t)gridDim.x * blockDim.x) {
    const uint4 w = philox4x32_10(make_uint4((uint32_t)j, t, 0u, (uint32_t)tag), key);
    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const float u0 = fmaf((float)ws[2 * p], 2.3283064365386963e-10f, 1.1641532182693481e-10f);
      const float u1 = fmaf((float)ws[2 * p + 1], 2.3283064365386963e-10f, 1.1641532182693481e-10f);
      const float rad = sqrtf(-2.0f * logf(u0));
      float sn, cs;
      sincospif(2.0f * u1, &sn, &cs);
      const int64_t e0 = 4 * j + 2 * p;
      if (e0 < count) out[e0] = scale * rad * cs;
      if (e0 + 1 < count) out[e0 + 1] = scale * rad * sn;
    }
  }
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

}  // namespace adasap
