// Per-element bodies shared by the input kernels of an iteration (the block
// sample, the start vector v0, the gathered block rows and the tensor-core
// operands of the block) and by k_head_prep, which does all of them in one
// launch.  Each body is the exact arithmetic of its own kernel, so the fused
// launch gives the same bits as the separate ones.
#pragma once
#include "tc_ptx.cuh"

namespace adasap {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
//   (hi0, lo0) = 0xD2511F53 * c0, (hi1, lo1) = 0xCD9E8D57 * c2,
//   c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0),
// with the key bumped by (0x9E3779B9, 0xBB67AE85) between rounds.
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

__host__ __device__ __forceinline__ uint2 seed_key(uint64_t seed) {
  return make_uint2((uint32_t)(seed & 0xFFFFFFFFull), (uint32_t)(seed >> 32));
}

// Half width h of the Feistel network on 2h bits, 2^(2h) >= n.
__host__ __forceinline__ int feistel_half_bits(int64_t n) {
  int k = 2;
  while (k < 62 && (1LL << k) < n) ++k;
  return (k + 1) / 2;
}

// B[i] = pi_t(i): the balanced 4-round Feistel permutation of [0, 2^(2h)) with
// round j mapping (L, R) -> (R, L ^ (word0(Philox(R, t, j, tag)) & mask)),
// applied until the value falls below n (cycle walking, Black & Rogaway,
// CT-RSA 2002; it ends because pi_t's cycle through i < n returns below n).
__device__ __forceinline__ int64_t feistel_index(int64_t i, int64_t n, int h, uint32_t t, int tag, uint2 key) {
  const uint32_t mask = (h >= 32) ? 0xFFFFFFFFu : ((1u << h) - 1u);
  uint64_t x = (uint64_t)i;
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
  return (int64_t)x;
}

// Normals 4 j .. 4 j + 3 of a stream at iteration t (those below count): Philox
// counter (j, t, 0, tag); word pairs (0, 1) and (2, 3) give two normals each by
// Box-Muller with u(w) = (w + 0.5) 2^-32.
__device__ __forceinline__ void normals4(int64_t j, uint32_t t, int tag, uint2 key, float scale, int64_t count,
                                         float* __restrict__ out) {
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

// Row j of the split column operands of the tensor-core kernels, canonical
// layout: b_j = [x'_src (d), 1, q_src, 0 ...] for a point (src >= 0), the
// padding row [0, 1, 1e20, 0 ...] for src < 0.
template <int KP>
__device__ __forceinline__ void build_tc_row(const float* __restrict__ X, const float* __restrict__ q, int64_t src,
                                             int d, int dp, int64_t j, float* __restrict__ hi, float* __restrict__ lo) {
  float bv[KP];
#pragma unroll
  for (int k = 0; k < KP; ++k) bv[k] = 0.0f;
  if (src >= 0) {
    for (int k = 0; k < d; ++k) bv[k] = X[src * dp + k];
    bv[d + 1] = q[src];
  } else {
    bv[d + 1] = 1e20f;
  }
  bv[d] = 1.0f;
#pragma unroll
  for (int k = 0; k < KP; ++k) {
    const float h = tf32_round(bv[k]);
    hi[tc_off<KP>(j, k)] = h;
    lo[tc_off<KP>(j, k)] = tf32_round(bv[k] - h);
  }
}

// Element (row j, column c) of the multi-right-hand-side B operand: chunk j / 32
// holds rows [32 (j / 32), 32 (j / 32) + 32) as the sp x 32 K-major operand, hi
// and (three passes) lo.
__device__ __forceinline__ void build_w_elem(float v, int64_t j, int c, int sp, int passes, float* __restrict__ whi,
                                             float* __restrict__ wlo) {
  const float h = tf32_round(v);
  const int64_t off = (j / 32) * (int64_t)sp * 32 + tc_off<32>(c, (int)(j % 32));
  whi[off] = h;
  if (passes == 3) wlo[off] = tf32_round(v - h);
}

}  // namespace adasap
