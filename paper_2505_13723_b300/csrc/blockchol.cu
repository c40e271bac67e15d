// Exact block solve of Alg. 1 (SAP): D = (K_BB + lambda I)^{-1} R.
//
//   H = sigma2 k(X_B, X_B) + lambda I formed explicitly in FP32 (difference-form
//       distances), padded to bp = 64 * ceil(b / 64) rows with the identity;
//   H = L L^T by a right-looking blocked Cholesky over 64 x 64 tiles: per
//       panel k, k_chol_diag factors the diagonal tile and inverts it,
//       k_chol_panel forms L_ik = A_ik L_kk^{-T} for the tiles below, and
//       k_chol_update applies A_IJ -= L_Ik L_Jk^T to the trailing tiles;
//   D by blocked forward and backward substitution with the inverted
//       diagonal tiles (one CTA: the substitution is a chain of b / 64 steps),
//       then refined twice: D += (L L^T)^{-1} (R - H D), with R - H D
//       accumulated in FP64 against a copy of H.
// The refinement removes the factorisation's rounding (FP32, growing with b),
// so D carries the accuracy of H itself.  A non-positive pivot sets the
// solver status (ENUMERIC, detail 7) and is replaced by 1, so the launch
// chain always completes.
#include <algorithm>

#include "internal.cuh"

namespace adasap {

constexpr int kCb = 64;   // tile (and panel) width

template <int KERN>
__global__ void k_form_h(const float* __restrict__ xb, int64_t b, int64_t bp, int dp, float sigma2, float lam,
                         float* __restrict__ H) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < bp * bp; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / bp, j = e - i * bp;
    float v;
    if (i < b && j < b) {
      float u = 0.0f;
      for (int k = 0; k < dp; ++k) {
        const float t = xb[i * dp + k] - xb[j * dp + k];
        u = fmaf(t, t, u);
      }
      v = sigma2 * kval<KERN>(u) + (i == j ? lam : 0.0f);
    } else {
      v = i == j ? 1.0f : 0.0f;
    }
    H[e] = v;
  }
}

// Diagonal tile k (64 x 64, 1024 threads, 4 entries each): Cholesky in shared
// memory, then the inverse of the factor (one thread per column).
__global__ void __launch_bounds__(1024) k_chol_diag(float* __restrict__ A, int64_t bp, int k,
                                                    float* __restrict__ Linv, DevScalars* sc) {
  __shared__ float T[kCb][kCb + 1];
  __shared__ float I[kCb][kCb + 1];
  const int64_t o = (int64_t)k * kCb;
  for (int e = threadIdx.x; e < kCb * kCb; e += 1024) {
    const int r = e / kCb, c = e % kCb;
    T[r][c] = A[(o + r) * bp + o + c];
    I[r][c] = 0.0f;
  }
  __syncthreads();
  for (int j = 0; j < kCb; ++j) {
    if (threadIdx.x == 0) {
      const float d = T[j][j];
      if (!(d > 0.0f)) {
        set_status(sc, ADASAP_ENUMERIC, 7);
        T[j][j] = 1.0f;
      } else {
        T[j][j] = sqrtf(d);
      }
    }
    __syncthreads();
    if ((int)threadIdx.x > j && (int)threadIdx.x < kCb) T[threadIdx.x][j] /= T[j][j];
    __syncthreads();
    for (int e = threadIdx.x; e < kCb * kCb; e += 1024) {
      const int r = e / kCb, c = e % kCb;
      if (r > j && c > j && c <= r) T[r][c] = fmaf(-T[r][j], T[c][j], T[r][c]);
    }
    __syncthreads();
  }
  if (threadIdx.x < kCb) {
    const int col = threadIdx.x;
    for (int i = col; i < kCb; ++i) {
      float acc = i == col ? 1.0f : 0.0f;
      for (int m = col; m < i; ++m) acc = fmaf(-T[i][m], I[m][col], acc);
      I[i][col] = acc / T[i][i];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kCb * kCb; e += 1024) {
    const int r = e / kCb, c = e % kCb;
    if (c <= r) A[(o + r) * bp + o + c] = T[r][c];
    Linv[(int64_t)k * kCb * kCb + e] = I[r][c];
  }
}

// Tiles (i, k) below the diagonal: L_ik = A_ik L_kk^{-T} (1024 threads, 4 outputs each).
__global__ void __launch_bounds__(1024) k_chol_panel(float* __restrict__ A, int64_t bp, int k,
                                                     const float* __restrict__ Linv) {
  __shared__ float T[kCb][kCb + 1];
  __shared__ float Li[kCb][kCb + 1];
  const int64_t oi = (int64_t)(k + 1 + blockIdx.x) * kCb, ok = (int64_t)k * kCb;
  for (int e = threadIdx.x; e < kCb * kCb; e += 1024) {
    const int r = e / kCb, c = e % kCb;
    T[r][c] = A[(oi + r) * bp + ok + c];
    Li[r][c] = Linv[(int64_t)k * kCb * kCb + e];
  }
  __syncthreads();
  const int c = threadIdx.x % kCb, r0 = threadIdx.x / kCb;   // rows r0 + 16 t
  float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll 8
  for (int m = 0; m < kCb; ++m) {
    const float l = Li[c][m];
#pragma unroll
    for (int t = 0; t < 4; ++t) acc[t] = fmaf(T[r0 + 16 * t][m], l, acc[t]);
  }
#pragma unroll
  for (int t = 0; t < 4; ++t) A[(oi + r0 + 16 * t) * bp + ok + c] = acc[t];
}

// Trailing tiles I >= J > k: A_IJ -= L_Ik L_Jk^T (256 threads, a 4 x 4 register tile each).
__global__ void __launch_bounds__(256) k_chol_update(float* __restrict__ A, int64_t bp, int k, int nt) {
  const int J = k + 1 + blockIdx.x, I = k + 1 + blockIdx.y;
  if (J > I) return;
  __shared__ float P[kCb][kCb + 1];
  __shared__ float Q[kCb][kCb + 1];
  const int64_t oI = (int64_t)I * kCb, oJ = (int64_t)J * kCb, ok = (int64_t)k * kCb;
  for (int e = threadIdx.x; e < kCb * kCb; e += 256) {
    const int r = e / kCb, c = e % kCb;
    P[r][c] = A[(oI + r) * bp + ok + c];
    Q[r][c] = A[(oJ + r) * bp + ok + c];
  }
  __syncthreads();
  const int tc = threadIdx.x % 16, tr = threadIdx.x / 16;   // rows tr + 16 a, columns tc + 16 b
  float acc[4][4] = {};
#pragma unroll 4
  for (int m = 0; m < kCb; ++m) {
    float pv[4], qv[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      pv[t] = P[tr + 16 * t][m];
      qv[t] = Q[tc + 16 * t][m];
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(pv[a], qv[b], acc[a][b]);
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) A[(oI + tr + 16 * a) * bp + oJ + tc + 16 * b] -= acc[a][b];
}

// D (+)= (L L^T)^{-1} R by blocked substitution, one CTA of 1024 threads; R and
// D are bp x s (row stride s), Y is bp x s scratch.  Forward: warp w sums rows w
// and w + 32 of the block over the lanes (coalesced along a row of L); backward:
// lane l owns rows l and l + 32 of the block and warp p one slice of the rows
// below (coalesced along a row of L, which is a column of L^T).
__global__ void __launch_bounds__(1024) k_chol_solve(const float* __restrict__ L, int64_t bp,
                                                     const float* __restrict__ Linv, const float* __restrict__ R,
                                                     int s, float* __restrict__ Y, float* __restrict__ D, int add) {
  __shared__ float part[kCb][33];
  __shared__ float tmp[kCb];
  const int lane = threadIdx.x % 32, p = threadIdx.x / 32;
  const int nt = (int)(bp / kCb);
  for (int col = 0; col < s; ++col) {
    // forward: Y_K = Linv_K (R_K - sum_{J<K} L_KJ Y_J)
    for (int K = 0; K < nt; ++K) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int64_t wrow = (int64_t)K * kCb + p + 32 * h;
        float acc = 0.0f;
        for (int64_t m = lane; m < (int64_t)K * kCb; m += 32) acc = fmaf(L[wrow * bp + m], Y[m * s + col], acc);
        acc = warp_sum(acc);
        if (lane == 0) tmp[p + 32 * h] = R[wrow * s + col] - acc;
      }
      __syncthreads();
      if (threadIdx.x < kCb) {
        const int rr = threadIdx.x;
        float y = 0.0f;
        for (int m = 0; m < kCb; ++m) y = fmaf(Linv[(int64_t)K * kCb * kCb + rr * kCb + m], tmp[m], y);
        Y[((int64_t)K * kCb + rr) * s + col] = y;
      }
      __syncthreads();
    }
    // backward: X_K = Linv_K^T (Y_K - sum_{J>K} L_JK^T X_J), written into Y
    for (int K = nt - 1; K >= 0; --K) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int64_t row = (int64_t)K * kCb + lane + 32 * h;
        float acc = 0.0f;
        for (int64_t m = (int64_t)(K + 1) * kCb + p; m < bp; m += 32) acc = fmaf(L[m * bp + row], Y[m * s + col], acc);
        part[lane + 32 * h][p] = acc;
      }
      __syncthreads();
      if (threadIdx.x < kCb) {
        const int rr = threadIdx.x;
        const int64_t row = (int64_t)K * kCb + rr;
        float t = Y[row * s + col];
        for (int q = 0; q < 32; ++q) t -= part[rr][q];
        tmp[rr] = t;
      }
      __syncthreads();
      if (threadIdx.x < kCb) {
        const int rr = threadIdx.x;
        const int64_t row = (int64_t)K * kCb + rr;
        float x = 0.0f;
        for (int m = 0; m < kCb; ++m) x = fmaf(Linv[(int64_t)K * kCb * kCb + m * kCb + rr], tmp[m], x);
        Y[row * s + col] = x;
        D[row * s + col] = add ? D[row * s + col] + x : x;
      }
      __syncthreads();
    }
  }
}

// E = R - H D with FP64 sums (one warp per row of H).
__global__ void k_h_residual(const float* __restrict__ H, int64_t bp, const float* __restrict__ D,
                             const float* __restrict__ R, int s, float* __restrict__ E) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < bp; i += nw) {
    for (int c = 0; c < s; ++c) {
      double acc = 0.0;
      for (int64_t j = lane; j < bp; j += 32) acc += (double)H[i * bp + j] * (double)D[j * s + c];
      acc = warp_sum(acc);
      if (lane == 0) E[i * s + c] = (float)((double)R[i * s + c] - acc);
    }
  }
}

// W[B[i]] -= D[i] (Alg. 1 update; no acceleration, unit step)
__global__ void k_block_sub(float* __restrict__ W, const int* __restrict__ B, int64_t b, int s,
                            const float* __restrict__ D) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < b * s; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / s;
    const int c = (int)(e - i * s);
    W[(int64_t)B[i] * s + c] -= D[e];
  }
}

int64_t chol_pad(int64_t b) { return (b + kCb - 1) / kCb * kCb; }

cudaError_t launch_form_h(int kern, const float* xb, int64_t b, int dp, float sigma2, float lam, float* H,
                          cudaStream_t st) {
  const int64_t bp = chol_pad(b);
  const int blocks = (int)std::min<int64_t>((bp * bp + 255) / 256, 148 * 16);
  if (kern == ADASAP_RBF) k_form_h<ADASAP_RBF><<<blocks, 256, 0, st>>>(xb, b, bp, dp, sigma2, lam, H);
  else if (kern == ADASAP_MATERN32) k_form_h<ADASAP_MATERN32><<<blocks, 256, 0, st>>>(xb, b, bp, dp, sigma2, lam, H);
  else k_form_h<ADASAP_MATERN52><<<blocks, 256, 0, st>>>(xb, b, bp, dp, sigma2, lam, H);
  return cudaGetLastError();
}

int64_t chol_linv_floats(int64_t b) { return chol_pad(b) * kCb; }

cudaError_t launch_block_chol(float* A, int64_t b, float* Linv, DevScalars* sc, cudaStream_t st) {
  const int64_t bp = chol_pad(b);
  const int nt = (int)(bp / kCb);
  for (int k = 0; k < nt; ++k) {
    k_chol_diag<<<1, 1024, 0, st>>>(A, bp, k, Linv, sc);
    const int rest = nt - k - 1;
    if (rest > 0) {
      k_chol_panel<<<rest, 1024, 0, st>>>(A, bp, k, Linv);
      k_chol_update<<<dim3(rest, rest), 256, 0, st>>>(A, bp, k, nt);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_chol_solve(const float* L, int64_t b, const float* Linv, const float* R, int s, float* Y,
                              float* D, int add, cudaStream_t st) {
  k_chol_solve<<<1, 1024, 0, st>>>(L, chol_pad(b), Linv, R, s, Y, D, add);
  return cudaGetLastError();
}

cudaError_t launch_h_residual(const float* H, int64_t b, const float* D, const float* R, int s, float* E,
                              cudaStream_t st) {
  const int64_t bp = chol_pad(b);
  const int blocks = (int)std::min<int64_t>((bp * 32 + 255) / 256, 148 * 8);
  k_h_residual<<<blocks, 256, 0, st>>>(H, bp, D, R, s, E);
  return cudaGetLastError();
}

cudaError_t launch_block_sub(float* W, const int* B, int64_t b, int s, const float* D, cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>((b * s + 255) / 256, 148 * 8);
  k_block_sub<<<std::max(blocks, 1), 256, 0, st>>>(W, B, b, s, D);
  return cudaGetLastError();
}

}  // namespace adasap
