// Measured throughput of the arithmetic pipes that bound the block-row product
// (special-function unit for ex2 / rsqrt / sqrt, FP32 FMA), for the roofline the
// benchmark reports.  Each thread runs kProbeChains independent dependency
// chains so that latency is hidden and only issue throughput counts; the SM
// clock over the run is taken from clock64 against the global timer.
#include <algorithm>

#include "tc_ptx.cuh"

namespace adasap {
namespace {

constexpr int kProbeChains = 8;
constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSm = 4;

template <int OP>
__global__ void __launch_bounds__(kProbeThreads) k_pipe_probe(int iters, float* sink, long long* clk) {
  float x[kProbeChains];
#pragma unroll
  for (int i = 0; i < kProbeChains; ++i) x[i] = 0.25f + 0.01f * i + 1e-6f * threadIdx.x;
  long long c0 = 0, t0 = 0;
  if (threadIdx.x == 0) {
    c0 = clock64();
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kProbeChains; ++i) {
      if (OP == 0) x[i] = ex2_approx(-x[i]);            // stays in [0.5, 1]
      else if (OP == 1) x[i] = rsqrt_approx(x[i]);      // alternates a, a^-1/2: stays finite
      else if (OP == 3) x[i] = sqrt_approx(x[i]);       // tends to 1 from below: stays finite
      else x[i] = fmaf(x[i], 0.999f, 1e-4f);
    }
  }
  float acc = 0.0f;
#pragma unroll
  for (int i = 0; i < kProbeChains; ++i) acc += x[i];
  if (acc == 12345.0f) *sink = acc;  // keeps the chains live
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    long long t1;
    const long long c1 = clock64();
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
    clk[0] = c1 - c0;
    clk[1] = t1 - t0;
  }
}

}  // namespace

cudaError_t measure_pipes(double* out4, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))) return e;
  float* sink = nullptr;
  long long* clk = nullptr;
  if ((e = cudaMalloc(&sink, sizeof(float)))) return e;
  if ((e = cudaMalloc(&clk, 2 * sizeof(long long)))) {
    cudaFree(sink);
    return e;
  }
  cudaEvent_t a = nullptr, b = nullptr;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  const int blocks = sms * kProbeBlocksPerSm;
  const int iters = 2048;
  for (int op = 0; op < 4 && e == cudaSuccess; ++op) {
    auto launch = [&]() {
      if (op == 0) k_pipe_probe<0><<<blocks, kProbeThreads, 0, st>>>(iters, sink, clk);
      else if (op == 1) k_pipe_probe<1><<<blocks, kProbeThreads, 0, st>>>(iters, sink, clk);
      else if (op == 2) k_pipe_probe<2><<<blocks, kProbeThreads, 0, st>>>(iters, sink, clk);
      else k_pipe_probe<3><<<blocks, kProbeThreads, 0, st>>>(iters, sink, clk);
    };
    launch();  // warm-up
    cudaEventRecord(a, st);
    launch();
    cudaEventRecord(b, st);
    long long h[2] = {0, 0};
    if ((e = cudaMemcpyAsync(h, clk, sizeof(h), cudaMemcpyDeviceToHost, st)) ||
        (e = cudaStreamSynchronize(st)) || (e = cudaGetLastError()))
      break;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, a, b);
    const double ghz = h[1] > 0 ? (double)h[0] / (double)h[1] : 0.0;   // cycles per ns of block 0
    const double ops = (double)blocks * kProbeThreads * kProbeChains * (double)iters;
    // operations per SM per cycle, over the whole launch at the measured clock
    out4[op] = (ms > 0.0f && ghz > 0.0) ? ops / ((double)sms * (double)ms * 1e6 * ghz) : 0.0;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(sink);
  cudaFree(clk);
  return e;
}

// Element-by-element evaluation of the epilogues' device functions (self-test support).
__global__ void k_eval_math(int fn, const float* __restrict__ x, int64_t n, float* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = fn == 0 ? sqrt_fma(x[i]) : sqrt_approx(x[i]);
}

cudaError_t launch_eval_math(int fn, const float* x, int64_t n, float* out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 148 * 16);
  k_eval_math<<<blocks, 256, 0, st>>>(fn, x, n, out);
  return cudaGetLastError();
}

// The failure path of the bounded waits, exercised without a fault: one thread
// waits on an mbarrier that nothing ever arrives on, with the same bounded wait
// the tensor-core kernels use; when the limit runs out it records code kWaitSelfTestCode
// in the context's error flag (as a timed-out tensor-core kernel does) and returns.
__global__ void k_wait_selftest(uint64_t limit_ns, int* err) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(&bar, 0u, nullptr, limit_ns)) tc_note_timeout(err, kWaitSelfTestCode);
}

cudaError_t launch_wait_selftest(uint64_t limit_ns, int* err, cudaStream_t st) {
  k_wait_selftest<<<1, 32, 0, st>>>(limit_ns, err);
  return cudaGetLastError();
}

}  // namespace adasap
