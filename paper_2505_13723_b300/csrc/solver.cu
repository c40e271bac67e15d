// C-ABI entry points (include/adasap.h): context set-up, the block-row product,
// the ADASAP iteration (Alg. 2) captured once as a CUDA graph and replayed,
// the posterior mean, the hyperparameter adjoint and the device sampler.
//
// One iteration is a graph with one two-branch section:
//   sample B, Omega, v0 -> gather X_B -> thin QR of Omega -> sketch K_BB Omega
//   (Step II) -> Gram matrices of the sketch                 (whole GPU)
//   fork:  branch 1 (high-priority stream, kBranchSms SMs): the factorisations
//            of Alg. 4 and the Woodbury factor
//          branch 2 (persistent CTAs on the other SMs): block residual
//            K_Bn Z + lambda Z_B - Y_B (Step I)
//   join -> randomized powering (Alg. 5) -> eta -> direction P^{-1} R
//           (App. C.2) -> NesterovAcc (Alg. 6) -> t += 1     (whole GPU)
// The branches are independent given B and Omega, so the latency-bound
// factorisations (mostly single-CTA launches) run beside the throughput-bound
// Step I on SMs that Step I leaves free, instead of waiting for its CTAs to
// retire.  The powering steps are short whole-GPU bursts (b x b products and
// two-launch Woodbury applies) after the join.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "internal.cuh"

using namespace adasap;

namespace adasap {
cudaError_t core_init();
}

// A product y = K(rows, X') w dispatched to the tensor-core kernel (s = 1,
// split precision) or to the FP32 SIMT kernels.
struct RowsPlan {
  bool tc;     // tensor-core kernel: rows_tc.cu (s == 1) or rows_tc_mrhs.cu (s >= 2)
  bool mrhs;
  int passes;  // contraction MMAs of the multi-RHS kernel: 3 (split W and K) or 1 (TF32)
  int nsplit;
  int ctas;    // persistent CTAs of the tensor-core kernel (0: one per SM)
  int64_t wop_floats;  // W operand scratch: hi + lo of the multi-RHS kernel, or the tile-prepared w
};

// SMs left to the factorisation branch while Step I runs (its launches are
// mostly single-CTA; Step I's persistent CTAs occupy the other SMs throughout)
constexpr int kBranchSms = 4;

static thread_local std::string g_last_error;

static void note_error(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
}

#define CT(x)                      \
  do {                             \
    cudaError_t e_ = (x);          \
    if (e_ != cudaSuccess) {       \
      note_error(e_, #x);          \
      return ADASAP_ECUDA;         \
    }                              \
  } while (0)

struct adasap_ctx {
  int device = 0;
  int64_t n = 0;
  int d = 0, dp = 0, kern = 0;
  float ell = 1.f, sigma2 = 1.f, lambda = 1.f;
  double kappa = 1.0;
  float* Xc = nullptr;      // n x dp, x' = kappa (x - mean) / ell
  float* qc = nullptr;      // n, ||x'||^2
  double* mean_dev = nullptr;
  cudaStream_t s0 = nullptr, s1 = nullptr;
  cudaEvent_t ev_in = nullptr, ev_fork = nullptr, ev_join = nullptr, ev_out = nullptr, ev_omega = nullptr;
  cudaEvent_t ev_t0 = nullptr, ev_t1 = nullptr;
  DevScalars* sc = nullptr;
  DevScalars* sc_host = nullptr;  // pinned
  void* ws = nullptr;             // kernel_rows workspace
  size_t ws_bytes = 0;
  int prec = 0;                   // ADASAP_PREC_FP32, ADASAP_PREC_TF32X3 or ADASAP_PREC_TF32
  int kp = 0;                     // K of the tensor-core operands (0: unavailable)
  int64_t npad = 0;
  float* tc_hi = nullptr;         // split column operands of X' (npad x kp, MMA layout)
  float* tc_lo = nullptr;
  int* err_dev = nullptr;         // device error flag of the tensor-core kernel
};

namespace {

// Device allocations of one call, freed together.
struct Arena {
  std::vector<void*> ptrs;
  cudaError_t err = cudaSuccess;
  template <class T>
  T* get(size_t count) {
    if (count == 0) count = 1;
    void* p = nullptr;
    const cudaError_t e = cudaMalloc(&p, count * sizeof(T));
    if (e != cudaSuccess) {
      if (err == cudaSuccess) err = e;
      return nullptr;
    }
    ptrs.push_back(p);
    return static_cast<T*>(p);
  }
  ~Arena() {
    for (void* p : ptrs) cudaFree(p);
  }
};

bool is_device_ptr(const void* p) {
  cudaPointerAttributes attr;
  const cudaError_t e = cudaPointerGetAttributes(&attr, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

adasap_status order_after(cudaStream_t user, cudaEvent_t ev, cudaStream_t mine) {
  CT(cudaEventRecord(ev, user));
  CT(cudaStreamWaitEvent(mine, ev, 0));
  return ADASAP_OK;
}

}  // namespace

extern "C" {

void adasap_default_opts(adasap_opts* o, int64_t n) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->b = n >= 100 ? n / 100 : (n > 0 ? n : 1);
  o->r = (int)std::min<int64_t>(std::min<int64_t>(100, o->b), kMaxRank);
  o->max_iters = 1000;
  o->tol = 0.0;
  o->power_iters = 10;
  o->mu = 0.0;
  o->nu = 0.0;
  o->precond = 0;
  o->literal = 0;
  o->seed = 0;
  o->check_every = 10;
  o->check_rows = 65536;
  o->eps = 0.0;
  o->tail_average = 0;
}

const char* adasap_status_string(adasap_status s) {
  switch (s) {
    case ADASAP_OK: return "ok";
    case ADASAP_EINVAL: return "invalid argument";
    case ADASAP_ENOMEM: return "device allocation failed";
    case ADASAP_ECUDA: return "CUDA runtime error";
    case ADASAP_ENUMERIC: return "Cholesky of an r x r core failed";
    case ADASAP_EDIVERGED: return "residual diverged";
    case ADASAP_ETIMEOUT: return "bounded device wait timed out";
    case ADASAP_ENOTCONVERGED: return "tolerance not reached within max_iters";
  }
  return "unknown status";
}

const char* adasap_last_error(void) { return g_last_error.c_str(); }

adasap_status adasap_create(const float* X, int64_t n, int d, int kernel, float ell, float sigma2, float lambda,
                            void* stream, adasap_ctx** out) {
  if (!out || !X || n < 1 || n >= (1LL << 31) || d < 1 || d > kMaxDim || kernel < 0 || kernel > 2 ||
      !(ell > 0.f) || !(sigma2 > 0.f) || !(lambda > 0.f))
    return ADASAP_EINVAL;
  *out = nullptr;
  adasap_ctx* c = new (std::nothrow) adasap_ctx();
  if (!c) return ADASAP_ENOMEM;
  auto fail = [&](adasap_status s) {
    adasap_destroy(c);
    return s;
  };
  cudaStream_t us = (cudaStream_t)stream;
  if (cudaGetDevice(&c->device) != cudaSuccess) return fail(ADASAP_ECUDA);
  if (core_init() != cudaSuccess) { note_error(cudaGetLastError(), "core_init"); return fail(ADASAP_ECUDA); }
  if (tc_init() != cudaSuccess) { note_error(cudaGetLastError(), "tc_init"); return fail(ADASAP_ECUDA); }
  if (tc_mrhs_init() != cudaSuccess) { note_error(cudaGetLastError(), "tc_mrhs_init"); return fail(ADASAP_ECUDA); }
  if (rf_init() != cudaSuccess) { note_error(cudaGetLastError(), "rf_init"); return fail(ADASAP_ECUDA); }
  c->n = n;
  c->d = d;
  c->dp = padded_dim(d);
  c->kern = kernel;
  c->ell = ell;
  c->sigma2 = sigma2;
  c->lambda = lambda;
  c->kappa = kernel_kappa(kernel);
  int lo = 0, hi = 0;
  if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess) return fail(ADASAP_ECUDA);
  if (cudaStreamCreateWithPriority(&c->s0, cudaStreamNonBlocking, lo) != cudaSuccess) return fail(ADASAP_ECUDA);
  if (cudaStreamCreateWithPriority(&c->s1, cudaStreamNonBlocking, hi) != cudaSuccess) return fail(ADASAP_ECUDA);
  cudaEvent_t* evs[] = {&c->ev_in, &c->ev_fork, &c->ev_join, &c->ev_out, &c->ev_omega};
  for (cudaEvent_t* e : evs)
    if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) return fail(ADASAP_ECUDA);
  if (cudaEventCreate(&c->ev_t0) != cudaSuccess || cudaEventCreate(&c->ev_t1) != cudaSuccess)
    return fail(ADASAP_ECUDA);
  if (cudaMalloc(&c->Xc, (size_t)n * c->dp * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&c->qc, (size_t)n * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&c->mean_dev, (size_t)d * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&c->sc, sizeof(DevScalars)) != cudaSuccess ||
      cudaMallocHost(&c->sc_host, sizeof(DevScalars)) != cudaSuccess)
    return fail(ADASAP_ENOMEM);
  if (order_after(us, c->ev_in, c->s0) != ADASAP_OK) return fail(ADASAP_ECUDA);
  {
    Arena ar;
    const float* Xd = X;
    if (!is_device_ptr(X)) {
      float* tmp = ar.get<float>((size_t)n * d);
      if (!tmp) return fail(ADASAP_ENOMEM);
      if (cudaMemcpyAsync(tmp, X, (size_t)n * d * sizeof(float), cudaMemcpyHostToDevice, c->s0) != cudaSuccess)
        return fail(ADASAP_ECUDA);
      Xd = tmp;
    }
    double* parts = ar.get<double>((size_t)kColsumBlocks * d);
    if (!parts) return fail(ADASAP_ENOMEM);
    if (launch_colsum(Xd, n, d, parts, c->s0) != cudaSuccess) return fail(ADASAP_ECUDA);
    std::vector<double> hp((size_t)kColsumBlocks * d), mean(d, 0.0);
    if (cudaMemcpyAsync(hp.data(), parts, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, c->s0) != cudaSuccess ||
        cudaStreamSynchronize(c->s0) != cudaSuccess)
      return fail(ADASAP_ECUDA);
    for (int b = 0; b < kColsumBlocks; ++b)
      for (int k = 0; k < d; ++k) mean[k] += hp[(size_t)b * d + k];
    for (int k = 0; k < d; ++k) mean[k] /= (double)n;
    if (cudaMemcpyAsync(c->mean_dev, mean.data(), d * sizeof(double), cudaMemcpyHostToDevice, c->s0) != cudaSuccess)
      return fail(ADASAP_ECUDA);
    if (launch_transform(Xd, n, d, c->dp, c->mean_dev, c->kappa / (double)ell, c->Xc, c->qc, c->s0) != cudaSuccess)
      return fail(ADASAP_ECUDA);
    c->kp = tc_kp(d);
    if (cudaMalloc(&c->err_dev, sizeof(int)) != cudaSuccess ||
        cudaMemsetAsync(c->err_dev, 0, sizeof(int), c->s0) != cudaSuccess)
      return fail(ADASAP_ENOMEM);
    if (c->kp > 0) {
      c->npad = tc_npad(n);
      if (cudaMalloc(&c->tc_hi, (size_t)c->npad * c->kp * sizeof(float)) != cudaSuccess ||
          cudaMalloc(&c->tc_lo, (size_t)c->npad * c->kp * sizeof(float)) != cudaSuccess)
        return fail(ADASAP_ENOMEM);
      if (launch_build_tc(c->Xc, c->qc, nullptr, n, d, c->dp, c->tc_hi, c->tc_lo, c->s0) != cudaSuccess)
        return fail(ADASAP_ECUDA);
      c->prec = ADASAP_PREC_TF32X3;
    }
    if (cudaStreamSynchronize(c->s0) != cudaSuccess) return fail(ADASAP_ECUDA);
  }
  *out = c;
  return ADASAP_OK;
}

void adasap_destroy(adasap_ctx* c) {
  if (!c) return;
  if (c->s0) cudaStreamSynchronize(c->s0);
  if (c->s1) cudaStreamSynchronize(c->s1);
  cudaFree(c->Xc);
  cudaFree(c->qc);
  cudaFree(c->mean_dev);
  cudaFree(c->sc);
  cudaFree(c->ws);
  cudaFree(c->tc_hi);
  cudaFree(c->tc_lo);
  cudaFree(c->err_dev);
  if (c->sc_host) cudaFreeHost(c->sc_host);
  cudaEvent_t evs[] = {c->ev_in, c->ev_fork, c->ev_join, c->ev_out, c->ev_omega, c->ev_t0, c->ev_t1};
  for (cudaEvent_t e : evs)
    if (e) cudaEventDestroy(e);
  if (c->s0) cudaStreamDestroy(c->s0);
  if (c->s1) cudaStreamDestroy(c->s1);
  delete c;
}

}  // extern "C"

namespace {

RowsArgs rows_over_x(const adasap_ctx* c, const float* xr, const float* qr, const int* ridx, int64_t m,
                     const float* w, int64_t ldw, float* part) {
  RowsArgs a;
  a.xr = xr;
  a.qr = qr;
  a.ridx = ridx;
  a.m = m;
  a.xc = c->Xc;
  a.qc = c->qc;
  a.ncols = c->n;
  a.w = w;
  a.ldw = ldw;
  a.part = part;
  a.cps = 0;
  a.sigma2 = c->sigma2;
  return a;
}

adasap_status grow_ws(adasap_ctx* c, size_t bytes) {
  if (bytes <= c->ws_bytes) return ADASAP_OK;
  cudaFree(c->ws);
  c->ws = nullptr;
  c->ws_bytes = 0;
  if (cudaMalloc(&c->ws, bytes) != cudaSuccess) return ADASAP_ENOMEM;
  c->ws_bytes = bytes;
  return ADASAP_OK;
}

RowsPlan plan_rows(const adasap_ctx* c, int64_t m, int64_t ncols, int s, int reserve_sms = 0) {
  RowsPlan p;
  p.tc = c->prec != ADASAP_PREC_FP32 && c->kp > 0;
  p.passes = c->prec == ADASAP_PREC_TF32 ? 1 : 3;
  p.mrhs = p.tc && s > 1;
  p.ctas = (p.tc && reserve_sms > 0) ? std::max(1, tc_slots() - reserve_sms) : 0;
  p.nsplit = !p.tc ? rows_nsplit(m, ncols, s, c->dp, false)
                   : (p.mrhs ? tc_mrhs_nsplit(m, ncols, p.ctas) : tc_plan_nsplit(m, ncols, p.ctas));
  p.wop_floats = p.mrhs ? 2 * tc_mrhs_wfloats(ncols, s) : (p.tc ? tc_wprep_floats(ncols, c->kern) : 0);
  return p;
}

// y-partials of K(rows, X') W over all n columns of the context
// (wop: p.wop_floats of scratch for the multi-RHS kernel's W operand, required there; for the
// single-RHS tensor-core kernel the tile-prepared w, optional; w has row stride s)
cudaError_t run_rows_over_x(const adasap_ctx* c, const RowsPlan& p, const float* xr, const float* qr, const int* ridx,
                            int64_t m, const float* w, int s, float* part, int self_mode, cudaStream_t st,
                            float* wop = nullptr) {
  if (p.mrhs) {
    if (!wop) return cudaErrorInvalidValue;
    float* whi = wop;
    float* wlo = wop + p.wop_floats / 2;
    cudaError_t e = launch_build_w_tc(w, s, c->n, s, p.passes, whi, wlo, st);
    if (e != cudaSuccess) return e;
    return launch_rows_tc_mrhs(c->kern, c->d, xr, qr, ridx, m, c->dp, c->tc_hi, c->tc_lo, c->n, self_mode, whi, wlo,
                               s, p.passes, part, p.nsplit, c->sigma2, c->err_dev, st, p.ctas);
  }
  if (p.tc) {
    if (wop) {
      cudaError_t e = launch_prep_w(c->kern, w, s, c->n, wop, st);
      if (e != cudaSuccess) return e;
    }
    return launch_rows_tc(c->kern, c->d, xr, qr, ridx, m, c->dp, c->tc_hi, c->tc_lo, c->n, self_mode, w, s, part,
                          p.nsplit, c->sigma2, c->err_dev, st, p.ctas, wop);
  }
  return launch_rows(c->kern, c->dp, rows_over_x(c, xr, qr, ridx, m, w, s, part), s, p.nsplit, false, st);
}

}  // namespace

extern "C" adasap_status adasap_set_precision(adasap_ctx* c, int prec) {
  if (!c || (prec != ADASAP_PREC_FP32 && prec != ADASAP_PREC_TF32X3 && prec != ADASAP_PREC_TF32)) return ADASAP_EINVAL;
  if (prec != ADASAP_PREC_FP32 && c->kp == 0) return ADASAP_EINVAL;
  c->prec = prec;
  return ADASAP_OK;
}

extern "C" adasap_status adasap_kernel_rows(adasap_ctx* c, const int64_t* B, int64_t b, const float* W, int s,
                                            float* out, void* stream) {
  if (!c || !B || !W || !out || b < 1 || b >= (1LL << 31) || s < 1 || s > kMaxRhs) return ADASAP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const RowsPlan p = plan_rows(c, b, c->n, s);
  const size_t idx_bytes = ((size_t)b * sizeof(int) + 255) & ~(size_t)255;
  const size_t part_bytes = ((size_t)p.nsplit * b * s * sizeof(float) + 255) & ~(size_t)255;
  const size_t wop_bytes = (size_t)p.wop_floats * sizeof(float);
  const adasap_status g = grow_ws(c, idx_bytes + part_bytes + wop_bytes);
  if (g != ADASAP_OK) return g;
  int* idx = (int*)c->ws;
  float* part = (float*)((char*)c->ws + idx_bytes);
  float* wop = p.wop_floats > 0 ? (float*)((char*)c->ws + idx_bytes + part_bytes) : nullptr;
  CT(launch_index32(B, b, c->n, idx, st));
  CT(run_rows_over_x(c, p, c->Xc, c->qc, idx, b, W, s, part, 1, st, wop));
  CT(launch_reduce(part, p.nsplit, b, s, 0, s, out, s, 0.f, nullptr, nullptr, 0, 0.f, nullptr, nullptr, 0, nullptr,
                   st));
  return ADASAP_OK;
}

extern "C" adasap_status adasap_predict(adasap_ctx* c, const float* Xtest, int64_t m, const float* W, int s,
                                        float* out, void* stream) {
  if (!c || !Xtest || !W || !out || m < 1 || m >= (1LL << 31) || s < 1 || s > kMaxRhs) return ADASAP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  Arena ar;
  const RowsPlan p = plan_rows(c, m, c->n, s);
  float* xt = ar.get<float>((size_t)m * c->dp);
  float* qt = ar.get<float>((size_t)m);
  float* part = ar.get<float>((size_t)p.nsplit * m * s);
  float* wop = p.wop_floats > 0 ? ar.get<float>((size_t)p.wop_floats) : nullptr;
  if (ar.err != cudaSuccess) return ADASAP_ENOMEM;
  CT(launch_transform(Xtest, m, c->d, c->dp, c->mean_dev, c->kappa / (double)c->ell, xt, qt, st));
  CT(run_rows_over_x(c, p, xt, qt, nullptr, m, W, s, part, 0, st, wop));
  CT(launch_reduce(part, p.nsplit, m, s, 0, s, out, s, 0.f, nullptr, nullptr, 0, 0.f, nullptr, nullptr, 0, nullptr,
                   st));
  CT(cudaStreamSynchronize(st));  // the arena frees its buffers on return
  return ADASAP_OK;
}

extern "C" adasap_status adasap_residual(adasap_ctx* c, const float* Y, const float* W, int s, double* rel,
                                         void* stream) {
  if (!c || !Y || !W || !rel || s < 1 || s > kMaxRhs) return ADASAP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = c->n;
  const int64_t mb = std::min<int64_t>(n, (int64_t)1 << 16);  // rows per chunk
  const RowsPlan p = plan_rows(c, mb, n, s);
  Arena ar;
  const size_t ns_ = (size_t)n * s;
  const float* Yd = Y;
  const float* Wd = W;
  float* ycopy = nullptr;
  float* wcopy = nullptr;
  if (!is_device_ptr(Y)) Yd = ycopy = ar.get<float>(ns_);
  if (!is_device_ptr(W)) Wd = wcopy = ar.get<float>(ns_);
  int* idx = ar.get<int>((size_t)mb);
  float* part = ar.get<float>((size_t)p.nsplit * mb * s);
  float* res = ar.get<float>((size_t)mb * s);
  float* wop = p.wop_floats > 0 ? ar.get<float>((size_t)p.wop_floats) : nullptr;
  double* sq = ar.get<double>(kReduceBlocks);
  double* acc = ar.get<double>(2);
  if (ar.err != cudaSuccess) return ADASAP_ENOMEM;
  if (ycopy) CT(cudaMemcpyAsync(ycopy, Y, ns_ * sizeof(float), cudaMemcpyHostToDevice, st));
  if (wcopy) CT(cudaMemcpyAsync(wcopy, W, ns_ * sizeof(float), cudaMemcpyHostToDevice, st));
  // ||Y||^2 (the reduce writes a copy of Y into a scratch it does not need: chunk by chunk)
  CT(cudaMemsetAsync(acc, 0, 2 * sizeof(double), st));
  for (int64_t i0 = 0; i0 < n; i0 += mb) {
    const int64_t m = std::min(mb, n - i0);
    CT(launch_reduce(Yd + i0 * s, 1, m, s, 0, s, res, s, 0.f, nullptr, nullptr, 0, 0.f, nullptr, nullptr, 0, sq, st));
    CT(launch_sum_blocks_add(sq, kReduceBlocks, acc + 1, st));
  }
  // ||(K + lambda I) W - Y||^2 over row chunks, each a batched block-row product
  for (int64_t i0 = 0; i0 < n; i0 += mb) {
    const int64_t m = std::min(mb, n - i0);
    CT(launch_iota32(idx, i0, m, st));
    CT(run_rows_over_x(c, p, c->Xc, c->qc, idx, m, Wd, s, part, 1, st, wop));
    CT(launch_reduce(part, p.nsplit, m, s, 0, s, res, s, c->lambda, Wd, idx, s, -1.f, Yd, idx, s, sq, st));
    CT(launch_sum_blocks_add(sq, kReduceBlocks, acc, st));
  }
  double h[2];
  CT(cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, st));
  CT(cudaStreamSynchronize(st));
  *rel = h[1] > 0.0 ? std::sqrt(h[0] / h[1]) : NAN;
  return ADASAP_OK;
}

extern "C" adasap_status adasap_hypergrad(adasap_ctx* c, const float* W, const float* G, int s, double* d_ell,
                                          double* d_sigma2, void* stream) {
  if (!c || !W || !G || !d_ell || !d_sigma2 || s < 1 || s > kMaxRhs) return ADASAP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  Arena ar;
  // the partials of a 1-column group may use more splits than a 2-column group
  const size_t part_elems = std::max((size_t)rows_nsplit(c->n, c->n, 2, c->dp, true) * 4,
                                     (size_t)rows_nsplit(c->n, c->n, 1, c->dp, true) * 2) * (size_t)c->n;
  float* part = ar.get<float>(part_elems);
  double* acc = ar.get<double>(2 * kReduceBlocks);
  if (ar.err != cudaSuccess) return ADASAP_ENOMEM;
  CT(cudaMemsetAsync(acc, 0, 2 * kReduceBlocks * sizeof(double), st));
  for (int c0 = 0; c0 < s; c0 += 2) {
    const int g = std::min(2, s - c0);
    const int ns = rows_nsplit(c->n, c->n, g, c->dp, true);
    CT(launch_rows(c->kern, c->dp, rows_over_x(c, c->Xc, c->qc, nullptr, c->n, W + c0, s, part), g, ns, true, st));
    CT(launch_adj_reduce(part, ns, c->n, g, G, s, c0, acc, st));
  }
  std::vector<double> h(2 * kReduceBlocks);
  CT(cudaMemcpyAsync(h.data(), acc, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  CT(cudaStreamSynchronize(st));
  double sk = 0.0, sg = 0.0;
  for (int i = 0; i < kReduceBlocks; ++i) {
    sk += h[2 * i];
    sg += h[2 * i + 1];
  }
  *d_sigma2 = sk / (double)c->sigma2;
  *d_ell = sg / (double)c->ell;
  return ADASAP_OK;
}

extern "C" adasap_status adasap_measure_pipes(double* out, int count, void* stream) {
  if (!out || count < 1) return ADASAP_EINVAL;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  CT(measure_pipes(v, (cudaStream_t)stream));
  for (int i = 0; i < count && i < 4; ++i) out[i] = v[i];
  return ADASAP_OK;
}

extern "C" adasap_status adasap_eval_math(int fn, const float* x, int64_t n, float* out, void* stream) {
  if ((fn != 0 && fn != 1) || n < 0 || (n > 0 && (!x || !out))) return ADASAP_EINVAL;
  CT(launch_eval_math(fn, x, n, out, (cudaStream_t)stream));
  return ADASAP_OK;
}

extern "C" adasap_status adasap_sample(uint64_t seed, int64_t t, int64_t n, int64_t b, int r, int64_t* B,
                                       float* Omega, float* v0, void* stream) {
  if (n < 1 || n >= (1LL << 31) || b < 1 || b > n || r < 0 || t < 0 || t >= (1LL << 32)) return ADASAP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (B) CT(launch_sample_block(seed, nullptr, t, n, b, 1, nullptr, B, st));
  if (Omega && r > 0) CT(launch_normals(seed, nullptr, t, b * (int64_t)r, 2, (float)(1.0 / std::sqrt((double)b)), Omega, st));
  if (v0) CT(launch_normals(seed, nullptr, t, b, 3, 1.0f, v0, st));
  return ADASAP_OK;
}


// ---------------------------------------------------------------------------
// ADASAP solver handle: device state, the captured iteration graph, residuals.
// ---------------------------------------------------------------------------
struct adasap_solver {
  adasap_ctx* c = nullptr;
  int s = 1;
  adasap_opts o{};
  bool sched = false;
  bool identity = false;           // no Nystrom sketch (ADASAP-I, or the exact solve)
  bool exact = false;              // Alg. 1 with the exact block solve (Cholesky of K_BB + lambda I)
  float *Hf = nullptr, *Hc = nullptr, *Linv = nullptr;   // factor, copy of H, inverted diagonal tiles
  float *Rp = nullptr, *Dp = nullptr, *Yp = nullptr, *Ep = nullptr;  // padded b x s blocks
  int r = 0;
  int64_t b = 0, mc = 0;
  int ns1 = 1, ns_sk = 1, ns_pw = 1, ns_c = 1;
  RowsPlan plan1{}, plan_c{};
  bool tc_pw = false;              // K_BB v products on the tensor cores
  bool sk_tc = false;              // sketch K_BB Omega on the tensor cores (multi-RHS kernel)
  float* wop1 = nullptr;           // W operand scratch of Step I / the residual check (multi-RHS)
  float* wsk = nullptr;            // Omega operand of the sketch (hi + lo)
  bool use_prep = false;           // the inputs of an iteration come from k_head_prep (one launch)
  bool head_grouped = false;       // the batch runs this system's sketch, split sum and Grams grouped
  HeadPrepArgs prep{};
  HeadPrepArgs* prep_dev = nullptr;
  float *XBhi = nullptr, *XBlo = nullptr;
  double beta = 0, gamma = 0, alpha = 0, eps = 0;
  int literal = 0;
  int64_t iters = 0;
  Arena ar;
  float *Y = nullptr, *W = nullptr, *V = nullptr, *Z = nullptr;
  int* B32 = nullptr;
  float *Om = nullptr, *v0 = nullptr, *XB = nullptr, *qB = nullptr, *R = nullptr, *D = nullptr;
  float* OmN = nullptr;   // Omega of the next iteration, orthonormalised one iteration ahead
  float* Wbar = nullptr;  // running sum of the tail iterates (opts.tail_average)
  int64_t T_sched = 0;    // iterations of a caller-supplied schedule
  const float* Oms_sched = nullptr;
  float *part1 = nullptr, *part2 = nullptr, *Ysk = nullptr, *a = nullptr, *h = nullptr, *vA = nullptr, *vB = nullptr;
  int* Cidx = nullptr;
  float *Rc = nullptr, *cpart = nullptr;
  double* sqb = nullptr;
  CoreBufs cb{};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  ~adasap_solver() {
    if (c && c->s0) cudaStreamSynchronize(c->s0);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  }
};

namespace {

adasap_status alloc_solver(adasap_solver* S) {
  adasap_ctx* c = S->c;
  Arena& ar = S->ar;
  const int64_t n = c->n, b = S->b;
  const int s = S->s, r = S->r, rr = std::max(r, 1);
  const size_t ns_ = (size_t)n * s;
  S->Y = ar.get<float>(ns_);
  S->W = ar.get<float>(ns_);
  S->V = ar.get<float>(ns_);
  S->Z = ar.get<float>(ns_);
  S->B32 = ar.get<int>(b);
  S->Om = ar.get<float>((size_t)b * rr);
  S->OmN = ar.get<float>((size_t)b * rr);
  if (S->o.tail_average) S->Wbar = ar.get<float>(ns_);
  S->v0 = ar.get<float>(b);
  S->XB = ar.get<float>((size_t)b * c->dp);
  S->qB = ar.get<float>(b);
  S->R = ar.get<float>((size_t)b * s);
  S->D = ar.get<float>((size_t)b * s);
  S->part1 = ar.get<float>((size_t)S->ns1 * b * s);
  if (S->tc_pw) {
    S->XBhi = ar.get<float>((size_t)tc_npad(b) * c->kp);
    S->XBlo = ar.get<float>((size_t)tc_npad(b) * c->kp);
  }
  S->part2 = ar.get<float>(std::max((size_t)S->ns_sk * b * rr, (size_t)S->ns_pw * b));
  const int64_t wop = std::max(S->plan1.wop_floats, S->plan_c.wop_floats);
  if (wop > 0) S->wop1 = ar.get<float>((size_t)wop);
  if (S->sk_tc) S->wsk = ar.get<float>((size_t)2 * tc_mrhs_wfloats(b, r));
  if (S->exact) {
    const size_t bp = (size_t)chol_pad(b);
    S->Hf = ar.get<float>(bp * bp);
    S->Hc = ar.get<float>(bp * bp);
    S->Linv = ar.get<float>((size_t)chol_linv_floats(b));
    S->Rp = ar.get<float>(bp * s);
    S->Dp = ar.get<float>(bp * s);
    S->Yp = ar.get<float>(bp * s);
    S->Ep = ar.get<float>(bp * s);
    if (ar.err != cudaSuccess) return ADASAP_ENOMEM;
    for (float* z : {S->Rp, S->Dp, S->Yp, S->Ep})
      if (cudaMemset(z, 0, bp * s * sizeof(float)) != cudaSuccess) return ADASAP_ECUDA;
  }
  S->Ysk = ar.get<float>((size_t)b * rr);
  S->a = ar.get<float>(b);
  S->h = ar.get<float>(b);
  S->vA = ar.get<float>(b);
  S->vB = ar.get<float>(b);
  S->Cidx = ar.get<int>(S->mc);
  S->Rc = ar.get<float>((size_t)S->mc * s);
  S->cpart = ar.get<float>((size_t)S->ns_c * S->mc * s);
  S->sqb = ar.get<double>(kReduceBlocks);
  CoreBufs& cb = S->cb;
  cb.r = r;
  cb.s = s;
  cb.b = b;
  cb.gram_chunks = gram_chunks_for(b);
  cb.gram_part = ar.get<float2>((size_t)cb.gram_chunks * 4 * rr * rr);
  cb.G = ar.get<double>((size_t)4 * rr * rr);
  cb.Lc = ar.get<double>((size_t)rr * rr);
  cb.Gnu = ar.get<double>((size_t)rr * rr);
  cb.Gyy = ar.get<double>((size_t)rr * rr);
  cb.X1 = ar.get<double>((size_t)rr * rr);
  cb.A = ar.get<double>((size_t)rr * rr);
  cb.V32 = ar.get<float>((size_t)rr * rr);
  cb.lam = ar.get<double>(rr);
  cb.T = ar.get<double>((size_t)rr * rr);
  cb.T32 = ar.get<float>((size_t)rr * rr);
  cb.S = ar.get<double>(rr);
  cb.keep = ar.get<double>(rr);
  cb.Minv = ar.get<float>((size_t)rr * rr);
  cb.Gu = ar.get<float>((size_t)rr * rr);
  cb.U = ar.get<float>((size_t)b * rr);
  cb.utv_chunks = utv_chunks_for(b);
  cb.utv_part = ar.get<double>((size_t)cb.utv_chunks * rr * s);
  cb.coef = ar.get<float>((size_t)rr * s);
  cb.qk = ar.get<float>((size_t)rr * s);
  cb.sq_part = ar.get<double>(kReduceBlocks);
  cb.dot_part = ar.get<double>(kReduceBlocks);
  cb.alpha = ar.get<double>(2);
  cb.Ident = ar.get<double>((size_t)rr * rr);
  cb.cis = ar.get<double>(rr);
  cb.wb_part = ar.get<float>(wb_part_floats(b));
  cb.wb_coef = ar.get<float>(kMaxRank + 1);
  cb.wb_count = ar.get<unsigned int>(1);
  if (cb.wb_count && cudaMemset(cb.wb_count, 0, sizeof(unsigned int)) != cudaSuccess) return ADASAP_ECUDA;
  // sampled block, Nystrom sketch on the tensor cores: the inputs of an iteration in one launch
  if (!S->sched && !S->identity && S->sk_tc && S->XBhi && ar.err == cudaSuccess) {
    HeadPrepArgs& p = S->prep;
    p.seed = S->o.seed;
    p.t_dev = &c->sc->t;
    p.n = n;
    p.b = b;
    p.npad = tc_npad(b);
    p.h = feistel_half_width(n);
    p.d = c->d;
    p.dp = c->dp;
    p.r = r;
    p.sp = tc_mrhs_sp(r);
    p.Xc = c->Xc;
    p.qc = c->qc;
    p.B32 = S->B32;
    p.XB = S->XB;
    p.qB = S->qB;
    p.XBhi = S->XBhi;
    p.XBlo = S->XBlo;
    p.v0 = S->v0;
    p.OmN = S->OmN;
    p.Om = S->Om;
    p.whi = S->wsk;
    p.wlo = S->wsk + tc_mrhs_wfloats(b, r);
    S->prep_dev = ar.get<HeadPrepArgs>(1);
    if (S->prep_dev && cudaMemcpy(S->prep_dev, &p, sizeof(p), cudaMemcpyHostToDevice) != cudaSuccess)
      return ADASAP_ECUDA;
    S->use_prep = S->prep_dev != nullptr;
  }
  return ar.err == cudaSuccess ? ADASAP_OK : ADASAP_ENOMEM;
}

// K_BB-shaped product operands: rows and columns both the gathered block
RowsArgs block_args(adasap_solver* S) {
  RowsArgs kb;
  kb.xr = S->XB; kb.qr = S->qB; kb.ridx = nullptr; kb.m = S->b;
  kb.xc = S->XB; kb.qc = S->qB; kb.ncols = S->b;
  kb.part = S->part2; kb.cps = 0; kb.sigma2 = S->c->sigma2;
  kb.w = nullptr; kb.ldw = 1;
  return kb;
}

// Draw Omega of iteration t + offset (t = the device counter) into OmN and
// orthonormalise it (Alg. 2 Step II with reading R2: thin QR).
cudaError_t next_omega(adasap_solver* S, int offset, cudaStream_t st) {
  adasap_ctx* c = S->c;
  const int64_t b = S->b;
  const int r = S->r;
  const long long* tdev = &c->sc->t;
  cudaError_t e;
  if (S->sched) e = launch_copy_omega(S->Oms_sched, tdev, offset, S->T_sched, b, r, S->OmN, st);
  else e = launch_normals(S->o.seed, tdev, offset, b * (int64_t)r, 2, (float)(1.0 / std::sqrt((double)b)), S->OmN, st);
  if (e != cudaSuccess) return e;
  return launch_orthonormalize(S->cb, S->OmN, S->Ysk, c->sc, st);
}

// ---- one iteration, recorded in phases ---------------------------------------
// The phases end where a batch of independent systems meets for a grouped
// launch: before Step I and before each K_BB a product of Alg. 5.  Each phase
// records on the system's own streams (s0, forking to s1 and joining back).
#define KR(x)                              \
  do {                                     \
    const cudaError_t e_ = (x);            \
    if (e_ != cudaSuccess) return e_;      \
  } while (0)

// sample, gather, sketch and Gram matrices; fork the factorisation branch to s1
// (prep_done: the batch has already run this system's k_head_prep; head_done: and its
// sketch, split sum and Gram matrices, in grouped launches)
cudaError_t rec_head(adasap_solver* S, const int64_t* Bs, const float* v0s, bool prep_done = false,
                     bool head_done = false) {
  adasap_ctx* c = S->c;
  cudaStream_t s0 = c->s0, s1 = c->s1;
  const int64_t n = c->n, b = S->b;
  const int r = S->r;
  CoreBufs& cb = S->cb;
  const long long* tdev = &c->sc->t;
  // sample B, Omega, v0 (Alg. 2; Alg. 5)
  // (Omega_t was drawn and orthonormalised one iteration ahead, into OmN)
  if (S->use_prep) {
    // B, the gathered rows and their operands, v0, Omega_t and its operand: one launch
    if (!prep_done) KR(launch_head_prep(S->prep_dev, 1, c->kp, head_prep_work(S->prep), s0));
  } else {
    if (S->sched) {
      KR(launch_copy_schedule(Bs, nullptr, v0s, tdev, n, b, r, S->B32, S->Om, S->v0, c->sc, s0));
    } else {
      KR(launch_sample_block(S->o.seed, tdev, 0, n, b, 1, S->B32, nullptr, s0));
      KR(launch_normals(S->o.seed, tdev, 0, b, 3, 1.0f, S->v0, s0));
    }
    if (!S->identity) KR(cudaMemcpyAsync(S->Om, S->OmN, (size_t)b * r * sizeof(float), cudaMemcpyDeviceToDevice, s0));
    KR(launch_gather(c->Xc, c->qc, S->B32, b, c->dp, S->XB, S->qB, s0));
  }
  if (!S->identity && !head_done) {
    // whole-GPU part of Steps II-III: sketch K_BB Omega and its Gram matrices
    if (S->sk_tc) {
      const int64_t wf = tc_mrhs_wfloats(b, r);
      if (!S->use_prep) {
        KR(launch_build_tc(c->Xc, c->qc, S->B32, b, c->d, c->dp, S->XBhi, S->XBlo, s0));
        KR(launch_build_w_tc(S->Om, r, b, r, 3, S->wsk, S->wsk + wf, s0));
      }
      KR(launch_rows_tc_mrhs(c->kern, c->d, S->XB, S->qB, nullptr, b, c->dp, S->XBhi, S->XBlo, b, 1, S->wsk,
                             S->wsk + wf, r, 3, S->part2, S->ns_sk, c->sigma2, c->err_dev, s0));
    } else {
      RowsArgs kb = block_args(S);
      kb.w = S->Om;
      kb.ldw = r;
      KR(launch_rows(c->kern, c->dp, kb, r, S->ns_sk, false, s0));
    }
    KR(launch_reduce(S->part2, S->ns_sk, b, r, 0, r, S->Ysk, r, 0.f, nullptr, nullptr, 0, 0.f, nullptr, nullptr, 0,
                     nullptr, s0));
    KR(launch_nystrom_grams(cb, S->Om, S->Ysk, s0));
  }
  KR(cudaEventRecord(c->ev_fork, s0));
  KR(cudaStreamWaitEvent(s1, c->ev_fork, 0));
  // branch 1: the factorisations of Alg. 4 and the Woodbury factor (App. C.2)
  if (!S->identity) {
    KR(launch_nystrom_core(cb, S->eps, c->lambda, c->sc, S->Om, S->Ysk, s1));
    KR(launch_woodbury_factor(cb, c->lambda, c->sc, s1));
  }
  if (S->tc_pw && !S->sk_tc) KR(launch_build_tc(c->Xc, c->qc, S->B32, b, c->d, c->dp, S->XBhi, S->XBlo, s1));
  KR(cudaEventRecord(c->ev_join, s1));
  if (!S->identity) {
    // Omega of iteration t + 1 and its thin QR, beside the power loop and the
    // direction (the sketch buffer serves as scratch: the Nystrom core is done
    // with it); the update waits for it before the iteration counter moves
    KR(next_omega(S, 1, s1));
    KR(cudaEventRecord(c->ev_omega, s1));
  }
  return cudaSuccess;
}

// the point at which Step I takes the residual (reading R1)
float* step1_point(adasap_solver* S) { return S->literal ? S->W : S->Z; }

// branch 2: the Step I block product, concurrent with branch 1
cudaError_t rec_step1(adasap_solver* S) {
  adasap_ctx* c = S->c;
  return run_rows_over_x(c, S->plan1, c->Xc, c->qc, S->B32, S->b, step1_point(S), S->s, S->part1, 1, c->s0,
                         S->wop1);
}

// block residual R = K_Bn P + lambda P_B - Y_B from the Step I partials; join branch 1
cudaError_t rec_step1_finish(adasap_solver* S) {
  adasap_ctx* c = S->c;
  const int s = S->s;
  float* P = step1_point(S);
  KR(launch_reduce(S->part1, S->ns1, S->b, s, 0, s, S->R, s, (float)c->lambda, P, S->B32, s, -1.f, S->Y, S->B32, s,
                   nullptr, c->s0));
  return cudaStreamWaitEvent(c->s0, c->ev_join, 0);
}

// Alg. 5 with the Nystrom preconditioner, carried as a_i = P^{-1/2} v_i: one
// apply (two launches) per H product
float* power_buf(adasap_solver* S, int i) { return (i & 1) ? S->vB : S->vA; }

cudaError_t rec_power_init(adasap_solver* S) {
  return launch_wb_single(S->cb, kInvSqrtNormalised, S->v0, power_buf(S, 0), S->c->sc, S->c->s0);
}

cudaError_t rec_power_rows(adasap_solver* S, int i) {
  adasap_ctx* c = S->c;
  float* acur = power_buf(S, i);
  if (S->tc_pw)
    return launch_rows_tc(c->kern, c->d, S->XB, S->qB, nullptr, S->b, c->dp, S->XBhi, S->XBlo, S->b, 1, acur, 1,
                          S->part2, S->ns_pw, c->sigma2, c->err_dev, c->s0);
  RowsArgs kb = block_args(S);
  kb.w = acur;
  kb.ldw = 1;
  return launch_rows(c->kern, c->dp, kb, 1, S->ns_pw, false, c->s0);
}

cudaError_t rec_power_apply(adasap_solver* S, int i) {
  adasap_ctx* c = S->c;
  const bool last = i == S->o.power_iters - 1;
  return launch_power_step(S->cb, last ? kRayleighEta : kInvUnit, S->part2, S->ns_pw, (float)c->lambda,
                           power_buf(S, i), S->h, power_buf(S, i + 1), c->sc, c->s0);
}

// Alg. 5 with the identity preconditioner (ADASAP-I)
cudaError_t rec_power_identity(adasap_solver* S) {
  adasap_ctx* c = S->c;
  cudaStream_t s0 = c->s0;
  const int64_t b = S->b;
  CoreBufs& cb = S->cb;
  const float* vcur = S->v0;
  float* vbuf[2] = {S->vA, S->vB};
  RowsArgs kb = block_args(S);
  kb.ldw = 1;
  for (int i = 0; i < S->o.power_iters; ++i) {
    const bool last = i == S->o.power_iters - 1;
    float* vnext = vbuf[i & 1];
    KR(launch_reduce(vcur, 1, b, 1, 0, 1, S->h, 1, 0.f, nullptr, nullptr, 0, 0.f, nullptr, nullptr, 0, cb.sq_part,
                     s0));
    KR(launch_woodbury_apply(cb, kInvSqrtNormalised, S->h, 1, S->a, false, false, nullptr, c->sc, s0));
    kb.w = S->a;
    if (S->tc_pw)
      KR(launch_rows_tc(c->kern, c->d, S->XB, S->qB, nullptr, b, c->dp, S->XBhi, S->XBlo, b, 1, S->a, 1, S->part2,
                        S->ns_pw, c->sigma2, c->err_dev, s0));
    else
      KR(launch_rows(c->kern, c->dp, kb, 1, S->ns_pw, false, s0));
    KR(launch_reduce(S->part2, S->ns_pw, b, 1, 0, 1, S->h, 1, (float)c->lambda, S->a, nullptr, 1, 0.f, nullptr,
                     nullptr, 0, nullptr, s0));
    KR(launch_woodbury_apply(cb, kInvSqrt, S->h, 1, vnext, true, last, last ? vcur : nullptr, c->sc, s0));
    vcur = vnext;
  }
  return launch_set_eta(cb, c->sc, S->identity, s0);
}

// Step IV-a: direction D = P^{-1} R
cudaError_t rec_direction(adasap_solver* S) {
  adasap_ctx* c = S->c;
  if (!S->identity && S->s == 1) return launch_wb_single(S->cb, kInv, S->R, S->D, c->sc, c->s0);
  return launch_woodbury_apply(S->cb, kInv, S->R, S->s, S->D, false, false, nullptr, c->sc, c->s0);
}

// Step IV-b: NesterovAcc; t += 1
cudaError_t rec_update(adasap_solver* S, double* trace) {
  adasap_ctx* c = S->c;
  cudaStream_t s0 = c->s0;
  const int s = S->s;
  KR(launch_nesterov(S->W, S->V, S->Z, c->n * (int64_t)s, (float)S->beta, (float)S->alpha, S->literal, s0));
  KR(launch_scatter(S->W, S->V, S->Z, S->B32, S->b, s, S->D, (float)S->gamma, (float)S->alpha, S->literal, c->sc,
                    s0));
  if (trace) KR(launch_trace(c->sc, trace, s0));
  if (!S->identity) KR(cudaStreamWaitEvent(s0, c->ev_omega, 0));
  return launch_tick(c->sc, s0);
}

// One iteration of Alg. 1 (SAP) with the exact block solve: the factorisation of
// K_BB + lambda I (branch s1) beside the Step I product at W_t (s0), then the
// refined substitution and W_B -= D.
cudaError_t rec_iteration_exact(adasap_solver* S, const int64_t* Bs, const float* v0s, double* trace) {
  adasap_ctx* c = S->c;
  cudaStream_t s0 = c->s0, s1 = c->s1;
  const int64_t n = c->n, b = S->b;
  const int s = S->s;
  const long long* tdev = &c->sc->t;
  if (S->sched) KR(launch_copy_schedule(Bs, nullptr, v0s, tdev, n, b, 0, S->B32, nullptr, S->v0, c->sc, s0));
  else KR(launch_sample_block(S->o.seed, tdev, 0, n, b, 1, S->B32, nullptr, s0));
  KR(launch_gather(c->Xc, c->qc, S->B32, b, c->dp, S->XB, S->qB, s0));
  KR(cudaEventRecord(c->ev_fork, s0));
  KR(cudaStreamWaitEvent(s1, c->ev_fork, 0));
  const size_t bp = (size_t)chol_pad(b);
  KR(launch_form_h(c->kern, S->XB, b, c->dp, c->sigma2, c->lambda, S->Hf, s1));
  KR(cudaMemcpyAsync(S->Hc, S->Hf, bp * bp * sizeof(float), cudaMemcpyDeviceToDevice, s1));
  KR(launch_block_chol(S->Hf, b, S->Linv, c->sc, s1));
  KR(cudaEventRecord(c->ev_join, s1));
  KR(run_rows_over_x(c, S->plan1, c->Xc, c->qc, S->B32, b, S->W, s, S->part1, 1, s0, S->wop1));
  KR(launch_reduce(S->part1, S->ns1, b, s, 0, s, S->Rp, s, (float)c->lambda, S->W, S->B32, s, -1.f, S->Y, S->B32, s,
                   nullptr, s0));
  KR(cudaStreamWaitEvent(s0, c->ev_join, 0));
  KR(launch_chol_solve(S->Hf, b, S->Linv, S->Rp, s, S->Yp, S->Dp, 0, s0));
  for (int k = 0; k < 2; ++k) {
    KR(launch_h_residual(S->Hc, b, S->Dp, S->Rp, s, S->Ep, s0));
    KR(launch_chol_solve(S->Hf, b, S->Linv, S->Ep, s, S->Yp, S->Dp, 1, s0));
  }
  KR(launch_block_sub(S->W, S->B32, b, s, S->Dp, s0));
  if (trace) KR(launch_trace(c->sc, trace, s0));
  return launch_tick(c->sc, s0);
}

// the whole iteration of one system
cudaError_t rec_iteration(adasap_solver* S, const int64_t* Bs, const float* v0s, double* trace) {
  if (S->exact) return rec_iteration_exact(S, Bs, v0s, trace);
  KR(rec_head(S, Bs, v0s));
  KR(rec_step1(S));
  KR(rec_step1_finish(S));
  // Alg. 5 after the join, on the whole GPU: v <- P^{-1/2} H P^{-1/2} v / ||v||, N times
  if (S->identity) {
    KR(rec_power_identity(S));
  } else {
    KR(rec_power_init(S));
    for (int i = 0; i < S->o.power_iters; ++i) {
      KR(rec_power_rows(S, i));
      KR(rec_power_apply(S, i));
    }
  }
  KR(rec_direction(S));
  return rec_update(S, trace);
}

// Record one ADASAP iteration on s0 (forking to s1) into S->graph.
cudaError_t capture_iteration(adasap_solver* S, const int64_t* Bs, const float* v0s, double* trace) {
  cudaStream_t s0 = S->c->s0;
  cudaError_t e = cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  const cudaError_t ce = rec_iteration(S, Bs, v0s, trace);
  e = cudaStreamEndCapture(s0, &S->graph);
  if (ce != cudaSuccess) return ce;
  if (e != cudaSuccess) return e;
  return cudaGraphInstantiateWithFlags(&S->exec, S->graph, cudaGraphInstantiateFlagUseNodePriority);
}

// Allocate the solver state, copy Y and W0, and draw the first Omega; the
// iteration graph is captured by the caller (one system, or a batch).
adasap_status solver_prepare(adasap_ctx* c, const float* Y, int s, const adasap_opts* o, const int64_t* Bs,
                             const float* Oms, const float* v0s, const float* W0, cudaStream_t us,
                             adasap_solver** out, int64_t T_sched, int reserve_sms, int share = 1) {
  if (!c || !Y || !o || !out || s < 1 || s > kMaxRhs) return ADASAP_EINVAL;
  *out = nullptr;
  const int64_t n = c->n, b = o->b;
  const bool exact = o->precond == 2;            // Alg. 1 (SAP): exact block solve
  const bool identity = o->precond == 1 || exact;  // no Nystrom sketch
  const int r = identity ? 0 : o->r;
  if (b < 1 || b > n || o->power_iters < 1 || o->precond < 0 || o->precond > 2) return ADASAP_EINVAL;
  if (exact && b > kMaxExactBlock) return ADASAP_EINVAL;
  if (!identity && (r < 1 || r > kMaxRank || r > b)) return ADASAP_EINVAL;
  if (Bs && (!v0s || (!identity && !Oms))) return ADASAP_EINVAL;
  adasap_solver* S = new (std::nothrow) adasap_solver();
  if (!S) return ADASAP_ENOMEM;
  S->c = c;
  S->s = s;
  S->o = *o;
  S->sched = Bs != nullptr;
  S->T_sched = T_sched;
  S->Oms_sched = Oms;
  S->identity = identity;
  S->exact = exact;
  S->r = r;
  S->b = b;
  const double lam = c->lambda;
  const double mu = o->mu > 0 ? o->mu : lam;
  const double nu = o->nu > 0 ? o->nu : (double)n / (double)b;
  S->beta = 1.0 - std::sqrt(mu / nu);
  S->gamma = 1.0 / std::sqrt(mu * nu);
  S->alpha = 1.0 / (1.0 + S->gamma * nu);
  S->eps = o->eps > 0 ? o->eps : std::ldexp(1.0, -23);
  S->literal = o->literal ? 1 : 0;
  S->mc = std::min<int64_t>(n, std::max<int64_t>(1, o->check_rows));
  S->plan1 = plan_rows(c, b, n, s, reserve_sms);
  S->plan_c = plan_rows(c, S->mc, n, s);
  S->tc_pw = c->prec != ADASAP_PREC_FP32 && c->kp > 0;
  S->ns1 = S->plan1.nsplit;
  S->sk_tc = S->tc_pw && !identity && r >= 2;
  // the sketch's column splits are planned for the SMs this system has: all of them
  // alone, its share of them when `share` systems run their heads at the same time
  // (one-tile items on every SM for each of 48 systems spread the sketches of a
  // batch over 0.3 ms)
  const int sk_ctas = share > 1 ? std::max(1, tc_slots() / share) : 0;
  S->ns_sk = identity ? 1 : (S->sk_tc ? tc_mrhs_nsplit(b, b, sk_ctas) : rows_nsplit(b, b, r, c->dp, false));
  S->ns_pw = S->tc_pw ? tc_plan_nsplit(b, b) : rows_nsplit(b, b, 1, c->dp, false);
  S->ns_c = S->plan_c.nsplit;
  adasap_status st = alloc_solver(S);
  if (st != ADASAP_OK) { delete S; return st; }
  auto fail = [&](cudaError_t e, const char* what) {
    note_error(e, what);
    delete S;
    return ADASAP_ECUDA;
  };
  cudaError_t e;
  const size_t bytes = (size_t)n * s * sizeof(float);
  if ((e = cudaEventRecord(c->ev_in, us)) || (e = cudaStreamWaitEvent(c->s0, c->ev_in, 0))) return fail(e, "order");
  if ((e = cudaMemcpyAsync(S->Y, Y, bytes, cudaMemcpyDefault, c->s0))) return fail(e, "copy Y");
  if (W0) e = cudaMemcpyAsync(S->W, W0, bytes, cudaMemcpyDefault, c->s0);
  else e = cudaMemsetAsync(S->W, 0, bytes, c->s0);
  if (e) return fail(e, "copy W0");
  if ((e = cudaMemsetAsync(c->sc, 0, sizeof(DevScalars), c->s0))) return fail(e, "memset");
  {
    const int rr = std::max(S->r, 1);
    std::vector<double> eye((size_t)rr * rr, 0.0);
    for (int i = 0; i < rr; ++i) eye[(size_t)i * rr + i] = 1.0;
    if ((e = cudaMemcpy(S->cb.Ident, eye.data(), eye.size() * sizeof(double), cudaMemcpyHostToDevice)))
      return fail(e, "identity");
  }
  // ||Y||_F^2 (the reduce copies Y into V, overwritten just below)
  if ((e = launch_reduce(S->Y, 1, n, s, 0, s, S->V, s, 0.f, nullptr, nullptr, 0, 0.f, nullptr, nullptr, 0, S->sqb,
                         c->s0)))
    return fail(e, "ysq");
  if ((e = launch_sum_blocks(S->sqb, kReduceBlocks, &c->sc->ysq, c->s0))) return fail(e, "ysq");
  if ((e = cudaMemcpyAsync(S->V, S->W, bytes, cudaMemcpyDeviceToDevice, c->s0))) return fail(e, "V0");
  if ((e = cudaMemcpyAsync(S->Z, S->W, bytes, cudaMemcpyDeviceToDevice, c->s0))) return fail(e, "Z0");
  // Omega of the first iteration (each iteration then prepares the next one's)
  if (!S->identity && !(S->sched && S->T_sched == 0) && (e = next_omega(S, 0, c->s0))) return fail(e, "first Omega");
  if ((e = cudaStreamSynchronize(c->s0))) return fail(e, "sync");
  *out = S;
  return ADASAP_OK;
}

adasap_status solver_begin(adasap_ctx* c, const float* Y, int s, const adasap_opts* o, const int64_t* Bs,
                           const float* Oms, const float* v0s, const float* W0, double* trace, cudaStream_t us,
                           adasap_solver** out, int64_t T_sched = 0) {
  adasap_status st = solver_prepare(c, Y, s, o, Bs, Oms, v0s, W0, us, out, T_sched, kBranchSms);
  if (st != ADASAP_OK) return st;
  const cudaError_t e = capture_iteration(*out, Bs, v0s, trace);
  if (e != cudaSuccess) {
    note_error(e, "graph capture");
    delete *out;
    *out = nullptr;
    return ADASAP_ECUDA;
  }
  return ADASAP_OK;
}

adasap_status solver_residual(adasap_solver* S, double* rel, cudaStream_t us) {
  adasap_ctx* c = S->c;
  const int s = S->s;
  const int64_t mc = S->mc;
  CT(cudaEventRecord(c->ev_in, us));
  CT(cudaStreamWaitEvent(c->s0, c->ev_in, 0));
  const int* cidx = nullptr;
  if (mc < c->n) {
    CT(launch_sample_block(S->o.seed, nullptr, S->iters, c->n, mc, 4, S->Cidx, nullptr, c->s0));
    cidx = S->Cidx;
  }
  CT(run_rows_over_x(c, S->plan_c, c->Xc, c->qc, cidx, mc, S->W, s, S->cpart, 1, c->s0, S->wop1));
  CT(launch_reduce(S->cpart, S->ns_c, mc, s, 0, s, S->Rc, s, c->lambda, S->W, cidx, s, -1.f, S->Y, cidx, s, S->sqb,
                   c->s0));
  CT(launch_sum_blocks(S->sqb, kReduceBlocks, &c->sc->resid_sq, c->s0));
  CT(cudaMemcpyAsync(c->sc_host, c->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->s0));
  int tc_err = 0;
  CT(cudaMemcpyAsync(&tc_err, c->err_dev, sizeof(int), cudaMemcpyDeviceToHost, c->s0));
  CT(cudaStreamSynchronize(c->s0));
  const DevScalars& hs = *c->sc_host;
  *rel = std::sqrt(hs.resid_sq * ((double)c->n / (double)mc) / hs.ysq);
  if (hs.status != 0) return (adasap_status)hs.status;
  if (tc_err != 0) return ADASAP_ETIMEOUT;   // a tensor-core kernel gave up a wait (its outputs are NaN)
  if (!std::isfinite(*rel) || *rel > 1e8) return ADASAP_EDIVERGED;
  return ADASAP_OK;
}

}  // namespace

extern "C" adasap_status adasap_solver_begin(adasap_ctx* c, const float* Y, int s, const adasap_opts* o,
                                             const float* W0, void* stream, adasap_solver** out) {
  try {
    return solver_begin(c, Y, s, o, nullptr, nullptr, nullptr, W0, nullptr, (cudaStream_t)stream, out);
  } catch (...) {
    return ADASAP_ENOMEM;
  }
}

extern "C" adasap_status adasap_solver_step(adasap_solver* S, int iters, void* stream) {
  if (!S || iters < 0) return ADASAP_EINVAL;
  for (int i = 0; i < iters; ++i) CT(cudaGraphLaunch(S->exec, (cudaStream_t)stream));
  S->iters += iters;
  return ADASAP_OK;
}

extern "C" adasap_status adasap_solver_residual(adasap_solver* S, double* rel, void* stream) {
  if (!S || !rel) return ADASAP_EINVAL;
  return solver_residual(S, rel, (cudaStream_t)stream);
}

extern "C" adasap_status adasap_solver_get_w(adasap_solver* S, float* W, void* stream) {
  if (!S || !W) return ADASAP_EINVAL;
  CT(cudaMemcpyAsync(W, S->W, (size_t)S->c->n * S->s * sizeof(float), cudaMemcpyDefault, (cudaStream_t)stream));
  return ADASAP_OK;
}

// Checkpoint and resume: (W, V, Z) and the iteration counter t are the whole
// state of Alg. 2 between iterations (the draws of iteration t depend only on the
// seed and t).
extern "C" adasap_status adasap_solver_get_state(adasap_solver* S, float* W, float* V, float* Z, int64_t* t,
                                                 void* stream) {
  if (!S || !W || !V || !Z || !t) return ADASAP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = (size_t)S->c->n * S->s * sizeof(float);
  long long tc = 0;
  CT(cudaMemcpyAsync(W, S->W, bytes, cudaMemcpyDefault, st));
  CT(cudaMemcpyAsync(V, S->V, bytes, cudaMemcpyDefault, st));
  CT(cudaMemcpyAsync(Z, S->Z, bytes, cudaMemcpyDefault, st));
  CT(cudaMemcpyAsync(&tc, &S->c->sc->t, sizeof(long long), cudaMemcpyDeviceToHost, st));
  CT(cudaStreamSynchronize(st));
  *t = (int64_t)tc;
  return ADASAP_OK;
}

extern "C" adasap_status adasap_solver_set_state(adasap_solver* S, const float* W, const float* V, const float* Z,
                                                 int64_t t, void* stream) {
  if (!S || !W || !V || !Z || t < 0 || t >= (1LL << 32) || (S->sched && t > S->T_sched)) return ADASAP_EINVAL;
  adasap_ctx* c = S->c;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = (size_t)c->n * S->s * sizeof(float);
  const long long tc = (long long)t;
  CT(cudaEventRecord(c->ev_in, st));
  CT(cudaStreamWaitEvent(c->s0, c->ev_in, 0));
  CT(cudaMemcpyAsync(S->W, W, bytes, cudaMemcpyDefault, c->s0));
  CT(cudaMemcpyAsync(S->V, V, bytes, cudaMemcpyDefault, c->s0));
  CT(cudaMemcpyAsync(S->Z, Z, bytes, cudaMemcpyDefault, c->s0));
  CT(cudaMemcpyAsync(&c->sc->t, &tc, sizeof(long long), cudaMemcpyHostToDevice, c->s0));
  // Omega of iteration t (each iteration then prepares the next one's)
  if (!S->identity && !(S->sched && t == S->T_sched)) CT(next_omega(S, 0, c->s0));
  CT(cudaStreamSynchronize(c->s0));
  S->iters = t;
  return ADASAP_OK;
}

extern "C" adasap_status adasap_solver_scalars(adasap_solver* S, double* eta, double* rho, int* status,
                                               void* stream) {
  if (!S) return ADASAP_EINVAL;
  adasap_ctx* c = S->c;
  CT(cudaEventRecord(c->ev_in, (cudaStream_t)stream));
  CT(cudaStreamWaitEvent(c->s0, c->ev_in, 0));
  CT(cudaMemcpyAsync(c->sc_host, c->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->s0));
  CT(cudaStreamSynchronize(c->s0));
  if (eta) *eta = c->sc_host->eta;
  if (rho) *rho = c->sc_host->rho;
  if (status) *status = c->sc_host->status;
  return ADASAP_OK;
}

extern "C" void adasap_solver_end(adasap_solver* S) { delete S; }

namespace {

adasap_status solve_loop(adasap_solver* S, float* W, adasap_stats* stats, int T_run, cudaStream_t us) {
  adasap_ctx* c = S->c;
  const adasap_opts& o = S->o;
  adasap_status st = ADASAP_OK;
  double rel = NAN;
  bool converged = false, checked_last = false;
  int it = 0;
  const size_t wbytes = (size_t)c->n * S->s * sizeof(float);
  const int64_t wcount = c->n * (int64_t)S->s;
  CT(cudaEventRecord(c->ev_t0, c->s0));
  if (o.tail_average) {
    // Alg. 1 / 2 tail averaging over exactly T_run iterations: mean(W_j, j = ceil(T/2) .. T)
    const int j0 = (T_run + 1) / 2;
    if (j0 == 0) CT(cudaMemcpyAsync(S->Wbar, S->W, wbytes, cudaMemcpyDeviceToDevice, c->s0));
    else CT(cudaMemsetAsync(S->Wbar, 0, wbytes, c->s0));
    for (it = 1; it <= T_run; ++it) {
      CT(cudaGraphLaunch(S->exec, c->s0));
      if (it >= j0) CT(launch_tail_add(S->W, S->Wbar, wcount, c->s0));
    }
    it = T_run;
    S->iters = it;
    CT(launch_tail_finish(S->Wbar, S->W, wcount, 1.0f / (float)(T_run - j0 + 1), c->s0));
  }
  while (!o.tail_average && it < T_run) {
    int k = T_run - it;
    if (!S->sched && o.check_every > 0) k = std::min(k, o.check_every - (it % o.check_every));
    for (int i = 0; i < k; ++i) CT(cudaGraphLaunch(S->exec, c->s0));
    it += k;
    S->iters = it;
    checked_last = false;
    if (!S->sched && o.check_every > 0 && it % o.check_every == 0) {
      st = solver_residual(S, &rel, c->s0);
      checked_last = true;
      if (st != ADASAP_OK) break;
      if (o.tol > 0 && rel <= o.tol) {
        converged = true;
        break;
      }
    }
  }
  CT(cudaEventRecord(c->ev_t1, c->s0));
  CT(cudaStreamSynchronize(c->s0));
  float ms = 0.f;
  CT(cudaEventElapsedTime(&ms, c->ev_t0, c->ev_t1));
  if (st == ADASAP_OK && !checked_last && !S->sched) {  // (with tail averaging: on the average)
    st = solver_residual(S, &rel, c->s0);
    if (st == ADASAP_OK && o.tol > 0 && rel <= o.tol) converged = true;
  }
  CT(cudaMemcpyAsync(c->sc_host, c->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->s0));
  CT(cudaMemcpyAsync(W, S->W, wbytes, cudaMemcpyDefault, c->s0));
  CT(cudaStreamSynchronize(c->s0));
  if (st == ADASAP_OK && c->sc_host->status != 0) st = (adasap_status)c->sc_host->status;
  if (stats) {
    stats->iters = it;
    stats->rel_resid = rel;
    stats->resid_exact = S->mc == c->n ? 1 : 0;
    stats->seconds = ms * 1e-3;
    stats->last_eta = c->sc_host->eta;
    stats->last_rho = c->sc_host->rho;
    stats->status_detail = c->sc_host->detail;
  }
  if (st == ADASAP_OK && !S->sched && !o.tail_average && o.tol > 0 && !converged) st = ADASAP_ENOTCONVERGED;
  CT(cudaEventRecord(c->ev_out, c->s0));
  CT(cudaStreamWaitEvent(us, c->ev_out, 0));
  return st;
}

}  // namespace

extern "C" adasap_status adasap_solve(adasap_ctx* c, const float* Y, int s, const adasap_opts* o, float* W,
                                      adasap_stats* stats, void* stream) {
  if (!W || !o || o->max_iters < 0) return ADASAP_EINVAL;
  try {
    adasap_solver* S = nullptr;
    adasap_status st = solver_begin(c, Y, s, o, nullptr, nullptr, nullptr, W, nullptr, (cudaStream_t)stream, &S);
    if (st != ADASAP_OK) return st;
    st = solve_loop(S, W, stats, o->max_iters, (cudaStream_t)stream);
    delete S;
    return st;
  } catch (...) {
    return ADASAP_ENOMEM;
  }
}

extern "C" adasap_status adasap_solve_scheduled(adasap_ctx* c, const float* Y, int s, const adasap_opts* o,
                                                const int64_t* B_sched, const float* Omega_sched,
                                                const float* v0_sched, int T, float* W, double* trace,
                                                adasap_stats* stats, void* stream) {
  if (!B_sched || !W || !o || T < 0) return ADASAP_EINVAL;
  try {
    adasap_solver* S = nullptr;
    adasap_status st =
        solver_begin(c, Y, s, o, B_sched, Omega_sched, v0_sched, W, trace, (cudaStream_t)stream, &S, T);
    if (st != ADASAP_OK) return st;
    st = solve_loop(S, W, stats, T, (cudaStream_t)stream);
    delete S;
    return st;
  } catch (...) {
    return ADASAP_ENOMEM;
  }
}

// ---------------------------------------------------------------------------
// Many independent systems (uneven n) iterated together: adasap_solve_batched.
// One graph holds one iteration of every active system, each on its own
// streams; the Step I products and the K_BB a products of Alg. 5 of all
// systems that share a kernel and operand width run as one grouped persistent
// tensor-core launch each, whose column split the batch autotunes.
// ---------------------------------------------------------------------------
namespace {

struct GroupedProduct {
  int kern = 0, kp = 0;
  std::vector<int> members;      // indices into Batch::S
  TcArgs* grp = nullptr;         // device, one per member
  int64_t* gstart = nullptr;     // device, prefix sums of the members' items
  int64_t nitems = 0;
  unsigned long long* sched = nullptr;   // device, the launch's item counters (zero between launches)
};

struct Batch {
  std::vector<adasap_solver*> S;
  std::vector<char> active, grouped;
  std::vector<int> ns1_max, nspw_max;   // split capacity of each system's partial buffers
  cudaStream_t ms = nullptr;
  cudaEvent_t ev = nullptr, ev_t0 = nullptr, ev_t1 = nullptr;
  int tpi1 = 32, tpipw = 4;             // column tiles per item of the grouped launches
  int ctas = 0;
  std::vector<GroupedProduct> step1, pw[2];
  // grouped Woodbury applies of the grouped systems: powering start, powering
  // steps on buffer 0 / 1, the last (Rayleigh) step, the direction
  WbArgs* wb[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  int* wb_start = nullptr;   // device prefix sums of the grouped systems' chunk counts
  int nwb = 0, wb_blocks = 0;
  // grouped k_head_prep of the active systems that take it, one table per
  // operand width (tc_kp 16, 32)
  HeadPrepArgs* prep[2] = {nullptr, nullptr};
  int nprep[2] = {0, 0};
  int64_t prep_work[2] = {0, 0};
  // the rest of the head of those systems, grouped: the sketches K_BB Omega (one
  // persistent launch per kernel, operand width and shared-memory plan), their split
  // sums and the two Gram matrices of Alg. 4's core
  struct SketchGroup {
    int kern = 0, kp = 0, n = 0;
    int64_t key = 0, nitems = 0;
    std::vector<unsigned char> first;   // host copy of the first argument block
    void* tab = nullptr;                // device argument blocks
    int64_t* gstart = nullptr;          // device prefix sums of the items
  };
  std::vector<SketchGroup> sk;
  SplitSumArgs* ssum = nullptr;
  GramArgs* gram[2] = {nullptr, nullptr};
  int nhead = 0, gram_chunks[2] = {0, 0}, gram_active[2] = {0, 0}, gram_c[2] = {0, 0};
  int64_t ssum_elems = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  void free_groups() {
    for (auto* v : {&step1, &pw[0], &pw[1]}) {
      for (GroupedProduct& g : *v) {
        cudaFree(g.grp);
        cudaFree(g.gstart);
        cudaFree(g.sched);
      }
      v->clear();
    }
    for (WbArgs*& w : wb) {
      cudaFree(w);
      w = nullptr;
    }
    cudaFree(wb_start);
    wb_start = nullptr;
    nwb = 0;
    for (int k = 0; k < 2; ++k) {
      cudaFree(prep[k]);
      prep[k] = nullptr;
      nprep[k] = 0;
      prep_work[k] = 0;
    }
    for (SketchGroup& g : sk) {
      cudaFree(g.tab);
      cudaFree(g.gstart);
    }
    sk.clear();
    cudaFree(ssum);
    ssum = nullptr;
    for (GramArgs*& g : gram) {
      cudaFree(g);
      g = nullptr;
    }
    nhead = 0;
    ssum_elems = 0;
    for (adasap_solver* x : S)
      if (x) x->head_grouped = false;
  }
  void free_graph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
  }
  ~Batch() {
    if (ms) cudaStreamSynchronize(ms);
    free_graph();
    free_groups();
    for (adasap_solver* x : S) delete x;
    if (ev) cudaEventDestroy(ev);
    if (ev_t0) cudaEventDestroy(ev_t0);
    if (ev_t1) cudaEventDestroy(ev_t1);
    if (ms) cudaStreamDestroy(ms);
  }
};

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// A system joins the grouped launches when both of its products run on the
// single-RHS tensor-core kernel.
bool groupable(const adasap_solver* S) {
  return !S->identity && !S->sched && S->s == 1 && S->plan1.tc && !S->plan1.mrhs && S->tc_pw;
}

// column tiles of the tensor-core kernel are 128 wide
int step1_splits(const adasap_solver* S, int tpi) { return (int)ceil_div(tc_npad(S->c->n) / 128, tpi); }
int power_splits(const adasap_solver* S, int tpi) { return (int)ceil_div(tc_npad(S->b) / 128, tpi); }

// Grouped launch descriptions for the active groupable systems; which = 0 Step I,
// 1 / 2 the K_BB a product on power buffer 0 / 1.
cudaError_t build_groups(Batch& bt, int which, int tpi, std::vector<GroupedProduct>& out) {
  std::vector<GroupedProduct> cls;
  std::vector<std::vector<TcArgs>> args;
  for (size_t i = 0; i < bt.S.size(); ++i) {
    if (!bt.active[i] || !bt.grouped[i]) continue;
    adasap_solver* S = bt.S[i];
    adasap_ctx* c = S->c;
    size_t k = 0;
    while (k < cls.size() && !(cls[k].kern == c->kern && cls[k].kp == c->kp)) ++k;
    if (k == cls.size()) {
      cls.emplace_back();
      cls.back().kern = c->kern;
      cls.back().kp = c->kp;
      args.emplace_back();
    }
    TcArgs a;
    if (which == 0)
      a = make_tc_args(c->d, c->Xc, c->qc, S->B32, S->b, c->dp, c->tc_hi, c->tc_lo, c->n, 1, step1_point(S), S->s,
                       S->part1, step1_splits(S, tpi), c->sigma2, c->err_dev);
    else
      a = make_tc_args(c->d, S->XB, S->qB, nullptr, S->b, c->dp, S->XBhi, S->XBlo, S->b, 1, power_buf(S, which - 1),
                       1, S->part2, power_splits(S, tpi), c->sigma2, c->err_dev);
    cls[k].members.push_back((int)i);
    args[k].push_back(a);
  }
  for (size_t k = 0; k < cls.size(); ++k) {
    std::vector<int64_t> start(1, 0);
    for (const TcArgs& a : args[k]) start.push_back(start.back() + tc_items(a));
    GroupedProduct& g = cls[k];
    g.nitems = start.back();
    cudaError_t e;
    if ((e = cudaMalloc(&g.grp, args[k].size() * sizeof(TcArgs))) ||
        (e = cudaMalloc(&g.gstart, start.size() * sizeof(int64_t))) ||
        (e = cudaMalloc(&g.sched, 2 * sizeof(unsigned long long))) ||
        (e = cudaMemset(g.sched, 0, 2 * sizeof(unsigned long long))) ||
        (e = cudaMemcpy(g.grp, args[k].data(), args[k].size() * sizeof(TcArgs), cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(g.gstart, start.data(), start.size() * sizeof(int64_t), cudaMemcpyHostToDevice))) {
      out.insert(out.end(), cls.begin(), cls.begin() + k + 1);
      return e;
    }
  }
  out.insert(out.end(), cls.begin(), cls.end());
  return cudaSuccess;
}

cudaError_t build_wb(Batch& bt) {
  std::vector<WbArgs> h[5];
  std::vector<int> start(1, 0);
  for (size_t i = 0; i < bt.S.size(); ++i) {
    if (!bt.active[i] || !bt.grouped[i]) continue;
    adasap_solver* S = bt.S[i];
    adasap_ctx* c = S->c;
    const int np = S->o.power_iters;
    const float lam = (float)c->lambda;
    h[0].push_back(wb_args_single(S->cb, kInvSqrtNormalised, S->v0, power_buf(S, 0), c->sc));
    for (int par = 0; par < 2; ++par)
      h[1 + par].push_back(wb_args_power(S->cb, kInvUnit, S->part2, S->ns_pw, lam, power_buf(S, par), S->h,
                                         power_buf(S, par + 1), c->sc));
    h[3].push_back(wb_args_power(S->cb, kRayleighEta, S->part2, S->ns_pw, lam, power_buf(S, np - 1), S->h,
                                 power_buf(S, np), c->sc));
    h[4].push_back(wb_args_single(S->cb, kInv, S->R, S->D, c->sc));
    start.push_back(start.back() + h[0].back().nchunk);   // the same chunking in all five tables
  }
  bt.nwb = (int)h[0].size();
  bt.wb_blocks = start.back();
  if (bt.nwb == 0) return cudaSuccess;
  for (int k = 0; k < 5; ++k) {
    KR(cudaMalloc(&bt.wb[k], h[k].size() * sizeof(WbArgs)));
    KR(cudaMemcpy(bt.wb[k], h[k].data(), h[k].size() * sizeof(WbArgs), cudaMemcpyHostToDevice));
  }
  KR(cudaMalloc(&bt.wb_start, start.size() * sizeof(int)));
  KR(cudaMemcpy(bt.wb_start, start.data(), start.size() * sizeof(int), cudaMemcpyHostToDevice));
  return cudaSuccess;
}

// Tables of the grouped k_head_prep (active systems with use_prep), by operand width.
cudaError_t build_prep(Batch& bt) {
  std::vector<HeadPrepArgs> h[2];
  for (size_t i = 0; i < bt.S.size(); ++i) {
    if (!bt.active[i] || !bt.S[i]->use_prep) continue;
    const int k = bt.S[i]->c->kp == 16 ? 0 : 1;
    h[k].push_back(bt.S[i]->prep);
    bt.prep_work[k] = std::max(bt.prep_work[k], head_prep_work(h[k].back()));
  }
  for (int k = 0; k < 2; ++k) {
    bt.nprep[k] = (int)h[k].size();
    if (h[k].empty()) continue;
    KR(cudaMalloc(&bt.prep[k], h[k].size() * sizeof(HeadPrepArgs)));
    KR(cudaMemcpy(bt.prep[k], h[k].data(), h[k].size() * sizeof(HeadPrepArgs), cudaMemcpyHostToDevice));
  }
  return cudaSuccess;
}

// Tables of the grouped heads: the active systems with k_head_prep and a tensor-core
// sketch; sketches by (kernel, operand width, shared-memory plan), then one table of
// split sums and one per Gram call of launch_nystrom_grams.
cudaError_t build_head(Batch& bt) {
  const size_t asz = mrhs_args_size();
  std::vector<std::vector<unsigned char>> blocks;
  std::vector<std::vector<int64_t>> starts;
  std::vector<SplitSumArgs> ss;
  std::vector<GramArgs> gr[2];
  for (size_t i = 0; i < bt.S.size(); ++i) {
    adasap_solver* S = bt.S[i];
    if (!bt.active[i] || !S->use_prep || !S->sk_tc) continue;
    adasap_ctx* c = S->c;
    const int64_t b = S->b;
    const int r = S->r;
    std::vector<unsigned char> blk(asz);
    const int64_t wf = tc_mrhs_wfloats(b, r);
    const int64_t items = mrhs_fill_args(blk.data(), c->d, S->XB, S->qB, nullptr, b, c->dp, S->XBhi, S->XBlo, b, 1,
                                         S->wsk, S->wsk + wf, r, 3, S->part2, S->ns_sk, c->sigma2, c->err_dev);
    if (items < 1) continue;
    const int64_t key = mrhs_plan_key(blk.data());
    size_t g = 0;
    while (g < bt.sk.size() && !(bt.sk[g].kern == c->kern && bt.sk[g].kp == c->kp && bt.sk[g].key == key)) ++g;
    if (g == bt.sk.size()) {
      bt.sk.emplace_back();
      bt.sk.back().kern = c->kern;
      bt.sk.back().kp = c->kp;
      bt.sk.back().key = key;
      bt.sk.back().first = blk;
      blocks.emplace_back();
      starts.emplace_back(1, 0);
    }
    blocks[g].insert(blocks[g].end(), blk.begin(), blk.end());
    starts[g].push_back(starts[g].back() + items);
    ++bt.sk[g].n;
    SplitSumArgs sa;
    sa.part = S->part2;
    sa.nsplit = S->ns_sk;
    sa.m = b;
    sa.s = r;
    sa.out = S->Ysk;
    ss.push_back(sa);
    bt.ssum_elems = std::max(bt.ssum_elems, b * r);
    // launch_nystrom_grams: [Omega | M Omega] (rows r), then M Omega with exact products
    CoreBufs& cb = S->cb;
    gr[0].push_back(gram_fill_args(S->Om, r, r, S->Ysk, r, r, b, cb.gram_part, cb.gram_chunks, cb.G, r));
    gr[1].push_back(gram_fill_args(S->Ysk, r, r, nullptr, 0, 0, b, cb.gram_part, cb.gram_chunks, cb.Gyy, 0));
    for (int k = 0; k < 2; ++k) {
      bt.gram_chunks[k] = std::max(bt.gram_chunks[k], gr[k].back().chunks);
      bt.gram_active[k] = std::max(bt.gram_active[k], gr[k].back().active);
      bt.gram_c[k] = std::max(bt.gram_c[k], gr[k].back().c);
    }
    S->head_grouped = true;
  }
  for (size_t g = 0; g < bt.sk.size(); ++g) {
    Batch::SketchGroup& G = bt.sk[g];
    G.nitems = starts[g].back();
    KR(cudaMalloc(&G.tab, blocks[g].size()));
    KR(cudaMalloc(&G.gstart, starts[g].size() * sizeof(int64_t)));
    KR(cudaMemcpy(G.tab, blocks[g].data(), blocks[g].size(), cudaMemcpyHostToDevice));
    KR(cudaMemcpy(G.gstart, starts[g].data(), starts[g].size() * sizeof(int64_t), cudaMemcpyHostToDevice));
  }
  bt.nhead = (int)ss.size();
  if (bt.nhead > 0) {
    KR(cudaMalloc(&bt.ssum, ss.size() * sizeof(SplitSumArgs)));
    KR(cudaMemcpy(bt.ssum, ss.data(), ss.size() * sizeof(SplitSumArgs), cudaMemcpyHostToDevice));
    for (int k = 0; k < 2; ++k) {
      KR(cudaMalloc(&bt.gram[k], gr[k].size() * sizeof(GramArgs)));
      KR(cudaMemcpy(bt.gram[k], gr[k].data(), gr[k].size() * sizeof(GramArgs), cudaMemcpyHostToDevice));
    }
  }
  return cudaSuccess;
}

cudaError_t launch_groups(const Batch& bt, const std::vector<GroupedProduct>& gs, cudaStream_t st) {
  for (const GroupedProduct& g : gs)
    KR(launch_rows_tc_grouped(g.kern, g.kp, g.grp, g.gstart, (int)g.members.size(), g.nitems,
                              bt.S[g.members[0]]->c->err_dev, bt.ctas, st, g.sched));
  return cudaSuccess;
}

// Splits of the grouped launches and the partial buffers sized for them.
void set_splits(Batch& bt) {
  for (size_t i = 0; i < bt.S.size(); ++i) {
    if (!bt.grouped[i]) continue;
    bt.S[i]->ns1 = step1_splits(bt.S[i], bt.tpi1);
    bt.S[i]->ns_pw = power_splits(bt.S[i], bt.tpipw);
  }
}

// Column tiles per item of each grouped product, by timing each candidate
// launch alone on the stream (the partial buffers are scratch until the first
// iteration writes them; B holds row 0 until the first sample).
adasap_status autotune(Batch& bt) {
  const int c1[] = {8, 16, 32, 64};
  const int cpw[] = {1, 2, 4, 8};
  for (int which = 0; which < 2; ++which) {
    float best = 1e30f;
    for (int tpi : (which == 0 ? c1 : cpw)) {
      std::vector<GroupedProduct> gs;
      cudaError_t e = build_groups(bt, which == 0 ? 0 : 1, tpi, gs);
      float ms = 0.f;
      if (e == cudaSuccess) {
        for (int rep = 0; rep < 5 && e == cudaSuccess; ++rep) {
          if (rep == 2) e = cudaEventRecord(bt.ev_t0, bt.ms);
          if (e == cudaSuccess) e = launch_groups(bt, gs, bt.ms);
        }
        if (e == cudaSuccess) e = cudaEventRecord(bt.ev_t1, bt.ms);
        if (e == cudaSuccess) e = cudaEventSynchronize(bt.ev_t1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, bt.ev_t0, bt.ev_t1);
      }
      for (GroupedProduct& g : gs) {
        cudaFree(g.grp);
        cudaFree(g.gstart);
        cudaFree(g.sched);
      }
      if (e != cudaSuccess) {
        note_error(e, "autotune");
        return ADASAP_ECUDA;
      }
      if (ms < best) {
        best = ms;
        (which == 0 ? bt.tpi1 : bt.tpipw) = tpi;
      }
    }
  }
  return ADASAP_OK;
}

// One iteration of every active system.
cudaError_t rec_batch(Batch& bt) {
  cudaStream_t ms = bt.ms;
  std::vector<adasap_solver*> act, grp;
  for (size_t i = 0; i < bt.S.size(); ++i)
    if (bt.active[i]) {
      act.push_back(bt.S[i]);
      if (bt.grouped[i]) grp.push_back(bt.S[i]);
    }
  auto fork = [&](const std::vector<adasap_solver*>& v) -> cudaError_t {
    KR(cudaEventRecord(bt.ev, ms));
    for (adasap_solver* S : v) KR(cudaStreamWaitEvent(S->c->s0, bt.ev, 0));
    return cudaSuccess;
  };
  auto join = [&](const std::vector<adasap_solver*>& v) -> cudaError_t {
    for (adasap_solver* S : v) {
      KR(cudaEventRecord(S->c->ev_out, S->c->s0));
      KR(cudaStreamWaitEvent(ms, S->c->ev_out, 0));
    }
    return cudaSuccess;
  };
  // the inputs of the iteration of every system that takes k_head_prep: one launch
  // per operand width for all of them, before the systems fork
  for (int k = 0; k < 2; ++k)
    if (bt.nprep[k] > 0) KR(launch_head_prep(bt.prep[k], bt.nprep[k], k == 0 ? 16 : 32, bt.prep_work[k], ms));
  // and the rest of their heads: sketches, split sums, Gram matrices (so that every
  // system's factorisation chain starts at the same time)
  if (bt.nhead > 0) {
    for (const Batch::SketchGroup& g : bt.sk)
      KR(launch_rows_tc_mrhs_grouped(g.kern, g.kp, g.first.data(), g.tab, g.gstart, g.n, g.nitems, ms));
    KR(launch_split_sum_grouped(bt.ssum, bt.nhead, bt.ssum_elems, ms));
    for (int k = 0; k < 2; ++k)
      KR(launch_gram_grouped(bt.gram[k], bt.nhead, bt.gram_chunks[k], bt.gram_active[k], bt.gram_c[k], k == 1, ms));
  }
  KR(fork(act));
  for (adasap_solver* S : act) KR(rec_head(S, nullptr, nullptr, S->use_prep, S->head_grouped));
  for (adasap_solver* S : act)
    if (!groupable(S)) KR(rec_step1(S));
  if (!grp.empty()) {
    KR(join(grp));
    KR(launch_groups(bt, bt.step1, ms));
    KR(fork(grp));
  }
  // the grouped systems' powering and direction run on the batch stream: one
  // grouped product and one grouped apply per powering step
  for (adasap_solver* S : act) {
    KR(rec_step1_finish(S));
    if (S->identity) KR(rec_power_identity(S));
    else if (!groupable(S)) KR(rec_power_init(S));
  }
  if (!grp.empty()) {
    KR(join(grp));
    KR(launch_wb_grouped(bt.wb[0], bt.wb_start, bt.nwb, bt.wb_blocks, kInvSqrtNormalised, ms));
  }
  const int np = act.empty() ? 0 : act[0]->o.power_iters;
  for (int i = 0; i < np; ++i) {
    for (adasap_solver* S : act)
      if (!S->identity && !groupable(S)) KR(rec_power_rows(S, i));
    if (!grp.empty()) {
      KR(launch_groups(bt, bt.pw[i & 1], ms));
      const bool last = i == np - 1;
      KR(launch_wb_grouped(bt.wb[last ? 3 : 1 + (i & 1)], bt.wb_start, bt.nwb, bt.wb_blocks,
                           last ? kRayleighEta : kInvUnit, ms));
    }
    for (adasap_solver* S : act)
      if (!S->identity && !groupable(S)) KR(rec_power_apply(S, i));
  }
  if (!grp.empty()) {
    KR(launch_wb_grouped(bt.wb[4], bt.wb_start, bt.nwb, bt.wb_blocks, kInv, ms));
    KR(fork(grp));
  }
  for (adasap_solver* S : act) {
    if (!groupable(S)) KR(rec_direction(S));
    KR(rec_update(S, nullptr));
  }
  return join(act);
}

adasap_status rebuild(Batch& bt) {
  bt.free_graph();
  bt.free_groups();
  cudaError_t e;
  if ((e = build_groups(bt, 0, bt.tpi1, bt.step1)) || (e = build_groups(bt, 1, bt.tpipw, bt.pw[0])) ||
      (e = build_groups(bt, 2, bt.tpipw, bt.pw[1])) || (e = build_wb(bt)) || (e = build_prep(bt)) ||
      (e = build_head(bt))) {
    note_error(e, "grouped launch tables");
    return ADASAP_ECUDA;
  }
  if ((e = cudaStreamBeginCapture(bt.ms, cudaStreamCaptureModeThreadLocal))) {
    note_error(e, "batch capture");
    return ADASAP_ECUDA;
  }
  const cudaError_t ce = rec_batch(bt);
  e = cudaStreamEndCapture(bt.ms, &bt.graph);
  if (ce != cudaSuccess || e != cudaSuccess) {
    note_error(ce != cudaSuccess ? ce : e, "batch capture");
    return ADASAP_ECUDA;
  }
  if ((e = cudaGraphInstantiateWithFlags(&bt.exec, bt.graph, cudaGraphInstantiateFlagUseNodePriority))) {
    note_error(e, "batch instantiate");
    return ADASAP_ECUDA;
  }
  return ADASAP_OK;
}

adasap_status solve_batched(int nsys, adasap_ctx* const* ctxs, const float* const* Y, int s,
                            const adasap_opts* opts, float* const* W, adasap_stats* stats, cudaStream_t us) {
  for (int i = 0; i < nsys; ++i) {
    if (!ctxs[i] || !Y[i] || !W[i] || opts[i].tail_average || opts[i].max_iters < 0 || opts[i].precond == 2 ||
        opts[i].power_iters != opts[0].power_iters)
      return ADASAP_EINVAL;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return ADASAP_EINVAL;  // one active solver per context
  }
  Batch bt;
  CT(cudaStreamCreateWithFlags(&bt.ms, cudaStreamNonBlocking));
  CT(cudaEventCreateWithFlags(&bt.ev, cudaEventDisableTiming));
  CT(cudaEventCreate(&bt.ev_t0));
  CT(cudaEventCreate(&bt.ev_t1));
  // persistent CTAs of the grouped launches: the rest of the GPU runs the
  // systems' factorisation branches (mostly single-CTA launches)
  const int reserve = std::min(32, std::max(kBranchSms, nsys / 4));
  bt.ctas = std::max(1, tc_slots() - reserve);
  bt.S.assign(nsys, nullptr);
  bt.active.assign(nsys, 1);
  bt.grouped.assign(nsys, 0);
  for (int i = 0; i < nsys; ++i) {
    const adasap_status st =
        solver_prepare(ctxs[i], Y[i], s, &opts[i], nullptr, nullptr, nullptr, W[i], us, &bt.S[i], 0, reserve, nsys);
    if (st != ADASAP_OK) return st;
    adasap_solver* S = bt.S[i];
    bt.grouped[i] = groupable(S);
    if (!bt.grouped[i]) continue;
    // partial buffers for the smallest split candidates; B = row 0 until the first sample
    const int64_t b = S->b;
    S->part1 = S->ar.get<float>((size_t)step1_splits(S, 8) * b);
    const size_t pw = std::max((size_t)power_splits(S, 1) * b, (size_t)S->ns_sk * b * S->r);
    S->part2 = S->ar.get<float>(pw);
    if (S->ar.err != cudaSuccess) return ADASAP_ENOMEM;
    CT(cudaMemset(S->B32, 0, (size_t)b * sizeof(int)));
  }
  CT(cudaDeviceSynchronize());
  int ngrouped = 0;
  for (int i = 0; i < nsys; ++i) ngrouped += bt.grouped[i];
  if (ngrouped > 0) {
    const adasap_status st = autotune(bt);
    if (st != ADASAP_OK) return st;
  }
  set_splits(bt);
  // iterate: every system leaves the batch at its own tolerance or max_iters
  std::vector<double> rel(nsys, NAN), secs(nsys, 0.0);
  std::vector<adasap_status> res(nsys, ADASAP_OK);
  std::vector<char> checked(nsys, 0), conv(nsys, 0);
  CT(cudaEventRecord(bt.ev_t0, bt.ms));
  int nactive = nsys;
  adasap_status st = ADASAP_OK;
  auto leave = [&](int i) -> adasap_status {
    CT(cudaEventRecord(bt.ev_t1, bt.ms));
    CT(cudaEventSynchronize(bt.ev_t1));
    float ms = 0.f;
    CT(cudaEventElapsedTime(&ms, bt.ev_t0, bt.ev_t1));
    secs[i] = ms * 1e-3;
    bt.active[i] = 0;
    --nactive;
    return ADASAP_OK;
  };
  for (int i = 0; i < nsys; ++i)
    if (opts[i].max_iters == 0 && (st = leave(i)) != ADASAP_OK) return st;
  if (nactive > 0 && (st = rebuild(bt)) != ADASAP_OK) return st;
  while (nactive > 0) {
    int64_t k = INT64_MAX;
    for (int i = 0; i < nsys; ++i) {
      if (!bt.active[i]) continue;
      const adasap_opts& o = bt.S[i]->o;
      int64_t ki = o.max_iters - bt.S[i]->iters;
      if (o.check_every > 0) ki = std::min<int64_t>(ki, o.check_every - bt.S[i]->iters % o.check_every);
      k = std::min(k, ki);
    }
    for (int64_t j = 0; j < k; ++j) CT(cudaGraphLaunch(bt.exec, bt.ms));
    bool changed = false;
    for (int i = 0; i < nsys; ++i) {
      if (!bt.active[i]) continue;
      adasap_solver* S = bt.S[i];
      S->iters += k;
      checked[i] = 0;
      const bool at_max = S->iters >= S->o.max_iters;
      const bool due = S->o.check_every > 0 && S->iters % S->o.check_every == 0;
      if (!due && !at_max) continue;
      if (due) {
        res[i] = solver_residual(S, &rel[i], bt.ms);
        checked[i] = 1;
        conv[i] = res[i] == ADASAP_OK && S->o.tol > 0 && rel[i] <= S->o.tol;
      }
      if (res[i] != ADASAP_OK || conv[i] || at_max) {
        if ((st = leave(i)) != ADASAP_OK) return st;
        changed = true;
      }
    }
    if (changed && nactive > 0 && (st = rebuild(bt)) != ADASAP_OK) return st;
  }
  CT(cudaStreamSynchronize(bt.ms));
  adasap_status worst = ADASAP_OK;
  for (int i = 0; i < nsys; ++i) {
    adasap_solver* S = bt.S[i];
    adasap_ctx* c = S->c;
    if (res[i] == ADASAP_OK && !checked[i]) {
      res[i] = solver_residual(S, &rel[i], bt.ms);
      conv[i] = res[i] == ADASAP_OK && S->o.tol > 0 && rel[i] <= S->o.tol;
    }
    CT(cudaMemcpyAsync(c->sc_host, c->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->s0));
    CT(cudaMemcpyAsync(W[i], S->W, (size_t)c->n * s * sizeof(float), cudaMemcpyDefault, c->s0));
    CT(cudaStreamSynchronize(c->s0));
    if (res[i] == ADASAP_OK && c->sc_host->status != 0) res[i] = (adasap_status)c->sc_host->status;
    if (res[i] == ADASAP_OK && S->o.tol > 0 && !conv[i]) res[i] = ADASAP_ENOTCONVERGED;
    if (stats) {
      stats[i].iters = (int)S->iters;
      stats[i].rel_resid = rel[i];
      stats[i].resid_exact = S->mc == c->n ? 1 : 0;
      stats[i].seconds = secs[i];
      stats[i].last_eta = c->sc_host->eta;
      stats[i].last_rho = c->sc_host->rho;
      stats[i].status_detail = c->sc_host->detail;
    }
    if (worst == ADASAP_OK || (worst == ADASAP_ENOTCONVERGED && res[i] != ADASAP_OK)) worst = res[i];
  }
  CT(cudaEventRecord(bt.ev, bt.ms));
  CT(cudaStreamWaitEvent(us, bt.ev, 0));
  return worst;
}

}  // namespace

extern "C" adasap_status adasap_solve_batched(int nsys, adasap_ctx* const* ctxs, const float* const* Y, int s,
                                              const adasap_opts* opts, float* const* W, adasap_stats* stats,
                                              void* stream) {
  if (nsys < 1 || !ctxs || !Y || !opts || !W || s < 1 || s > kMaxRhs) return ADASAP_EINVAL;
  try {
    return solve_batched(nsys, ctxs, Y, s, opts, W, stats, (cudaStream_t)stream);
  } catch (...) {
    return ADASAP_ENOMEM;
  }
}

// ---------------------------------------------------------------------------
// Pathwise conditioning (Sec. 2.1): random-feature prior draws, the s-column
// solve, the samples at test points, and their test metrics.
// ---------------------------------------------------------------------------
extern "C" adasap_status adasap_rf_prior(adasap_ctx* c, const float* Xq, int64_t m, const float* z, const float* u,
                                         const float* phase, const float* theta, int q, int s, float* F,
                                         void* stream) {
  if (!c || !Xq || !z || !phase || !theta || !F || m < 1 || m >= (1LL << 31) || q < 1 || s < 1 || s > kMaxRhs ||
      (c->kern != ADASAP_RBF && !u))
    return ADASAP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  Arena ar;
  float* xt = ar.get<float>((size_t)m * c->dp);
  float* qt = ar.get<float>((size_t)m);
  float* om = ar.get<float>((size_t)q * c->dp);
  float* cph = ar.get<float>((size_t)q);
  if (ar.err != cudaSuccess) return ADASAP_ENOMEM;
  CT(launch_transform(Xq, m, c->d, c->dp, c->mean_dev, c->kappa / (double)c->ell, xt, qt, st));
  CT(launch_rf_prep(z, u, phase, q, c->d, c->dp, c->kern, c->mean_dev, c->ell, c->kappa, om, cph, st));
  CT(launch_rf_apply(xt, m, c->dp, om, cph, theta, q, s, (float)std::sqrt(2.0 * c->sigma2 / q), nullptr, nullptr, 0,
                     0, 0.f, F, s, 0, st));
  CT(cudaStreamSynchronize(st));  // the arena frees its buffers on return
  return ADASAP_OK;
}

extern "C" adasap_status adasap_pathwise(adasap_ctx* c, const float* y, const float* Xtest, int64_t m,
                                         const float* z, const float* u, const float* phase, const float* theta,
                                         int q, const float* zeta, int ns, int with_mean, const adasap_opts* o,
                                         float* out, float* W, adasap_stats* stats, void* stream) {
  const int sc = ns + (with_mean ? 1 : 0);
  if (!c || !y || !Xtest || !z || !phase || !theta || !zeta || !o || !out || !W || m < 1 || m >= (1LL << 31) ||
      q < 1 || ns < 1 || sc > kMaxRhs || (c->kern != ADASAP_RBF && !u))
    return ADASAP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = c->n;
  const int off = with_mean ? 1 : 0;
  const float scale = (float)std::sqrt(2.0 * c->sigma2 / q);
  Arena ar;
  float* R = ar.get<float>((size_t)n * sc);
  float* om = ar.get<float>((size_t)q * c->dp);
  float* cph = ar.get<float>((size_t)q);
  float* xt = ar.get<float>((size_t)m * c->dp);
  float* qt = ar.get<float>((size_t)m);
  if (ar.err != cudaSuccess) return ADASAP_ENOMEM;
  CT(launch_rf_prep(z, u, phase, q, c->d, c->dp, c->kern, c->mean_dev, c->ell, c->kappa, om, cph, st));
  // right-hand sides: [y,] y - f_j(X) - zeta_j
  if (with_mean)
    CT(launch_reduce(y, 1, n, 1, 0, 1, R, sc, 0.f, nullptr, nullptr, 0, 0.f, nullptr, nullptr, 0, nullptr, st));
  CT(launch_rf_apply(c->Xc, n, c->dp, om, cph, theta, q, ns, -scale, y, zeta, ns, 0, -1.f, R, sc, off, st));
  // W = (K + lambda I)^{-1} R by ADASAP (one solve for all columns)
  const adasap_status s1 = adasap_solve(c, R, sc, o, W, stats, stream);
  if (s1 != ADASAP_OK && s1 != ADASAP_ENOTCONVERGED) return s1;
  // samples: k(X*, X) W [+ f(X*) on the sample columns]
  const adasap_status s2 = adasap_predict(c, Xtest, m, W, sc, out, stream);
  if (s2 != ADASAP_OK) return s2;
  CT(launch_transform(Xtest, m, c->d, c->dp, c->mean_dev, c->kappa / (double)c->ell, xt, qt, st));
  CT(launch_rf_apply(xt, m, c->dp, om, cph, theta, q, ns, scale, nullptr, out, sc, off, 1.f, out, sc, off, st));
  CT(cudaStreamSynchronize(st));
  return s1;
}

extern "C" adasap_status adasap_rmse_nll(const float* mean, int64_t ld_mean, const float* samples,
                                         int64_t ld_samples, int s, const float* ytest, int64_t m, double noise,
                                         double* rmse, double* nll, void* stream) {
  if (!mean || !samples || !ytest || !rmse || !nll || m < 1 || s < 2 || ld_mean < 1 || ld_samples < s ||
      !(noise >= 0.0))
    return ADASAP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int blocks = (int)std::min<int64_t>((m + 255) / 256, 296);
  Arena ar;
  double* parts = ar.get<double>((size_t)2 * blocks);
  if (ar.err != cudaSuccess) return ADASAP_ENOMEM;
  CT(launch_rmse_nll(mean, ld_mean, samples, ld_samples, s, ytest, m, noise, parts, blocks, st));
  std::vector<double> h((size_t)2 * blocks);
  CT(cudaMemcpyAsync(h.data(), parts, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  CT(cudaStreamSynchronize(st));
  double se = 0.0, nl = 0.0;
  for (int b = 0; b < blocks; ++b) {
    se += h[2 * b];
    nl += h[2 * b + 1];
  }
  *rmse = std::sqrt(se / (double)m);
  *nll = nl / (double)m;
  return ADASAP_OK;
}

// ---------------------------------------------------------------------------
// Device-side failures of bounded waits (the paper has no counterpart).
// ---------------------------------------------------------------------------
extern "C" adasap_status adasap_check_device(adasap_ctx* c, int* code, void* stream) {
  if (!c) return ADASAP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  CT(cudaEventRecord(c->ev_in, st));
  CT(cudaStreamWaitEvent(c->s0, c->ev_in, 0));
  int h = 0;
  CT(cudaMemcpyAsync(&h, c->err_dev, sizeof(int), cudaMemcpyDeviceToHost, c->s0));
  CT(cudaMemsetAsync(c->err_dev, 0, sizeof(int), c->s0));
  CT(cudaStreamSynchronize(c->s0));
  if (code) *code = h;
  return h != 0 ? ADASAP_ETIMEOUT : ADASAP_OK;
}

extern "C" adasap_status adasap_wait_selftest(adasap_ctx* c, uint64_t limit_ns, void* stream) {
  if (!c || limit_ns > 1000000000ull) return ADASAP_EINVAL;
  CT(launch_wait_selftest(limit_ns, c->err_dev, (cudaStream_t)stream));
  return ADASAP_OK;
}

extern "C" adasap_status adasap_schedule_check(int64_t m, int64_t ncols, int max_ctas, int* nsplit, int* flat) {
  if (m < 1 || ncols < 1 || !nsplit || !flat) return ADASAP_EINVAL;
  return tc_schedule_check(m, ncols, max_ctas, nsplit, flat) == 0 ? ADASAP_OK : ADASAP_ENUMERIC;
}

extern "C" adasap_status adasap_solver_graph_kernels(adasap_solver* S, int* count) {
  if (!S || !count || !S->graph) return ADASAP_EINVAL;
  size_t nn = 0;
  CT(cudaGraphGetNodes(S->graph, nullptr, &nn));
  std::vector<cudaGraphNode_t> nodes(nn);
  CT(cudaGraphGetNodes(S->graph, nodes.data(), &nn));
  int k = 0;
  for (size_t i = 0; i < nn; ++i) {
    cudaGraphNodeType t;
    CT(cudaGraphNodeGetType(nodes[i], &t));
    k += t == cudaGraphNodeTypeKernel;
  }
  *count = k;
  return ADASAP_OK;
}

extern "C" adasap_status adasap_solver_diag(adasap_solver* S, double* out, int count, void* stream) {
  if (!S || !out || count < 1) return ADASAP_EINVAL;
  adasap_ctx* c = S->c;
  CT(cudaEventRecord(c->ev_in, (cudaStream_t)stream));
  CT(cudaStreamWaitEvent(c->s0, c->ev_in, 0));
  CT(cudaMemcpyAsync(c->sc_host, c->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->s0));
  int tc_err = 0;
  CT(cudaMemcpyAsync(&tc_err, c->err_dev, sizeof(int), cudaMemcpyDeviceToHost, c->s0));
  CT(cudaStreamSynchronize(c->s0));
  const DevScalars& h = *c->sc_host;
  const double vals[] = {h.delta, h.rho, h.eta, h.lam_hat, (double)h.chol_retries, (double)h.jacobi_sweeps,
                         (double)h.status, (double)h.detail, (double)h.t, (double)tc_err};
  for (int i = 0; i < count && i < (int)(sizeof(vals) / sizeof(vals[0])); ++i) out[i] = vals[i];
  return ADASAP_OK;
}

// ---------------------------------------------------------------------------
// adasap_kernel_rows_noalloc: the block-row product for callers that cannot
// allocate device memory while they run.
//
// Its scratch (the int32 copy of B and the per-split partial sums) lives in the
// file-scope array below instead of the context's growable workspace, so the
// call itself makes no allocation.  The array is part of the library's device
// image: every GPU that loads the library holds these kNoallocScratchBytes
// until the process exits.  In host code the array's name is only a host-side
// stand-in; its device address is looked up once per device, on the first call
// made on that device, with cudaGetSymbolAddress.
// ---------------------------------------------------------------------------
namespace {
constexpr size_t kNoallocScratchBytes = (size_t)8 << 20;
constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoallocMaxDevices] = {};
}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

extern "C" adasap_status adasap_kernel_rows_noalloc(adasap_ctx* c, const int64_t* B, int64_t b, const float* W,
                                                    int s, float* out, void* stream) {
  if (!c || !B || !W || !out || b < 1 || b >= (1LL << 31) || s < 1 || s > kMaxRhs) return ADASAP_EINVAL;
  int dev = -1;
  CT(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoallocMaxDevices) {
    g_last_error = "adasap_kernel_rows_noalloc: device index " + std::to_string(dev) +
                   " is beyond the per-device address table (devices 0.." + std::to_string(kNoallocMaxDevices - 1) +
                   ")";
    return ADASAP_EINVAL;
  }
  if (dev != c->device) {
    g_last_error = "adasap_kernel_rows_noalloc: the context's device must be the current device";
    return ADASAP_EINVAL;
  }
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        note_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        return ADASAP_ECUDA;
      }
      g_noalloc_ptr[dev] = p;
    }
    base = g_noalloc_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  RowsPlan p = plan_rows(c, b, c->n, s);
  if (p.mrhs) {  // the multi-RHS kernel needs W-operand scratch: keep the CUDA-core kernel here
    p.tc = p.mrhs = false;
    p.ctas = 0;
    p.wop_floats = 0;
    p.nsplit = rows_nsplit(b, c->n, s, c->dp, false);
  }
  const size_t idx_bytes = ((size_t)b * sizeof(int) + 255) & ~(size_t)255;
  const size_t part_bytes = (size_t)p.nsplit * b * s * sizeof(float);
  if (idx_bytes + part_bytes > kNoallocScratchBytes) {
    g_last_error = "adasap_kernel_rows_noalloc: needs " + std::to_string(idx_bytes + part_bytes) +
                   " bytes of scratch, the static array holds " + std::to_string(kNoallocScratchBytes) +
                   "; use adasap_kernel_rows or a smaller b * s";
    return ADASAP_EINVAL;
  }
  // Every byte read below is written first in this call (the index copy, then one
  // partial per split and row), so nothing has to be cleared.
  int* idx = static_cast<int*>(base);
  float* part = reinterpret_cast<float*>(static_cast<unsigned char*>(base) + idx_bytes);
  CT(launch_index32(B, b, c->n, idx, st));
  CT(run_rows_over_x(c, p, c->Xc, c->qc, idx, b, W, s, part, 1, st));
  CT(launch_reduce(part, p.nsplit, b, s, 0, s, out, s, 0.f, nullptr, nullptr, 0, 0.f, nullptr, nullptr, 0, nullptr,
                   st));
  return ADASAP_OK;
}
