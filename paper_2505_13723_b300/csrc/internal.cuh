// Internal launchers of the ADASAP CUDA path.  Host code in solver.cu composes
// them; each launcher is defined next to its kernels.
#pragma once
#include "common.cuh"

namespace adasap {

constexpr int kMaxRank = 128;   // r <= 128 (one CTA holds r x r FP64 in shared memory)
constexpr int kMaxRhs = 128;    // s <= 128
constexpr int kMaxDim = 64;     // d <= 64

// Padded feature width used for the device copy of X (multiple of 4).
int padded_dim(int d);
// kappa of the pre-scaling x' = kappa (x - mean) / ell (see common.cuh).
double kernel_kappa(int kern);

// Operand description of one kernel-times-matrix product
//   part[p][i][:] = sigma2 * sum_{j in split p} k(x'_{row i}, x'_j) * w[j][:]
// Rows: row i has data xr[src*DP .. +DP) and squared norm qr[src] with
// src = ridx ? ridx[i] : i (ridx[i] < 0 marks an invalid row: NaN output).
// Columns: xc (ncols x DP), qc (ncols).  W rows are indexed like columns.
struct RowsArgs {
  const float* xr;
  const float* qr;
  const int* ridx;
  int64_t m;
  const float* xc;
  const float* qc;
  int64_t ncols;
  const float* w;
  int64_t ldw;
  float* part;
  int64_t cps;  // columns per split
  float sigma2;
};

// Number of column splits for an m-row product (fills the GPU without a tail).
int rows_nsplit(int64_t m, int64_t ncols, int s, int dp, bool adjoint);
// Launch the fused distance + kernel epilogue + contraction (K1/K2 engine).
// s <= 4 (or adjoint): register-blocked narrow kernel; otherwise the
// tiled kernel with a shared-memory kernel tile.  part: nsplit x m x s
// (x 2s for the adjoint: [k-sums | g-sums]).
cudaError_t launch_rows(int kern, int dp, const RowsArgs& a, int s, int nsplit, bool adjoint,
                        cudaStream_t st);
// out[i*ldo + c] = sum_p part[(p*m + i)*na + coff + c] + beta*A[ai*lda + c] + gamma*B[bi*ldb + c]
// (ai = aidx ? aidx[i] : i, same for bi); FP64 sums.  If blocksq != NULL each of
// kReduceBlocks blocks writes its sum of out^2 there.
constexpr int kReduceBlocks = 296;
cudaError_t launch_reduce(const float* part, int nsplit, int64_t m, int na, int coff, int s,
                          float* out, int64_t ldo, float beta, const float* A, const int* aidx,
                          int64_t lda, float gamma, const float* B, const int* bidx, int64_t ldb,
                          double* blocksq, cudaStream_t st);
// out rows i < m: x'[idx[i]] (DP floats) and q[idx[i]]
cudaError_t launch_gather(const float* X, const float* q, const int* idx, int64_t m, int dp,
                          float* out, float* qout, cudaStream_t st);
// Column sums (FP64) of raw X (n x d): per-block partials [nb][d].
constexpr int kColsumBlocks = 148;
cudaError_t launch_colsum(const float* X, int64_t n, int d, double* partials, cudaStream_t st);
// x' = kappa (x - mean) / ell, padded to dp; q = ||x'||^2 (FP64 then rounded).
cudaError_t launch_transform(const float* X, int64_t n, int d, int dp, const double* mean_dev,
                             double scale, float* out, float* q, cudaStream_t st);
// out[i] = start + i (int32 row indices of a contiguous row range)
cudaError_t launch_iota32(int* out, int64_t start, int64_t m, cudaStream_t st);
// int64 indices -> int32, entries outside [0, n) become -1.
cudaError_t launch_index32(const int64_t* in, int64_t m, int64_t n, int* out, cudaStream_t st);

// ---- exact block solve of Alg. 1 (blockchol.cu) ------------------------------------
constexpr int64_t kMaxExactBlock = 8192;   // b of the exact solve (two bp x bp FP32 matrices)
int64_t chol_pad(int64_t b);               // b rounded up to the 64-row tile
int64_t chol_linv_floats(int64_t b);       // floats of the inverted diagonal tiles
// H = sigma2 k(X_B, X_B) + lambda I (bp x bp, identity padding) from the gathered block
cudaError_t launch_form_h(int kern, const float* xb, int64_t b, int dp, float sigma2, float lam, float* H,
                          cudaStream_t st);
// blocked Cholesky in place (lower triangle of A), inverted diagonal tiles in Linv
cudaError_t launch_block_chol(float* A, int64_t b, float* Linv, DevScalars* sc, cudaStream_t st);
// D = (L L^T)^{-1} R (add = 0) or D += (L L^T)^{-1} R (add = 1); R, D, Y: bp x s
cudaError_t launch_chol_solve(const float* L, int64_t b, const float* Linv, const float* R, int s, float* Y,
                              float* D, int add, cudaStream_t st);
// E = R - H D, FP64 sums
cudaError_t launch_h_residual(const float* H, int64_t b, const float* D, const float* R, int s, float* E,
                              cudaStream_t st);
// W[B[i]] -= D[i]
cudaError_t launch_block_sub(float* W, const int* B, int64_t b, int s, const float* D, cudaStream_t st);

// ---- random-feature prior and pathwise conditioning (pathwise.cu) -------------------
cudaError_t rf_init();
// omega (q x dp) and phase constants for points in the context's x' form.
cudaError_t launch_rf_prep(const float* z, const float* u, const float* phase, int q, int d, int dp, int kern,
                           const double* mean, double ell, double kappa, float* omega, float* cphase,
                           cudaStream_t st);
// out[i][coff + j] = scale * sum_l theta[l][j] cos(omega_l . x_i + c_l) + (y ? y[i] : 0)
//                    + gz * zin[i][zoff + j]   (zin may alias out)
cudaError_t launch_rf_apply(const float* x, int64_t m, int dp, const float* omega, const float* cphase,
                            const float* theta, int q, int s, float scale, const float* y, const float* zin,
                            int64_t ldz, int zoff, float gz, float* out, int64_t ldo, int coff, cudaStream_t st);
// per-block [sum err^2, sum nll] of the test metrics (blocks x 2 doubles)
cudaError_t launch_rmse_nll(const float* mean, int64_t ldm, const float* smp, int64_t lds, int s, const float* yt,
                            int64_t m, double noise, double* parts, int blocks, cudaStream_t st);

// ---- tensor-core block-row product (rows_tc.cu) ------------------------------------
// One block-row product on the tensor cores (rows_tc.cu): rows (x', q) with an
// optional row index, the column operands in the split canonical layout, w.
struct TcArgs {
  const float* xr;   // rows, x' form (m rows of stride dp), or gathered block
  const float* qr;
  const int* ridx;   // row -> source row (NULL: identity); < 0 marks an invalid row
  int64_t m;
  int dp, d;
  const float* bhi;  // columns: split operands in the canonical layout (npad rows)
  const float* blo;
  int64_t ncols;
  int self_mode;     // 1: column j is the same point as the row's source index
  const float* w;
  int64_t ldw;
  float* part;       // nsplit x m
  int64_t cps;       // columns per split (multiple of 128)
  int nsplit;
  float sigma2;
  int* err;          // set to 1 on a wait timeout
  int flat;          // 1: equal tile runs per CTA (one product only; nsplit = tc_flat_slots)
  const float* wp;   // w prepared per 128-column tile by launch_prep_w (NULL: the kernel stages w itself)
  // grouped launches: {next item, CTAs done}, zero between launches (NULL: static order)
  unsigned long long* sched;
};
TcArgs make_tc_args(int d, const float* xr, const float* qr, const int* ridx, int64_t m, int dp, const float* bhi,
                    const float* blo, int64_t ncols, int self_mode, const float* w, int64_t ldw, float* part,
                    int nsplit, float sigma2, int* err);
int64_t tc_items(const TcArgs& a);   // (row tile, split) items of one product
// Several independent products (grp[g], device) in one persistent launch of at
// most `ctas` CTAs; gstart (device, ngrp + 1) is the prefix sum of tc_items.
// sched (device, 2 counters, zero; NULL: static order): the CTAs take their items
// after the first from a shared counter, so that CTAs slowed by other work on
// their SMs take fewer; the last CTA to finish zeroes the counters again.
cudaError_t launch_rows_tc_grouped(int kern, int kp, const TcArgs* grp, const int64_t* gstart, int ngrp,
                                   int64_t nitems, int* err, int ctas, cudaStream_t st,
                                   unsigned long long* sched = nullptr);
// K of the augmented MMA operands (16 or 32; 0 if d + 2 > 32) and padded row count.
int tc_kp(int d);
int64_t tc_npad(int64_t n);
cudaError_t tc_init();
// Resident CTAs of the tensor-core kernel (one per SM) and its column split for
// an m x ncols product spread over min(slots, max_ctas) persistent CTAs (0: all).
int tc_slots();
int tc_nsplit(int64_t m, int64_t ncols, int max_ctas = 0);
// Partial slots of the flat schedule (equal tile runs per CTA) when it is the
// cheaper one, else 0; launch_rows_tc takes that schedule when nsplit equals it.
int tc_flat_slots(int64_t m, int64_t ncols, int max_ctas = 0);
// tc_flat_slots if non-zero, else tc_nsplit: the split count for launch_rows_tc.
int tc_plan_nsplit(int64_t m, int64_t ncols, int max_ctas = 0);
// Host walk of the flat schedule (0: consistent); see adasap_schedule_check.
int tc_schedule_check(int64_t m, int64_t ncols, int max_ctas, int* nsplit, int* flat);
// Split (hi, lo) column operands in the MMA layout for X' (or rows gidx of X').
cudaError_t launch_build_tc(const float* X, const float* q, const int* gidx, int64_t n, int d, int dp, float* hi,
                            float* lo, cudaStream_t st);
// part[p][i] = sigma2 * sum_{j in split p} k(x'_{row i}, x'_j) w[j] (s = 1).
cudaError_t launch_rows_tc(int kern, int d, const float* xr, const float* qr, const int* ridx, int64_t m, int dp,
                           const float* bhi, const float* blo, int64_t ncols, int self_mode, const float* w,
                           int64_t ldw, float* part, int nsplit, float sigma2, int* err, cudaStream_t st,
                           int max_ctas = 0, const float* wp = nullptr);
// w (ncols entries, stride ldw) laid out for the tensor-core kernel's bulk copies: per
// 128-column tile t, wp[t][0][:] = w, and for the Matern kernels wp[t][1][:] = w / log2(e),
// wp[t][2][:] = w / (3 log2(e)^2); zero past ncols.  tc_wprep_floats: floats of wp.
int64_t tc_wprep_floats(int64_t ncols, int kern);
cudaError_t launch_prep_w(int kern, const float* w, int64_t ldw, int64_t ncols, float* wp, cudaStream_t st);

// ---- multi-RHS tensor-core product (rows_tc_mrhs.cu) ------------------------------
// Padded accumulator width for s right-hand sides, and the floats of one W
// operand (hi or lo) for n rows.
int tc_mrhs_sp(int s);
int64_t tc_mrhs_wfloats(int64_t n, int s);
cudaError_t tc_mrhs_init();
int tc_mrhs_nsplit(int64_t m, int64_t ncols, int max_ctas = 0);
// Grouped multi-RHS products (several independent products in one persistent
// launch): mrhs_fill_args writes the argument block of one product, as
// launch_rows_tc_mrhs would launch it, into host memory (mrhs_args_size() bytes)
// and returns its (row tile, split) items (-1 for invalid sizes); products launched
// together need the same kernel, tc_kp and mrhs_plan_key (shared-memory plan).
size_t mrhs_args_size();
int64_t mrhs_fill_args(void* out, int d, const float* xr, const float* qr, const int* ridx, int64_t m, int dp,
                       const float* bhi, const float* blo, int64_t ncols, int self_mode, const float* whi,
                       const float* wlo, int s, int passes, float* part, int nsplit, float sigma2, int* err);
int64_t mrhs_plan_key(const void* args);
// first: host copy of grp[0]; grp (device, ngrp blocks), gstart (device, ngrp + 1 prefix sums of the items)
cudaError_t launch_rows_tc_mrhs_grouped(int kern, int kp, const void* first, const void* grp, const int64_t* gstart,
                                        int ngrp, int64_t nitems, cudaStream_t st);
// W (n x s, row stride ldw) -> chunked canonical B operands (hi; lo when passes == 3).
cudaError_t launch_build_w_tc(const float* W, int64_t ldw, int64_t n, int s, int passes, float* whi, float* wlo,
                              cudaStream_t st);
// part[p][i][c] = sigma2 * sum_{j in split p} k(x'_{row i}, x'_j) W[j][c] on the tensor cores.
cudaError_t launch_rows_tc_mrhs(int kern, int d, const float* xr, const float* qr, const int* ridx, int64_t m, int dp,
                                const float* bhi, const float* blo, int64_t ncols, int self_mode, const float* whi,
                                const float* wlo, int s, int passes, float* part, int nsplit, float sigma2, int* err,
                                cudaStream_t st, int max_ctas = 0);

// ---- pipe throughput probe (probe.cu): ex2, rsqrt, FFMA per SM per cycle -------------
cudaError_t measure_pipes(double* out4, cudaStream_t st);   // ex2, rsqrt, FFMA, sqrt
// out[i] = f(x[i]): fn 0 the FMA-pipe square root (sqrt_fma), 1 sqrt.approx
cudaError_t launch_eval_math(int fn, const float* x, int64_t n, float* out, cudaStream_t st);
// A bounded wait that no arrival completes: records kWaitSelfTestCode in err after limit_ns.
constexpr int kWaitSelfTestCode = 99;
cudaError_t launch_wait_selftest(uint64_t limit_ns, int* err, cudaStream_t st);

// ---- sampler (Philox4x32-10; definitions in sampler.cu) -------------------------
// Inputs of one iteration of one system, in one launch (k_head_prep): the
// block B (Feistel sample), its gathered rows and tensor-core operands, the
// start vector v0, Omega_t (copied from the buffer it was prepared in one
// iteration ahead) and the sketch's split B operand from Omega_t.  Each part
// has the same arithmetic as its own kernel (launch_sample_block, tag 1;
// launch_normals, tag 3; launch_gather; launch_build_tc; launch_build_w_tc,
// three passes).  A table of these, one per system, is launched at once with
// blockIdx.y selecting the system.
// out (m x s) = sum over nsplit partial blocks of part (nsplit x m x s), for one
// system of a grouped launch (launch_split_sum_grouped: blockIdx.y = system).
struct SplitSumArgs {
  const float* part;
  int nsplit;
  int64_t m;
  int s;
  float* out;
};
cudaError_t launch_split_sum_grouped(const SplitSumArgs* tab, int nsys, int64_t max_elems, cudaStream_t st);

// One Gram call of launch_gram for one system of a grouped launch (the host
// fills it with gram_fill_args; launch_gram_grouped: blockIdx.z / y = system).
struct GramArgs {
  const float* A1;
  int64_t ld1;
  int c1;
  const float* A2;
  int64_t ld2;
  int c2;
  int64_t m, chunk_rows;
  int rows, chunks, active, c;
  float2* part;
  double* G;
};
GramArgs gram_fill_args(const float* A1, int64_t ld1, int c1, const float* A2, int64_t ld2, int c2, int64_t m,
                        float2* part, int chunks, double* G, int rows);
// tab: device, nsys entries; max_chunks / max_active / max_c: maxima over the table
cudaError_t launch_gram_grouped(const GramArgs* tab, int nsys, int max_chunks, int max_active, int max_c, bool exact,
                                cudaStream_t st);

struct HeadPrepArgs {
  uint64_t seed;
  const long long* t_dev;   // iteration counter
  int64_t n, b, npad;       // points, block size, tc_npad(b)
  int h;                    // Feistel half width for n
  int d, dp, r, sp;         // sp = tc_mrhs_sp(r)
  const float* Xc;
  const float* qc;
  int* B32;
  float* XB;
  float* qB;
  float* XBhi;
  float* XBlo;
  float* v0;
  const float* OmN;
  float* Om;
  float* whi;
  float* wlo;
};
int64_t head_prep_work(const HeadPrepArgs& a);   // work items of one system
// tab: device array of nsys entries, all with tc_kp(d) == kp
cudaError_t launch_head_prep(const HeadPrepArgs* tab, int nsys, int kp, int64_t max_work, cudaStream_t st);
int feistel_half_width(int64_t n);
cudaError_t launch_sample_block(uint64_t seed, const long long* t_dev, int64_t t_host, int64_t n,
                                int64_t b, int stream_tag, int* B32, int64_t* B64, cudaStream_t st);
// Iteration counter of the draw: (*t_dev if t_dev else 0) + t_host.
cudaError_t launch_normals(uint64_t seed, const long long* t_dev, int64_t t_host, int64_t count,
                           int stream_tag, float scale, float* out, cudaStream_t st);
// Omega of schedule iteration *t_dev + offset (skipped when that is >= T).
cudaError_t launch_copy_omega(const float* Om_s, const long long* t_dev, int offset, int64_t T, int64_t b, int r,
                              float* Om, cudaStream_t st);
// Copy iteration t (read from t_dev) of a schedule into the working buffers.
cudaError_t launch_copy_schedule(const int64_t* Bs, const float* Om_s, const float* v0s,
                                 const long long* t_dev, int64_t n, int64_t b, int r, int* B32,
                                 float* Om, float* v0, DevScalars* sc, cudaStream_t st);

// ---- Nystrom core, Woodbury, Nesterov (core.cu) ---------------------------------
struct CoreBufs {
  int r, s;
  int64_t b;
  // Gram workspace
  float2* gram_part;  // [gram_chunks][2r][2r] (hi, lo) partial pairs
  int gram_chunks;
  double* G;          // 2r x 2r
  double* Lc;         // r x r lower Cholesky of the Nystrom core
  double* Gnu;        // r x r  Y_nu^T Y_nu
  double* Gyy;        // r x r  Y^T Y with exact products
  double* X1;         // r x r  scratch
  double* A;          // r x r  B^T B
  float* V32;         // r x r  eigenvectors (FP32 Jacobi)
  double* lam;        // r      Rayleigh quotients
  double* T;          // r x r  U = Y_nu T
  float* T32;         // r x r  FP32 right factor of the latest k_make_u (T, or (L^{-1})^T in the QR)
  double* S;          // r      Nystrom eigenvalues (descending)
  double* keep;       // r      1 if S_i > 0 else 0
  float* Minv;        // r x r  (rho S^-1 + U^T U)^-1 on the kept pairs
  float* Gu;          // r x r  U^T U
  float* U;           // b x r
  double* utv_part;   // [utv_chunks][r][s]
  int utv_chunks;
  float* coef;        // r x s
  float* qk;          // r x s: keep . (U^T v) of the multi-RHS inverse apply
  double* sq_part;    // [kReduceBlocks] sums of squares / dots
  double* dot_part;   // [kReduceBlocks]
  double* alpha;      // scalar apply coefficient
  double* Ident;      // r x r identity
  double* cis;        // r  (S_k + rho)^{-1/2} - rho^{-1/2}
  float* wb_part;     // wb_part_floats(b): per-chunk partials of the single-RHS applies
  float* wb_coef;     // [kMaxRank + 1] apply coefficients and alpha
  unsigned int* wb_count;  // finished-block counter (zero between launches)
};
int wb_chunks_for(int64_t b);
size_t wb_part_floats(int64_t b);  // floats of CoreBufs::wb_part for block size b
int gram_chunks_for(int64_t b);
int utv_chunks_for(int64_t b);
cudaError_t launch_gram(const float* A1, int64_t ld1, int c1, const float* A2, int64_t ld2, int c2,
                        int64_t m, float2* part, int chunks, double* G, bool exact, cudaStream_t st,
                        int rows = 0 /* entries with min(i, j) >= rows are not needed (0: all) */);
cudaError_t launch_orthonormalize(CoreBufs& cb, float* Om, float* tmp, DevScalars* sc, cudaStream_t st);
// Gram matrices of the sketch (whole-GPU launches): G = [Omega | Y]^T [Omega | Y], Gyy = Y^T Y (exact products)
cudaError_t launch_nystrom_grams(CoreBufs& cb, const float* Om, const float* Ysk, cudaStream_t st);
// Alg. 4 from the Gram matrices on: Cholesky, eigenpairs, S, rho, U (mostly single-CTA launches)
cudaError_t launch_nystrom_core(CoreBufs& cb, double eps, double lam, DevScalars* sc,
                                const float* Om, const float* Ysk, cudaStream_t st);
cudaError_t launch_woodbury_factor(CoreBufs& cb, double lam, DevScalars* sc, cudaStream_t st);
// P^{-1/2}-type or P^{-1}-type apply of App. C.2 in three launches:
//   utv: part = U^T v (per chunk); coef: small FP64 work; apply: out = alpha v + U coef.
// kInvUnit and kRayleighEta are the powering steps of Alg. 5 (single-RHS applies only).
enum ApplyMode { kInvSqrt = 0, kInvSqrtNormalised = 1, kInv = 2, kInvUnit = 3, kRayleighEta = 4 };
cudaError_t launch_woodbury_apply(CoreBufs& cb, int mode, const float* v, int s, float* out,
                                  bool want_sq, bool want_dot, const float* dotv, DevScalars* sc,
                                  cudaStream_t st);
cudaError_t launch_set_eta(CoreBufs& cb, DevScalars* sc, int identity, cudaStream_t st);
// One single-RHS Woodbury apply (kInvSqrtNormalised or kInv): two whole-GPU launches.
cudaError_t launch_wb_single(CoreBufs& cb, int mode, const float* v, float* out, DevScalars* sc, cudaStream_t st);
// Arguments of one two-launch Woodbury apply (core.cu), and the grouped form:
// the applies of several systems (g: device array) in one pair of launches of
// max_chunks x ngrp blocks (max_chunks >= every g[i].nchunk); all share `mode`.
struct WbArgs {
  const float* U;
  int64_t b;
  int r;
  int mode;
  const float* v;       // input rows (kInvSqrtNormalised, kInv)
  const float* part;    // nsplit x b partial products (kInvUnit, kRayleighEta)
  int nsplit;
  const float* a;       // current powering iterate
  float lam;
  float* hbuf;          // b floats: h of the powering step, for launch B
  const double* keep;
  const float* Minv;
  const float* Gu;      // U^T U (FP32)
  const double* S;
  const double* cis;
  DevScalars* sc;
  float* out;
  float* wpart;         // nchunk x kWbSlotsP partials (16-byte aligned)
  float* wcoef;         // coef[0..r) and alpha at [kMaxRank] (written by the last block of launch A)
  unsigned int* count;  // blocks of launch A done (reset by its last block)
  int nchunk;
  int64_t per;          // rows per chunk
};
WbArgs wb_args_single(CoreBufs& cb, int mode, const float* v, float* out, DevScalars* sc);
WbArgs wb_args_power(CoreBufs& cb, int mode, const float* part, int nsplit, float lam, const float* acur,
                     float* hbuf, float* anext, DevScalars* sc);
// start: device prefix sums of the systems' chunk counts (ngrp + 1 entries, the last = nblocks)
cudaError_t launch_wb_grouped(const WbArgs* g, const int* start, int ngrp, int nblocks, int mode, cudaStream_t st);
// One powering step of Alg. 5 on h = sum_p part[p] + lam * acur (nsplit x b partials):
//   kInvUnit:     anext = P^{-1} h / sqrt(h^T P^{-1} h)  (h kept in hbuf)
//   kRayleighEta: sc->lam_hat = acur . h, sc->eta = 1 / lam_hat
cudaError_t launch_power_step(CoreBufs& cb, int mode, const float* part, int nsplit, float lam, const float* acur,
                              float* hbuf, float* anext, DevScalars* sc, cudaStream_t st);
cudaError_t launch_nesterov(float* W, float* V, float* Z, int64_t count, float beta, float alpha,
                            int literal, cudaStream_t st);
cudaError_t launch_scatter(float* W, float* V, float* Z, const int* B, int64_t b, int s,
                           const float* D, float gamma, float alpha, int literal, DevScalars* sc,
                           cudaStream_t st);
cudaError_t launch_tail_add(const float* W, float* Wbar, int64_t count, cudaStream_t st);
cudaError_t launch_tail_finish(const float* Wbar, float* W, int64_t count, float inv, cudaStream_t st);
cudaError_t launch_sum_blocks(const double* parts, int count, double* dst, cudaStream_t st);
cudaError_t launch_sum_blocks_add(const double* parts, int count, double* dst, cudaStream_t st);   // *dst += sum
cudaError_t launch_trace(DevScalars* sc, double* trace, cudaStream_t st);
cudaError_t launch_tick(DevScalars* sc, cudaStream_t st);
cudaError_t launch_scale_copy(const float* src, float* dst, int64_t count, cudaStream_t st);
cudaError_t launch_adj_reduce(const float* part, int nsplit, int64_t m, int s, const float* G,
                              int64_t ldg, int coff, double* blockacc, cudaStream_t st);

}  // namespace adasap
