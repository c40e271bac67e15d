// Block-row kernel product on the 5th-generation tensor cores (tcgen05 + TMEM).
//
// The same product as k_rows_narrow (Alg. 2 Step I, K_Bn w; the K_BB v products
// of Alg. 5; the posterior mean), with the squared distances formed by MMAs:
//   a_i = [-2 x'_i, q_i, 1, 0...],  b_j = [x'_j, 1, q_j, 0...]   (K = KP >= d + 2)
//   u_ij = a_i . b_j = q_i + q_j - 2 x'_i . x'_j = ||x'_i - x'_j||^2
// FP32 accuracy is recovered with a TF32 hi/lo split of both operands and three
// MMAs, hi.hi + hi.lo + lo.hi (the dropped lo.lo term is 2^-22 relative); a
// row paired with its own column (the diagonal of K_BB / K_Bn) gets u = 0.
//
// CTA = 128 rows x a column range, 640 threads, persistent over (row tile,
// column split) items, or over equal runs of tiles (the flat schedule, for
// small products):
//   warp 0       copy producer: bulk copies (cp.async.bulk, the TMA engine) of
//                128-column operand tiles into an 8-stage shared-memory ring
//                (5 at KP = 32), as fast as the MMAs free the stages
//   warps 1, 3   MMA issuers, one thread each: warp 1 the even tiles, warp 3 the
//                odd ones (tcgen05.mma kind::tf32, M = 128, N = 128, K = 8 per
//                instruction); warp 1 owns the TMEM allocation (4 x 128 FP32
//                distance columns, the whole TMEM).  One issuer spent about as long
//                in its two barrier waits per tile as in issuing the tile's six
//                MMAs, so the tensor pipe idled half the time.
//   warp 2       w producer: the w values of each tile (loaded two tiles ahead)
//                into an 8-stage w ring, twice as deep as the TMEM ring, so that
//                the w of a tile is in place before its TMEM buffer is
//   warps 4..19  epilogue in four groups of four warps: group g takes every
//                fourth tile (TMEM buffer g); warp w tcgen05.ld-s the 32 rows of
//                TMEM lane quadrant w % 4, all 128 columns, releases the buffer
//                once its last load has landed, applies the RBF / Matern
//                epilogue and contracts with w in registers
// (One warp staging both the copies and w gated every tile on that warp's
// serial chain of barrier waits, copy issues and w stores: about 1,500 clocks
// per tile, three times the special-function pipe's time for an RBF tile.)
// Operands live in shared memory in the no-swizzle K-major canonical layout:
// 8-row core groups of 16-byte K chunks (LBO = 128 B between K chunks,
// SBO = 32 * KP B between 8-row groups).  The column operands are prebuilt in
// that layout in global memory (padded to a multiple of 128 rows), so a tile
// is one contiguous copy.  Every mbarrier wait is bounded: on timeout the CTA
// raises an error flag, drains its own copies and MMAs, frees TMEM and writes
// NaN partials.  The grouped form takes the items of several independent
// products (for example the block-row products of many GP systems) in one
// launch.
#include <algorithm>
#include <vector>

#include "prep.cuh"
#include "tc_ptx.cuh"

namespace adasap {

// Epilogue: 16 warps, warp w covering TMEM lane quadrant w % 4 and the 32-column
// group (w - 4) / 4 of every 128-column tile.
constexpr int kTcEpiWarps = 16;
constexpr int kTcThreadsV2 = 32 * (4 + kTcEpiWarps);   // producer, MMA, 2 idle, epilogue
constexpr int kTcWArrays = 3;                          // w, w / log2e, w / (3 log2e^2)

constexpr int kTcBufs = 4;                             // TMEM distance buffers
constexpr int kTcWStages = 2 * kTcBufs;                // w ring
constexpr int kTcWPre = 4;                             // tiles of w held in registers ahead of the ring
constexpr uint32_t kTcTmemCols = kTcBufs * kTcN;       // 512: the whole TMEM of the SM

template <int KP>
struct TcSmem {
  static constexpr int OPF = kTcM * KP;  // floats per 128-row operand tile
  // column-operand ring depth: copies are issued this many tiles ahead of the MMAs,
  // enough to cover the copy latency under load (shared memory: 8 x 16 KB at KP = 16,
  // 5 x 32 KB at KP = 32)
  static constexpr int kStages = KP == 16 ? 8 : 5;
  static constexpr size_t ops_bytes = (size_t)(2 + 2 * kStages) * OPF * sizeof(float);
  static constexpr size_t w_bytes = (size_t)kTcWStages * kTcWArrays * kTcN * sizeof(float);   // [stage][array][128]
  static constexpr size_t red_bytes = (size_t)4 * kTcM * sizeof(float);                   // column-group partials
  static constexpr size_t bytes = ops_bytes + w_bytes + red_bytes + 64 * sizeof(uint64_t) + 64 + 1024;
};

// Matern epilogues: of every 8 consecutive entries of a chunk, this many take
// their square root on the FMA pipe (sqrt_fma) instead of the special-function
// unit, whose sqrt issues at half its ex2 rate on this GPU (15.8 against 31.5 per
// SM per clock): per entry that unit then needs (1 - k/8)/15.8 + 1/31.5 clocks
// instead of 1/15.8 + 1/31.5, for about fourteen more issued instructions per
// moved sqrt.  Measured on the Step I launch (10^4 x 2^20 entries): Matern-3/2
// 4.02 ms at k = 0, 3.85 at k = 1, 4.03 at k = 2; Matern-5/2, whose epilogue
// issues more instructions per entry, 4.14 at k = 0 and 1 and slower above.
// With the Newton steps of two entries packed into f32x2 instructions (half the
// issue cost per moved sqrt) k = 2 measured 3.84 against 3.86 ms and k = 3, 4
// slower: past one in eight the kernel is not bound by one pipe but by how well
// its 4 epilogue warps per scheduler hide the special-function latency.
template <int KERN>
__host__ __device__ constexpr int sqrt_fma_per8() { return KERN == ADASAP_MATERN32 ? 1 : 0; }

// Per-entry epilogue on the scaled distance v = log2(e)^2 u (M32, M52) or u (RBF),
// accumulating k(u) w / sigma2 into acc; wl = w / log2(e), w3 = w / (3 log2(e)^2):
//   RBF  k = 2^-u
//   M32  k = (1 + a) e^-a   = 2^-a' (1 + a' / log2 e),              a' = sqrt(v)
//   M52  k = (1 + a + a^2/3) e^-a = 2^-a' (1 + a'/log2 e + a'^2 / (3 log2^2 e))
// sw: a' from sqrt_fma (FMA pipe) instead of sqrt.approx (special-function unit);
// a compile-time constant at every call (unrolled loops).
template <int KERN>
__device__ __forceinline__ float tc_term(float v, float w, float wl, float w3, float acc, bool sw = false) {
  // RBF: for a near-duplicate pair u may come out below 0 by the rounding of q_i + q_j - 2 x_i.x_j
  // (about 2^-22 (q_i + q_j)); 2^{-u} is then 1 + O(1e-6), inside the product's tolerance, so the
  // RBF term needs no clamp
  if (KERN == ADASAP_RBF) return fmaf(ex2_approx(-v), w, acc);
  const float ap = sw ? sqrt_fma(v) : sqrt_approx(fmaxf(v, 0.0f));   // a' (clamped at 0 or 1e-30)
  const float e = ex2_approx(-ap);
  if (KERN == ADASAP_MATERN32) return fmaf(e, fmaf(ap, wl, w), acc);
  return fmaf(e, fmaf(ap, fmaf(ap, w3, wl), w), acc);
}

// Epilogue of one 128 x 128 distance tile for one warp: its 32 rows (one TMEM lane
// quadrant, tq) against the tile's 128 columns, as four 32-column TMEM loads; the
// tile's w arrays start at wt.  After the last load has landed the distance
// buffer is released to the MMA issuers (tempty).  Returns this thread's sum of
// k(u) w / sigma2 over the tile.
//
// RBF takes one of two forms per tile, chosen by one vote of the warp:
// Fast form: no column of the tile is a row's own point, so every entry goes
// through tc_term unchanged, summed into four independent chains (with one
// special-function op and one FMA per entry, a single chain leaves the FMA
// latency exposed), two loads' worth of code unrolled.  Against a test of
// every 32-column chunk this cut the instructions per entry from 4.25 to 3.6
// and the Step I launch (10^4 x 2^20 entries) from 2.05 to 1.72 ms.
template <int KERN>
__host__ __device__ constexpr int tc_fast_chains() { return KERN == ADASAP_RBF ? 4 : 1; }

template <int KERN>
__device__ __forceinline__ float tc_tile_fast(uint32_t tq, const float* __restrict__ wt, uint64_t* tempty_bar,
                                              int lane) {
  constexpr int NC = tc_fast_chains<KERN>();
  float ta[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll(KERN == ADASAP_RBF ? 2 : 1)
  for (int cc = 0; cc < kTcN / 32; ++cc) {
    uint32_t u[32];
    TMEM_LD32(tq + (uint32_t)(cc * 32), u);
    TMEM_WAIT32(u);
    if (cc == kTcN / 32 - 1) {
      // the last load of the tile has landed: the distance buffer is free for the next MMA
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty_bar);
    }
    const float* wst = wt + cc * 32;
#pragma unroll
    for (int i4 = 0; i4 < 8; ++i4) {
      const float4 w4 = *reinterpret_cast<const float4*>(wst + 4 * i4);
      float4 l4 = w4, t4 = w4;
      if (KERN != ADASAP_RBF) l4 = *reinterpret_cast<const float4*>(wst + kTcN + 4 * i4);
      if (KERN == ADASAP_MATERN52) t4 = *reinterpret_cast<const float4*>(wst + 2 * kTcN + 4 * i4);
      // entry 4 i4 + e of the chunk; (4 i4 + e) % 8 < sqrt_fma_per8 takes the FMA-pipe sqrt
      const int h = 4 * (i4 & 1);
      ta[0 % NC] = tc_term<KERN>(__uint_as_float(u[4 * i4 + 0]), w4.x, l4.x, t4.x, ta[0 % NC], h + 0 < sqrt_fma_per8<KERN>());
      ta[1 % NC] = tc_term<KERN>(__uint_as_float(u[4 * i4 + 1]), w4.y, l4.y, t4.y, ta[1 % NC], h + 1 < sqrt_fma_per8<KERN>());
      ta[2 % NC] = tc_term<KERN>(__uint_as_float(u[4 * i4 + 2]), w4.z, l4.z, t4.z, ta[2 % NC], h + 2 < sqrt_fma_per8<KERN>());
      ta[3 % NC] = tc_term<KERN>(__uint_as_float(u[4 * i4 + 3]), w4.w, l4.w, t4.w, ta[3 % NC], h + 3 < sqrt_fma_per8<KERN>());
    }
  }
  return NC == 1 ? ta[0] : (ta[0] + ta[1]) + (ta[2] + ta[3]);
}

// Self form: the tile holds the own point gi (a global column index, -1 for none)
// of at least one of the warp's rows; that entry is taken at u = 0 exactly (the
// split distance leaves a rounding residue of about 2^-22 (q_i + q_j) there).
// Such tiles are rare: one row tile in ctiles for a product of a point set with
// itself, about 32 * 128 / n of the tiles for gathered rows against all n points.
template <int KERN>
__device__ __forceinline__ float tc_tile_self(uint32_t tq, const float* __restrict__ wt, uint64_t* tempty_bar,
                                           int lane, int64_t jt, int64_t gi) {
  float ta = 0.0f;
#pragma unroll 1
  for (int cc = 0; cc < kTcN / 32; ++cc) {
    uint32_t u[32];
    TMEM_LD32(tq + (uint32_t)(cc * 32), u);
    TMEM_WAIT32(u);
    if (cc == kTcN / 32 - 1) {
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty_bar);
    }
    const float* wst = wt + cc * 32;
    const int64_t jb = jt + cc * 32;
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      const float v = (jb + i == gi) ? 0.0f : __uint_as_float(u[i]);
      ta = tc_term<KERN>(v, wst[i], wst[kTcN + i], wst[2 * kTcN + i], ta);
    }
  }
  return ta;
}

// Matern epilogues: one chain and a test of every 32-column chunk for the rows'
// own points (same u = 0 rule).  Their two special-function ops per entry hide
// the chain's latency, and this form measured faster for them than the
// per-tile choice above (Matern-3/2 Step I, 10^4 x 2^20 entries: 3.87 against
// 4.07 ms).
template <int KERN>
__device__ __forceinline__ float tc_tile_chunked(uint32_t tq, const float* __restrict__ wt, uint64_t* tempty_bar,
                                                 int lane, int64_t jt, int64_t gi) {
  float ta = 0.0f;
#pragma unroll 1
  for (int cc = 0; cc < kTcN / 32; ++cc) {
    uint32_t u[32];
    TMEM_LD32(tq + (uint32_t)(cc * 32), u);
    TMEM_WAIT32(u);
    if (cc == kTcN / 32 - 1) {
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty_bar);
    }
    const float* wst = wt + cc * 32;
    const int64_t jb = jt + cc * 32;
    if (__any_sync(0xffffffffu, gi >= jb && gi < jb + 32)) {
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const float v = (jb + i == gi) ? 0.0f : __uint_as_float(u[i]);
        ta = tc_term<KERN>(v, wst[i], wst[kTcN + i], wst[2 * kTcN + i], ta);
      }
    } else {
#pragma unroll
      for (int i4 = 0; i4 < 8; ++i4) {
        const float4 w4 = *reinterpret_cast<const float4*>(wst + 4 * i4);
        const float4 l4 = *reinterpret_cast<const float4*>(wst + kTcN + 4 * i4);
        float4 t4 = w4;
        if (KERN == ADASAP_MATERN52) t4 = *reinterpret_cast<const float4*>(wst + 2 * kTcN + 4 * i4);
        // entry 4 i4 + e of the chunk; (4 i4 + e) % 8 < sqrt_fma_per8 takes the FMA-pipe sqrt
        const int h = 4 * (i4 & 1);
        ta = tc_term<KERN>(__uint_as_float(u[4 * i4 + 0]), w4.x, l4.x, t4.x, ta, h + 0 < sqrt_fma_per8<KERN>());
        ta = tc_term<KERN>(__uint_as_float(u[4 * i4 + 1]), w4.y, l4.y, t4.y, ta, h + 1 < sqrt_fma_per8<KERN>());
        ta = tc_term<KERN>(__uint_as_float(u[4 * i4 + 2]), w4.z, l4.z, t4.z, ta, h + 2 < sqrt_fma_per8<KERN>());
        ta = tc_term<KERN>(__uint_as_float(u[4 * i4 + 3]), w4.w, l4.w, t4.w, ta, h + 3 < sqrt_fma_per8<KERN>());
      }
    }
  }
  return ta;
}

// One run of the flat schedule: CTA x of G takes the flattened tiles
// [x T / G, (x + 1) T / G) of the row-tile-major sequence of all T tiles
// (ctiles per row tile); the run starting at fpos (< fend, the end of the
// share) lies in row tile `rtile`, covers its column tiles [tb, te), writes
// partial slot x - (first CTA of the row tile) -- the largest y with
// y T / G <= rtile * ctiles -- and ends the row tile when te == ctiles.
struct TcFlatRun {
  int64_t rtile, tb, te, slot;
  bool row_end;
};
__host__ __device__ __forceinline__ TcFlatRun tc_flat_run(int64_t x, int64_t G, int64_t T, int64_t ctiles,
                                                          int64_t fpos, int64_t fend) {
  TcFlatRun run;
  run.rtile = fpos / ctiles;
  run.tb = fpos % ctiles;
  run.te = run.tb + (fend - fpos) < ctiles ? run.tb + (fend - fpos) : ctiles;
  run.slot = x - ((run.rtile * ctiles + 1) * G - 1) / T;
  run.row_end = run.te == ctiles;
  return run;
}

// GROUPED: the items of several independent products (one TcArgs each; item
// ranges gstart[g] .. gstart[g + 1]) in one persistent launch.
template <int KERN, int KP, bool GROUPED>
__global__ void __launch_bounds__(kTcThreadsV2, 1)
    k_rows_tc(TcArgs a0, const TcArgs* __restrict__ grp, const int64_t* __restrict__ gstart, int ngrp) {
  using L = TcSmem<KP>;
  constexpr int OPF = L::OPF;
  constexpr int kTcStages = L::kStages;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
  float* sAhi = reinterpret_cast<float*>(base);
  float* sAlo = sAhi + OPF;
  float* sB = sAlo + OPF;  // [stage][hi, lo][OPF]
  float* sw = reinterpret_cast<float*>(base + L::ops_bytes);                 // [stage][array][128]
  float* red = reinterpret_cast<float*>(base + L::ops_bytes + L::w_bytes);   // [group][128]
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + L::ops_bytes + L::w_bytes + L::red_bytes);
  uint64_t* full = bars;                     // [kTcStages] column tiles landed (copies)
  uint64_t* empty = bars + kTcStages;        // [kTcStages] column tile stage consumed by the MMAs
  uint64_t* tfull = bars + 2 * kTcStages;    // [kTcBufs] distance buffer ready
  uint64_t* tempty = tfull + kTcBufs;        // [kTcBufs] distance buffer read (4 epilogue warps)
  uint64_t* wfull = tfull + 2 * kTcBufs;     // [kTcWStages] w stage written
  uint64_t* wempty = wfull + kTcWStages;     // [kTcWStages] w stage read (4 epilogue warps)
  uint64_t* drain = wempty + kTcWStages;     // [2] one per MMA issuer
  uint32_t* tslot = reinterpret_cast<uint32_t*>(drain + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // the row operand carries log2(e)^2 for the Matern kernels (see tc_term)
  const float rscale = (KERN == ADASAP_RBF) ? 1.0f : kLog2e * kLog2e;

  // ---- set-up once per CTA: barriers, TMEM --------------------------------------
  if (tid == 0) {
    for (int i = 0; i < kTcStages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < kTcBufs; ++i) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], kTcEpiWarps / kTcBufs);   // the four warps of group i
    }
    for (int i = 0; i < kTcWStages; ++i) {
      mbar_init(&wfull[i], 1);
      mbar_init(&wempty[i], kTcEpiWarps / kTcBufs);   // the four warps of the group taking that tile
    }
    mbar_init(&drain[0], 1);
    mbar_init(&drain[1], 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(kTcTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;
  // the item count only after the set-up (with it before the barrier the Matern
  // instantiations measured 1.6% slower)
  const int64_t nitems = GROUPED ? gstart[ngrp] : (a0.m + kTcM - 1) / kTcM * a0.nsplit;

  // Items (row tile, column split) are taken in grid-stride order with the row
  // tile varying fastest, so the CTAs running at one time share column tiles in
  // L2 (grouped launches with counters: the same global order, each CTA's items
  // after its first from the counter).  The pipeline phases run on across items
  // (gt counts this CTA's tiles).
  uint32_t gt = 0, ndrain = 0;
  // Flat mode (one product): CTA x takes the tiles [x T / G, (x + 1) T / G) of the
  // row-tile-major sequence of all T tiles (G CTAs, T >= G), as runs within one
  // row tile each.  A run's partials go to slot x - (first CTA of its row tile);
  // the CTA that ends a row tile zeroes the slots after its own, so every slot
  // of every row is written.
  const bool flat = !GROUPED && a0.flat;
  // grouped launches with counters: items after the first from the shared counter
  // (the same items in the same global order, so the outputs are unchanged)
  const bool dyn = GROUPED && a0.sched != nullptr;
  __shared__ int64_t s_next;
  const int64_t ctiles = (a0.ncols + kTcN - 1) / kTcN;
  const int64_t ftotal = flat ? (a0.m + kTcM - 1) / kTcM * ctiles : 0;
  int64_t fpos = flat ? (int64_t)blockIdx.x * ftotal / gridDim.x : 0;
  const int64_t fend = flat ? ((int64_t)blockIdx.x + 1) * ftotal / gridDim.x : 0;
  for (int64_t item = blockIdx.x; flat ? fpos < fend : item < nitems;
       item = dyn ? s_next : item + gridDim.x) {
    int sys = 0;
    if (GROUPED) {  // the product this item belongs to: last g with gstart[g] <= item
      int hi = ngrp - 1;
      while (sys < hi) {
        const int mid = (sys + hi + 1) >> 1;
        if (gstart[mid] <= item) sys = mid;
        else hi = mid - 1;
      }
    }
    const TcArgs& a = GROUPED ? grp[sys] : a0;
    const int64_t li = GROUPED ? item - gstart[sys] : item;
    const int64_t rtiles = (a.m + kTcM - 1) / kTcM;
    int64_t rtile, split, c0, c1;
    bool row_end = false;
    if (flat) {
      const TcFlatRun run = tc_flat_run(blockIdx.x, gridDim.x, ftotal, ctiles, fpos, fend);
      rtile = run.rtile;
      split = run.slot;
      c0 = run.tb * kTcN;
      c1 = min(a.ncols, run.te * kTcN);
      row_end = run.row_end;
      fpos += run.te - run.tb;
    } else {
      rtile = li % rtiles;
      split = li / rtiles;
      c0 = split * a.cps;
      c1 = min(a.ncols, c0 + a.cps);
    }
    const int64_t row0 = rtile * kTcM;
    // after an abort the remaining items only write NaN partials (the flag is read
    // after a block barrier, so every role agrees)
    const int ntiles = (c1 > c0 && !*abort_flag) ? (int)((c1 - c0 + kTcN - 1) / kTcN) : 0;
    // row operands (hi/lo split) of this item's row tile
    if (tid < kTcM) {
      const int64_t ri = row0 + tid;
      float av[KP];
#pragma unroll
      for (int k = 0; k < KP; ++k) av[k] = 0.0f;
      bool ok = ri < a.m;
      int64_t src = ri;
      if (ok && a.ridx) {
        const int id = a.ridx[ri];
        ok = id >= 0;
        src = id;
      }
      if (ok) {
        for (int k = 0; k < a.d; ++k) av[k] = -2.0f * rscale * a.xr[src * a.dp + k];
        av[a.d] = rscale * a.qr[src];
        av[a.d + 1] = rscale;
      } else {
        av[a.d] = 1e20f;  // padded or invalid row: u is huge, the kernel value 0
        av[a.d + 1] = 1.0f;
      }
#pragma unroll
      for (int k = 0; k < KP; ++k) {
        const float hi = tf32_round(av[k]);
        const float lo = tf32_round(av[k] - hi);
        sAhi[tc_off<KP>(tid, k)] = hi;
        sAlo[tc_off<KP>(tid, k)] = lo;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();

    if (warp == 0) {
      // ---- copy producer: column tiles by bulk copy (lane 0), each as soon as the
      // MMAs have freed its stage ------------------------------------------------------
      if (lane == 0) {
        int xi = 0;  // column tiles issued
        for (; xi < ntiles; ++xi) {
          const uint32_t gx = gt + (uint32_t)xi;
          const int st = gx % kTcStages;
          if (!mbar_wait(&empty[st], ((gx / kTcStages) & 1u) ^ 1u, abort_flag)) {
            *abort_flag = 1;
            tc_note_timeout(a.err, 1);
            break;
          }
          mbar_arrive_expect_tx(&full[st], 2u * OPF * sizeof(float));
          const int64_t off = (c0 + (int64_t)xi * kTcN) * KP;
          bulk_g2s(sB + (st * 2 + 0) * OPF, a.bhi + off, OPF * sizeof(float), &full[st]);
          bulk_g2s(sB + (st * 2 + 1) * OPF, a.blo + off, OPF * sizeof(float), &full[st]);
        }
        if (*abort_flag) {
          // our copies still write shared memory: wait (bounded) for the last ones
          for (int x = max(0, xi - kTcStages); x < xi; ++x) {
            const uint32_t gx = gt + (uint32_t)x;
            mbar_wait(&full[gx % kTcStages], (gx / kTcStages) & 1u, nullptr);
          }
        }
      }
    } else if (warp == 2 && a.wp) {
      // ---- w producer, prepared w: one bulk copy of each tile's w arrays (lane 0)
      // into the w ring, once the epilogue is done with the stage's previous tile -------
      if (lane == 0) {
        constexpr uint32_t wbytes = (KERN == ADASAP_RBF ? 1u : (uint32_t)kTcWArrays) * kTcN * sizeof(float);
        const float* wsrc = a.wp + (c0 / kTcN) * (wbytes / sizeof(float));
        int wi = 0;  // tiles issued
        for (; wi < ntiles; ++wi) {
          const uint32_t g = gt + (uint32_t)wi;
          const int ws = g % kTcWStages;
          if (!mbar_wait(&wempty[ws], ((g / kTcWStages) & 1u) ^ 1u, abort_flag)) {
            *abort_flag = 1;
            tc_note_timeout(a.err, 4);
            break;
          }
          mbar_arrive_expect_tx(&wfull[ws], wbytes);
          bulk_g2s(sw + ws * kTcWArrays * kTcN, wsrc + (int64_t)wi * (wbytes / sizeof(float)), wbytes, &wfull[ws]);
        }
        if (*abort_flag) {
          // our copies still write shared memory: wait (bounded) for the last ones
          for (int x = max(0, wi - kTcWStages); x < wi; ++x) {
            const uint32_t gx = gt + (uint32_t)x;
            mbar_wait(&wfull[gx % kTcWStages], (gx / kTcWStages) & 1u, nullptr);
          }
        }
      }
    } else if (warp == 2) {
      // ---- w producer, w as given (any stride or alignment): w of every tile into
      // the w ring (whole warp), once the epilogue is done with the stage's previous
      // tile (kTcWStages tiles back) -------------------------------------------------
      bool ok = true;
      // w of tile t (zero past the split), loaded kTcWPre tiles ahead so that the
      // global load latency overlaps the waits and stores of the tiles in between
      // (one 16-byte load per lane where w is contiguous and 16-byte aligned)
      const bool vec = a.ldw == 1 && ((reinterpret_cast<uintptr_t>(a.w) & 15u) == 0);
      auto load_w = [&](int t, float (&wv)[4]) {
        const int64_t jb = c0 + (int64_t)t * kTcN + 4 * lane;
        if (vec && t < ntiles && jb + 3 < c1) {
          const float4 q = __ldg(reinterpret_cast<const float4*>(a.w + jb));
          wv[0] = q.x, wv[1] = q.y, wv[2] = q.z, wv[3] = q.w;
          return;
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) wv[e] = (t < ntiles && jb + e < c1) ? __ldg(a.w + (jb + e) * a.ldw) : 0.0f;
      };
      float wq[kTcWPre][4];
#pragma unroll
      for (int k = 0; k < kTcWPre; ++k) load_w(k, wq[k]);
      for (int t = 0; ok && t < ntiles; ++t) {
        const uint32_t g = gt + (uint32_t)t;
        const int ws = g % kTcWStages;
        if (lane == 0) {
          ok = mbar_wait(&wempty[ws], ((g / kTcWStages) & 1u) ^ 1u, abort_flag);
          if (!ok) {
            *abort_flag = 1;
            tc_note_timeout(a.err, 4);
          }
        }
        ok = __shfl_sync(0xffffffffu, (int)ok, 0) != 0;
        if (!ok) break;
        float wv[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          wv[e] = wq[0][e];
#pragma unroll
          for (int k = 0; k + 1 < kTcWPre; ++k) wq[k][e] = wq[k + 1][e];
        }
        load_w(t + kTcWPre, wq[kTcWPre - 1]);
        float* wst = sw + ws * kTcWArrays * kTcN;
        *reinterpret_cast<float4*>(wst + 4 * lane) = make_float4(wv[0], wv[1], wv[2], wv[3]);
        if (KERN != ADASAP_RBF) {
          const float il = 1.0f / kLog2e, i3 = 1.0f / (3.0f * kLog2e * kLog2e);
          *reinterpret_cast<float4*>(wst + kTcN + 4 * lane) =
              make_float4(wv[0] * il, wv[1] * il, wv[2] * il, wv[3] * il);
          *reinterpret_cast<float4*>(wst + 2 * kTcN + 4 * lane) =
              make_float4(wv[0] * i3, wv[1] * i3, wv[2] * i3, wv[3] * i3);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&wfull[ws]);
      }
    } else if (warp == 1 || warp == 3) {
      // ---- MMA issuers: tiles g = gt + t with g % 2 == iss ----------------------------
      const int iss = warp == 1 ? 0 : 1;
      if (lane == 0) {
        int issued = 0;
        for (int t = (int)(((uint32_t)iss + 2u - gt % 2u) % 2u); t < ntiles; t += 2) {
          const uint32_t g = gt + (uint32_t)t;
          const int st = g % kTcStages, buf = g % kTcBufs;
          if (!mbar_wait(&full[st], (g / kTcStages) & 1u, abort_flag) ||
              !mbar_wait(&tempty[buf], ((g / kTcBufs) & 1u) ^ 1u, abort_flag)) {
            *abort_flag = 1;
            tc_note_timeout(a.err, 2);
            break;
          }
          tc_fence_after();
          const uint32_t dt = tbase + (uint32_t)(buf * kTcN);
          const uint32_t a_hi = smem_u32(sAhi), a_lo = smem_u32(sAlo);
          const uint32_t b_hi = smem_u32(sB + (st * 2 + 0) * OPF), b_lo = smem_u32(sB + (st * 2 + 1) * OPF);
          uint32_t acc = 0;
#pragma unroll
          for (int pass = 0; pass < 3; ++pass) {
            const uint32_t A = pass == 2 ? a_lo : a_hi;
            const uint32_t B = pass == 1 ? b_lo : b_hi;
#pragma unroll
            for (int ks = 0; ks < KP / 8; ++ks) {
              tc_mma_tf32(dt, smem_desc(A + 256u * ks, 128u, 32u * KP), smem_desc(B + 256u * ks, 128u, 32u * KP),
                          kIdescTf32, acc);
              acc = 1;
            }
          }
          tc_commit(&empty[st]);
          tc_commit(&tfull[buf]);
          issued = t + 1;
        }
        if (issued > 0) {
          // all MMAs of this issuer in this item complete before the row operands are
          // rewritten (next item) or TMEM is released (end)
          tc_commit(&drain[iss]);
          mbar_wait(&drain[iss], ndrain & 1u, nullptr);
          ++ndrain;
        }
      }
    } else if (warp >= 4) {
      // ---- epilogue: 32 rows (TMEM quadrant) x 32 columns (group) per warp ---------
      const int qd = warp & 3, cg = (warp - 4) >> 2;
      const int rl = qd * 32 + lane;
      const int64_t ri = row0 + rl;
      int64_t gi = -1;
      bool bad = false;
      if (ri < a.m) {
        const int64_t src = a.ridx ? (int64_t)a.ridx[ri] : ri;
        bad = src < 0;
        if (a.self_mode) gi = src;
      }
      float acc = 0.0f, cmp = 0.0f;
      // group cg takes the tiles g = gt + t with g % kTcBufs == cg (TMEM buffer and w
      // stage cg), all 128 columns of its quadrant's rows, so the four groups work
      // on four consecutive tiles at once and one group's TMEM-load latency hides
      // behind the others' arithmetic
      const int t0 = (int)(((uint32_t)cg + kTcBufs - gt % kTcBufs) % kTcBufs);
      for (int t = t0; t < ntiles; t += kTcBufs) {
        const uint32_t gg = gt + (uint32_t)t;
        const uint32_t ph = (gg / kTcBufs) & 1u;
        const int ws = gg % kTcWStages;
        if (!mbar_wait(&tfull[cg], ph, abort_flag) || !mbar_wait(&wfull[ws], (gg / kTcWStages) & 1u, abort_flag)) {
          *abort_flag = 1;
          tc_note_timeout(a.err, 3);
          break;
        }
        tc_fence_after();
        const uint32_t tq = tbase + ((uint32_t)(qd * 32) << 16) + (uint32_t)(cg * kTcN);
        const float* wt = sw + ws * kTcWArrays * kTcN;
        const int64_t jt = c0 + (int64_t)t * kTcN;
        float tacc;
        if (KERN == ADASAP_RBF) {
          // one vote per tile decides whether any of the warp's rows meets its own point here
          tacc = __any_sync(0xffffffffu, gi >= jt && gi < jt + kTcN) ? tc_tile_self<KERN>(tq, wt, &tempty[cg], lane, jt, gi)
                                                                     : tc_tile_fast<KERN>(tq, wt, &tempty[cg], lane);
        } else {
          tacc = tc_tile_chunked<KERN>(tq, wt, &tempty[cg], lane, jt, gi);
        }
        // the w stage of this tile is free again
        __syncwarp();
        if (lane == 0) mbar_arrive(&wempty[ws]);
        const float y = tacc - cmp;
        const float tt = acc + y;
        cmp = (tt - acc) - y;
        acc = tt;
      }
      // combine the four groups' partial sums of each row
      red[cg * kTcM + rl] = acc - cmp;
      asm volatile("bar.sync 1, %0;" ::"r"(32 * kTcEpiWarps) : "memory");
      if (cg == 0 && ri < a.m) {
        // group cg summed the tiles t = cg - gt (mod 4) of this item; under the shared
        // counter the four classes are added in class order, so that the result does
        // not depend on which CTA (and so which gt) took the item
        static_assert(kTcBufs == 4, "four epilogue groups");
        const int c0 = dyn ? (int)(gt % kTcBufs) : 0;
        const float tot = (red[(c0 & 3) * kTcM + rl] + red[((c0 + 1) & 3) * kTcM + rl]) +
                          (red[((c0 + 2) & 3) * kTcM + rl] + red[((c0 + 3) & 3) * kTcM + rl]);
        a.part[split * a.m + ri] = (bad || *abort_flag) ? __int_as_float(0x7fc00000) : a.sigma2 * tot;
        if (row_end)
          for (int64_t s2 = split + 1; s2 < a.nsplit; ++s2) a.part[s2 * a.m + ri] = 0.0f;
      }
    }
    gt += (uint32_t)ntiles;
    if (dyn && tid == 0) s_next = (int64_t)atomicAdd(a0.sched, 1ull) + gridDim.x;
    // item boundary: the row operands, both TMEM buffers and red[] are free again
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  if (dyn && tid == 0) {
    // every CTA has taken its last item when the count of finished CTAs completes:
    // the last one zeroes the counters for the next launch
    __threadfence();
    if (atomicAdd(a0.sched + 1, 1ull) == (unsigned long long)gridDim.x - 1ull) {
      a0.sched[0] = 0ull;
      a0.sched[1] = 0ull;
    }
  }
  if (warp == 0 && lane == 0 && *abort_flag) tc_note_timeout(a0.err, 9);
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(kTcTmemCols) : "memory");
  }
}

// ---------------------------------------------------------------------------
// Split column operands in the canonical layout, npad = multiple of 128 rows:
//   b_j = [x'_j (d), 1, q_j, 0...] for j < n; padding rows [0, 1, 1e20, 0...].
// With gidx, row j takes the point gidx[j] (a gathered block).
template <int KP>
__global__ void k_build_tc(const float* __restrict__ X, const float* __restrict__ q, const int* __restrict__ gidx,
                           int64_t n, int64_t npad, int d, int dp, float* __restrict__ hi, float* __restrict__ lo) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < npad; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t src = j < n ? (gidx ? (int64_t)max(gidx[j], 0) : j) : -1;
    build_tc_row<KP>(X, q, src, d, dp, j, hi, lo);
  }
}

// w per 128-column tile (see launch_prep_w): A arrays of 128 floats per tile
template <int A>
__global__ void k_prep_w(const float* __restrict__ w, int64_t ldw, int64_t ncols, int64_t npad,
                         float* __restrict__ wp) {
  const float il = 1.0f / kLog2e, i3 = 1.0f / (3.0f * kLog2e * kLog2e);
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < npad; j += (int64_t)gridDim.x * blockDim.x) {
    const float v = j < ncols ? w[j * ldw] : 0.0f;
    float* o = wp + (j / kTcN) * (A * kTcN) + (j % kTcN);
    o[0] = v;
    if (A == 3) {
      o[kTcN] = v * il;
      o[2 * kTcN] = v * i3;
    }
  }
}

int tc_kp(int d) { return d + 2 <= 16 ? 16 : (d + 2 <= 32 ? 32 : 0); }
int64_t tc_npad(int64_t n) { return (n + kTcN - 1) / kTcN * kTcN; }

int64_t tc_wprep_floats(int64_t ncols, int kern) {
  return tc_npad(ncols) * (kern == ADASAP_RBF ? 1 : kTcWArrays);
}

cudaError_t launch_prep_w(int kern, const float* w, int64_t ldw, int64_t ncols, float* wp, cudaStream_t st) {
  const int64_t npad = tc_npad(ncols);
  const int blocks = (int)std::min<int64_t>((npad + 255) / 256, 148 * 8);
  if (kern == ADASAP_RBF) k_prep_w<1><<<blocks, 256, 0, st>>>(w, ldw, ncols, npad, wp);
  else k_prep_w<kTcWArrays><<<blocks, 256, 0, st>>>(w, ldw, ncols, npad, wp);
  return cudaGetLastError();
}

cudaError_t launch_build_tc(const float* X, const float* q, const int* gidx, int64_t n, int d, int dp, float* hi,
                            float* lo, cudaStream_t st) {
  const int kp = tc_kp(d);
  const int64_t npad = tc_npad(n);
  const int blocks = (int)std::min<int64_t>((npad + 255) / 256, 148 * 8);
  if (kp == 16) k_build_tc<16><<<blocks, 256, 0, st>>>(X, q, gidx, n, npad, d, dp, hi, lo);
  else if (kp == 32) k_build_tc<32><<<blocks, 256, 0, st>>>(X, q, gidx, n, npad, d, dp, hi, lo);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

static int g_tc_slots = 0;  // resident CTAs of k_rows_tc per SM x SMs

template <int KERN, int KP>
static cudaError_t tc_setup() {
  const int bytes = (int)std::max<size_t>(TcSmem<KP>::bytes, 80 * 1024);
  cudaError_t e = cudaFuncSetAttribute(k_rows_tc<KERN, KP, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_rows_tc<KERN, KP, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t tc_init() {
  cudaError_t e;
  if ((e = tc_setup<0, 16>()) || (e = tc_setup<1, 16>()) || (e = tc_setup<2, 16>()) || (e = tc_setup<0, 32>()) ||
      (e = tc_setup<1, 32>()) || (e = tc_setup<2, 32>()))
    return e;
  int per_sm = 0, dev = 0, sms = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rows_tc<1, 16, false>, kTcThreadsV2,
                                                         std::max<size_t>(TcSmem<16>::bytes, 80 * 1024))))
    return e;
  if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))) return e;
  g_tc_slots = std::max(1, per_sm) * sms;
  return cudaSuccess;
}

// Column splits: whole 128-column tiles; items (row tile x split) are spread
// over min(slots, max_ctas) persistent CTAs.
int tc_slots() { return g_tc_slots > 0 ? g_tc_slots : 148; }

int tc_nsplit(int64_t m, int64_t ncols, int max_ctas) {
  const int64_t rt = (m + kTcM - 1) / kTcM;
  const int64_t tiles = (ncols + kTcN - 1) / kTcN;
  const int64_t slots = (max_ctas > 0 && max_ctas < tc_slots()) ? max_ctas : tc_slots();
  // An item costs its column tiles plus a start-up of about two tiles (row
  // operands, pipeline fill and drain); minimise items per CTA x item cost.
  constexpr double kStartupTiles = 2.0;
  int64_t best = 1;
  double best_cost = 1e300;
  for (int64_t ns = 1; ns <= std::min<int64_t>(tiles, 4096); ++ns) {
    const int64_t tot = rt * ns;
    const int64_t waves = (tot + slots - 1) / slots;
    if (waves > 64) break;
    const int64_t tps = (tiles + ns - 1) / ns;
    const double cost = (double)waves * ((double)tps + kStartupTiles);
    if (cost < best_cost - 1e-9) {
      best_cost = cost;
      best = ns;
    }
  }
  return (int)best;
}

// Flat mode (see the kernel): the partial slots a row needs when the T tiles of
// the product are cut into G equal runs, or 0 when that is not cheaper than the
// best (row tile x split) items (same cost model: a run costs its tiles plus a
// start-up of two tiles; a CTA's share meets at most ceil((P - 1) / tiles) + 1
// row tiles, and a row tile at most 1 + ceil((tiles - 1) / floor(T / G)) CTAs).
// Only for products of at most 64 tiles per CTA: with more, the item order (row
// tile fastest) lets the CTAs running at one time share column tiles in L2,
// which equal runs give up, and the waves it rounds to cost little.
int tc_flat_slots(int64_t m, int64_t ncols, int max_ctas) {
  const int64_t rt = (m + kTcM - 1) / kTcM;
  const int64_t tiles = (ncols + kTcN - 1) / kTcN;
  const int64_t G = (max_ctas > 0 && max_ctas < tc_slots()) ? max_ctas : tc_slots();
  const int64_t T = rt * tiles;
  if (T < 2 * G || T > 64 * G) return 0;
  const int64_t P = (T + G - 1) / G, pmin = T / G;
  const double flat_cost = (double)P + 2.0 * (double)((P - 1 + tiles - 1) / tiles + 1);
  const int64_t ns = tc_nsplit(m, ncols, max_ctas);
  const double gs_cost = (double)((rt * ns + G - 1) / G) * ((double)((tiles + ns - 1) / ns) + 2.0);
  if (!(flat_cost < gs_cost)) return 0;
  return (int)std::min<int64_t>(G, 1 + (tiles - 1 + pmin - 1) / pmin);
}

int tc_plan_nsplit(int64_t m, int64_t ncols, int max_ctas) {
  const int fs = tc_flat_slots(m, ncols, max_ctas);
  return fs > 0 ? fs : tc_nsplit(m, ncols, max_ctas);
}

// Host walk of the schedule launch_rows_tc takes for an m x ncols product on
// min(slots, max_ctas) CTAs: with the flat schedule every tile must be covered
// once and every (row tile, slot) written once, through the kernel's own run
// decoding (tc_flat_run).
int tc_schedule_check(int64_t m, int64_t ncols, int max_ctas, int* nsplit, int* flat) {
  const int ns = tc_plan_nsplit(m, ncols, max_ctas);
  const int fs = tc_flat_slots(m, ncols, max_ctas);
  *nsplit = ns;
  *flat = fs > 0 && ns == fs;
  if (!*flat) return 0;  // items (row tile, split): item li writes slot li / rtiles of its rows
  const int64_t rt = (m + kTcM - 1) / kTcM, ctiles = (ncols + kTcN - 1) / kTcN, T = rt * ctiles;
  const int64_t G = (max_ctas > 0 && max_ctas < tc_slots()) ? max_ctas : tc_slots();
  std::vector<int> tiles((size_t)T, 0), slots((size_t)(rt * ns), 0);
  for (int64_t x = 0; x < G; ++x) {
    int64_t fpos = x * T / G;
    const int64_t fend = (x + 1) * T / G;
    if (fend <= fpos) return 1;  // a CTA without tiles would leave its slot unwritten
    while (fpos < fend) {
      const TcFlatRun run = tc_flat_run(x, G, T, ctiles, fpos, fend);
      if (run.slot < 0 || run.slot >= ns || run.te <= run.tb) return 2;
      for (int64_t t = run.tb; t < run.te; ++t) ++tiles[(size_t)(run.rtile * ctiles + t)];
      ++slots[(size_t)(run.rtile * ns + run.slot)];
      if (run.row_end)
        for (int64_t s2 = run.slot + 1; s2 < ns; ++s2) ++slots[(size_t)(run.rtile * ns + s2)];
      fpos += run.te - run.tb;
    }
  }
  for (int c : tiles)
    if (c != 1) return 3;
  for (int c : slots)
    if (c != 1) return 4;
  return 0;
}

template <int KERN, int KP, bool G>
static cudaError_t launch_tc_k(const TcArgs& a, const TcArgs* grp, const int64_t* gstart, int ngrp, int ctas,
                               cudaStream_t st) {
  k_rows_tc<KERN, KP, G><<<ctas, kTcThreadsV2, std::max<size_t>(TcSmem<KP>::bytes, 80 * 1024), st>>>(a, grp, gstart,
                                                                                                     ngrp);
  return cudaGetLastError();
}

template <bool G>
static cudaError_t launch_tc_any(int kern, int kp, const TcArgs& a, const TcArgs* grp, const int64_t* gstart,
                                 int ngrp, int ctas, cudaStream_t st) {
  if (kp == 16) {
    if (kern == 0) return launch_tc_k<0, 16, G>(a, grp, gstart, ngrp, ctas, st);
    if (kern == 1) return launch_tc_k<1, 16, G>(a, grp, gstart, ngrp, ctas, st);
    return launch_tc_k<2, 16, G>(a, grp, gstart, ngrp, ctas, st);
  }
  if (kp == 32) {
    if (kern == 0) return launch_tc_k<0, 32, G>(a, grp, gstart, ngrp, ctas, st);
    if (kern == 1) return launch_tc_k<1, 32, G>(a, grp, gstart, ngrp, ctas, st);
    return launch_tc_k<2, 32, G>(a, grp, gstart, ngrp, ctas, st);
  }
  return cudaErrorInvalidValue;
}

TcArgs make_tc_args(int d, const float* xr, const float* qr, const int* ridx, int64_t m, int dp, const float* bhi,
                    const float* blo, int64_t ncols, int self_mode, const float* w, int64_t ldw, float* part,
                    int nsplit, float sigma2, int* err) {
  TcArgs a;
  a.xr = xr; a.qr = qr; a.ridx = ridx; a.m = m; a.dp = dp; a.d = d;
  a.bhi = bhi; a.blo = blo; a.ncols = ncols; a.self_mode = self_mode;
  a.w = w; a.ldw = ldw; a.part = part; a.sigma2 = sigma2; a.err = err;
  const int64_t tiles = (ncols + kTcN - 1) / kTcN;
  a.cps = (tiles + nsplit - 1) / nsplit * kTcN;
  a.nsplit = nsplit;
  a.flat = 0;
  a.wp = nullptr;
  a.sched = nullptr;
  return a;
}

int64_t tc_items(const TcArgs& a) { return (a.m + kTcM - 1) / kTcM * (int64_t)a.nsplit; }

cudaError_t launch_rows_tc(int kern, int d, const float* xr, const float* qr, const int* ridx, int64_t m, int dp,
                           const float* bhi, const float* blo, int64_t ncols, int self_mode, const float* w,
                           int64_t ldw, float* part, int nsplit, float sigma2, int* err, cudaStream_t st,
                           int max_ctas, const float* wp) {
  if (m <= 0 || ncols <= 0) return cudaSuccess;
  TcArgs a = make_tc_args(d, xr, qr, ridx, m, dp, bhi, blo, ncols, self_mode, w, ldw, part, nsplit, sigma2, err);
  a.wp = wp;
  const int slots = (max_ctas > 0 && max_ctas < tc_slots()) ? max_ctas : tc_slots();
  int ctas = (int)std::min<int64_t>(tc_items(a), slots);
  // the flat schedule when the caller's slot count is the one it needs (either
  // schedule writes every slot of every row)
  const int fs = tc_flat_slots(m, ncols, max_ctas);
  if (fs > 0 && nsplit == fs) {
    a.flat = 1;
    ctas = slots;
  }
  return launch_tc_any<false>(kern, tc_kp(d), a, nullptr, nullptr, 0, ctas, st);
}

cudaError_t launch_rows_tc_grouped(int kern, int kp, const TcArgs* grp, const int64_t* gstart, int ngrp,
                                   int64_t nitems, int* err, int ctas, cudaStream_t st, unsigned long long* sched) {
  if (ngrp < 1 || nitems <= 0) return cudaSuccess;
  TcArgs a0 = {};
  a0.err = err;
  a0.sched = sched;
  return launch_tc_any<true>(kern, kp, a0, grp, gstart, ngrp, (int)std::min<int64_t>(nitems, ctas), st);
}

}  // namespace adasap
