// Multi-right-hand-side block-row product on the 5th-generation tensor cores:
//   part[p][i][c] = sigma2 * sum_{j in split p} k(x'_{row i}, x'_j) W[j][c],   c < s, 2 <= s <= 128
// (Alg. 2 Step I with s columns, the Step II sketch K_BB Omega with s = r, the
// posterior mean of s samples).  Both contractions run on the tensor cores:
//   1. squared distances of a 128 x 128 tile by the TF32-split MMAs of
//      rows_tc.cu (a_i = [-2 x'_i, q_i, 1], b_j = [x'_j, 1, q_j]) into TMEM;
//   2. the epilogue warps turn them into kernel values, split those into TF32
//      hi/lo and store them as 32-column chunks in shared memory (the A operand
//      of a second MMA, no-swizzle K-major layout);
//   3. each chunk is multiplied by the matching 32-row chunk of W (the B
//      operand, prebuilt hi/lo in the same layout by k_build_w_tc) into a
//      128 x s_pad FP32 accumulator in TMEM:
//        passes = 3: K_hi W_hi + K_hi W_lo + K_lo W_hi   (FP32-level accuracy)
//        passes = 1: K_hi W_hi                           (TF32 inputs)
// Kernel values are split into TF32 hi/lo by integer operations (tf32_split) rather
// than cvt.rna.tf32.f32: same rounding, and measured faster (RBF, 4,096 x 262,144
// entries, s = 64: 1.87 -> 1.63 ms with the RBF-only fast path below).  Variants
// that kept the kernel-value chunks in TMEM as the A operand (tcgen05.st, then
// tcgen05.mma with A in tensor memory), or split the epilogue into four warpgroups,
// measured no faster: a TF32 MMA of M = 128, K = 8 takes about 90 clocks here, so
// the 48 contraction MMAs of a tile set its time.
// The accumulators span one column split (at most kMrhsMaxCols columns, the even
// and odd tiles in two accumulators, so that the FP32 accumulation in the tensor
// cores stays below the product's tolerance even for sums of one sign); the
// splits are summed in double-float by k_reduce.
//
// CTA = 128 rows, 384 threads, one CTA per SM, persistent over (row tile,
// split) items like rows_tc.cu:
//   warp 0       producer: bulk copies of the column operand tiles (1- or
//                2-stage ring) and of the W chunks (2-slot ring), in the order the
//                MMAs consume them
//   warp 1       TMEM owner and distance MMA issuer
//   warp 3       contraction MMA issuer (two issuing threads: one was itself the
//                limit, at about 90 clocks an MMA)
//   warps 4..11  epilogue: warpgroup g forms chunks 2g, 2g + 1 of every tile in
//                its own chunk slot (one producer per slot, so that a parity wait
//                can never alias a phase two uses back), then reads its half of
//                the accumulator
// TMEM: columns [0, 256) two distance buffers, [256, 256 + s_pad) and
// [384, 384 + s_pad) the accumulators of the even and odd tiles (512 allocated).  Every wait is bounded; on a timeout the CTA
// raises the error flag, drains its copies and MMAs, frees TMEM and writes NaN.
#include <algorithm>
#include <cstring>

#include "prep.cuh"
#include "tc_ptx.cuh"

namespace adasap {

namespace {

constexpr int kCh = 32;                     // columns per contraction chunk
static_assert(kCh == 32, "build_w_elem lays out chunks of 32 rows");
constexpr int kChPerTile = kTcN / kCh;      // 4
constexpr int kWSlots = 2;                  // W chunk ring
// K chunk slots: one or two per epilogue warpgroup (two where shared memory allows:
// the warpgroup then writes its second chunk of a tile while the MMAs read the first)
constexpr size_t kMrhsSmemMax = 232448;     // opt-in shared memory per CTA
// The MMAs take a tile's chunks in the order j = 0..3 -> chunk column 2 (j & 1) + (j >> 1):
// warpgroup 0's first, warpgroup 1's first, warpgroup 0's second, warpgroup 1's second.
__host__ __device__ constexpr int chunk_col(int j) { return 2 * (j & 1) + (j >> 1); }
constexpr uint32_t kMrhsTmemCols = 512;
constexpr uint32_t kAccCol = 256;           // first accumulator column (even tiles)
constexpr uint32_t kAccCol2 = 384;          // second accumulator (odd tiles): two sums of half the terms each
constexpr int64_t kMrhsMaxCols = 4096;      // columns accumulated in TMEM per item (2048 per accumulator)

struct MrhsArgs {
  const float* xr;
  const float* qr;
  const int* ridx;
  int64_t m;
  int dp, d;
  const float* bhi;    // column distance operands (npad rows, canonical layout)
  const float* blo;
  int64_t ncols;
  int self_mode;
  const float* whi;    // W chunks: [npad / 32][s_pad x 32] canonical, hi and lo
  const float* wlo;
  int s, sp;           // right-hand sides and the padded accumulator width (multiple of 16)
  int passes;          // 3 (split) or 1
  int nks;             // K chunk slots per epilogue warpgroup (1 or 2)
  int nx;              // column operand stages (1 or 2)
  float* part;         // nsplit x m x s
  int64_t cps;         // columns per split (multiple of 128)
  int nsplit;
  float sigma2;
  int* err;
};

// Shared-memory plan (bytes from a 128-byte aligned base)
struct MrhsSmem {
  size_t a, x, k, kslot, w, bars, total;   // kslot: floats per K slot
  __host__ __device__ MrhsSmem(int kp, int sp, int passes, int nks, int nx = 2) {
    const size_t opf = (size_t)kTcM * kp * sizeof(float);
    kslot = (size_t)(passes == 3 ? 2 : 1) * kTcM * kCh;
    a = 0;                                                      // row operands hi, lo
    x = a + 2 * opf;                                            // [2 stages][hi, lo] column tiles
    k = x + (size_t)2 * nx * opf;                               // [2 nks slots][hi(, lo)] 128 x 32 chunks
    w = k + (size_t)2 * nks * kslot * sizeof(float);            // [kWSlots][hi, lo] sp x 32 chunks
    bars = w + (size_t)kWSlots * 2 * sp * kCh * sizeof(float);
    total = bars + 32 * sizeof(uint64_t) + 64 + 128;
  }
};

// GROUPED: the items of several independent products (one MrhsArgs each, item
// ranges gstart[g] .. gstart[g + 1]) in one persistent launch; they share the
// shared-memory plan (s padding, passes, slot and stage counts), taken from a0.
template <int KERN, int KP, bool GROUPED>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_rows_tc_mrhs(MrhsArgs a0, const MrhsArgs* __restrict__ grp, const int64_t* __restrict__ gstart, int ngrp) {
  constexpr int OPF = kTcM * KP;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
  const MrhsSmem L(KP, a0.sp, a0.passes, a0.nks, a0.nx);
  float* sAhi = reinterpret_cast<float*>(base + L.a);
  float* sAlo = sAhi + OPF;
  float* sX = reinterpret_cast<float*>(base + L.x);   // [st][hi, lo][OPF]
  float* sK = reinterpret_cast<float*>(base + L.k);   // [slot][hi(, lo)][128 * 32]
  float* sW = reinterpret_cast<float*>(base + L.w);   // [slot][hi, lo][sp * 32]
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + L.bars);
  uint64_t* full = bars;         // [2] column tiles landed
  uint64_t* empty = bars + 2;    // [2] column tile stage free
  uint64_t* tfull = bars + 4;    // [2] distance buffer ready
  uint64_t* tempty = bars + 6;   // [2] distance buffer read (8 epilogue warps)
  uint64_t* kfull = bars + 8;    // [2 nks] K chunk written (4 warps of one warpgroup)
  uint64_t* kempty = bars + 12;  // [2 nks] K chunk consumed
  uint64_t* wfull = bars + 16;   // [2] W chunk landed
  uint64_t* wempty = bars + 18;  // [2] W chunk consumed
  uint64_t* ofull = bars + 20;   // accumulator of the item complete
  uint64_t* drain = bars + 21;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 22);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int sp = a0.sp;
  const uint32_t wbytes = (uint32_t)(sp * kCh * sizeof(float));

  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], 8);
      mbar_init(&wfull[i], 1);
      mbar_init(&wempty[i], 1);
    }
    for (int i = 0; i < 4; ++i) {
      mbar_init(&kfull[i], 4);
      mbar_init(&kempty[i], 1);
    }
    mbar_init(ofull, 1);
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(kMrhsTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;
  const int64_t nitems = GROUPED ? gstart[ngrp] : (a0.m + kTcM - 1) / kTcM * a0.nsplit;

  uint32_t gt = 0, nof = 0, ndrain = 0;
  for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
    int sys = 0;
    if (GROUPED) {  // the product this item belongs to: last g with gstart[g] <= item
      int hi = ngrp - 1;
      while (sys < hi) {
        const int mid = (sys + hi + 1) >> 1;
        if (gstart[mid] <= item) sys = mid;
        else hi = mid - 1;
      }
    }
    const MrhsArgs& a = GROUPED ? grp[sys] : a0;
    const int64_t li = GROUPED ? item - gstart[sys] : item;
    const int64_t rtiles = (a.m + kTcM - 1) / kTcM;
    const int64_t rtile = li % rtiles, split = li / rtiles;
    const int64_t row0 = rtile * kTcM;
    const int64_t c0 = split * a.cps;
    const int64_t c1 = min(a.ncols, c0 + a.cps);
    const int ntiles = (c1 > c0 && !*abort_flag) ? (int)((c1 - c0 + kTcN - 1) / kTcN) : 0;
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
        for (int k = 0; k < a.d; ++k) av[k] = -2.0f * a.xr[src * a.dp + k];
        av[a.d] = a.qr[src];
      } else {
        av[a.d] = 1e20f;
      }
      av[a.d + 1] = 1.0f;
#pragma unroll
      for (int k = 0; k < KP; ++k) {
        const float hi = tf32_round(av[k]);
        sAhi[tc_off<KP>(tid, k)] = hi;
        sAlo[tc_off<KP>(tid, k)] = tf32_round(av[k] - hi);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();

    if (warp == 0) {
      // ---- producer: X(0); then per tile t: X(t + 1), W(t, 0..3) -----------------
      if (lane == 0) {
        int xi = 0;         // column tiles issued
        int64_t wi = 0;     // W chunks issued (item-local)
        bool ok = true;
        auto issue_x = [&](int t) -> bool {
          const uint32_t g = gt + (uint32_t)t;
          const int st = (int)(g % (uint32_t)a.nx);
          if (!mbar_wait(&empty[st], ((g / (uint32_t)a.nx) & 1u) ^ 1u, abort_flag)) {
            tc_note_timeout(a.err, 11);
            return false;
          }
          mbar_arrive_expect_tx(&full[st], 2u * OPF * sizeof(float));
          const int64_t off = (c0 + (int64_t)t * kTcN) * KP;
          bulk_g2s(sX + (st * 2 + 0) * OPF, a.bhi + off, OPF * sizeof(float), &full[st]);
          bulk_g2s(sX + (st * 2 + 1) * OPF, a.blo + off, OPF * sizeof(float), &full[st]);
          return true;
        };
        if (ntiles > 0) ok = issue_x(0), xi = ok ? 1 : 0;
        for (int t = 0; ok && t < ntiles; ++t) {
          if (t + 1 < ntiles) {
            if (!(ok = issue_x(t + 1))) break;
            xi = t + 2;
          }
          for (int j = 0; j < kChPerTile; ++j) {
            const uint32_t q = (gt + (uint32_t)t) * kChPerTile + (uint32_t)j;  // consumption index
            const int sl = q & 1;
            if (!mbar_wait(&wempty[sl], ((q >> 1) & 1u) ^ 1u, abort_flag)) {
              tc_note_timeout(a.err, 12);
              ok = false;
              break;
            }
            mbar_arrive_expect_tx(&wfull[sl], (a.passes == 3 ? 2u : 1u) * wbytes);
            const int64_t chunk = (c0 + (int64_t)t * kTcN) / kCh + chunk_col(j);
            bulk_g2s(sW + (sl * 2 + 0) * sp * kCh, a.whi + chunk * sp * kCh, wbytes, &wfull[sl]);
            if (a.passes == 3) bulk_g2s(sW + (sl * 2 + 1) * sp * kCh, a.wlo + chunk * sp * kCh, wbytes, &wfull[sl]);
            ++wi;
          }
        }
        if (!ok) {
          *abort_flag = 1;
          // our copies still write shared memory: wait (bounded) for the last of each ring
          for (int t = max(0, xi - a.nx); t < xi; ++t) {
            const uint32_t g = gt + (uint32_t)t;
            mbar_wait(&full[g % (uint32_t)a.nx], (g / (uint32_t)a.nx) & 1u, nullptr);
          }
          for (int64_t k = (wi > 2 ? wi - 2 : 0); k < wi; ++k) {
            const uint32_t q = gt * kChPerTile + (uint32_t)k;
            mbar_wait(&wfull[q & 1], (q >> 1) & 1u, nullptr);
          }
        }
      }
    } else if (warp == 1) {
      // ---- distance MMA issuer: dist(t) for every tile of the item, each once its
      // column tile has landed and the epilogue has read that distance buffer's
      // previous tile ------------------------------------------------------------------
      if (lane == 0) {
        bool ok = true, any = false;
        const uint32_t a_hi = smem_u32(sAhi), a_lo = smem_u32(sAlo);
        for (int t = 0; ok && t < ntiles; ++t) {
          const uint32_t g = gt + (uint32_t)t;
          const int st = (int)(g % (uint32_t)a.nx), buf = g & 1;
          const uint32_t ph = (g >> 1) & 1u;
          if (!mbar_wait(&full[st], (g / (uint32_t)a.nx) & 1u, abort_flag) ||
              !mbar_wait(&tempty[buf], ph ^ 1u, abort_flag)) {
            tc_note_timeout(a.err, 13);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t dt = tbase + (uint32_t)(buf * kTcN);
          const uint32_t b_hi = smem_u32(sX + (st * 2 + 0) * OPF), b_lo = smem_u32(sX + (st * 2 + 1) * OPF);
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
          any = true;
        }
        if (!ok) *abort_flag = 1;
        if (any) {
          // every distance MMA of this issuer completes before the row operands are
          // rewritten (next item) or TMEM is released (end)
          tc_commit(drain);
          mbar_wait(drain, ndrain & 1u, nullptr);
          ++ndrain;
        }
      }
    } else if (warp == 3) {
      // ---- contraction MMA issuer: contr(t, 0..3) for every tile.  A second issuing
      // thread beside the distance MMAs: one thread issuing all 54 MMAs of a tile was
      // itself the limit (its chain of waits, descriptor arithmetic and issues) -------
      if (lane == 0) {
        bool ok = true;
        // accumulate flags of the even and odd tiles' accumulators, as two scalars (an
        // array indexed by t & 1 went to local memory, in the issue chain of every MMA)
        uint32_t acc_even = 0u, acc_odd = 0u;
        const uint32_t idesc = tc_idesc_tf32(sp);
        const uint32_t dacc = tbase + kAccCol;
        for (int t = 0; ok && t < ntiles; ++t) {
          for (int j = 0; j < kChPerTile; ++j) {
            const uint32_t gg = gt + (uint32_t)t;
            const uint32_t q = gg * kChPerTile + (uint32_t)j;   // W ring: consumption index
            const int wsl = q & 1;
            // chunk j comes from warpgroup j & 1 (its chunk j >> 1 of the tile)
            const int ksl = a.nks == 2 ? 2 * (j & 1) + (j >> 1) : (j & 1);
            const uint32_t ku = a.nks == 2 ? gg : 2u * gg + (uint32_t)(j >> 1);  // use of that slot
            if (!mbar_wait(&kfull[ksl], ku & 1u, abort_flag)) {
              tc_note_timeout(a.err, 14);
              ok = false;
              break;
            }
            if (!mbar_wait(&wfull[wsl], (q >> 1) & 1u, abort_flag)) {
              tc_note_timeout(a.err, 18);
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t k_hi = smem_u32(sK + ksl * L.kslot);
            const uint32_t k_lo = k_hi + (uint32_t)(kTcM * kCh * sizeof(float));
            const uint32_t w_hi = smem_u32(sW + (wsl * 2 + 0) * sp * kCh);
            const uint32_t w_lo = smem_u32(sW + (wsl * 2 + 1) * sp * kCh);
            // descriptors built once per chunk; K step ks starts 256 bytes further on,
            // i.e. 16 more in the descriptor's start-address field (address >> 4, 14
            // bits: shared addresses stay below 2^18 bytes, so the field never carries)
            const uint64_t dkh = smem_desc(k_hi, 128u, 32u * kCh), dkl = smem_desc(k_lo, 128u, 32u * kCh);
            const uint64_t dwh = smem_desc(w_hi, 128u, 32u * kCh), dwl = smem_desc(w_lo, 128u, 32u * kCh);
            const uint32_t dt = dacc + (uint32_t)(t & 1) * (kAccCol2 - kAccCol);
            uint32_t acc = (t & 1) ? acc_odd : acc_even;
#pragma unroll
            for (int ks = 0; ks < kCh / 8; ++ks) {
              tc_mma_tf32(dt, dkh + 16u * ks, dwh + 16u * ks, idesc, acc);   // K_hi W_hi
              acc = 1u;
            }
            if (a.passes == 3) {
#pragma unroll
              for (int ks = 0; ks < kCh / 8; ++ks) tc_mma_tf32(dt, dkh + 16u * ks, dwl + 16u * ks, idesc, 1u);  // K_hi W_lo
#pragma unroll
              for (int ks = 0; ks < kCh / 8; ++ks) tc_mma_tf32(dt, dkl + 16u * ks, dwh + 16u * ks, idesc, 1u);  // K_lo W_hi
            }
            if (t & 1) acc_odd = 1u;
            else acc_even = 1u;
            tc_commit(&kempty[ksl]);
            tc_commit(&wempty[wsl]);
          }
        }
        if (!ok) *abort_flag = 1;
        // the accumulator is complete once every contraction MMA above has finished
        // (items with tiles only: both roles count those in nof); the epilogue reads it
        // before the item's closing barrier, so this issuer needs no drain of its own
        if (ntiles > 0) tc_commit(ofull);
      }
    } else if (warp >= 4) {
      // ---- epilogue ------------------------------------------------------------------
      const int g = (warp - 4) >> 2, qd = warp & 3;
      const int rl = qd * 32 + lane;
      const int64_t ri = row0 + rl;
      int64_t gi = -1;
      bool bad = false;
      if (ri < a.m) {
        const int64_t src = a.ridx ? (int64_t)a.ridx[ri] : ri;
        bad = src < 0;
        if (a.self_mode) gi = src;
      }
      for (int t = 0; t < ntiles; ++t) {
        const uint32_t gg = gt + (uint32_t)t;
        const int buf = gg & 1;
        if (!mbar_wait(&tfull[buf], (gg >> 1) & 1u, abort_flag)) {
          *abort_flag = 1;
          tc_note_timeout(a.err, 15);
          break;
        }
        tc_fence_after();
        uint32_t u0[32], u1[32];
        const uint32_t taddr = tbase + ((uint32_t)(qd * 32) << 16) + (uint32_t)(buf * kTcN + g * 64);
        TMEM_LD32(taddr, u0);
        TMEM_LD32(taddr + 32u, u1);
        TMEM_WAIT32(u0);
        TMEM_WAIT32(u1);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[buf]);
        bool stop = false;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int c = 2 * g + h;
          const int sl = a.nks == 2 ? 2 * g + h : g;                   // this warpgroup's slot
          const uint32_t ku = a.nks == 2 ? gg : 2u * gg + (uint32_t)h;  // its use of the slot
          if (!mbar_wait(&kempty[sl], (ku & 1u) ^ 1u, abort_flag)) {
            tc_note_timeout(a.err, 16);
            stop = true;
            break;
          }
          const int64_t jb = c0 + (int64_t)t * kTcN + c * kCh;
          float* khi = sK + sl * L.kslot;
          float* klo = khi + kTcM * kCh;
          const uint32_t* u = h ? u1 : u0;
          // RBF chunks without the row's own column skip the per-entry test and clamp (the
          // RBF term needs no clamp); the Matern chunks keep them (measured faster there)
          const bool fast = KERN == ADASAP_RBF && !__any_sync(0xffffffffu, gi >= jb && gi < jb + kCh);
          if (fast) {
#pragma unroll
            for (int k4 = 0; k4 < kCh / 4; ++k4) {
              float hv[4], lv[4];
#pragma unroll
              for (int e = 0; e < 4; ++e) tf32_split(kval<KERN>(__uint_as_float(u[4 * k4 + e])), hv[e], lv[e]);
              const int off = (rl >> 3) * (8 * kCh) + k4 * 32 + (rl & 7) * 4;
              *reinterpret_cast<float4*>(khi + off) = make_float4(hv[0], hv[1], hv[2], hv[3]);
              if (a.passes == 3) *reinterpret_cast<float4*>(klo + off) = make_float4(lv[0], lv[1], lv[2], lv[3]);
            }
          } else {
#pragma unroll
            for (int k4 = 0; k4 < kCh / 4; ++k4) {
              float hv[4], lv[4];
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const int k = 4 * k4 + e;
                const float uu = (jb + k == gi) ? 0.0f : fmaxf(__uint_as_float(u[k]), 0.0f);
                tf32_split(kval<KERN>(uu), hv[e], lv[e]);
              }
              const int off = (rl >> 3) * (8 * kCh) + k4 * 32 + (rl & 7) * 4;
              *reinterpret_cast<float4*>(khi + off) = make_float4(hv[0], hv[1], hv[2], hv[3]);
              if (a.passes == 3) *reinterpret_cast<float4*>(klo + off) = make_float4(lv[0], lv[1], lv[2], lv[3]);
            }
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          __syncwarp();
          if (lane == 0) mbar_arrive(&kfull[sl]);
        }
        if (stop) {
          *abort_flag = 1;
          break;
        }
      }
      // ---- the item's accumulator: warpgroup g reads 16-column groups g, g + 2, ...
      const bool have = ntiles == 0 || mbar_wait(ofull, nof & 1u, abort_flag);
      if (!have) tc_note_timeout(a.err, 17);
      tc_fence_after();
      const bool nan_out = bad || !have || *abort_flag;
      for (int cg16 = g; cg16 < sp / 16; cg16 += 2) {
        uint32_t v[16];
        if (ntiles > 0) {
          TMEM_LD16(tbase + ((uint32_t)(qd * 32) << 16) + kAccCol + (uint32_t)(cg16 * 16), v);
          TMEM_WAIT16(v);
          if (ntiles > 1) {   // the odd tiles' accumulator
            uint32_t v2[16];
            TMEM_LD16(tbase + ((uint32_t)(qd * 32) << 16) + kAccCol2 + (uint32_t)(cg16 * 16), v2);
            TMEM_WAIT16(v2);
#pragma unroll
            for (int e = 0; e < 16; ++e) v[e] = __float_as_uint(__uint_as_float(v[e]) + __uint_as_float(v2[e]));
          }
        } else {
#pragma unroll
          for (int e = 0; e < 16; ++e) v[e] = 0u;  // an empty split contributes zero
        }
        if (ri < a.m) {
          float* dst = a.part + (split * a.m + ri) * a.s;
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int c = cg16 * 16 + e;
            if (c < a.s) dst[c] = nan_out ? __int_as_float(0x7fc00000) : a.sigma2 * __uint_as_float(v[e]);
          }
        }
      }
      tc_fence_before();
    }
    gt += (uint32_t)ntiles;
    nof += ntiles > 0 ? 1u : 0u;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  if (warp == 0 && lane == 0 && *abort_flag) tc_note_timeout(a0.err, 19);
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(kMrhsTmemCols)
                 : "memory");
  }
}

// W operand chunks: chunk q holds rows j in [32 q, 32 q + 32) of W as the
// sp x 32 K-major B operand (element (c, j - 32 q) at tc_off<32>), hi and lo.
__global__ void k_build_w_tc(const float* __restrict__ W, int64_t ldw, int64_t n, int s, int sp, int64_t npad,
                             int passes, float* __restrict__ whi, float* __restrict__ wlo) {
  const int64_t total = npad * sp;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / sp;
    const int c = (int)(e - j * sp);
    build_w_elem((j < n && c < s) ? W[j * ldw + c] : 0.0f, j, c, sp, passes, whi, wlo);
  }
}

template <int KERN, int KP>
cudaError_t mrhs_setup(int sp_max) {
  const size_t need = MrhsSmem(KP, sp_max, 3, 1).total;   // the largest plan launched
  const int bytes = (int)std::max(need, kMrhsSmemMax);
  cudaError_t e = cudaFuncSetAttribute(k_rows_tc_mrhs<KERN, KP, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_rows_tc_mrhs<KERN, KP, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// The argument block of one product as launched (shared-memory plan included).
MrhsArgs make_mrhs_args(int d, const float* xr, const float* qr, const int* ridx, int64_t m, int dp,
                        const float* bhi, const float* blo, int64_t ncols, int self_mode, const float* whi,
                        const float* wlo, int s, int passes, float* part, int nsplit, float sigma2, int* err) {
  MrhsArgs a;
  a.xr = xr; a.qr = qr; a.ridx = ridx; a.m = m; a.dp = dp; a.d = d;
  a.bhi = bhi; a.blo = blo; a.ncols = ncols; a.self_mode = self_mode;
  a.whi = whi; a.wlo = wlo; a.s = s; a.sp = tc_mrhs_sp(s); a.passes = passes;
  const int kp = tc_kp(d);
  // two K slots per warpgroup (the epilogue writes a tile's second chunk while the
  // MMAs read the first) before a second column-operand stage (a contraction tile is
  // long enough to reload the one stage behind the distance MMA)
  a.nks = 2;
  a.nx = 2;
  if (MrhsSmem(kp, a.sp, passes, 2, 2).total > kMrhsSmemMax) a.nx = 1;
  if (MrhsSmem(kp, a.sp, passes, 2, 1).total > kMrhsSmemMax) a.nks = 1, a.nx = 2;
  a.part = part; a.sigma2 = sigma2; a.err = err;
  const int64_t tiles = (ncols + kTcN - 1) / kTcN;
  a.cps = (tiles + nsplit - 1) / nsplit * kTcN;
  a.nsplit = nsplit;
  return a;
}

template <bool G>
cudaError_t launch_mrhs_any(int kern, int kp, const MrhsArgs& a, const MrhsArgs* grp, const int64_t* gstart, int ngrp,
                            int ctas, cudaStream_t st) {
  const size_t smem = MrhsSmem(kp, a.sp, a.passes, a.nks, a.nx).total;
#define ADASAP_MRHS(KE, KPV) k_rows_tc_mrhs<KE, KPV, G><<<ctas, kTcThreads, smem, st>>>(a, grp, gstart, ngrp)
  if (kp == 16) {
    if (kern == 0) ADASAP_MRHS(0, 16);
    else if (kern == 1) ADASAP_MRHS(1, 16);
    else ADASAP_MRHS(2, 16);
  } else if (kp == 32) {
    if (kern == 0) ADASAP_MRHS(0, 32);
    else if (kern == 1) ADASAP_MRHS(1, 32);
    else ADASAP_MRHS(2, 32);
  } else {
    return cudaErrorInvalidValue;
  }
#undef ADASAP_MRHS
  return cudaGetLastError();
}

}  // namespace

int tc_mrhs_sp(int s) { return (s + 15) / 16 * 16; }

int64_t tc_mrhs_wfloats(int64_t n, int s) { return tc_npad(n) * tc_mrhs_sp(s); }

cudaError_t tc_mrhs_init() {
  cudaError_t e;
  if ((e = mrhs_setup<0, 16>(kMaxRhs)) || (e = mrhs_setup<1, 16>(kMaxRhs)) || (e = mrhs_setup<2, 16>(kMaxRhs)) ||
      (e = mrhs_setup<0, 32>(kMaxRhs)) || (e = mrhs_setup<1, 32>(kMaxRhs)) || (e = mrhs_setup<2, 32>(kMaxRhs)))
    return e;
  return cudaSuccess;
}

int tc_mrhs_nsplit(int64_t m, int64_t ncols, int max_ctas) {
  // as tc_nsplit, with at most kMrhsMaxCols columns accumulated per item
  const int64_t rt = (m + kTcM - 1) / kTcM;
  const int64_t tiles = (ncols + kTcN - 1) / kTcN;
  const int64_t slots = (max_ctas > 0 && max_ctas < tc_slots()) ? max_ctas : tc_slots();
  const int64_t min_ns = (tiles + kMrhsMaxCols / kTcN - 1) / (kMrhsMaxCols / kTcN);
  constexpr double kStartupTiles = 2.0;
  int64_t best = std::max<int64_t>(1, min_ns);
  double best_cost = 1e300;
  for (int64_t ns = std::max<int64_t>(1, min_ns); ns <= std::min<int64_t>(tiles, 4096); ++ns) {
    const int64_t tot = rt * ns;
    const int64_t waves = (tot + slots - 1) / slots;
    if (waves > 64 && ns > min_ns) break;
    const int64_t tps = (tiles + ns - 1) / ns;
    const double cost = (double)waves * ((double)tps + kStartupTiles);
    if (cost < best_cost - 1e-9) {
      best_cost = cost;
      best = ns;
    }
  }
  return (int)best;
}

cudaError_t launch_build_w_tc(const float* W, int64_t ldw, int64_t n, int s, int passes, float* whi, float* wlo,
                              cudaStream_t st) {
  const int sp = tc_mrhs_sp(s);
  const int64_t npad = tc_npad(n);
  const int blocks = (int)std::min<int64_t>((npad * sp + 255) / 256, 148 * 16);
  k_build_w_tc<<<blocks, 256, 0, st>>>(W, ldw, n, s, sp, npad, passes, whi, wlo);
  return cudaGetLastError();
}

cudaError_t launch_rows_tc_mrhs(int kern, int d, const float* xr, const float* qr, const int* ridx, int64_t m, int dp,
                                const float* bhi, const float* blo, int64_t ncols, int self_mode, const float* whi,
                                const float* wlo, int s, int passes, float* part, int nsplit, float sigma2, int* err,
                                cudaStream_t st, int max_ctas) {
  if (m <= 0 || ncols <= 0) return cudaSuccess;
  if (s < 1 || s > kMaxRhs || (passes != 1 && passes != 3)) return cudaErrorInvalidValue;
  const MrhsArgs a = make_mrhs_args(d, xr, qr, ridx, m, dp, bhi, blo, ncols, self_mode, whi, wlo, s, passes, part,
                                    nsplit, sigma2, err);
  const int64_t nitems = (m + kTcM - 1) / kTcM * (int64_t)nsplit;
  const int slots = (max_ctas > 0 && max_ctas < tc_slots()) ? max_ctas : tc_slots();
  const int ctas = (int)std::min<int64_t>(nitems, slots);
  return launch_mrhs_any<false>(kern, tc_kp(d), a, nullptr, nullptr, 0, ctas, st);
}

size_t mrhs_args_size() { return sizeof(MrhsArgs); }

int64_t mrhs_fill_args(void* out, int d, const float* xr, const float* qr, const int* ridx, int64_t m, int dp,
                       const float* bhi, const float* blo, int64_t ncols, int self_mode, const float* whi,
                       const float* wlo, int s, int passes, float* part, int nsplit, float sigma2, int* err) {
  if (m <= 0 || ncols <= 0 || s < 1 || s > kMaxRhs || (passes != 1 && passes != 3) || nsplit < 1) return -1;
  const MrhsArgs a = make_mrhs_args(d, xr, qr, ridx, m, dp, bhi, blo, ncols, self_mode, whi, wlo, s, passes, part,
                                    nsplit, sigma2, err);
  std::memcpy(out, &a, sizeof(a));
  return (m + kTcM - 1) / kTcM * (int64_t)nsplit;
}

int64_t mrhs_plan_key(const void* args) {
  MrhsArgs a;
  std::memcpy(&a, args, sizeof(a));
  return (((int64_t)a.sp * 4 + a.passes) * 4 + a.nks) * 4 + a.nx;
}

cudaError_t launch_rows_tc_mrhs_grouped(int kern, int kp, const void* first, const void* grp, const int64_t* gstart,
                                        int ngrp, int64_t nitems, cudaStream_t st) {
  if (ngrp < 1 || nitems < 1) return cudaSuccess;
  MrhsArgs a0;
  std::memcpy(&a0, first, sizeof(a0));
  const int ctas = (int)std::min<int64_t>(nitems, tc_slots());
  return launch_mrhs_any<true>(kern, kp, a0, static_cast<const MrhsArgs*>(grp), gstart, ngrp, ctas, st);
}

}  // namespace adasap
