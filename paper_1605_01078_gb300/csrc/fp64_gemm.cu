// FP64 product kernel: the general operation of Eq. 4 on GB300.
//
// One persistent launch runs every product M_r of one or more problems (the Figure 1
// table, its Kronecker square of Figure 2, or its cube) over work units (problem,
// product r, BT x BT output tile of the block, k-steps of 8), BT = 128 or 64.  Each
// thread block is warp-specialised:
//
//   producer warps (4)  stage the 1..8 source tiles of A (blocks X_s) and of B
//       (blocks V_t) of a k-step into a shared-memory ring -- with TMA box loads
//       (cp.async.bulk.tensor, completion on an mbarrier) when the operands are
//       16-byte aligned, else with zero-filling 8-byte cp.async; transposed operands
//       with the other box orientation -- and form the operand sums
//       sum_s delta_s X_s and sum_t eps_t V_t into a ring of "summed" tiles: the
//       packing-time sums of Section 3.4, with no temporary in global memory.
//       Columns past the block edge h_k read as zero (the zero padding of Section
//       3.3); TMA zero-fills past the matrix edge.
//   consumer warps (8)  accumulate M_tile += A_sum * B_sum with FP64 fused
//       multiply-adds on a (BT/16) x (BT/16) register tile per thread and, after the
//       last k-step of a partial sum, add gamma_q * alpha * M_tile into every C block q
//       the product updates -- the fused scatter of the micro-kernel (Section 3.4).
//       A partial sum covers at most accumulation_chunk_k(L) of k (256, or 128 at
//       three levels): a register accumulator that ran over all of h_k would add
//       thousands of terms in sequence, and its rounding error, growing with the
//       length of that sequence, set the error of the large products (about 2.4e-12
//       of max|A| max|B| at 16384^3 with two levels, measured).  Chunks start from zero
//       and are added into C, which shortens every sequential sum to the chunk length
//       plus the number of chunks.  The two halves of the consumer warps flush half a
//       chunk apart, so the chunk flushes overlap the other half's multiply-adds.
//
// C updates are device atomics (red.global.add.f64) for every schedule; a store into a
// temporary is a clear followed by adds.  The two groups hand tiles over through
// mbarriers, with each summed slot's (problem, product, tile, last step) in shared
// memory; every wait is bounded (about one second of clock cycles), after which the
// kernel records STRASSEN_ERR_TIMEOUT in a device status word and returns instead of
// hanging.  A single launch gives each block one stream-K range (or its tiles under
// the owner schedule); a batched launch lets blocks claim whole work units, longest
// first, from a global counter.
//
// GB300 design notes.  FP64 runs at about 2 FMA lanes per clock per SM (measured
// 1.20 TFLOP/s for the whole GPU; DMMA is slower at 1.06), so this kernel is bound by
// the FP64 pipe by two orders of magnitude over HBM.  The design therefore keeps the
// FP64 pipe fed with nothing but the product's FMAs in the consumer warps (staging,
// address arithmetic, operand sums and barrier traffic live in the producer warps),
// forms each operand sum once per staged tile with an integer-pipe binary64 addition
// (int_fadd.h, bit-identical to DADD), uses sign-bit flips for negation, and
// balances work across the 152 SMs exactly (stream-K ranges of the (unit, k-step)
// space).  Atomic C updates (red.global.add.f64) execute in the L2, off the SM's FP64
// pipe.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "int_fadd.h"
#include "internal.h"

namespace sgb {
namespace {

__constant__ PlanTables c_plans = kPlanTables;
__device__ int g_fp64_status;  // STRASSEN_ERR_TIMEOUT once a bounded wait gave up

// Block tile BT x BT x BK: BT = 128 (tile id 0) or 64 (tile id 1, for small blocks where
// 128-wide tiles would mostly compute padding).  The consumers are 16 x 16 threads with
// a (BT/16) x (BT/16) register tile each.
constexpr int BK = 8;
constexpr int kTileIds = kNumTiles;
constexpr int tile_edge(int tile_id) { return tile_id == 0 ? 128 : 64; }
// Cost model of the tile choice (FMA-equivalents): a 64-wide k-step costs
// kSmallTileFactor times its FMAs, and every k-step a fixed overhead for the hand-over
// between the warp groups.
constexpr double kStepOverheadFma = 2000.0;
constexpr int kConsumers = 256;  // 8 warps: 16 x 16 threads
constexpr int kProducers = 128;  // 4 warps: staging and operand sums
constexpr int kThreads = kConsumers + kProducers;
constexpr int NS = 4;  // ring of summed tiles
// Ring of raw source tiles: two slots (the load of the next k-step overlaps the sums of
// this one) while MAXT source tiles per operand fit twice in shared memory; one slot
// for the eight-term products of three levels with 128-wide tiles.  One k-step of the
// consumers takes about 64K clocks of FP64 work per SM (128-wide tiles), so a producer
// that loads (about 1 us) and then sums (a few us) each step still runs ahead of them
// through the summed ring.
template <int MAXT, int BT>
constexpr int raw_slots() { return (MAXT >= 8 && BT >= 128) ? 1 : 2; }
constexpr long long kWaitLimitCycles = 2000000000LL;  // ~1 s at 2 GHz
// Register split (setmaxnreg): the block is launched with kLaunchRegs per thread;
// the producer warpgroup gives registers back and the two consumer warpgroups take
// them.  The shares add up exactly to the launch total, so the increase never waits
// on registers that do not exist.
constexpr int kLaunchRegs = 168, kProducerRegs = 88, kConsumerRegs = 208;
static_assert(kProducers * kProducerRegs + kConsumers * kConsumerRegs == kThreads * kLaunchRegs,
              "register split must add up to the launch allocation");

struct alignas(128) ProbDesc {
  CUtensorMap tmA, tmB;
  const double* A;
  const double* B;
  double* C;
  int64_t lda, ldb, ldc;
  int64_t a_rows, a_cols, b_rows, b_cols, c_rows, c_cols;
  int64_t hm, hn, hk;
  int64_t iter_begin;  // first iteration of this problem in the stream-K space
  int64_t claim_begin;  // batched: index of this problem's first claim
  int64_t units;        // batched: work units of this problem
  int32_t units_per_claim;  // batched: whole units per claim (short units go several to a claim)
  int32_t plan_row;    // table row of the first product of this problem
  int32_t nprod;
  int32_t m_target;
  int32_t epi;
  int32_t tiles_m, tiles_n, ksteps;
  int32_t use_tma;
  int32_t flush_steps;       // k-steps per accumulation chunk (partial sums leave the registers)
  int32_t trans_a, trans_b;  // op(A) = A^T (A stored k x m), op(B) = B^T (B stored n x k)
  int32_t tri;               // level 0: 0 all of C, 1 only j <= i, 2 only j >= i (local to C)
  int32_t target_row0;       // first table row of the launch's level (for inner targets)
  int32_t inner_row0;        // inner targets: first row of the (L-1)-level table, else -1
  int32_t inner_count;       // inner targets: 7^(L-1)
  double alpha;              // the product is scaled by alpha in the scatter
};

struct KArgs {
  ProbDesc single;         // the problem when not batched
  const ProbDesc* descs;   // device array when batched
  unsigned long long* chunk_counter;  // batched: next unit to claim (cleared before the launch)
  int nprob;
  int sched;
  int64_t total;           // stream-K: iterations of all problems; owner: tile positions
  int64_t nchunks;         // batched: claims (each one or more whole units of one problem)
  int64_t dp_rounds;       // single stream-K launch: rounds of whole units before the split tail
};

// What the producers tell the consumers about the k-step in a summed slot.
struct StepMeta {
  int p, r, t;  // problem, product, tile of the step
  int flags;    // kStepLast, kStepFlush0, kStepFlush1 (see step_flags); kStepEnd: no step
};
constexpr int kStepLast = 1, kStepEnd = 2, kStepFlush0 = 4, kStepFlush1 = 8;

template <int MAXT, int BT>
struct Smem {
  static constexpr int BM = BT, BN = BT;
  static constexpr int NR = raw_slots<MAXT, BT>();
  static constexpr int kRawA = MAXT * BM * BK;  // doubles per ring slot
  static constexpr int kRawB = MAXT * BK * BN;
  static constexpr size_t kBytes =
      sizeof(double) * (size_t)(NR * (kRawA + kRawB) + NS * BK * (BM + BN) + (kConsumers / 32) * 2 * BN) +
      sizeof(uint64_t) * (2 * NR + 2 * NS) + sizeof(StepMeta) * NS + 16;
  static_assert(kBytes <= 227 * 1024, "shared memory per block");
};

// ---------------------------------------------------------------- PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with the given parity; false when the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          long long limit = kWaitLimitCycles) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(smem_u32(smem)), "l"(gmem), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_mbar_arrive(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ double flip_sign(double x, int neg) {
  return __longlong_as_double(__double_as_longlong(x) ^ ((long long)neg << 63));
}
__device__ __forceinline__ void record_timeout() { atomicExch(&g_fp64_status, STRASSEN_ERR_TIMEOUT); }

// ---------------------------------------------------------------- work cursor

// Walks this block's sequence of (problem, product, tile, k-step) without divisions
// after the start.  Producers and consumers each keep one.
struct Cursor {
  int p, r, t, ks;
  int64_t left;  // steps left, including the current one
};

template <bool BATCHED>
__device__ __forceinline__ const ProbDesc& desc_of(const KArgs& a, int p) {
  if constexpr (BATCHED) return a.descs[p];
  else return a.single;
}

// Cursor on range `id` of the work: a batched launch claims one whole unit per id;
// single launches have one range per block (a stream-K share, or the block's tile
// positions under the owner schedule).
template <bool BATCHED>
__device__ Cursor range_cursor(const KArgs& a, int64_t id) {
  Cursor c;
  c.p = 0; c.r = 0; c.t = 0; c.ks = 0; c.left = 0;
  if (BATCHED || a.sched == kSchedStreamK) {
    int64_t beg, end;
    int p = 0;
    if constexpr (BATCHED) {
      // Claim `id` holds whole units of one problem: p is the last problem whose first
      // claim is <= id.
      int lo = 0, hi = a.nprob - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (a.descs[mid].claim_begin <= id) lo = mid; else hi = mid - 1;
      }
      p = lo;
      const ProbDesc& dp = a.descs[p];
      const int64_t u0 = (id - dp.claim_begin) * dp.units_per_claim;
      const int64_t u1 = u0 + dp.units_per_claim < dp.units ? u0 + dp.units_per_claim : dp.units;
      beg = dp.iter_begin + u0 * dp.ksteps;
      end = dp.iter_begin + u1 * dp.ksteps;
    } else {
      // Claims 0 .. dp_rounds - 1: whole units, round-robin over the blocks, so the
      // blocks of one round work on neighbouring tiles of the same product at the same
      // k (their operand tiles meet in the L2); the last claim: an even share of the
      // remaining units' iterations (stream-K), which balances the tail.
      const int64_t ksteps = a.single.ksteps;
      if (id < a.dp_rounds) {
        beg = (id * gridDim.x + blockIdx.x) * ksteps;
        end = beg + ksteps;
      } else {
        const int64_t tb = a.dp_rounds * gridDim.x * ksteps, len = a.total - tb;
        beg = tb + (len * blockIdx.x) / gridDim.x;
        end = tb + (len * (blockIdx.x + 1)) / gridDim.x;
      }
    }
    c.left = end - beg;
    if (c.left > 0) {
      const ProbDesc& d = desc_of<BATCHED>(a, p);
      const int64_t local = beg - d.iter_begin;
      const int64_t u = local / d.ksteps;
      const int tiles = d.tiles_m * d.tiles_n;
      c.p = p;
      c.ks = (int)(local - u * d.ksteps);
      c.r = (int)(u / tiles);
      c.t = (int)(u - (int64_t)c.r * tiles);
    }
  } else {
    const ProbDesc& d = desc_of<BATCHED>(a, 0);
    const int64_t owned = (a.total > id) ? (a.total - 1 - id) / gridDim.x + 1 : 0;
    c.left = owned * d.nprod * d.ksteps;
    c.t = (int)id;
  }
  return c;
}

// Flags of a k-step: kStepLast when it ends this block's part of the unit (the unit's
// last k-step, or the end of a stream-K share); kStepFlush0 / kStepFlush1 when it ends
// an accumulation chunk of consumer group 0 / 1.  Both groups flush every flush_steps
// k-steps, group 1 half a chunk later than group 0, so that while one group adds its
// partial sums into C the other keeps the FP64 pipe busy.
template <bool BATCHED>
__device__ __forceinline__ int step_flags(const KArgs& a, const Cursor& c) {
  const ProbDesc& d = desc_of<BATCHED>(a, c.p);
  int f = 0;
  if (c.ks == d.ksteps - 1 || ((BATCHED || a.sched == kSchedStreamK) && c.left == 1)) f |= kStepLast;
  const int kk = c.ks + 1, fs = d.flush_steps;
  if (kk % fs == 0) f |= kStepFlush0;
  if ((kk + fs / 2) % fs == 0) f |= kStepFlush1;
  return f;
}

template <bool BATCHED>
__device__ __forceinline__ void cursor_next(const KArgs& a, Cursor& c) {
  const ProbDesc& d = desc_of<BATCHED>(a, c.p);
  --c.left;
  if (++c.ks < d.ksteps) return;
  c.ks = 0;
  if (BATCHED || a.sched == kSchedStreamK) {
    if (++c.t < d.tiles_m * d.tiles_n) return;
    c.t = 0;
    if (++c.r < d.nprod) return;
    c.r = 0;
    ++c.p;
  } else {
    if (++c.r < d.nprod) return;
    c.r = 0;
    c.t += gridDim.x;
  }
}

// ---------------------------------------------------------------- kernel

template <int MAXT, bool BATCHED, int BT>
__global__ void __launch_bounds__(kThreads, 1) fp64_strassen_kernel(const __grid_constant__ KArgs a) {
  using S = Smem<MAXT, BT>;
  constexpr int NR = S::NR;
  constexpr int BM = BT, BN = BT, TM = BT / 16, TN = BT / 16;
  extern __shared__ __align__(128) double smem[];
  double* rawA = smem;                    // [NR][MAXT][BM][BK]   (TMA box layout: row, k)
  double* rawB = rawA + NR * S::kRawA;    // [NR][MAXT][BK][BN]
  double* sumA = rawB + NR * S::kRawB;    // [NS][BK][BM]         (k-major for the consumers)
  double* sumB = sumA + NS * BK * BM;     // [NS][BK][BN]
  double* epi_stage = sumB + NS * BK * BN;  // [consumer warp][2][BN]
  uint64_t* bars = reinterpret_cast<uint64_t*>(epi_stage + (kConsumers / 32) * 2 * BN);
  uint64_t* raw_full = bars;              // count kProducers (+ TMA bytes)
  uint64_t* raw_empty = bars + NR;        // count kProducers
  uint64_t* sum_full = bars + 2 * NR;     // count kProducers
  uint64_t* sum_empty = bars + 2 * NR + NS;  // count kConsumers
  StepMeta* meta = reinterpret_cast<StepMeta*>(bars + 2 * NR + 2 * NS);  // [NS], written by producer 0
  uint64_t* claim_full = reinterpret_cast<uint64_t*>(meta + NS);          // count 1
  uint64_t* claim_empty = claim_full + 1;                                 // count kProducers - 1
  unsigned long long* claim_slot = reinterpret_cast<unsigned long long*>(claim_full + 2);

  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int i = 0; i < NR; ++i) { mbar_init(&raw_full[i], kProducers); mbar_init(&raw_empty[i], kProducers); }
    for (int i = 0; i < NS; ++i) { mbar_init(&sum_full[i], kProducers); mbar_init(&sum_empty[i], kConsumers); }
    mbar_init(claim_full, 1);
    mbar_init(claim_empty, kProducers - 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  }
  if constexpr (BATCHED) {
    // Descriptors were written by a copy before the launch: make the tensor maps
    // visible to the TMA unit.
    if (tid == kConsumers) {
      for (int p = 0; p < a.nprob; ++p) {
        if (!a.descs[p].use_tma) continue;
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;\n" ::"l"(&a.descs[p].tmA) : "memory");
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;\n" ::"l"(&a.descs[p].tmB) : "memory");
      }
    }
  }
  __syncthreads();

  Cursor cur;  // the producers' sum cursor
  cur.p = 0; cur.r = 0; cur.t = 0; cur.ks = 0; cur.left = 0;

  if (tid >= kConsumers) {
    // ======================= producers =======================
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;\n" ::"n"(kProducerRegs));
    const int pt = tid - kConsumers;
    Cursor cl = cur;  // load cursor (NR - 1 steps ahead of the sum cursor)
    bool timed_out = false;
    // Ranges of the work this block claims: a single launch has one per block; a
    // batched launch claims chunks from a global counter until none are left, so blocks
    // that meet cheaper iterations simply take more chunks.  Producer 0 claims and
    // hands the id to the other producers through shared memory (bounded waits on two
    // mbarriers).  The load cursor claims; the sum cursor follows through a two-entry
    // queue (the load cursor runs at most one step, so at most one range, ahead).
    int64_t fifo[2] = {0, 0};
    int fin = 0, fout = 0, nclaims = 0;
    bool claims_done = false;
    auto claim = [&]() -> int64_t {
      if constexpr (BATCHED) {
        if (pt == 0) {
          if (nclaims > 0 && !mbar_wait(claim_empty, (uint32_t)((nclaims - 1) & 1))) { timed_out = true; return -1; }
          *claim_slot = atomicAdd(a.chunk_counter, 1ULL);
          mbar_arrive(claim_full);
        }
        if (!mbar_wait(claim_full, (uint32_t)(nclaims & 1))) { timed_out = true; return -1; }
        const unsigned long long c = *claim_slot;
        if (pt != 0) mbar_arrive(claim_empty);
        ++nclaims;
        return c < (unsigned long long)a.nchunks ? (int64_t)c : -1;
      } else if (a.sched == kSchedStreamK) {
        return nclaims <= a.dp_rounds ? (int64_t)nclaims++ : -1;
      } else {
        return nclaims++ == 0 ? (int64_t)blockIdx.x : -1;
      }
    };
    auto advance_load = [&]() -> bool {
      while (cl.left <= 0) {
        if (claims_done || timed_out) return false;
        const int64_t id = claim();
        if (id < 0) { claims_done = true; return false; }
        cl = range_cursor<BATCHED>(a, id);
        if (cl.left > 0) fifo[(fin++) & 1] = id;
      }
      return true;
    };

    auto issue = [&](const Cursor& c, int slot) {
      const ProbDesc& d = desc_of<BATCHED>(a, c.p);
      // The descriptor's fields in registers: in a batched launch it lives in global
      // memory, and every copy instruction below (asm with a memory clobber) would
      // otherwise make the compiler load the fields again.
      const int64_t hm = d.hm, hn = d.hn, hk = d.hk;
      const int row = d.plan_row + c.r;
      const int na = min((int)c_plans.na[row], MAXT), nb = min((int)c_plans.nb[row], MAXT);
      const int tiles_n = d.tiles_n;
      const int tm = c.t / tiles_n, tn = c.t - (c.t / tiles_n) * tiles_n;
      const int trans_a = d.trans_a, trans_b = d.trans_b;
      double* ra = rawA + slot * S::kRawA;
      double* rb = rawB + slot * S::kRawB;
      if (d.use_tma) {
        if (pt == 0) {
          const CUtensorMap* tmA = &d.tmA;
          const CUtensorMap* tmB = &d.tmB;
          mbar_arrive_expect_tx(&raw_full[slot], (uint32_t)((na * BM * BK + nb * BK * BN) * sizeof(double)));
          for (int t = 0; t < na; ++t) {
            const uint8_t code = c_plans.ta[row][t];
            const int rr = (int)(term_bi(code) * hm + (int64_t)tm * BM), kc = (int)(term_bj(code) * hk + (int64_t)c.ks * BK);
            // A box [BM][BK] (row, k), or for A^T the stored box [BK][BM] (k, row)
            if (trans_a) tma_load_2d(ra + t * BM * BK, tmA, rr, kc, &raw_full[slot]);
            else tma_load_2d(ra + t * BM * BK, tmA, kc, rr, &raw_full[slot]);
          }
          for (int t = 0; t < nb; ++t) {
            const uint8_t code = c_plans.tb[row][t];
            const int kr = (int)(term_bi(code) * hk + (int64_t)c.ks * BK), cc = (int)(term_bj(code) * hn + (int64_t)tn * BN);
            // B box [BK][BN] (k, col), or for B^T the stored box [BN][BK] (col, k)
            if (trans_b) tma_load_2d(rb + t * BK * BN, tmB, kr, cc, &raw_full[slot]);
            else tma_load_2d(rb + t * BK * BN, tmB, cc, kr, &raw_full[slot]);
          }
        } else {
          mbar_arrive(&raw_full[slot]);
        }
      } else {
        {
        const double* A = d.A;
        const int64_t lda = d.lda, a_rows = d.a_rows, a_cols = d.a_cols;
        for (int t = 0; t < na; ++t) {
          const uint8_t code = c_plans.ta[row][t];
          const int64_t r0 = (int64_t)term_bi(code) * hm, c0 = (int64_t)term_bj(code) * hk;
#pragma unroll
          for (int q = 0; q < (BM * BK) / kProducers; ++q) {
            const int e = pt + q * kProducers;
            // raw layout [BM][BK], or [BK][BM] for A^T (the layout of the TMA box)
            const int i = trans_a ? e % BM : e / BK, kk = trans_a ? e / BM : e % BK;
            const int64_t li = (int64_t)tm * BM + i, lk = (int64_t)c.ks * BK + kk;
            const int64_t gr = r0 + li, gc = c0 + lk;  // element (gr, gc) of op(A)
            const bool ok = li < hm && lk < hk && gr < a_rows && gc < a_cols;
            const double* src = trans_a ? A + gc * lda + gr : A + gr * lda + gc;
            cp_async8(ra + t * BM * BK + e, ok ? src : A, ok ? 8 : 0);
          }
        }
        }
        {
        const double* B = d.B;
        const int64_t ldb = d.ldb, b_rows = d.b_rows, b_cols = d.b_cols;
        for (int t = 0; t < nb; ++t) {
          const uint8_t code = c_plans.tb[row][t];
          const int64_t r0 = (int64_t)term_bi(code) * hk, c0 = (int64_t)term_bj(code) * hn;
#pragma unroll
          for (int q = 0; q < (BN * BK) / kProducers; ++q) {
            const int e = pt + q * kProducers;
            // raw layout [BK][BN], or [BN][BK] for B^T
            const int kk = trans_b ? e % BK : e / BN, jj = trans_b ? e / BK : e % BN;
            const int64_t lk = (int64_t)c.ks * BK + kk, lj = (int64_t)tn * BN + jj;
            const int64_t gr = r0 + lk, gc = c0 + lj;  // element (gr, gc) of op(B)
            const bool ok = lk < hk && lj < hn && gr < b_rows && gc < b_cols;
            const double* src = trans_b ? B + gc * ldb + gr : B + gr * ldb + gc;
            cp_async8(rb + t * BK * BN + e, ok ? src : B, ok ? 8 : 0);
          }
        }
        }
        cp_async_mbar_arrive(&raw_full[slot]);
      }
    };

    // Loads run NR - 1 steps ahead of the sums: step s + NR - 1 is issued into the
    // slot that step s - 1 has released.
    constexpr int kAhead = NR - 1;
    int64_t issued = 0, landed = 0;
    for (; issued < kAhead && advance_load(); ++issued) {
      issue(cl, (int)issued);
      cursor_next<BATCHED>(a, cl);
    }
    int64_t s = 0;
    for (; !timed_out; ++s) {
      if (advance_load()) {
        const int slot1 = (int)(issued % NR);
        const int64_t use1 = issued / NR;
        if (use1 > 0 && !mbar_wait(&raw_empty[slot1], (uint32_t)((use1 - 1) & 1))) {
          timed_out = true;
          break;
        }
        issue(cl, slot1);
        ++issued;
        cursor_next<BATCHED>(a, cl);
      }
      if (timed_out || s >= issued) break;  // no step s: this block's work is done
      if (cur.left <= 0) cur = range_cursor<BATCHED>(a, fifo[(fout++) & 1]);
      const int slot = (int)(s % NR);
      const int q = (int)(s % NS);
      if (!mbar_wait(&raw_full[slot], (uint32_t)((s / NR) & 1))) {
        timed_out = true;
        break;
      }
      ++landed;
      if (s >= NS && !mbar_wait(&sum_empty[q], (uint32_t)(((s / NS) - 1) & 1))) {
        timed_out = true;
        break;
      }
      // Operand sums of this k-step, masked to the block's k extent.
      const ProbDesc& d = desc_of<BATCHED>(a, cur.p);
      const int row = d.plan_row + cur.r;
      const int na = min((int)c_plans.na[row], MAXT), nb = min((int)c_plans.nb[row], MAXT);
      const int64_t dhk = d.hk;
      const int dtrans_a = d.trans_a, dtrans_b = d.trans_b;
      // The sums run on binary64 bit patterns with the integer-pipe addition: no
      // floating-point value (or instruction) appears in the producer's path.
      const uint64_t* ra = reinterpret_cast<const uint64_t*>(rawA + slot * S::kRawA);
      const uint64_t* rb = reinterpret_cast<const uint64_t*>(rawB + slot * S::kRawB);
      uint64_t* sa = reinterpret_cast<uint64_t*>(sumA + q * BK * BM);
      uint64_t* sb = reinterpret_cast<uint64_t*>(sumB + q * BK * BN);
      const int64_t k0 = (int64_t)cur.ks * BK;
      // Each producer thread owns EPT consecutive k of row pt % BM of the A tile
      // (contiguous in the raw box) and of column pt % BN of the B tile.  The sums run
      // term by term over all of the thread's elements, so its EPT chains of additions
      // are independent and interleave; each chain still adds the terms left to right.
      constexpr int EPT = BM * BK / kProducers;
      static_assert(BM == BN && EPT * kProducers == BM * BK && EPT % 2 == 0, "producer element mapping");
      const int pr = pt % BM, koff = (pt / BM) * EPT;
      // Raw tiles of A^T and B^T arrive k-major ([BK][BM]) and column-major ([BN][BK]):
      // the same element (row pr, k koff + i) is then read with the other strides.
      {
        uint64_t v[EPT];
        const uint64_t s0 = (uint64_t)term_neg(c_plans.ta[row][0]) << 63;
        if (!dtrans_a) {
          const ulonglong2* r0 = reinterpret_cast<const ulonglong2*>(ra + pr * BK + koff);
#pragma unroll
          for (int h = 0; h < EPT / 2; ++h) {
            const ulonglong2 w = r0[h];
            v[2 * h] = w.x ^ s0;
            v[2 * h + 1] = w.y ^ s0;
          }
          for (int t = 1; t < na; ++t) {
            const uint64_t st = (uint64_t)term_neg(c_plans.ta[row][t]) << 63;
            const ulonglong2* rt = reinterpret_cast<const ulonglong2*>(ra + t * BM * BK + pr * BK + koff);
#pragma unroll
            for (int h = 0; h < EPT / 2; ++h) {
              const ulonglong2 w = rt[h];
              v[2 * h] = int_fadd_bits(v[2 * h], w.x ^ st);
              v[2 * h + 1] = int_fadd_bits(v[2 * h + 1], w.y ^ st);
            }
          }
        } else {
#pragma unroll
          for (int i = 0; i < EPT; ++i) v[i] = ra[(koff + i) * BM + pr] ^ s0;
          for (int t = 1; t < na; ++t) {
            const uint64_t st = (uint64_t)term_neg(c_plans.ta[row][t]) << 63;
            const uint64_t* rt = ra + t * BM * BK + pr;
#pragma unroll
            for (int i = 0; i < EPT; ++i) v[i] = int_fadd_bits(v[i], rt[(koff + i) * BM] ^ st);
          }
        }
#pragma unroll
        for (int i = 0; i < EPT; ++i) sa[(koff + i) * BM + pr] = (k0 + koff + i < dhk) ? v[i] : 0;
      }
      {
        uint64_t v[EPT];
        const uint64_t s0 = (uint64_t)term_neg(c_plans.tb[row][0]) << 63;
        if (!dtrans_b) {
#pragma unroll
          for (int i = 0; i < EPT; ++i) v[i] = rb[(koff + i) * BN + pr] ^ s0;
          for (int t = 1; t < nb; ++t) {
            const uint64_t st = (uint64_t)term_neg(c_plans.tb[row][t]) << 63;
            const uint64_t* rt = rb + t * BK * BN + pr;
#pragma unroll
            for (int i = 0; i < EPT; ++i) v[i] = int_fadd_bits(v[i], rt[(koff + i) * BN] ^ st);
          }
        } else {
          const ulonglong2* r0 = reinterpret_cast<const ulonglong2*>(rb + pr * BK + koff);
#pragma unroll
          for (int h = 0; h < EPT / 2; ++h) {
            const ulonglong2 w = r0[h];
            v[2 * h] = w.x ^ s0;
            v[2 * h + 1] = w.y ^ s0;
          }
          for (int t = 1; t < nb; ++t) {
            const uint64_t st = (uint64_t)term_neg(c_plans.tb[row][t]) << 63;
            const ulonglong2* rt = reinterpret_cast<const ulonglong2*>(rb + t * BK * BN + pr * BK + koff);
#pragma unroll
            for (int h = 0; h < EPT / 2; ++h) {
              const ulonglong2 w = rt[h];
              v[2 * h] = int_fadd_bits(v[2 * h], w.x ^ st);
              v[2 * h + 1] = int_fadd_bits(v[2 * h + 1], w.y ^ st);
            }
          }
        }
#pragma unroll
        for (int i = 0; i < EPT; ++i) sb[(koff + i) * BN + pr] = (k0 + koff + i < dhk) ? v[i] : 0;
      }
      if (pt == 0) meta[q] = StepMeta{cur.p, cur.r, cur.t, step_flags<BATCHED>(a, cur)};
      mbar_arrive(&sum_full[q]);
      mbar_arrive(&raw_empty[slot]);
      cursor_next<BATCHED>(a, cur);
    }
    if (!timed_out) {
      // End marker for the consumers in the next summed slot.
      const int q = (int)(s % NS);
      if (s >= NS && !mbar_wait(&sum_empty[q], (uint32_t)(((s / NS) - 1) & 1))) {
        timed_out = true;
      } else {
        if (pt == 0) meta[q] = StepMeta{0, 0, 0, kStepEnd};
        mbar_arrive(&sum_full[q]);
      }
    }
    if (timed_out) {
      record_timeout();
      // Let the copies this block still has in flight land (bounded) before leaving.
      for (int64_t s2 = landed; s2 < issued; ++s2) mbar_wait(&raw_full[s2 % NR], (uint32_t)((s2 / NR) & 1));
      asm volatile("cp.async.wait_all;\n" ::: "memory");
    }
    return;
  }

  // ======================= consumers =======================
  asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;\n" ::"n"(kConsumerRegs));
  const int tx = tid % (BN / TN), ty = tid / (BN / TN);
  // Consumer group of the accumulation chunks: warps 0-3 and 4-7 (warps w and w + 4
  // share an SM sub-partition, so each sub-partition keeps one computing warp while
  // the other flushes).
  const int flush_bit = (tid >> 5) < 4 ? kStepFlush0 : kStepFlush1;
  double acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;

  for (int64_t s = 0;; ++s) {
    const int q = (int)(s % NS);
    if (!mbar_wait(&sum_full[q], (uint32_t)((s / NS) & 1))) {
      record_timeout();
      return;
    }
    if (meta[q].flags & kStepEnd) break;
    const double* sa = sumA + q * BK * BM;
    const double* sb = sumB + q * BK * BN;
    // One k at a time: 64 independent FMAs per k already cover the FP64 pipe's
    // latency, and not unrolling keeps the register tile free of hoisted fragments.
#pragma unroll 1
    for (int kk = 0; kk < BK; ++kk) {
      double av[TM], bv[TN];
      const double2* pa0 = reinterpret_cast<const double2*>(sa + kk * BM + ty * (TM / 2));
      const double2* pa1 = reinterpret_cast<const double2*>(sa + kk * BM + BM / 2 + ty * (TM / 2));
      const double2* pb0 = reinterpret_cast<const double2*>(sb + kk * BN + tx * (TN / 2));
      const double2* pb1 = reinterpret_cast<const double2*>(sb + kk * BN + BN / 2 + tx * (TN / 2));
#pragma unroll
      for (int v = 0; v < TM / 4; ++v) {
        const double2 x0 = pa0[v], x1 = pa1[v];
        av[2 * v] = x0.x; av[2 * v + 1] = x0.y;
        av[TM / 2 + 2 * v] = x1.x; av[TM / 2 + 2 * v + 1] = x1.y;
      }
#pragma unroll
      for (int v = 0; v < TN / 4; ++v) {
        const double2 y0 = pb0[v], y1 = pb1[v];
        bv[2 * v] = y0.x; bv[2 * v + 1] = y0.y;
        bv[TN / 2 + 2 * v] = y1.x; bv[TN / 2 + 2 * v + 1] = y1.y;
      }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    // The step's metadata is read after the multiply-adds (it holds no registers
    // during them) and before the slot is released.
    const StepMeta m = meta[q];
    mbar_arrive(&sum_empty[q]);

    if (m.flags & (kStepLast | flush_bit)) {
      // Scatter epilogue: C_q += gamma_q * M_tile for every target of the product.
      // The tile leaves the registers one row group at a time through a per-warp
      // staging buffer, so that each warp issues coalesced atomics over whole tile rows
      // (and the register tile is not held twice).
      const ProbDesc& d = desc_of<BATCHED>(a, m.p);
      // The C coefficients: the product's own row, or for the inner products of a
      // hybrid plan the row of the (L-1)-level table it comes from (product index
      // 7^(L-1) a + b of the L-level table is inner product b of outer product a).
      const int row = d.inner_row0 < 0 ? d.plan_row + m.r
                                       : d.inner_row0 + (d.plan_row + m.r - d.target_row0) % d.inner_count;
      const int nc = d.m_target ? 1 : (int)c_plans.nc[row];
      const int tm = m.t / d.tiles_n, tn = m.t - (m.t / d.tiles_n) * d.tiles_n;
      const int warp = tid >> 5, lane = tid & 31;
      // The BLAS form's alpha scales the partial sum here; alpha = 1 (the plain
      // operation) skips the multiplies, which would otherwise take FP64-pipe slots
      // from the multiply-adds at every flush.
      if (d.alpha != 1.0) {
        const double alpha = d.alpha;
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] *= alpha;
      }
      double* stage = epi_stage + warp * (2 * BN);
      const int half = ty - 2 * warp;  // which of the warp's two thread rows
#pragma unroll
      for (int i = 0; i < TM; ++i) {
        double2* dst0 = reinterpret_cast<double2*>(stage + half * BN + tx * (TN / 2));
        double2* dst1 = reinterpret_cast<double2*>(stage + half * BN + BN / 2 + tx * (TN / 2));
#pragma unroll
        for (int v = 0; v < TN / 4; ++v) {
          dst0[v] = make_double2(acc[i][2 * v], acc[i][2 * v + 1]);
          dst1[v] = make_double2(acc[i][TN / 2 + 2 * v], acc[i][TN / 2 + 2 * v + 1]);
        }
        __syncwarp();
        // Local tile rows of this row group for the warp's two thread rows.
        const int rr0 = (i < TM / 2) ? (2 * warp) * (TM / 2) + i : BM / 2 + (2 * warp) * (TM / 2) + (i - TM / 2);
        const int rr1 = rr0 + TM / 2;
#pragma unroll 1
        for (int t = 0; t < nc; ++t) {
          const uint8_t code = d.m_target ? term_code(0, 0, 0) : c_plans.tc[row][t];
          const int neg = term_neg(code);
          const int64_t row0 = (int64_t)term_bi(code) * d.hm + (int64_t)tm * BM;
          const int64_t col0 = (int64_t)term_bj(code) * d.hn + (int64_t)tn * BN;
          const int64_t row_lim = min(d.hm - (int64_t)tm * BM, d.c_rows - row0);
          const int col_lim = (int)min(d.hn - (int64_t)tn * BN, d.c_cols - col0);
          // Row pointers and the triangle bound in registers (a batched launch reads
          // its descriptor from global memory, and each atomic below would otherwise
          // make the compiler load the fields again).  The triangle test compares the
          // tile-local column with gi - col0 (lower: j <= i, upper: j >= i).
          const int64_t ldc = d.ldc;
          double* const c_r0 = d.C + (row0 + rr0) * ldc + col0;
          double* const c_r1 = d.C + (row0 + rr1) * ldc + col0;
          const int tri = d.tri;
          const int64_t diag0 = row0 + rr0 - col0, diag1 = row0 + rr1 - col0;  // gi - col0 of the two rows
          const bool ok0 = rr0 < row_lim, ok1 = rr1 < row_lim;
#pragma unroll
          for (int q = 0; q < (2 * BN) / 32; ++q) {
            const int e = lane + 32 * q;
            const int h = e / BN, col = e - (e / BN) * BN;
            const int64_t dg = h ? diag1 : diag0;
            const bool in_tri = tri == 0 || (tri == 1 ? col <= dg : col >= dg);
            if ((h ? ok1 : ok0) && col < col_lim && in_tri)
              // red.global.add.f64, performed in the L2 (off the FP64 pipe).  Each C
              // element of a tile is always updated by the same thread, in product
              // order, so one owner per tile gives a deterministic result.
              atomicAdd((h ? c_r1 : c_r0) + col, flip_sign(stage[e], neg));
          }
        }
        __syncwarp();
      }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;
    }
  }
}

// ---------------------------------------------------------------- host side

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

struct DeviceState {
  bool ready = false;
  cudaError_t err = cudaSuccess;
  int sms = 0;
};
constexpr int kMaxDev = 64;
DeviceState g_dev[kMaxDev];
std::mutex g_mu;

template <int MAXT, bool BATCHED, int BT>
const void* kernel_fn() {
  return (const void*)fp64_strassen_kernel<MAXT, BATCHED, BT>;
}

// Kernel instance by the largest term count of the launch's products -- class c holds
// up to 2^c source tiles per operand (c = 0..3) -- and by the tile id.
constexpr int kTermClasses = kMaxLevels + 1;
template <bool BATCHED, int BT>
const void* pick_kernel_bt(int maxt_class) {
  switch (maxt_class) {
    case 0: return kernel_fn<1, BATCHED, BT>();
    case 1: return kernel_fn<2, BATCHED, BT>();
    case 2: return kernel_fn<4, BATCHED, BT>();
    default: return kernel_fn<8, BATCHED, BT>();
  }
}
const void* pick_kernel(int maxt_class, bool batched, int tile_id) {
  if (tile_id == 0) return batched ? pick_kernel_bt<true, 128>(maxt_class) : pick_kernel_bt<false, 128>(maxt_class);
  return batched ? pick_kernel_bt<true, 64>(maxt_class) : pick_kernel_bt<false, 64>(maxt_class);
}
template <int BT>
size_t smem_bytes_bt(int maxt_class) {
  switch (maxt_class) {
    case 0: return Smem<1, BT>::kBytes;
    case 1: return Smem<2, BT>::kBytes;
    case 2: return Smem<4, BT>::kBytes;
    default: return Smem<8, BT>::kBytes;
  }
}
size_t smem_bytes(int maxt_class, int tile_id) {
  return tile_id == 0 ? smem_bytes_bt<128>(maxt_class) : smem_bytes_bt<64>(maxt_class);
}

cudaError_t ensure_device(int* sms_out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceState& st = g_dev[dev];
  if (!st.ready) {
    st.ready = true;
    st.err = cudaDeviceGetAttribute(&st.sms, cudaDevAttrMultiProcessorCount, dev);
    for (int c = 0; c < kTermClasses && st.err == cudaSuccess; ++c)
      for (int b = 0; b < 2 && st.err == cudaSuccess; ++b)
        for (int t = 0; t < kTileIds && st.err == cudaSuccess; ++t)
          st.err = cudaFuncSetAttribute(pick_kernel(c, b != 0, t), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem_bytes(c, t));
    if (!g_encode && st.err == cudaSuccess) {
      cudaDriverEntryPointQueryResult q;
      void* fn = nullptr;
      if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
              cudaSuccess &&
          q == cudaDriverEntryPointSuccess)
        g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
      else
        cudaGetLastError();  // no TMA descriptors: every problem takes the cp.async path
    }
  }
  *sms_out = st.sms;
  return st.err;
}

int term_class_of(int levels, int prod_begin, int nprod) {
  int mx = 1;
  for (int r = prod_begin; r < prod_begin + nprod; ++r) {
    const int row = kPlanOffset[levels] + r;
    mx = std::max(mx, (int)std::max(kPlanTables.na[row], kPlanTables.nb[row]));
  }
  return mx <= 1 ? 0 : (mx <= 2 ? 1 : (mx <= 4 ? 2 : 3));
}

bool encode_2d(CUtensorMap* map, const double* base, int64_t rows, int64_t cols, int64_t ld, int box_cols,
               int box_rows) {
  if (!g_encode) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * sizeof(double))};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, (void*)base, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Fills a device descriptor from a launch with the tile edge of L.tile.  TMA is used
// when every box coordinate the kernel will issue is 16-byte aligned in the innermost
// dimension and the operands' base addresses and row strides are 16-byte multiples.
void fill_desc(const Fp64Launch& L, ProbDesc* d) {
  const int BT = tile_edge(L.tile);
  std::memset(d, 0, sizeof(*d));
  d->A = L.A; d->B = L.B; d->C = L.C;
  d->lda = L.lda; d->ldb = L.ldb; d->ldc = L.ldc;
  d->a_rows = L.a_rows; d->a_cols = L.a_cols; d->b_rows = L.b_rows; d->b_cols = L.b_cols;
  d->c_rows = L.c_rows; d->c_cols = L.c_cols;
  d->hm = L.hm; d->hn = L.hn; d->hk = L.hk;
  const int nprod = L.nprod < 0 ? kPlanCount[L.levels] - L.prod_begin : L.nprod;
  d->plan_row = kPlanOffset[L.levels] + L.prod_begin;
  d->nprod = nprod;
  d->m_target = L.m_target;
  d->epi = L.epi;
  d->tiles_m = (int)((L.hm + BT - 1) / BT);
  d->tiles_n = (int)((L.hn + BT - 1) / BT);
  d->ksteps = (int)((L.hk + BK - 1) / BK);
  d->trans_a = L.trans_a;
  d->trans_b = L.trans_b;
  d->tri = L.levels == 0 ? L.tri : 0;
  d->target_row0 = kPlanOffset[L.levels];
  d->inner_row0 = (L.inner_targets && L.levels >= 2) ? kPlanOffset[L.levels - 1] : -1;
  d->inner_count = L.levels >= 1 ? kPlanCount[L.levels - 1] : 1;
  d->alpha = L.alpha;
  d->flush_steps = accumulation_chunk_k(L.levels) / BK;
  // The innermost TMA coordinate is a block offset along k (A), n (B), m (A^T) or k
  // (B^T) plus a multiple of the tile: those block edges must be even.
  const bool edges_even = L.levels == 0 || (L.hk % 2 == 0 && L.hn % 2 == 0 && (!L.trans_a || L.hm % 2 == 0));
  const bool aligned = ((uintptr_t)L.A % 16 == 0) && ((uintptr_t)L.B % 16 == 0) && (L.lda % 2 == 0) &&
                       (L.ldb % 2 == 0) && edges_even &&
                       L.a_cols < (1LL << 31) && L.a_rows < (1LL << 31) && L.b_cols < (1LL << 31) &&
                       L.b_rows < (1LL << 31);
  // Tensor maps over the stored matrices: A (m x k) or A^T's storage (k x m), B (k x n)
  // or B^T's storage (n x k).
  const bool ma = L.trans_a ? encode_2d(&d->tmA, L.A, L.a_cols, L.a_rows, L.lda, BT, BK)
                            : encode_2d(&d->tmA, L.A, L.a_rows, L.a_cols, L.lda, BK, BT);
  const bool mb = L.trans_b ? encode_2d(&d->tmB, L.B, L.b_cols, L.b_rows, L.ldb, BK, BT)
                            : encode_2d(&d->tmB, L.B, L.b_rows, L.b_cols, L.ldb, BT, BK);
  d->use_tma = aligned && ma && mb;
}

}  // namespace

int device_sm_count() {
  int sms = 0;
  ensure_device(&sms);
  return sms;
}

// Estimated time (FMA-equivalents on the busiest SM) of a launch with a tile and a
// schedule: every k-step of a tile costs its padded FMAs (64-wide tiles carry a small
// penalty for their larger share of staging work per FMA) plus a fixed hand-over
// overhead; stream-K spreads the (unit, k-step) iterations evenly, the owner schedule
// gives whole tile positions (all products, all of k) to one block each.
static double estimate(const Fp64Launch& L, int sched, int nprod, int sms, int tile_id) {
  const int BT = tile_edge(tile_id);
  const double tiles_m = (double)((L.hm + BT - 1) / BT), tiles_n = (double)((L.hn + BT - 1) / BT);
  const double ksteps = (double)((L.hk + BK - 1) / BK);
  const double step = (double)BT * BT * BK * (tile_id == 0 ? 1.0 : small_tile_factor(L.levels)) + kStepOverheadFma;
  if (sched == kSchedStreamK) return step * std::ceil(nprod * tiles_m * tiles_n * ksteps / sms);
  return step * ksteps * nprod * std::ceil(tiles_m * tiles_n / sms);
}

double fp64_launch_estimate(const Fp64Launch& L, int tile_id, int sms) {
  const int nprod = L.nprod < 0 ? kPlanCount[L.levels] - L.prod_begin : L.nprod;
  return estimate(L, kSchedStreamK, nprod, sms, tile_id);
}

static int choose_fp64_tile(const Fp64Launch& L, int sms) {
  const int nprod = L.nprod < 0 ? kPlanCount[L.levels] - L.prod_begin : L.nprod;
  const double t0 = estimate(L, kSchedStreamK, nprod, sms, 0);
  const double t1 = estimate(L, kSchedStreamK, nprod, sms, 1);
  return t1 < t0 ? 1 : 0;
}

void choose_fp64_schedule(Fp64Launch* L, int prefer_deterministic) {
  int sms = 0;
  ensure_device(&sms);
  if (sms <= 0) sms = 1;
  if (L->tile < 0 || L->tile >= kTileIds) L->tile = choose_fp64_tile(*L, sms);
  const int nprod = L->nprod < 0 ? kPlanCount[L->levels] - L->prod_begin : L->nprod;
  const double so = estimate(*L, kSchedOwner, nprod, sms, L->tile);
  const double ss = estimate(*L, kSchedStreamK, nprod, sms, L->tile);
  // Owner scheduling is deterministic (one writer per C tile, fixed product order):
  // keep it unless stream-K is more than 3% faster by the estimate.
  const bool owner = prefer_deterministic || so <= ss * 1.03;
  L->sched = owner ? kSchedOwner : kSchedStreamK;
}

cudaError_t launch_fp64(const Fp64Launch& L, cudaStream_t stream) {
  int sms = 0;
  cudaError_t e = ensure_device(&sms);
  if (e != cudaSuccess) return e;
  if (L.levels < 0 || L.levels > kMaxLevels) return cudaErrorInvalidValue;
  KArgs args;
  std::memset(&args, 0, sizeof(args));
  Fp64Launch Lt = L;
  if (Lt.tile < 0 || Lt.tile >= kTileIds) Lt.tile = choose_fp64_tile(Lt, sms);
  fill_desc(Lt, &args.single);
  const ProbDesc& d = args.single;
  if (d.nprod <= 0 || d.ksteps <= 0 || d.tiles_m <= 0 || d.tiles_n <= 0) return cudaSuccess;
  args.nprob = 1;
  args.sched = L.sched;
  const int64_t tiles = (int64_t)d.tiles_m * d.tiles_n;
  int64_t grid;
  if (L.sched == kSchedStreamK) {
    args.total = (int64_t)d.nprod * tiles * d.ksteps;
    grid = std::min<int64_t>(sms, args.total);
    args.dp_rounds = ((int64_t)d.nprod * tiles) / grid;  // whole-unit rounds; the rest is split
  } else {
    args.total = tiles;
    grid = std::min<int64_t>(sms, tiles);
  }
  const int cls = term_class_of(L.levels, L.prod_begin, d.nprod);
  void* kargs[] = {&args};
  return cudaLaunchKernel(pick_kernel(cls, false, Lt.tile), dim3((unsigned)grid), dim3(kThreads), kargs,
                          smem_bytes(cls, Lt.tile), stream);
}

// ---------------------------------------------------------------- batched

namespace {

// The work list of a batched call travels as kernel parameters (captured by value
// when the call is captured in a CUDA graph) to a small kernel that copies the
// descriptors -- TMA tensor maps encoded on the host included -- into the device
// array the persistent kernel reads.
constexpr int kDescPerExpand = (32000 - 64) / (int)sizeof(ProbDesc);
constexpr int kClaimSteps = 32;
struct ExpandArgs {
  ProbDesc* out;
  unsigned long long* counter;  // cleared when not null
  int count;
  ProbDesc d[kDescPerExpand];
};

__global__ void expand_batch_kernel(const __grid_constant__ ExpandArgs a) {
  if (a.counter != nullptr && threadIdx.x == 0) *a.counter = 0ULL;
  const int words = (int)(sizeof(ProbDesc) / sizeof(uint4));
  for (int w = threadIdx.x; w < a.count * words; w += blockDim.x) {
    const int i = w / words, o = w - (w / words) * words;
    reinterpret_cast<uint4*>(&a.out[i])[o] = reinterpret_cast<const uint4*>(&a.d[i])[o];
  }
  // The tensor maps were written through the generic proxy; the persistent kernel
  // acquires them for the tensor-map proxy before use.
  asm volatile("fence.proxy.tensormap::generic.release.gpu;\n" ::: "memory");
}

// A kernel whose only thread waits on an mbarrier that nothing completes, with the
// given limit: exercises the bounded-wait path (status word set, kernel returns).
__global__ void wait_timeout_check_kernel(long long limit) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  if (!mbar_wait(&bar, 0, limit)) record_timeout();
}

}  // namespace

// Descriptors, then the chunk counter.
size_t fp64_batched_scratch_bytes(int count) { return sizeof(ProbDesc) * (size_t)std::max(count, 1) + 256; }

cudaError_t launch_fp64_batched(const Fp64Launch* probs, int count, void* scratch, cudaStream_t stream) {
  int sms = 0;
  cudaError_t e = ensure_device(&sms);
  if (e != cudaSuccess) return e;
  // One tile edge for the whole launch: the callers' choice when they agree, else the
  // one with the smaller summed estimate.
  int tile = probs[0].tile;
  for (int i = 1; i < count; ++i)
    if (probs[i].tile != tile) tile = -1;
  if (tile < 0 || tile >= kTileIds) {
    double est[kTileIds] = {0.0, 0.0};
    for (int i = 0; i < count; ++i)
      for (int t = 0; t < kTileIds; ++t) est[t] += fp64_launch_estimate(probs[i], t, 1);
    tile = est[1] < est[0] ? 1 : 0;
  }
  std::vector<ProbDesc> descs;
  descs.reserve(count);
  int cls = 0;
  for (int i = 0; i < count; ++i) {
    ProbDesc d;
    Fp64Launch L = probs[i];
    L.epi = kEpiAtomicAdd;
    L.sched = kSchedStreamK;
    L.tile = tile;
    fill_desc(L, &d);
    if (d.nprod <= 0 || d.ksteps <= 0 || d.tiles_m <= 0 || d.tiles_n <= 0) continue;
    cls = std::max(cls, term_class_of(L.levels, L.prod_begin, d.nprod));
    descs.push_back(d);
  }
  // Longest units first (a claim is one whole unit, so the last claims, which set the
  // tail, are the shortest); within a problem the units go product by product, tile by
  // tile, so the blocks that run at the same time work on neighbouring tiles of one
  // product at about the same k and share operand tiles in the L2.
  std::stable_sort(descs.begin(), descs.end(), [](const ProbDesc& x, const ProbDesc& y) { return x.ksteps > y.ksteps; });
  // A claim takes whole units of one problem, enough for at least kClaimSteps k-steps, so
  // that the claim hand-over (a global atomic and a handshake between the producers) is
  // paid rarely on problems with short units (three levels of a small product).
  int64_t total = 0, claims = 0;
  for (ProbDesc& d : descs) {
    d.iter_begin = total;
    d.claim_begin = claims;
    d.units = (int64_t)d.nprod * d.tiles_m * d.tiles_n;
    d.units_per_claim = std::max(1, kClaimSteps / d.ksteps);
    claims += (d.units + d.units_per_claim - 1) / d.units_per_claim;
    total += d.units * d.ksteps;
  }
  if (descs.empty()) return cudaSuccess;
  ProbDesc* dev = (ProbDesc*)scratch;
  unsigned long long* counter = reinterpret_cast<unsigned long long*>(dev + std::max(count, 1));
  ExpandArgs* ea = new (std::nothrow) ExpandArgs;
  if (!ea) return cudaErrorMemoryAllocation;
  for (size_t off = 0; off < descs.size() && e == cudaSuccess; off += kDescPerExpand) {
    ea->out = dev + off;
    ea->counter = off == 0 ? counter : nullptr;
    ea->count = (int)std::min<size_t>(kDescPerExpand, descs.size() - off);
    std::memcpy(ea->d, descs.data() + off, sizeof(ProbDesc) * ea->count);
    void* xargs[] = {ea};
    e = cudaLaunchKernel((const void*)expand_batch_kernel, dim3(1), dim3(256), xargs, 0, stream);
  }
  delete ea;
  if (e != cudaSuccess) return e;
  KArgs args;
  std::memset(&args, 0, sizeof(args));
  args.descs = dev;
  args.chunk_counter = counter;
  args.nprob = (int)descs.size();
  args.sched = kSchedStreamK;
  args.total = total;
  args.nchunks = claims;  // blocks claim until none are left
  const int64_t grid = std::min<int64_t>(sms, args.nchunks);
  void* kargs[] = {&args};
  return cudaLaunchKernel(pick_kernel(cls, true, tile), dim3((unsigned)grid), dim3(kThreads), kargs,
                          smem_bytes(cls, tile), stream);
}

namespace {

// Diagnostic: count pairs where the integer-pipe addition differs bitwise from the
// hardware DADD.  Pairs come from a counter-based hash (splitmix64) of (seed, index),
// mixing arbitrary bit patterns, moderate values and near-cancelling neighbours.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ULL;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
  return x ^ (x >> 31);
}

__global__ void int_fadd_check_kernel(long long count, unsigned long long seed, unsigned long long* mismatches) {
  unsigned long long local = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long r1 = splitmix64(seed ^ (2 * (unsigned long long)i));
    const unsigned long long r2 = splitmix64(seed ^ (2 * (unsigned long long)i + 1));
    double a, b;
    switch (r1 & 3) {
      case 0:  // arbitrary bit patterns
        a = __longlong_as_double((long long)r1);
        b = __longlong_as_double((long long)r2);
        break;
      case 1:  // neighbours: heavy cancellation
        a = __longlong_as_double((long long)((r1 & 0x800fffffffffffffULL) | 0x3ff0000000000000ULL));
        b = __longlong_as_double((long long)(((unsigned long long)__double_as_longlong(a) ^ (r2 & 0xfffULL)) ^
                                             (r2 & 0x8000000000000000ULL)));
        break;
      case 2:  // subnormals and tiny normals
        a = __longlong_as_double((long long)(r1 & 0x801fffffffffffffULL));
        b = __longlong_as_double((long long)(r2 & 0x801fffffffffffffULL));
        break;
      default:  // moderate values with exponent gaps up to 70
        a = scalbn((double)(r1 >> 11) * 0x1p-53, (int)(r2 % 60) - 30);
        b = scalbn((double)(r2 >> 11) * 0x1p-53 * ((r1 >> 1) & 1 ? 1.0 : -1.0), (int)(r2 % 60) - 30 - (int)(r1 % 71));
        break;
    }
    for (int neg = 0; neg < 2; ++neg) {
      const double want = neg ? __dsub_rn(a, b) : __dadd_rn(a, b);
      const double got = int_fadd(a, b, neg != 0);
      const bool same = (want != want) ? (got != got) : (__double_as_longlong(want) == __double_as_longlong(got));
      if (!same) ++local;
    }
  }
  if (local) atomicAdd(mismatches, local);
}

}  // namespace

cudaError_t check_int_fadd(long long count, unsigned long long seed, unsigned long long* mismatches_host,
                           cudaStream_t stream) {
  unsigned long long* d = nullptr;
  cudaError_t e = cudaMallocAsync(&d, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(d, 0, sizeof(unsigned long long), stream);
  if (e == cudaSuccess) {
    int_fadd_check_kernel<<<std::max(device_sm_count(), 1) * 4, 256, 0, stream>>>(count, seed, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(mismatches_host, d, sizeof(unsigned long long), cudaMemcpyDeviceToHost, stream);
  cudaFreeAsync(d, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  return e;
}

cudaError_t launch_wait_timeout_check(long long limit_cycles, cudaStream_t stream) {
  wait_timeout_check_kernel<<<1, 32, 0, stream>>>(limit_cycles);
  return cudaGetLastError();
}

int fp64_device_status(cudaStream_t stream) {
  if (cudaStreamSynchronize(stream) != cudaSuccess) return STRASSEN_ERR_CUDA;
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_fp64_status, sizeof(int)) != cudaSuccess) return STRASSEN_ERR_CUDA;
  if (v != 0) {
    const int zero = 0;
    if (cudaMemcpyToSymbol(g_fp64_status, &zero, sizeof(int)) != cudaSuccess) return STRASSEN_ERR_CUDA;
  }
  return v;
}

}  // namespace sgb
