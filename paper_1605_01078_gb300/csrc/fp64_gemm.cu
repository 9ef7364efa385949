// FP64 product kernel: the general operation of Eq. 4 on GB300.
//
// One persistent launch runs every product M_r of a plan (Figure 1 / Figure 2 table)
// over a set of work units (product r, output tile of the block, k-steps).  Per k-step
// a thread block
//   1. stages the 1..4 source tiles of A (blocks X_s) and of B (blocks V_t) into a
//      shared-memory ring with cp.async (8-byte copies, zero-filled outside the block
//      and outside the matrix: the virtual padding of Section 3.3),
//   2. forms the operand sums sum_s delta_s X_s and sum_t eps_t V_t from that ring into
//      a double-buffered "summed" tile (the packing-time sums of Section 3.4: no
//      temporary in global memory),
//   3. accumulates M_tile += A_sum * B_sum with FP64 fused multiply-adds in registers
//      (an 8x8 or 4x4 register tile per thread),
// and after the last k-step of a unit adds gamma_q * M_tile into every C block q the
// product updates (the fused scatter of the micro-kernel, Section 3.4).
//
// GB300 design notes.  FP64 runs at about 2 FMA lanes per clock per SM (measured
// 1.20 TFLOP/s for the whole GPU, DMMA 1.06), so every kernel here is bound by the
// FP64 pipe by more than two orders of magnitude over HBM: the design minimises FP64
// instructions (operand sums are formed once per staged tile, C updates once per unit,
// negations are sign-bit flips) and balances work across the 152 SMs exactly
// (stream-K ranges of the (unit, k-step) space), instead of chasing memory traffic.
// Atomic C updates (red.global.add.f64) execute in the L2, not in the SM's FP64 pipe.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "internal.h"

namespace sgb {
namespace {

struct KParams {
  const double* A;
  const double* B;
  double* C;
  int64_t lda, ldb, ldc;
  int64_t a_rows, a_cols, b_rows, b_cols, c_rows, c_cols;
  int64_t hm, hn, hk;
  int64_t total;  // stream-K: nprod * tiles * ksteps iterations; owner: tile positions
  int nprod;
  int tiles_m, tiles_n, ksteps;
  int epi, sched;
  uint8_t na[kMaxProducts], nb[kMaxProducts], nc[kMaxProducts];
  uint8_t ta[kMaxProducts][kMaxTerms], tb[kMaxProducts][kMaxTerms], tc[kMaxProducts][kMaxTerms];
};

__device__ __forceinline__ double flip_sign(double x, int neg) {
  return __longlong_as_double(__double_as_longlong(x) ^ ((long long)neg << 63));
}

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

struct Step {
  int r, tm, tn, ks;
  bool last;  // last k-step of this unit inside this block's range: run the epilogue
};

// Local step j of this block -> (product, tile, k-step).
__device__ __forceinline__ Step decode(const KParams& p, int64_t beg, int64_t end, int64_t j) {
  Step s;
  const int tiles = p.tiles_m * p.tiles_n;
  if (p.sched == kSchedStreamK) {
    const int64_t g = beg + j;
    const int64_t u = g / p.ksteps;
    s.ks = (int)(g - u * p.ksteps);
    s.r = (int)(u / tiles);
    const int t = (int)(u - (int64_t)s.r * tiles);
    s.tm = t / p.tiles_n;
    s.tn = t - s.tm * p.tiles_n;
    s.last = (s.ks == p.ksteps - 1) || (g == end - 1);
  } else {
    const int64_t per_tile = (int64_t)p.nprod * p.ksteps;
    const int64_t q = j / per_tile;
    const int64_t rem = j - q * per_tile;
    s.r = (int)(rem / p.ksteps);
    s.ks = (int)(rem - (int64_t)s.r * p.ksteps);
    const int t = (int)(blockIdx.x + q * gridDim.x);
    s.tm = t / p.tiles_n;
    s.tn = t - s.tm * p.tiles_n;
    s.last = (s.ks == p.ksteps - 1);
  }
  return s;
}

template <int BM, int BN, int BK, int TM, int TN, int MAXT, int NS>
struct Cfg {
  static constexpr int kThreads = (BM / TM) * (BN / TN);
  static constexpr int kRawA = MAXT * BK * BM;  // doubles per stage
  static constexpr int kRawB = MAXT * BK * BN;
  static constexpr size_t kSmem = sizeof(double) * (size_t)(NS * (kRawA + kRawB) + 2 * BK * (BM + BN));
};

template <int BM, int BN, int BK, int TM, int TN, int MAXT, int NS>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
fp64_strassen_kernel(const __grid_constant__ KParams p) {
  using C_ = Cfg<BM, BN, BK, TM, TN, MAXT, NS>;
  constexpr int NT = C_::kThreads;
  static_assert((BM * BK) % NT == 0 && (BN * BK) % NT == 0, "tile/thread mismatch");
  extern __shared__ __align__(16) double smem[];
  double* rawA = smem;                         // [NS][MAXT][BK][BM]
  double* rawB = rawA + NS * C_::kRawA;        // [NS][MAXT][BK][BN]
  double* sumA = rawB + NS * C_::kRawB;        // [2][BK][BM]
  double* sumB = sumA + 2 * BK * BM;           // [2][BK][BN]

  const int tid = threadIdx.x;
  // This block's share of the work.
  int64_t beg = 0, end = 0, count = 0;
  if (p.sched == kSchedStreamK) {
    beg = (p.total * (int64_t)blockIdx.x) / gridDim.x;
    end = (p.total * (int64_t)(blockIdx.x + 1)) / gridDim.x;
    count = end - beg;
  } else {
    const int64_t owned = (p.total > blockIdx.x) ? (p.total - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    count = owned * p.nprod * p.ksteps;
  }
  if (count <= 0) return;

  // Issue the cp.async copies of the source tiles of step j into ring slot j % NS.
  auto load_step = [&](int64_t j) {
    const Step s = decode(p, beg, end, j);
    const int slot = (int)(j % NS);
    double* ra = rawA + slot * C_::kRawA;
    double* rb = rawB + slot * C_::kRawB;
    const int na = min((int)p.na[s.r], MAXT), nb = min((int)p.nb[s.r], MAXT);
    for (int t = 0; t < na; ++t) {
      const uint8_t code = p.ta[s.r][t];
      const int64_t r0 = (int64_t)term_bi(code) * p.hm, c0 = (int64_t)term_bj(code) * p.hk;
#pragma unroll
      for (int q = 0; q < (BM * BK) / NT; ++q) {
        const int e = tid + q * NT;
        const int i = e / BK, kk = e - (e / BK) * BK;
        const int64_t li = (int64_t)s.tm * BM + i, lk = (int64_t)s.ks * BK + kk;
        const int64_t gr = r0 + li, gc = c0 + lk;
        const bool ok = li < p.hm && lk < p.hk && gr < p.a_rows && gc < p.a_cols;
        const double* src = ok ? p.A + gr * p.lda + gc : p.A;
        cp_async8(ra + (t * BK + kk) * BM + i, src, ok ? 8 : 0);
      }
    }
    for (int t = 0; t < nb; ++t) {
      const uint8_t code = p.tb[s.r][t];
      const int64_t r0 = (int64_t)term_bi(code) * p.hk, c0 = (int64_t)term_bj(code) * p.hn;
#pragma unroll
      for (int q = 0; q < (BN * BK) / NT; ++q) {
        const int e = tid + q * NT;
        const int kk = e / BN, jj = e - (e / BN) * BN;
        const int64_t lk = (int64_t)s.ks * BK + kk, lj = (int64_t)s.tn * BN + jj;
        const int64_t gr = r0 + lk, gc = c0 + lj;
        const bool ok = lk < p.hk && lj < p.hn && gr < p.b_rows && gc < p.b_cols;
        const double* src = ok ? p.B + gr * p.ldb + gc : p.B;
        cp_async8(rb + (t * BK + kk) * BN + jj, src, ok ? 8 : 0);
      }
    }
  };

  // Operand sums of step j: summed tile = sum_t sign_t * source tile t.
  auto sum_step = [&](int64_t j) {
    const Step s = decode(p, beg, end, j);
    const int slot = (int)(j % NS);
    const double* ra = rawA + slot * C_::kRawA;
    const double* rb = rawB + slot * C_::kRawB;
    double* sa = sumA + (int)(j & 1) * BK * BM;
    double* sb = sumB + (int)(j & 1) * BK * BN;
    const int na = min((int)p.na[s.r], MAXT), nb = min((int)p.nb[s.r], MAXT);
#pragma unroll
    for (int q = 0; q < (BM * BK) / NT; ++q) {
      const int e = tid + q * NT;
      double v = flip_sign(ra[e], term_neg(p.ta[s.r][0]));
      for (int t = 1; t < na; ++t) {
        const double x = ra[t * BK * BM + e];
        v = term_neg(p.ta[s.r][t]) ? v - x : v + x;
      }
      sa[e] = v;
    }
#pragma unroll
    for (int q = 0; q < (BN * BK) / NT; ++q) {
      const int e = tid + q * NT;
      double v = flip_sign(rb[e], term_neg(p.tb[s.r][0]));
      for (int t = 1; t < nb; ++t) {
        const double x = rb[t * BK * BN + e];
        v = term_neg(p.tb[s.r][t]) ? v - x : v + x;
      }
      sb[e] = v;
    }
  };

  // Register tile: rows {ty*TM/2 + i, BM/2 + ty*TM/2 + i}, cols likewise.
  const int tx = tid % (BN / TN), ty = tid / (BN / TN);
  double acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int jn = 0; jn < TN; ++jn) acc[i][jn] = 0.0;

  auto row_of = [&](int i) { return (i < TM / 2) ? ty * (TM / 2) + i : BM / 2 + ty * (TM / 2) + (i - TM / 2); };
  auto col_of = [&](int jn) { return (jn < TN / 2) ? tx * (TN / 2) + jn : BN / 2 + tx * (TN / 2) + (jn - TN / 2); };

  auto epilogue = [&](const Step& s) {
    const int nc = p.nc[s.r];
    for (int t = 0; t < nc; ++t) {
      const uint8_t code = p.tc[s.r][t];
      const int neg = term_neg(code);
      const int64_t r0 = (int64_t)term_bi(code) * p.hm, c0 = (int64_t)term_bj(code) * p.hn;
#pragma unroll
      for (int i = 0; i < TM; ++i) {
        const int64_t li = (int64_t)s.tm * BM + row_of(i);
        const int64_t gr = r0 + li;
        if (li >= p.hm || gr >= p.c_rows) continue;
        double* crow = p.C + gr * p.ldc;
#pragma unroll
        for (int jn = 0; jn < TN; ++jn) {
          const int64_t lj = (int64_t)s.tn * BN + col_of(jn);
          const int64_t gc = c0 + lj;
          if (lj >= p.hn || gc >= p.c_cols) continue;
          if (p.epi == kEpiAtomicAdd) {
            atomicAdd(crow + gc, flip_sign(acc[i][jn], neg));
          } else if (p.epi == kEpiRmw) {
            crow[gc] = neg ? crow[gc] - acc[i][jn] : crow[gc] + acc[i][jn];
          } else {
            crow[gc] = flip_sign(acc[i][jn], neg);
          }
        }
      }
    }
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int jn = 0; jn < TN; ++jn) acc[i][jn] = 0.0;
  };

  // Prologue: fill NS-1 ring slots, then form the sums of step 0.
#pragma unroll
  for (int q = 0; q < NS - 1; ++q) {
    if (q < count) load_step(q);
    cp_async_commit();
  }
  cp_async_wait<NS - 2>();
  __syncthreads();
  sum_step(0);

  for (int64_t j = 0; j < count; ++j) {
    if (j + NS - 1 < count) load_step(j + NS - 1);
    cp_async_commit();
    cp_async_wait<NS - 2>();  // step j+1 has landed (this thread's copies)
    __syncthreads();          // ... everyone's; summed[j&1] complete; summed[(j+1)&1] free
    if (j + 1 < count) sum_step(j + 1);
    const double* sa = sumA + (int)(j & 1) * BK * BM;
    const double* sb = sumB + (int)(j & 1) * BK * BN;
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[TM], b[TN];
      const double2* pa0 = reinterpret_cast<const double2*>(sa + kk * BM + ty * (TM / 2));
      const double2* pa1 = reinterpret_cast<const double2*>(sa + kk * BM + BM / 2 + ty * (TM / 2));
      const double2* pb0 = reinterpret_cast<const double2*>(sb + kk * BN + tx * (TN / 2));
      const double2* pb1 = reinterpret_cast<const double2*>(sb + kk * BN + BN / 2 + tx * (TN / 2));
#pragma unroll
      for (int v = 0; v < TM / 4; ++v) {
        const double2 x0 = pa0[v], x1 = pa1[v];
        a[2 * v] = x0.x; a[2 * v + 1] = x0.y;
        a[TM / 2 + 2 * v] = x1.x; a[TM / 2 + 2 * v + 1] = x1.y;
      }
#pragma unroll
      for (int v = 0; v < TN / 4; ++v) {
        const double2 y0 = pb0[v], y1 = pb1[v];
        b[2 * v] = y0.x; b[2 * v + 1] = y0.y;
        b[TN / 2 + 2 * v] = y1.x; b[TN / 2 + 2 * v + 1] = y1.y;
      }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int jn = 0; jn < TN; ++jn) acc[i][jn] = fma(a[i], b[jn], acc[i][jn]);
    }
    const Step s = decode(p, beg, end, j);
    if (s.last) epilogue(s);
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------- host side

struct TileInfo {
  int bm, bn, bk, threads, maxt;
  size_t smem;
  const void* fn[3];  // by MAXT class: 1, 2, 4 terms
  int occ[3];
};

template <int BM, int BN, int BK, int TM, int TN, int NS>
TileInfo make_tile_info() {
  TileInfo t;
  t.bm = BM; t.bn = BN; t.bk = BK;
  t.threads = (BM / TM) * (BN / TN);
  t.maxt = 4;
  t.smem = Cfg<BM, BN, BK, TM, TN, 4, NS>::kSmem;
  t.fn[0] = (const void*)fp64_strassen_kernel<BM, BN, BK, TM, TN, 1, NS>;
  t.fn[1] = (const void*)fp64_strassen_kernel<BM, BN, BK, TM, TN, 2, NS>;
  t.fn[2] = (const void*)fp64_strassen_kernel<BM, BN, BK, TM, TN, 4, NS>;
  t.occ[0] = t.occ[1] = t.occ[2] = 0;
  return t;
}

template <int BM, int BN, int BK, int TM, int TN, int NS>
size_t smem_for(int cls) {
  return cls == 0 ? Cfg<BM, BN, BK, TM, TN, 1, NS>::kSmem
                  : cls == 1 ? Cfg<BM, BN, BK, TM, TN, 2, NS>::kSmem : Cfg<BM, BN, BK, TM, TN, 4, NS>::kSmem;
}

constexpr int kNumTiles = 2;
// Tile 0: 128x128 block tile, 8x8 per thread, 256 threads.  Tile 1: 64x64, 4x4.
TileInfo g_tiles[kNumTiles];
size_t g_smem[kNumTiles][3];
std::once_flag g_once;
int g_sms = 0;
cudaError_t g_init_err = cudaSuccess;

void init_tiles() {
  g_tiles[0] = make_tile_info<128, 128, 4, 8, 8, 3>();
  g_tiles[1] = make_tile_info<64, 64, 4, 4, 4, 3>();
  for (int c = 0; c < 3; ++c) {
    g_smem[0][c] = smem_for<128, 128, 4, 8, 8, 3>(c);
    g_smem[1][c] = smem_for<64, 64, 4, 4, 4, 3>(c);
  }
  int dev = 0;
  g_init_err = cudaGetDevice(&dev);
  if (g_init_err != cudaSuccess) return;
  g_init_err = cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
  if (g_init_err != cudaSuccess) return;
  for (int t = 0; t < kNumTiles; ++t)
    for (int c = 0; c < 3; ++c) {
      g_init_err = cudaFuncSetAttribute(g_tiles[t].fn[c], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)g_smem[t][c]);
      if (g_init_err != cudaSuccess) return;
      int occ = 0;
      g_init_err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, g_tiles[t].fn[c],
                                                                 g_tiles[t].threads, g_smem[t][c]);
      if (g_init_err != cudaSuccess) return;
      g_tiles[t].occ[c] = std::max(occ, 1);
    }
}

int term_class(const Plan& pl, int only) {
  int mx = 1;
  for (int r = 0; r < pl.nprod; ++r) {
    if (only >= 0 && r != only) continue;
    mx = std::max(mx, (int)std::max(pl.na[r], pl.nb[r]));
  }
  return mx <= 1 ? 0 : (mx <= 2 ? 1 : 2);
}

}  // namespace

int fp64_num_tiles() { return kNumTiles; }

int device_sm_count() {
  std::call_once(g_once, init_tiles);
  return g_sms;
}

// Estimated cost (FP64-pipe cycles summed over SMs, arbitrary units) of running the
// launch with tile t and schedule `sched`, counting padded-tile FMAs, operand-sum adds
// (about 1.2 FMA each, measured) and the wave quantisation of owner scheduling.
static double estimate(const Fp64Launch& L, int t, int sched, int nprod, double avg_extra_terms) {
  const TileInfo& ti = g_tiles[t];
  const int64_t tiles_m = (L.hm + ti.bm - 1) / ti.bm, tiles_n = (L.hn + ti.bn - 1) / ti.bn;
  const int64_t ksteps = (L.hk + ti.bk - 1) / ti.bk;
  const double fma_per_unit = (double)ti.bm * ti.bn * ti.bk * ksteps;
  const double add_per_unit = 1.2 * avg_extra_terms * (double)(ti.bm + ti.bn) * ti.bk * ksteps;
  const double unit = fma_per_unit + add_per_unit;
  const double slots = (double)g_sms;  // the FP64 pipe is per SM: balance over SMs
  const double units = (double)nprod * tiles_m * tiles_n;
  if (sched == kSchedStreamK) return unit * units / slots;
  const double positions = (double)tiles_m * tiles_n;
  return unit * nprod * std::ceil(positions / slots);
}

void choose_fp64_schedule(Fp64Launch* L, int prefer_deterministic) {
  std::call_once(g_once, init_tiles);
  const Plan& pl = *L->plan;
  int nprod = L->only_product >= 0 ? 1 : pl.nprod;
  double extra = 0;
  for (int r = 0; r < pl.nprod; ++r) {
    if (L->only_product >= 0 && r != L->only_product) continue;
    extra += (pl.na[r] - 1) * 0.5 + (pl.nb[r] - 1) * 0.5;
  }
  extra /= nprod;
  double best = 1e300;
  int bt = 0, bs = kSchedOwner;
  for (int t = 0; t < kNumTiles; ++t)
    for (int s = 0; s < 2; ++s) {
      if (prefer_deterministic && s == kSchedStreamK) continue;
      // Stream-K needs atomic accumulation; a plain store epilogue cannot use it.
      if (s == kSchedStreamK && L->epi == kEpiStore) continue;
      // Owner scheduling pays full waves; prefer it (deterministic) within 2%.
      const double c = estimate(*L, t, s, nprod, extra) * (s == kSchedOwner ? 0.98 : 1.0);
      if (c < best) { best = c; bt = t; bs = s; }
    }
  L->tile = bt;
  L->sched = (ScheduleKind)bs;
  if (bs == kSchedStreamK) L->epi = kEpiAtomicAdd;
  else if (L->epi == kEpiAtomicAdd) L->epi = kEpiRmw;
}

cudaError_t launch_fp64(const Fp64Launch& L, cudaStream_t stream) {
  std::call_once(g_once, init_tiles);
  if (g_init_err != cudaSuccess) return g_init_err;
  if (L.tile < 0 || L.tile >= kNumTiles) return cudaErrorInvalidValue;
  const TileInfo& ti = g_tiles[L.tile];
  const Plan& pl = *L.plan;
  KParams p;
  std::memset(&p, 0, sizeof(p));
  p.A = L.A; p.B = L.B; p.C = L.C;
  p.lda = L.lda; p.ldb = L.ldb; p.ldc = L.ldc;
  p.a_rows = L.a_rows; p.a_cols = L.a_cols;
  p.b_rows = L.b_rows; p.b_cols = L.b_cols;
  p.c_rows = L.c_rows; p.c_cols = L.c_cols;
  p.hm = L.hm; p.hn = L.hn; p.hk = L.hk;
  int np = 0;
  for (int r = 0; r < pl.nprod; ++r) {
    if (L.only_product >= 0 && r != L.only_product) continue;
    p.na[np] = pl.na[r]; p.nb[np] = pl.nb[r]; p.nc[np] = pl.nc[r];
    std::memcpy(p.ta[np], pl.ta[r], kMaxTerms);
    std::memcpy(p.tb[np], pl.tb[r], kMaxTerms);
    std::memcpy(p.tc[np], pl.tc[r], kMaxTerms);
    ++np;
  }
  if (np == 0) return cudaErrorInvalidValue;
  p.nprod = np;
  p.tiles_m = (int)((L.hm + ti.bm - 1) / ti.bm);
  p.tiles_n = (int)((L.hn + ti.bn - 1) / ti.bn);
  p.ksteps = (int)((L.hk + ti.bk - 1) / ti.bk);
  p.epi = L.epi;
  p.sched = L.sched;
  if (L.sched == kSchedStreamK && L.epi != kEpiAtomicAdd) return cudaErrorInvalidValue;
  const int cls = term_class(pl, L.only_product);
  const int64_t tiles = (int64_t)p.tiles_m * p.tiles_n;
  int64_t grid;
  const int64_t resident = (int64_t)g_sms * ti.occ[cls];
  if (L.sched == kSchedStreamK) {
    p.total = (int64_t)np * tiles * p.ksteps;
    grid = std::min<int64_t>(resident, p.total);
  } else {
    p.total = tiles;
    grid = std::min<int64_t>(resident, tiles);
  }
  if (grid <= 0) return cudaSuccess;
  void* args[] = {&p};
  return cudaLaunchKernel(ti.fn[cls], dim3((unsigned)grid), dim3(ti.threads), args, g_smem[L.tile][cls],
                          stream);
}

}  // namespace sgb
