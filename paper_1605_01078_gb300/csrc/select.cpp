// Variant selection: which member of the family (classical, 1, 2 or 3 levels of ABC,
// AB or Naive) to run for a shape.  Section 4.2 of the paper proposes its performance
// model for exactly this choice, by problem size and thread count.
//
// Order of precedence in strassen_select():
//   1. an exhaustive-measurement record for the exact shape (strassen_tune_record);
//   2. the learned selector (an MLP over log2 m, log2 n, log2 k, the dtype and this
//      model's prediction for every candidate, which it corrects), when one is loaded
//      (strassen_selector_load) and enabled for the dtype;
//   3. the analytic model below.
//
// The analytic model restates the paper's T = T_a + T_m for this GPU: T_a counts the
// FP64 operations the kernels actually execute -- multiply-adds of the padded 128 x 128
// x 8 or 64 x 64 x 8 tiles (the GPU's analogue of the m_R x n_R micro-tile), the operand-sum and C
// additions of Naive and AB's separate kernels (the staging sums of ABC and AB run on
// the integer pipe and cost no FP64 time) -- at the FP64 pipe rate; T_m counts the extra
// passes of AB and Naive over their temporaries at the HBM rate; and each kernel launch
// costs a fixed overhead.  The FP64 rate comes from the device's SM count and clock.
// For the split-precision dtype the model is ozaki_model_seconds (tensor-core slice
// products plus the HBM passes of the splits and the recombination).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>
#include <unordered_map>

#include "internal.h"

namespace sgb {
namespace {

constexpr double kFmaPerClkPerSm = 2.0;             // FP64 pipe: 2 FMA / clk / SM (measured)
constexpr double kAddCost = 1.2;                    // a DADD costs about 1.2 DFMA (measured)
constexpr double kStageAddCost = 0.0;               // staging sums run on the integer pipe
constexpr double kBytesPerSec = 6.8e12;             // HBM, measured copy bandwidth
constexpr double kLaunchSec = 4e-6;
constexpr int kBK = 8;

double ceil_to(double x, double q) { return std::ceil(x / q) * q; }

struct Key {
  int64_t m, n, k;
  int dtype;
  bool operator==(const Key& o) const { return m == o.m && n == o.n && k == o.k && dtype == o.dtype; }
};
struct KeyHash {
  size_t operator()(const Key& k) const {
    uint64_t h = 1469598103934665603ull;
    for (uint64_t v : {(uint64_t)k.m, (uint64_t)k.n, (uint64_t)k.k, (uint64_t)k.dtype}) {
      h ^= v;
      h *= 1099511628211ull;
    }
    return (size_t)h;
  }
};
struct Choice {
  int levels, variant, tile;
};

std::mutex g_sel_mu;
std::unordered_map<Key, Choice, KeyHash> g_records;

// FP64 multiply-adds per second of the current device: SM count and peak SM clock
// from the device attributes (cached per device; GB300 values when no device answers).
double fma_per_sec() {
  static std::mutex mu;
  static double cache[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return kFmaPerClkPerSm * 152 * 2.07e9;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (cache[dev] == 0.0) {
    int sms = 0, khz = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) != cudaSuccess || sms <= 0 || khz <= 0) {
      cudaGetLastError();
      sms = 152;
      khz = 2070000;
    }
    cache[dev] = kFmaPerClkPerSm * sms * (khz * 1e3);
  }
  return cache[dev];
}

}  // namespace

double model_seconds(int64_t m, int64_t n, int64_t k, int levels, int variant, int tile) {
  Plan pl;
  if (!make_plan(levels, &pl) || tile < 0 || tile >= kNumTiles) return 1e30;
  const double edge = (double)tile_edge_of(tile);
  const double hm = (double)block_edge(m, levels), hn = (double)block_edge(n, levels),
               hk = (double)block_edge(k, levels);
  const double pm = ceil_to(hm, edge), pn = ceil_to(hn, edge), pk = ceil_to(hk, kBK);
  const double tile_factor = tile == 0 ? 1.0 : small_tile_factor(levels);
  double fma = 0, adds = 0, bytes = 0, launches = 0;
  if (levels == 0) {
    fma = pm * pn * pk;
    launches = 1;
  } else if (variant == STRASSEN_ABC || variant == STRASSEN_AB) {
    // Operand sums are re-formed for every tile, (na-1)/BN + (nb-1)/BM additions per
    // multiply-add, but on the integer pipe of the producer warps (kStageAddCost).
    for (int r = 0; r < pl.nprod; ++r) {
      fma += pm * pn * pk;
      adds += kStageAddCost / kAddCost * pm * pn * pk *
              ((pl.na[r] - 1) / edge + (pl.nb[r] - 1) / edge);
    }
    if (variant == STRASSEN_ABC) {
      launches = 1;
    } else {  // AB: clear M, product into M, C updates from M
      for (int r = 0; r < pl.nprod; ++r) {
        adds += pl.nc[r] * hm * hn;
        bytes += 8.0 * hm * hn * (1 + 1 + 2 * pl.nc[r]);
      }
      launches = 3.0 * pl.nprod;
    }
  } else {  // Naive: operand sums once, classical product into M, C updates
    for (int r = 0; r < pl.nprod; ++r) {
      fma += pm * pn * pk;
      adds += (pl.na[r] - 1) * hm * hk + (pl.nb[r] - 1) * hk * hn + pl.nc[r] * hm * hn;
      bytes += 8.0 * ((pl.na[r] + 1) * hm * hk + (pl.nb[r] + 1) * hk * hn + hm * hn * (2 + 2 * pl.nc[r]));
    }
    launches = 5.0 * pl.nprod;
  }
  return (tile_factor * fma + kAddCost * adds) / fma_per_sec() + bytes / kBytesPerSec + launches * kLaunchSec;
}

double model_seconds_dtype(int64_t m, int64_t n, int64_t k, int levels, int variant, int tile, int dtype) {
  if (dtype == STRASSEN_F64_OZ_BF16) return ozaki_model_seconds(m, n, k, levels);
  return model_seconds(m, n, k, levels, variant, tile);
}

void model_select(int64_t m, int64_t n, int64_t k, int* levels, int* variant, int* tile) {
  auto best_tile = [&](int L, int v, int* t_out) {
    double b = 1e300;
    for (int t = 0; t < kNumTiles; ++t) {
      const double x = model_seconds(m, n, k, L, v, t);
      if (x < b) { b = x; *t_out = t; }
    }
    return b;
  };
  int bt = 0;
  double best = best_tile(0, STRASSEN_ABC, &bt);
  int bl = 0, bv = STRASSEN_ABC;
  for (int L = 1; L <= kMaxLevels; ++L) {
    if (((int64_t)1 << L) > m || ((int64_t)1 << L) > n || ((int64_t)1 << L) > k) break;
    for (int v : {STRASSEN_ABC, STRASSEN_AB, STRASSEN_NAIVE}) {
      int t = 0;
      const double x = best_tile(L, v, &t);
      if (x < best * 0.99) {  // prefer fewer levels / ABC within 1%
        best = x;
        bl = L;
        bv = v;
        bt = t;
      }
    }
  }
  *levels = bl;
  *variant = bv;
  *tile = bt;
}

bool record_lookup(int64_t m, int64_t n, int64_t k, int dtype, int* levels, int* variant, int* tile) {
  std::lock_guard<std::mutex> lock(g_sel_mu);
  auto it = g_records.find(Key{m, n, k, dtype});
  if (it == g_records.end()) return false;
  *levels = it->second.levels;
  *variant = it->second.variant;
  *tile = it->second.tile;
  return true;
}

void record_store(int64_t m, int64_t n, int64_t k, int dtype, int levels, int variant, int tile) {
  std::lock_guard<std::mutex> lock(g_sel_mu);
  g_records[Key{m, n, k, dtype}] = Choice{levels, variant, tile};
}

void record_clear() {
  std::lock_guard<std::mutex> lock(g_sel_mu);
  g_records.clear();
}

}  // namespace sgb
