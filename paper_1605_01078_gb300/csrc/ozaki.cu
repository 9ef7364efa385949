// Split-precision FP64 products on the tensor cores (dtype STRASSEN_F64_OZ_BF16).
//
// Each Strassen product M_r = (sum_s delta_s X_s)(sum_t eps_t V_t) of Eq. 4 is
// computed from integer slices of its two FP64 operands (the error-free splitting of
// Ozaki, Ogita, Oishi and Rump, carried out on integer digits):
//
//   1. split (oz_split_rows; oz_colmax + oz_split_cols): form the operand sum; scale each
//      row of X^ (column of V^) by 2^-e so that it lies in (-1/2, 1/2), with e the
//      smallest integer such that the row maximum is below 2^(e-1); round to the
//      integer N = rint(x 2^(56 - e)) -- an exact scaling followed by round-to-nearest-
//      even, done here with integer operations on the bits of x -- and cut N into
//      S = 7 balanced base-256 digits (most significant first, d = floor((N + 2^(q-1))
//      / 2^q)), |d| <= 128: exact in BF16 (8 significant bits);
//   2. slice products (oz_gemm, tcgen05 + TMEM): for every weight w = s + t <= 8 (28
//      digit pairs) the exact integer G_w = sum_{s+t=w} D_s^X D_t^V.  BF16 x BF16
//      products of digits (|.| <= 2^14) are exact in FP32 and every FP32 accumulation
//      chunk holds at most 1024 of them (every partial sum an integer of magnitude at
//      most 2^24, representable in FP32), so the tensor-core accumulator stays exact;
//      the epilogue warps convert each chunk to int32 and sum the chunks of a weight
//      (at most 16384 k per segment keeps the sum below 2^31);
//   3. recombine + scatter (oz_recombine_local up to two levels, oz_recombine_scatter
//      at three): T = sum_w G_w 2^(8(8-w)) exactly in
//      128-bit integers (Horner over w, segments added), M = RN(T) 2^(e_i + f_j - 64)
//      with a single round-to-nearest-even conversion (integer operations), and
//      C_q = C_q + gamma_q M_r for every product in table order (the ABC scatter, one
//      owner thread per C element).
//
// GB300 notes.  FP64 arithmetic runs at about 2 lanes per clock per SM here, so the
// split and recombine steps use integer arithmetic for everything but the operand sums
// and the final C additions (digits are converted from 32-bit integers: a 64-bit
// integer conversion would run on the FP64 pipe); the products run on the BF16 tensor cores (tcgen05.mma
// kind::f16, accumulators in tensor memory) fed by TMA with 128-byte swizzle.  One CTA
// pair (cta_group::2) computes a 256 x 256 tile: each SM stages 128 rows of A's and 128
// rows of B's digit tile, 32 KB per k-block of 64, where a lone CTA with a 128 x 256
// tile needs 48 KB for the same products (at the full tensor rate more than the ~60 B
// per clock an SM received from the L2 in that kernel).  Every chunk drains the whole
// accumulator through tcgen05.ld: with chunks of 256 products the drains held the tensor
// pipe near two thirds busy, with 1024 they cost a few percent.  int32 chunk sums keep
// each CTA's 128 x 256 accumulator set in the epilogue warps' registers.  INT8 slices are not
// used: the INT8 tensor rate of this part (measured 150 TOP/s) is far below its BF16
// rate (1950 TFLOP/s).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "internal.h"

namespace sgb {
namespace {

__constant__ PlanTables c_oz_plans = kPlanTables;
__device__ int g_oz_status;

constexpr int kS = 7;          // digits per operand
constexpr int kB = 8;          // bits per digit: |d| <= 128, exact in BF16
constexpr int kGroups = kS;    // weights w = s + t = 2 .. kS + 1
// A CTA pair (a cluster of two CTAs, tcgen05 cta_group::2) computes one kPairM x kTN
// tile: each CTA stages kTM rows of the A digit tile and kHalfN rows of the B digit tile
// and holds kTM x kTN of the accumulator in its tensor memory.
constexpr int kTM = 128, kPairM = 256, kTN = 256, kHalfN = 128, kTK = 64;  // kTK bf16 = one 128-byte row
constexpr int kStages = 6;
constexpr int kStageBytes = (kTM + kHalfN) * 128;  // one CTA's share of a k-block
constexpr int kChunkItems = 16;  // k-blocks of 64 per exact FP32 chunk: 1024 products, |sum| <= 2^24
constexpr int kSegKB = 256;      // k-blocks per k segment: int32 group sums stay below 2^31
constexpr int kGroupRows = 8;    // pair-tile rows per group of the unit order (L2 reuse)
constexpr int kThreads = 384;    // warp 0 TMA, warp 1 MMA + TMEM, warps 4..11 epilogue
constexpr int kEpiThreads = 256, kEpiWarps = kEpiThreads / 32;
constexpr long long kWaitLimit = 2000000000LL;
constexpr int kPaceChunk = 16;          // k-block loads per pacing step
constexpr long long kPaceLimit = 10000;  // longest pause of one pacing step (about one step's MMAs)
constexpr int kLaunchRegs = 168, kLowRegs = 40, kHighRegs = 232;
static_assert(128 * kLowRegs + 256 * kHighRegs == kThreads * kLaunchRegs, "register split");

// ---------------------------------------------------------------- integer helpers

// Smallest e with |x| < 2^(e-1) for the magnitude bits `mag` of a finite double
// (0 for zero).
__device__ __forceinline__ int scale_exponent(unsigned long long mag) {
  if (mag == 0) return 0;
  const int E = (int)(mag >> 52);
  if (E > 0) return E - 1021;
  return (64 - __clzll((long long)mag)) - 1073;  // subnormal
}

// rint(x * 2^(56 - e)) as an integer, computed on the bits of x (|x| < 2^(e-1)).
__device__ __forceinline__ long long scaled_rint(unsigned long long bits, int e) {
  const unsigned long long mag = bits & 0x7fffffffffffffffULL;
  if (mag == 0) return 0;
  int E = (int)(mag >> 52);
  unsigned long long M = mag & ((1ULL << 52) - 1);
  if (E == 0) E = 1; else M |= (1ULL << 52);
  // x = M 2^(E - 1075), so x 2^(56 - e) = M 2^(E - 1019 - e)
  const int sh = E - 1019 - e;
  unsigned long long q;
  if (sh >= 0) {
    q = sh < 64 ? (M << sh) : 0;
  } else {
    const int r = -sh;
    if (r >= 63) {
      q = 0;
    } else {
      q = M >> r;
      const unsigned long long rem = M & ((1ULL << r) - 1), half = 1ULL << (r - 1);
      if (rem > half || (rem == half && (q & 1ULL))) q += 1;
    }
  }
  return (bits >> 63) ? -(long long)q : (long long)q;
}

// The S digits of N, most significant first: d = floor((N + 2^(q-1)) / 2^q).
__device__ __forceinline__ void digits_of(long long N, float* d) {
#pragma unroll
  for (int s = 1; s < kS; ++s) {
    const int q = kB * (kS - s);
    const long long v = (N + (1LL << (q - 1))) >> q;
    N -= v * (1LL << q);
    d[s - 1] = (float)(int)v;  // |v| <= 128: a 32-bit conversion (a 64-bit one runs on the FP64 pipe)
  }
  d[kS - 1] = (float)(int)N;
}

__device__ __forceinline__ unsigned long long mag_bits(unsigned long long bits) {
  return bits & 0x7fffffffffffffffULL;
}

// Bits of the operand sum x = sum_t sign_t * src[block_t](r, c), masked to the source
// extent, added left to right.  The split kernels leave the FP64 pipe idle otherwise,
// so the additions use it (DADD); the integer pipe carries the digit extraction.
__device__ __forceinline__ unsigned long long operand_sum(const double* src, int64_t ld, int64_t rows,
                                                          int64_t cols, int64_t h_r, int64_t h_c,
                                                          const uint8_t* terms, int nterms, int64_t r, int64_t c,
                                                          int trans) {
  const unsigned long long* s64 = reinterpret_cast<const unsigned long long*>(src);
  double v = 0.0;
  for (int t = 0; t < nterms; ++t) {
    const uint8_t code = terms[t];
    const int64_t gr = (int64_t)term_bi(code) * h_r + r, gc = (int64_t)term_bj(code) * h_c + c;
    unsigned long long x = 0;
    if (r < h_r && c < h_c && gr < rows && gc < cols) x = trans ? s64[gc * ld + gr] : s64[gr * ld + gc];
    x ^= (unsigned long long)term_neg(code) << 63;
    v = t == 0 ? __longlong_as_double((long long)x) : __dadd_rn(v, __longlong_as_double((long long)x));
  }
  return (unsigned long long)__double_as_longlong(v);
}

// ---------------------------------------------------------------- split kernels

struct SplitArgs {
  const double* src;
  int64_t ld, rows, cols;   // source matrix (A: m x k, B: k x n)
  int64_t h_r, h_c;         // block edges along the source's rows and columns
  int64_t h_out, h_outp;    // output rows (h_m or h_n) and padded rows
  int64_t h_k, h_kp;        // reduction length and padded length
  int plan_off;             // table row of product 0
  int trans;                // the source is stored transposed (element (r, c) at src[c * ld + r])
  __nv_bfloat16* slices;    // [P][S][h_outp][h_kp]
  int* exps;                // [P][h_outp]
  unsigned long long* vsum; // B side: [P][h_k][h_out] bits of the operand sums with more than one
                            // term, written by oz_colmax and read by oz_split_cols (null: none)
};

// Blocks are numbered with the product fastest (block b: product b % P, tile b / P), so
// that the products reading the same rows or columns of A or B run together and all but
// the first read them from the L2.  `n_products` is P.

// One block per output row i of X^ (rows of A's operand sum) and product.
__global__ void oz_split_rows(const __grid_constant__ SplitArgs a, int n_products) {
  extern __shared__ unsigned long long rowbuf[];  // h_k binary64 bit patterns
  __shared__ unsigned long long red[32];
  const int p = (int)(blockIdx.x % (unsigned)n_products);
  const int64_t i = blockIdx.x / (unsigned)n_products;
  const int row = a.plan_off + p;
  const int nt = c_oz_plans.na[row];
  uint8_t terms[kMaxTerms];
  for (int t = 0; t < kMaxTerms; ++t) terms[t] = c_oz_plans.ta[row][t];
  __nv_bfloat16* out = a.slices + ((int64_t)p * kS * a.h_outp + i) * a.h_kp;
  const int64_t slice_stride = a.h_outp * a.h_kp;
  if (i >= a.h_out) {  // padding rows
    for (int64_t k = threadIdx.x; k < a.h_kp; k += blockDim.x)
      for (int s = 0; s < kS; ++s) out[s * slice_stride + k] = __float2bfloat16(0.0f);
    if (threadIdx.x == 0) a.exps[(int64_t)p * a.h_outp + i] = 0;
    return;
  }
  unsigned long long mx = 0;
  for (int64_t k = threadIdx.x; k < a.h_k; k += blockDim.x) {
    const unsigned long long x = operand_sum(a.src, a.ld, a.rows, a.cols, a.h_r, a.h_c, terms, nt, i, k, a.trans);
    rowbuf[k] = x;
    mx = max(mx, mag_bits(x));
  }
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    unsigned long long v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0;
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) red[0] = v;
  }
  __syncthreads();
  const int e = scale_exponent(red[0]);
  if (threadIdx.x == 0) a.exps[(int64_t)p * a.h_outp + i] = e;
  for (int64_t k = threadIdx.x; k < a.h_kp; k += blockDim.x) {
    float d[kS];
    digits_of(k < a.h_k ? scaled_rint(rowbuf[k], e) : 0, d);
#pragma unroll
    for (int s = 0; s < kS; ++s) out[s * slice_stride + k] = __float2bfloat16(d[s]);
  }
}

// Column maxima of V^ (B's operand sum) for the per-column scales: one block per 64
// columns x kColMaxRows rows of the reduction dimension and product; partial
// maxima of the magnitude bits meet in `colmax_bits` (cleared before) by atomicMax
// (magnitude order equals the order of the bit patterns of non-negative doubles).
constexpr int kColMaxRows = 256;

__global__ void __launch_bounds__(256) oz_colmax(const __grid_constant__ SplitArgs a,
                                                 unsigned long long* colmax_bits, int n_products, int col_tiles) {
  __shared__ unsigned long long red[4][64];
  const int p = (int)(blockIdx.x % (unsigned)n_products);
  const unsigned blk = blockIdx.x / (unsigned)n_products;
  const int64_t j0 = (int64_t)(blk % (unsigned)col_tiles) * 64;
  const int64_t kb = (int64_t)(blk / (unsigned)col_tiles) * kColMaxRows;
  const int64_t ke = kb + kColMaxRows < a.h_k ? kb + kColMaxRows : a.h_k;
  const int row = a.plan_off + p;
  const int nt = c_oz_plans.nb[row];
  uint8_t terms[kMaxTerms];
  for (int t = 0; t < kMaxTerms; ++t) terms[t] = c_oz_plans.tb[row][t];
  const int tid = threadIdx.x, c = tid & 63, ph = tid >> 6;
  unsigned long long mx = 0;
  // Sums of several terms are kept for oz_split_cols, which then reads one value
  // instead of forming the sum again.
  unsigned long long* keep = (nt > 1 && a.vsum) ? a.vsum + (int64_t)p * a.h_k * a.h_out : nullptr;
  if (j0 + c < a.h_out)
    for (int64_t k = kb + ph; k < ke; k += 4) {
      const unsigned long long x = operand_sum(a.src, a.ld, a.rows, a.cols, a.h_r, a.h_c, terms, nt, k, j0 + c, a.trans);
      if (keep) keep[k * a.h_out + j0 + c] = x;
      mx = max(mx, mag_bits(x));
    }
  red[ph][c] = mx;
  __syncthreads();
  if (tid < 64) {
    const unsigned long long v = max(max(red[0][tid], red[1][tid]), max(red[2][tid], red[3][tid]));
    if (v != 0 && j0 + tid < a.h_out) atomicMax(&colmax_bits[(int64_t)p * a.h_outp + j0 + tid], v);
  }
}

// One block per 64 output columns j x 64 reduction indices k of V^ and product: the
// digits of the scaled column entries, written transposed ([j][k], k contiguous)
// through a shared-memory tile.  The blocks of the first 64 k also store the scale
// exponents.
constexpr int kColTilePitch = 64 + 8;  // bf16 per tile row (padding against bank conflicts)
constexpr size_t kSplitColsSmem = sizeof(__nv_bfloat16) * kS * 64 * kColTilePitch;

__global__ void __launch_bounds__(256) oz_split_cols(const __grid_constant__ SplitArgs a,
                                                     const unsigned long long* colmax_bits, int n_products,
                                                     int col_tiles) {
  __shared__ int ecol[64];
  extern __shared__ __align__(16) __nv_bfloat16 tile_raw[];  // [kS][64][kColTilePitch]
  auto tile = [&](int s, int c, int k) -> __nv_bfloat16& { return tile_raw[(s * 64 + c) * kColTilePitch + k]; };
  const int p = (int)(blockIdx.x % (unsigned)n_products);
  const unsigned blk = blockIdx.x / (unsigned)n_products;
  const int64_t j0 = (int64_t)(blk % (unsigned)col_tiles) * 64;
  const int64_t k_tile = blk / (unsigned)col_tiles;
  const int64_t k0 = k_tile * 64;
  const int row = a.plan_off + p;
  const int nt = c_oz_plans.nb[row];
  uint8_t terms[kMaxTerms];
  for (int t = 0; t < kMaxTerms; ++t) terms[t] = c_oz_plans.tb[row][t];
  const int tid = threadIdx.x;
  if (tid < 64) {
    const int64_t j = j0 + tid;
    const int e = j < a.h_out ? scale_exponent(colmax_bits[(int64_t)p * a.h_outp + j]) : 0;
    ecol[tid] = e;
    if (k_tile == 0 && j < a.h_outp) a.exps[(int64_t)p * a.h_outp + j] = e;
  }
  __syncthreads();
  const int64_t slice_stride = a.h_outp * a.h_kp;
  __nv_bfloat16* out = a.slices + (int64_t)p * kS * slice_stride;
  {
    for (int q = 0; q < 16; ++q) {
      const int e = tid + 256 * q;
      const int kk = e >> 6, cc = e & 63;
      const int64_t k = k0 + kk, j = j0 + cc;
      float d[kS];
      long long N = 0;
      if (j < a.h_out && k < a.h_k) {
        const unsigned long long x =
            (nt > 1 && a.vsum) ? a.vsum[((int64_t)p * a.h_k + k) * a.h_out + j]
                               : operand_sum(a.src, a.ld, a.rows, a.cols, a.h_r, a.h_c, terms, nt, k, j, a.trans);
        N = scaled_rint(x, ecol[cc]);
      }
      digits_of(N, d);
#pragma unroll
      for (int s = 0; s < kS; ++s) tile(s, cc, kk) = __float2bfloat16(d[s]);
    }
    __syncthreads();
    // 64 columns x 64 k per digit; each thread writes 16 consecutive k of one column.
    const int cc = tid >> 2, part = tid & 3;
    if (j0 + cc < a.h_outp) {
      for (int s = 0; s < kS; ++s) {
        __nv_bfloat16* dst = out + s * slice_stride + (j0 + cc) * a.h_kp + k0 + part * 16;
        const uint4* srcv = reinterpret_cast<const uint4*>(&tile(s, cc, part * 16));
        uint4* dstv = reinterpret_cast<uint4*>(dst);
        dstv[0] = srcv[0];
        dstv[1] = srcv[1];
      }
    }
  }
}

// ---------------------------------------------------------------- tcgen05 helpers

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// Arrival on the barrier at shared::cluster address `addr` (this CTA's or the peer's).
// The default CTA-scope release suffices: the only accesses it orders across the pair
// are tensor-memory reads, which tcgen05.fence::before_thread_sync orders before it (a
// cluster-scope release would also wait for the thread's earlier global stores).
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t addr) {
  asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];\n" ::"r"(addr) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try(bar, parity))
    if (clock64() - t0 > kWaitLimit) return false;
  return true;
}
__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_index() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;\n" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_total() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%nclusterid.x;\n" : "=r"(r));
  return r;
}
// shared::cluster address of this CTA's variable `p` in the cluster CTA `rank`.
__device__ __forceinline__ uint32_t cluster_addr(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
// TMA tile load into this CTA's shared memory whose completion is counted on the
// barrier at shared::cluster address `bar` (the leading CTA's barrier of the pair).
__device__ __forceinline__ void tma_2d_pair(void* dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cta.global.tile.mbarrier::complete_tx::bytes.cta_group::2"
      " [%0], [%1, {%2, %3}], [%4];\n" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
// Shared-memory matrix descriptor: K-major operand tile with 128-byte swizzle, rows of
// 128 bytes, 8-row swizzle atoms 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// Instruction descriptor of kind::f16: D = F32, A = B = BF16, both K-major, M = 256
// (rows 0-127 from the even CTA of the pair, 128-255 from the odd one), N = 256 (B rows
// 0-127 staged by the even CTA, 128-255 by the odd one).
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTN >> 3) << 17) |
                            ((uint32_t)(kPairM >> 4) << 24);

// One pair MMA (issued by the even CTA): D[tmem of both CTAs] (+)= A B^T over K = 16.
__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accum)
      : "memory");
}
// Arrival, once the MMAs issued so far complete, on the barrier at this offset in both CTAs.
__device__ __forceinline__ void umma_commit_pair(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;\n" ::"r"(
          smem_u32(bar)),
      "h"((uint16_t)3)
      : "memory");
}
// The same on this CTA's barrier only.
__device__ __forceinline__ void umma_commit_local(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr)
      : "memory");
}

// ---------------------------------------------------------------- slice-product kernel

struct GemmArgs {
  CUtensorMap tmA;  // DX of all products as rows [P*S*h_mp] x cols [h_kp], bf16, box 64 x 128
  CUtensorMap tmB;  // DV of all products as rows [P*S*h_np] x cols [h_kp], bf16, box 64 x 256
  int* G;           // [nseg][P][kGroups][h_mp][h_np] exact group sums G_w (w = 2 .. kS + 1) per k segment
  int P, tiles_m, tiles_n, nkb;
  int nseg;         // k segments of seg_kb <= kSegKB k-blocks (each segment's sums fit in int32)
  int seg_kb;
  int64_t h_mp, h_np;
  unsigned* pace;   // [0] pacing steps counted by the running pairs, [1] running pairs (zeroed before the launch)
};

// Number of digit pairs (s, t) with s + t = w, 1 <= s, t <= S.
__host__ __device__ constexpr int pairs_of(int w) {
  return (w - 1 < kS ? w - 1 : kS) - (w - kS > 1 ? w - kS : 1) + 1;
}

// Conversion of an FP32 chunk value (an integer, |v| <= 2^24) to int32: exact.  (Adding
// 1.5 * 2^23 and taking the bit pattern, one FADD, is exact only for |v| <= 2^22, which
// would cap a chunk at 256 products and drain the accumulator four times as often.)
__device__ __forceinline__ uint32_t f32_int(uint32_t bits) { return (uint32_t)__float2int_rz(__uint_as_float(bits)); }

// Work unit u = (product p, pair tile t, k segment g): a 256 x 256 block of every G_w of
// product p over the k-blocks of segment g (stored per segment; the recombination adds
// the segments), computed by one CTA pair (a cluster of two CTAs).  In each CTA warp 0
// issues TMA loads of the CTA's 128 rows of the A digit tile and 128 rows of the B digit
// tile into a 6-stage ring, counted on the even CTA's barrier; the even CTA's warp 1
// issues tcgen05.mma (cta_group::2, M = 256, N = 256, K = 16) into a double-buffered FP32
// accumulator (2 x 256 columns of each CTA's tensor memory: rows 0-127 in the even CTA,
// 128-255 in the odd one) and signals both CTAs; in each CTA eight epilogue warps turn
// every chunk of at most 1024 digit products (|sum| <= 2^24, exact in FP32) into int32
// and sum the chunks of a weight w in registers; at the end of each weight the exact G_w
// rows of the CTA go to global memory.  Each SM receives 32 KB of operands per 128 x 256
// x 64 share of the products, two thirds of what one CTA computing a 128 x 256 tile
// alone must load.
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1) oz_gemm(const __grid_constant__ GemmArgs a) {
  extern __shared__ __align__(1024) uint8_t sm_raw[];
  // 1024-byte aligned stage ring for the 128-byte swizzle (the same offsets in both CTAs)
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(sm_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* stA = sm;                               // [kStages][128 rows][128 B]
  uint8_t* stB = sm + kStages * kTM * 128;         // [kStages][128 rows][128 B]
  uint64_t* bars = reinterpret_cast<uint64_t*>(stB + kStages * kHalfN * 128);
  uint64_t* full = bars;                   // even CTA: both CTAs' loads of a stage landed
  uint64_t* empty = bars + kStages;        // both CTAs: the MMAs reading a stage completed
  uint64_t* tfull = bars + 2 * kStages;    // both CTAs: an accumulator buffer is complete
  uint64_t* tempty = bars + 2 * kStages + 2;  // even CTA: both CTAs' epilogues read a buffer
  uint64_t* drain = bars + 2 * kStages + 4;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kStages + 5);

  const uint32_t rank = cluster_ctarank();  // 0: issues the MMAs of the pair
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages; ++i) { mbar_init(&full[i], 1); mbar_init(&empty[i], 1); }
    for (int i = 0; i < 2; ++i) { mbar_init(&tfull[i], 1); mbar_init(&tempty[i], 2 * kEpiWarps); }
    mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  }
  if (warp == 1) {
    // collective over the pair: the same 512 columns in both CTAs
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], 512;\n" ::"r"(smem_u32(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();  // both CTAs' barriers initialised and tensor memory allocated
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  const int tiles = a.tiles_m * a.tiles_n;
  const int units = a.P * tiles * a.nseg;
  const int u_first = (int)cluster_index(), u_step = (int)cluster_total();
  // Unit u -> (product, pair tile, k segment).  Within a product the tiles go in groups
  // of kGroupRows tile rows, column by column inside a group, so that the units running
  // at the same time share their A digit rows and B digit columns in the L2.
  auto unit_of = [&](int u, int* p, int* tm, int* tn, int* kb0, int* kb1) {
    const int per_p = tiles * a.nseg;
    *p = u / per_p;
    const int rem = u - *p * per_p;
    const int t = rem / a.nseg, g = rem - (rem / a.nseg) * a.nseg;
    const int group = t / (kGroupRows * a.tiles_n);
    const int first = group * kGroupRows;
    const int rows = a.tiles_m - first < kGroupRows ? a.tiles_m - first : kGroupRows;
    const int in = t - group * kGroupRows * a.tiles_n;
    *tm = first + in % rows;
    *tn = in / rows;
    *kb0 = g * a.seg_kb;
    *kb1 = (g + 1) * a.seg_kb < a.nkb ? (g + 1) * a.seg_kb : a.nkb;
  };

  if (warp < 4) {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;\n" ::"n"(kLowRegs));
    if (warp == 0 && lane == 0) {
      // ------------------------------------------------ TMA producer (both CTAs)
      const uint32_t full0 = cluster_addr(full, 0);
      // Pacing (even CTA): the pairs that run together read the same digit tiles, and
      // the L2 keeps them only while the pairs stay close along k.  Every kPaceChunk
      // loads in the whole waves a pair counts a step in a.pace[0] and pauses (at most
      // kPaceLimit cycles; correctness never depends on it) while it is more than one
      // step ahead of the average running pair.  A pair joins at the current average
      // (one that starts late, its SMs busy with other work, holds nobody back) and on
      // leaving the whole waves takes its steps out again; the last, partial wave is
      // not paced.
      const int whole_waves_end = (units / u_step) * u_step;
      volatile unsigned* pace_v = a.pace;
      uint32_t it = 0, paced = 0;
      bool joined = false;
      if (rank == 0 && u_first < whole_waves_end) {
        const unsigned before = atomicAdd(&a.pace[1], 1u);
        paced = before > 0 ? pace_v[0] / before : 0u;
        atomicAdd(&a.pace[0], paced);
        joined = true;
      }
      bool bad = false;
      for (int u = u_first; u < units && !bad; u += u_step) {
        int p, tm, tn, kb0, kb1;
        unit_of(u, &p, &tm, &tn, &kb0, &kb1);
        if (joined && u >= whole_waves_end) {
          atomicSub(&a.pace[0], paced);
          atomicSub(&a.pace[1], 1u);
          joined = false;
        }
        const bool pace = joined;
        for (int w = 2; w <= kS + 1 && !bad; ++w) {
          const int s_lo = w - kS > 1 ? w - kS : 1, s_hi = w - 1 < kS ? w - 1 : kS;
          for (int s = s_lo; s <= s_hi && !bad; ++s) {
            const int tt = w - s;
            const int ya = (int)(((int64_t)p * kS + (s - 1)) * a.h_mp + (int64_t)tm * kPairM + kTM * rank);
            const int yb = (int)(((int64_t)p * kS + (tt - 1)) * a.h_np + (int64_t)tn * kTN + kHalfN * rank);
            for (int kb = kb0; kb < kb1; ++kb, ++it) {
              const int st = it % kStages;
              const uint32_t use = it / kStages;
              if (pace && (it % kPaceChunk) == 0) {
                ++paced;
                unsigned total = atomicAdd(&a.pace[0], 1u) + 1u, running = pace_v[1];
                const long long t0 = clock64();
                while ((unsigned long long)(paced - 1) * running > (unsigned long long)total &&
                       clock64() - t0 < kPaceLimit) {
                  __nanosleep(128);
                  total = pace_v[0];
                  running = pace_v[1];
                }
              }
              if (use > 0 && !mbar_wait(&empty[st], (use - 1) & 1)) { bad = true; break; }
              if (rank == 0) mbar_expect_tx(&full[st], 2 * kStageBytes);
              tma_2d_pair(stA + st * kTM * 128, &a.tmA, kb * kTK, ya, full0 + 8u * st);
              tma_2d_pair(stB + st * kHalfN * 128, &a.tmB, kb * kTK, yb, full0 + 8u * st);
            }
          }
        }
      }
      if (joined) {
        atomicSub(&a.pace[0], paced);
        atomicSub(&a.pace[1], 1u);
      }
      if (bad) {
        atomicExch(&g_oz_status, STRASSEN_ERR_TIMEOUT);
        const long long t0 = clock64();  // let copies in flight land before leaving
        while (clock64() - t0 < 2000000) {}
      }
    } else if (warp == 1 && lane == 0 && rank == 0) {
      // ------------------------------------------------ MMA issuer (even CTA)
      uint32_t it = 0, ch = 0;
      bool bad = false;
      for (int u = u_first; u < units && !bad; u += u_step) {
        int p, tm, tn, kb0, kb1;
        unit_of(u, &p, &tm, &tn, &kb0, &kb1);
        for (int w = 2; w <= kS + 1 && !bad; ++w) {
          const int n_items = pairs_of(w) * (kb1 - kb0);
          for (int c0 = 0; c0 < n_items && !bad; c0 += kChunkItems, ++ch) {
            const int buf = ch & 1;
            const uint32_t use = ch >> 1;
            if (use > 0 && !mbar_wait(&tempty[buf], (use - 1) & 1)) { bad = true; break; }
            tc_fence_after();
            const int c1 = c0 + kChunkItems < n_items ? c0 + kChunkItems : n_items;
            for (int i = c0; i < c1; ++i, ++it) {
              const int st = it % kStages;
              if (!mbar_wait(&full[st], (it / kStages) & 1)) { bad = true; break; }
              tc_fence_after();
              const uint64_t ad = sw128_desc(smem_u32(stA + st * kTM * 128));
              const uint64_t bd = sw128_desc(smem_u32(stB + st * kHalfN * 128));
#pragma unroll
              for (int k = 0; k < kTK / 16; ++k)
                umma(tmem + buf * kTN, ad + 2 * k, bd + 2 * k, (i > c0 || k > 0) ? 1u : 0u);
              umma_commit_pair(&empty[st]);
            }
            umma_commit_pair(&tfull[buf]);
          }
        }
      }
      // Wait (bounded) until every issued MMA has completed before tensor memory is released.
      umma_commit_local(drain);
      mbar_wait(drain, 0);
      if (bad) {
        atomicExch(&g_oz_status, STRASSEN_ERR_TIMEOUT);
      }
    }
  } else {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;\n" ::"n"(kHighRegs));
    // ------------------------------------------------ epilogue warps (both CTAs)
    const int ew = warp - 4;
    const int g = warp & 3;         // TMEM lane quarter this warp may read
    const int half = ew >> 2;       // column half (128 columns) of the tile
    const uint32_t tempty0 = cluster_addr(tempty, 0);
    uint32_t ch = 0;
    bool bad = false;
    uint32_t R[128];  // int32 group sums (unsigned arithmetic: the true sums fit in int32)
    for (int u = u_first; u < units && !bad; u += u_step) {
      int p, tm, tn, kb0, kb1;
      unit_of(u, &p, &tm, &tn, &kb0, &kb1);
      const int64_t row = (int64_t)tm * kPairM + kTM * rank + 32 * g + lane;
      const int64_t col0 = (int64_t)tn * kTN + 128 * half;
      for (int w = 2; w <= kS + 1 && !bad; ++w) {
#pragma unroll
        for (int q = 0; q < 128; ++q) R[q] = 0;
        const int n_items = pairs_of(w) * (kb1 - kb0);
        for (int c0 = 0; c0 < n_items; c0 += kChunkItems, ++ch) {
          const int buf = ch & 1;
          if (!mbar_wait(&tfull[buf], (ch >> 1) & 1)) { bad = true; break; }
          tc_fence_after();
          const uint32_t base = tmem + ((uint32_t)(32 * g) << 16) + buf * kTN + 128 * half;
#pragma unroll
          for (int q = 0; q < 4; ++q) {  // 32 columns per wait
            uint32_t v[32];
            tmem_ld32(base + 32 * q, v);
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
            for (int i = 0; i < 32; ++i) R[32 * q + i] += f32_int(v[i]);
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive_cluster(tempty0 + 8u * buf);
        }
        if (bad) break;
        const int seg = kb0 / a.seg_kb;
        int* dst = a.G + ((((int64_t)seg * a.P + p) * kGroups + (w - 2)) * a.h_mp + row) * a.h_np + col0;
        int4* d4 = reinterpret_cast<int4*>(dst);
#pragma unroll
        for (int q = 0; q < 32; ++q) d4[q] = make_int4((int)R[4 * q], (int)R[4 * q + 1], (int)R[4 * q + 2], (int)R[4 * q + 3]);
      }
    }
    if (bad) {
      atomicExch(&g_oz_status, STRASSEN_ERR_TIMEOUT);
    }
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();  // nothing of either CTA is still read or written by the other
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, 512;\n" ::"r"(tmem) : "memory");
  }
}

// ---------------------------------------------------------------- recombine + scatter

struct RecombineArgs {
  double* C;
  int64_t ldc, m, n;
  int64_t hm, hn, h_mp, h_np;
  int levels, P;
  int plan_off;   // table row of product 0 of the level
  double alpha;   // C_q += gamma_q alpha M
  const int* G;   // [nseg][P][kGroups][h_mp][h_np]
  int nseg;
  const int* e;   // [P][h_mp]
  const int* f;   // [P][h_np]
  // The products that update C block q (= qi 2^L + qj), in table order: entries
  // [first[q], first[q + 1]) of `upd`, each 2 r + (gamma < 0).
  int first[kMaxTerms * kMaxTerms + 1];
  uint16_t upd[1728];  // 12^3: the C updates of the deepest table
};

// RN(T) * 2^scale for the 128-bit two's complement integer T = th * 2^64 + tl, with
// integer operations (one rounding).
__device__ double round_i128(long long th, unsigned long long tl, int scale) {
  if (th == 0 && tl == 0) return 0.0;
  const bool neg = th < 0;
  unsigned long long mh = (unsigned long long)th, ml = tl;
  if (neg) {  // magnitude
    ml = ~ml + 1;
    mh = ~mh + (ml == 0 ? 1 : 0);
  }
  const int nb = mh ? 128 - __clzll((long long)mh) : 64 - __clzll((long long)ml);
  unsigned long long mant;
  int sh = 0;
  if (nb <= 53) {
    mant = ml;
  } else {
    sh = nb - 53;
    // mant = M >> sh, rem = M mod 2^sh
    unsigned long long rem_hi, rem_lo;
    if (sh >= 64) {
      mant = mh >> (sh - 64);
      rem_hi = (sh - 64) ? (mh & ((1ULL << (sh - 64)) - 1)) : 0;
      rem_lo = ml;
    } else {
      mant = (ml >> sh) | (sh ? (mh << (64 - sh)) : 0);
      rem_hi = 0;
      rem_lo = ml & ((1ULL << sh) - 1);
    }
    // compare rem with half = 2^(sh-1)
    int cmp;
    if (sh - 1 >= 64) {
      const unsigned long long hh = 1ULL << (sh - 1 - 64);
      cmp = rem_hi > hh ? 1 : (rem_hi < hh ? -1 : (rem_lo > 0 ? 1 : 0));
    } else {
      const unsigned long long hl = 1ULL << (sh - 1);
      cmp = rem_hi > 0 ? 1 : (rem_lo > hl ? 1 : (rem_lo < hl ? -1 : 0));
    }
    if (cmp > 0 || (cmp == 0 && (mant & 1ULL))) {
      mant += 1;
      if (mant == (1ULL << 53)) { mant >>= 1; sh += 1; }
    }
  }
  // value = mant * 2^(sh + scale), mant < 2^53
  const int mb = 64 - __clzll((long long)mant);     // bits of mant
  const int E = (mb - 1) + sh + scale + 1023;       // biased exponent of the result
  if (E >= 1 && E <= 2046) {
    const unsigned long long frac = (mant << (53 - mb)) & ((1ULL << 52) - 1);
    return __longlong_as_double((long long)(((unsigned long long)neg << 63) | ((unsigned long long)E << 52) | frac));
  }
  const double v = scalbn((double)mant, sh + scale);  // outside the normal range
  return neg ? -v : v;
}

// T = sum_w G_w 2^(b (S + 1 - w)) of product r at (i, j), summed over the k segments,
// as a 128-bit two's complement integer (th, tl).
__device__ __forceinline__ void group_total(const RecombineArgs& a, int r, int64_t i, int64_t j, long long* th_out,
                                            unsigned long long* tl_out) {
  const int64_t plane = a.h_mp * a.h_np;
  const int* g = a.G + (int64_t)r * kGroups * plane + i * a.h_np + j;
  const int64_t seg_stride = (int64_t)a.P * kGroups * plane;
  long long gw[kGroups];
#pragma unroll
  for (int w = 0; w < kGroups; ++w) {
    long long v = g[(int64_t)w * plane];
    for (int sg = 1; sg < a.nseg; ++sg) v += g[sg * seg_stride + (int64_t)w * plane];
    gw[w] = v;
  }
  if (a.nseg <= 128) {
    // |G_w| < 128 * 2^31: T_hi = G_2 2^16 + G_3 2^8 + G_4 and
    // T_lo = G_5 2^24 + G_6 2^16 + G_7 2^8 + G_8 fit in int64; T = T_hi 2^32 + T_lo.
    const long long t_hi = gw[0] * (1LL << 16) + gw[1] * (1LL << 8) + gw[2];
    const long long t_lo = gw[3] * (1LL << 24) + gw[4] * (1LL << 16) + gw[5] * (1LL << 8) + gw[6];
    long long th = t_hi >> 32;
    unsigned long long tl = (unsigned long long)t_hi << 32;
    const unsigned long long nl = tl + (unsigned long long)t_lo;
    th += (t_lo >> 63) + (nl < tl ? 1 : 0);
    *th_out = th;
    *tl_out = nl;
    return;
  }
  long long th = 0;  // Horner over w in 128-bit integers
  unsigned long long tl = 0;
#pragma unroll
  for (int w = 0; w < kGroups; ++w) {
    th = (long long)(((unsigned long long)th << kB) | (tl >> (64 - kB)));
    tl <<= kB;
    const unsigned long long nl = tl + (unsigned long long)gw[w];
    th += (gw[w] >> 63) + (nl < tl ? 1 : 0);
    tl = nl;
  }
  *th_out = th;
  *tl_out = tl;
}

// One block per C row (grid-stride): for every block column qj the products that
// update C block (qi, qj) are added in table order, gamma alpha RN(T) 2^(e_i + f_j - 64)
// each; the threads of the block take consecutive columns.
__global__ void __launch_bounds__(256) oz_recombine_scatter(const __grid_constant__ RecombineArgs a) {
  static_assert(kGroups == 7 && kB == 8, "the two-word split of T assumes seven 8-bit groups");
  const int Pn = 1 << a.levels;
  for (int64_t gr = blockIdx.x; gr < a.m; gr += gridDim.x) {
    const int qi = (int)(gr / a.hm);
    const int64_t i = gr - (int64_t)qi * a.hm;
    for (int qj = 0; qj < Pn; ++qj) {
      const int q = qi * Pn + qj;
      const int u0 = a.first[q], u1 = a.first[q + 1];
      const int64_t c0 = (int64_t)qj * a.hn;
      const int64_t cols = (c0 + a.hn < a.n ? c0 + a.hn : a.n) - c0;
      for (int64_t j = threadIdx.x; j < cols; j += blockDim.x) {
        double* cp = a.C + gr * a.ldc + c0 + j;
        double c = *cp;
        for (int u = u0; u < u1; ++u) {
          const int r = a.upd[u] >> 1;
          long long th;
          unsigned long long tl;
          group_total(a, r, i, j, &th, &tl);
          const double M = round_i128(th, tl,
                                      a.e[(int64_t)r * a.h_mp + i] + a.f[(int64_t)r * a.h_np + j] - kB * (kS + 1));
          const double aM = a.alpha == 1.0 ? M : a.alpha * M;  // no FP64 multiply for alpha = 1
          c = (a.upd[u] & 1) ? c - aM : c + aM;
        }
        *cp = c;
      }
    }
  }
}

// Up to two levels (at most 16 C blocks): one thread per local position (i, j) of the
// blocks, holding that position of every C block in registers.  Each product's M_r is
// recombined once (its seven group sums read once) and added into each of its target
// blocks; the products run in table order, so every C element receives its additions
// in exactly the order of oz_recombine_scatter, which reads each product's group sums
// once per target instead.
template <int NBLK>
__global__ void __launch_bounds__(256, 3) oz_recombine_local(const __grid_constant__ RecombineArgs a) {
  const int Pn = 1 << a.levels;
  const int64_t positions = a.hm * a.hn;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < positions;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / a.hn, j = e - (e / a.hn) * a.hn;
    double c[NBLK];
    unsigned valid = 0;
#pragma unroll
    for (int q = 0; q < NBLK; ++q) {
      c[q] = 0.0;
      if (q < Pn * Pn) {
        const int64_t gr = (int64_t)(q / Pn) * a.hm + i, gc = (int64_t)(q % Pn) * a.hn + j;
        if (gr < a.m && gc < a.n) {
          valid |= 1u << q;
          c[q] = a.C[gr * a.ldc + gc];
        }
      }
    }
    if (valid) {
      for (int r = 0; r < a.P; ++r) {
        const int row = a.plan_off + r;
        const int nc = c_oz_plans.nc[row];
        unsigned hit = 0;
        for (int t = 0; t < nc; ++t) {
          const uint8_t code = c_oz_plans.tc[row][t];
          hit |= 1u << (term_bi(code) * Pn + term_bj(code));
        }
        if (!(hit & valid)) continue;
        long long th;
        unsigned long long tl;
        group_total(a, r, i, j, &th, &tl);
        const double M = round_i128(th, tl, a.e[(int64_t)r * a.h_mp + i] + a.f[(int64_t)r * a.h_np + j] - kB * (kS + 1));
        const double aM = a.alpha == 1.0 ? M : a.alpha * M;  // no FP64 multiply for alpha = 1
        for (int t = 0; t < nc; ++t) {
          const uint8_t code = c_oz_plans.tc[row][t];
          const int qq = term_bi(code) * Pn + term_bj(code);
#pragma unroll
          for (int q = 0; q < NBLK; ++q)
            if (q == qq) c[q] = term_neg(code) ? c[q] - aM : c[q] + aM;
        }
      }
#pragma unroll
      for (int q = 0; q < NBLK; ++q) {
        if ((valid >> q) & 1u) {
          const int64_t gr = (int64_t)(q / Pn) * a.hm + i, gc = (int64_t)(q % Pn) * a.hn + j;
          a.C[gr * a.ldc + gc] = c[q];
        }
      }
    }
  }
}

// ---------------------------------------------------------------- host side

PFN_cuTensorMapEncodeTiled_v12000 g_oz_encode = nullptr;
std::once_flag g_oz_once;
cudaError_t g_oz_init = cudaSuccess;
size_t oz_gemm_smem() { return (size_t)kStages * kStageBytes + 1024 + 256; }

// CTA pairs the slice-product grid plans its waves for (two SMs each).
int pair_slots(int sms) { return std::max(sms / 2, 1); }

// CTA pairs of oz_gemm that can be resident at once on the current device (at most one
// pair per two SMs; fewer where the SMs of a GPU cluster do not pair up).
int resident_pairs(int sms) {
  static std::mutex mu;
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); dev = 0; }
  std::lock_guard<std::mutex> lock(mu);
  if (dev >= 0 && dev < 64 && cached[dev] > 0) return cached[dev];
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3(2 * pair_slots(sms));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = oz_gemm_smem();
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, (const void*)oz_gemm, &cfg) != cudaSuccess || n <= 0) {
    cudaGetLastError();
    n = pair_slots(sms);
  }
  n = std::min(n, pair_slots(sms));
  if (dev >= 0 && dev < 64) cached[dev] = n;
  return n;
}

void oz_init() {
  cudaDriverEntryPointQueryResult q;
  void* fn = nullptr;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess) {
    cudaGetLastError();
    g_oz_init = cudaErrorNotSupported;
    return;
  }
  g_oz_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  g_oz_init = cudaFuncSetAttribute((const void*)oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)oz_gemm_smem());
  if (g_oz_init == cudaSuccess)
    g_oz_init = cudaFuncSetAttribute((const void*)oz_split_cols, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kSplitColsSmem);
}

bool encode_bf16(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int box_rows) {
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(cols * 2)};
  cuuint32_t box[2] = {(cuuint32_t)kTK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return g_oz_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int64_t round_up(int64_t x, int64_t q) { return (x + q - 1) / q * q; }

// Number of k segments: enough that every segment's int32 group sums stay below 2^31
// (at most kSegKB k-blocks), and more while the units would make fewer than six waves
// on the GPU and each segment keeps at least 16 k-blocks (the segments are separate
// units and balance the waves; the recombination adds them).
int plan_segments(int64_t units_per_seg, int64_t nkb, int sms) {
  int64_t nseg = (nkb + kSegKB - 1) / kSegKB;
  while (units_per_seg * nseg < 6LL * sms && nkb / (nseg + 1) >= 16) ++nseg;
  return (int)nseg;
}

}  // namespace

int64_t ozaki_workspace_bytes(int64_t m, int64_t n, int64_t k, int levels) {
  const int64_t P = kPlanCount[levels];
  const int64_t hmp = round_up(block_edge(m, levels), kPairM), hnp = round_up(block_edge(n, levels), kTN),
                hkp = round_up(block_edge(k, levels), kTK);
  const int64_t nseg =
      plan_segments(P * (hmp / kPairM) * (hnp / kTN), hkp / kTK, pair_slots(std::max(device_sm_count(), 1)));
  const int64_t hk = block_edge(k, levels), hn = block_edge(n, levels);
  const int64_t vsum = levels > 0 ? P * hk * hn * 8 + 256 : 0;  // B operand sums kept between the two B passes
  return P * kS * (hmp + hnp) * hkp * 2 + P * (hmp + hnp) * 4 + nseg * kGroups * P * hmp * hnp * 4 + P * hnp * 8 +
         256 + vsum + 4096;
}

double ozaki_model_seconds(int64_t m, int64_t n, int64_t k, int levels) {
  if (m <= 0 || n <= 0 || k <= 0 || levels < 0 || levels > kMaxLevels) return 1e30;
  const int sms = std::max(device_sm_count(), 1);
  const int64_t P = kPlanCount[levels];
  const int64_t hm = block_edge(m, levels), hn = block_edge(n, levels), hk = block_edge(k, levels);
  const int64_t hmp = round_up(hm, kPairM), hnp = round_up(hn, kTN), hkp = round_up(hk, kTK);
  const int slots = pair_slots(sms);
  const int64_t nseg = plan_segments(P * (hmp / kPairM) * (hnp / kTN), hkp / kTK, slots);
  int64_t ta = 0, tb = 0, tc = 0;
  for (int r = 0; r < P; ++r) {
    const int row = kPlanOffset[levels] + r;
    ta += kPlanTables.na[row];
    tb += kPlanTables.nb[row];
    tc += kPlanTables.nc[row];
  }
  int pairs = 0;
  for (int w = 2; w <= kS + 1; ++w) pairs += pairs_of(w);
  // Slice products at the tensor rate the kernel reaches on large shapes (0.8 of the
  // BF16 dense peak of about 12.7K flops per clock per SM at 2 GHz, two SMs per unit),
  // in whole waves of CTA pairs.
  const double units = (double)P * (hmp / kPairM) * (hnp / kTN) * nseg;
  const double waves = std::ceil(units / slots);
  const double unit_flops = (double)pairs * 2.0 * kPairM * kTN * ((double)hkp / nseg);
  const double t_mma = waves * unit_flops / (2.0 * 0.8 * 12700.0 * 2.0e9);
  // HBM passes: operand reads per term (B twice: column maxima, then digits), digit
  // writes and reads, group-sum writes and reads, C read and write.
  const double bytes = 8.0 * (ta * hm * hk + 2.0 * tb * hk * hn) + 2.0 * 2.0 * kS * P * (hmp + hnp) * hkp +
                       2.0 * 4.0 * nseg * kGroups * P * hmp * hnp + 4.0 * kGroups * nseg * (double)tc * hm * hn +
                       16.0 * m * n;
  return t_mma + bytes / 6.8e12 + 5 * 4e-6;
}

int ozaki_device_status() {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_oz_status, sizeof(int)) != cudaSuccess) return STRASSEN_ERR_CUDA;
  if (v != 0) {
    const int zero = 0;
    if (cudaMemcpyToSymbol(g_oz_status, &zero, sizeof(int)) != cudaSuccess) return STRASSEN_ERR_CUDA;
  }
  return v;
}

cudaError_t run_ozaki(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B, int64_t ldb,
                      double* C, int64_t ldc, int levels, void* ws, cudaStream_t stream, int trans_a, int trans_b,
                      double alpha, cudaEvent_t* stage_events) {
  std::call_once(g_oz_once, oz_init);
  if (g_oz_init != cudaSuccess) return g_oz_init;
  int sms = device_sm_count();
  if (sms <= 0) sms = 1;
  const int P = kPlanCount[levels];
  const int64_t hm = block_edge(m, levels), hn = block_edge(n, levels), hk = block_edge(k, levels);
  const int64_t hmp = round_up(hm, kPairM), hnp = round_up(hn, kTN), hkp = round_up(hk, kTK);
  uint8_t* w = (uint8_t*)ws;
  __nv_bfloat16* DX = (__nv_bfloat16*)w;                       w += (size_t)P * kS * hmp * hkp * 2;
  __nv_bfloat16* DV = (__nv_bfloat16*)w;                       w += (size_t)P * kS * hnp * hkp * 2;
  int* ex = (int*)w;                                           w += (size_t)P * hmp * 4;
  int* fx = (int*)w;                                           w += (size_t)P * hnp * 4;
  w = (uint8_t*)(((uintptr_t)w + 255) & ~(uintptr_t)255);
  const int nseg = plan_segments((int64_t)P * (hmp / kPairM) * (hnp / kTN), hkp / kTK, pair_slots(sms));
  int* G = (int*)w;                                            w += (size_t)nseg * kGroups * P * hmp * hnp * 4;
  unsigned long long* colmax = (unsigned long long*)w;  // [P][h_np] magnitude bits
  w += (size_t)P * hnp * 8;
  w = (uint8_t*)(((uintptr_t)w + 255) & ~(uintptr_t)255);
  unsigned* pace = (unsigned*)w;  // the slice-product kernel's pacing counter
  w += 256;
  unsigned long long* vsum = levels > 0 ? (unsigned long long*)w : nullptr;  // [P][h_k][h_n]

  SplitArgs sa;
  sa.src = A; sa.ld = lda; sa.rows = m; sa.cols = k; sa.h_r = hm; sa.h_c = hk;
  sa.h_out = hm; sa.h_outp = hmp; sa.h_k = hk; sa.h_kp = hkp;
  sa.plan_off = kPlanOffset[levels]; sa.slices = DX; sa.exps = ex; sa.trans = trans_a;
  sa.vsum = nullptr;
  const size_t row_smem = (size_t)hk * sizeof(double);
  if (row_smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute((const void*)oz_split_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)row_smem);
    if (e != cudaSuccess) return e;
  }
  if (stage_events && cudaEventRecord(stage_events[0], stream) != cudaSuccess) return cudaGetLastError();
  oz_split_rows<<<(unsigned)(hmp * P), 256, row_smem, stream>>>(sa, P);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;

  SplitArgs sb;
  sb.src = B; sb.ld = ldb; sb.rows = k; sb.cols = n; sb.h_r = hk; sb.h_c = hn;
  sb.h_out = hn; sb.h_outp = hnp; sb.h_k = hk; sb.h_kp = hkp;
  sb.plan_off = kPlanOffset[levels]; sb.slices = DV; sb.exps = fx; sb.trans = trans_b;
  sb.vsum = vsum;
  e = cudaMemsetAsync(colmax, 0, sizeof(unsigned long long) * (size_t)P * hnp, stream);
  if (e != cudaSuccess) return e;
  oz_colmax<<<(unsigned)((hnp / 64) * ((hk + kColMaxRows - 1) / kColMaxRows) * P), 256, 0, stream>>>(
      sb, colmax, P, (int)(hnp / 64));
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  oz_split_cols<<<(unsigned)((hnp / 64) * (hkp / 64) * P), 256, kSplitColsSmem, stream>>>(sb, colmax, P,
                                                                                           (int)(hnp / 64));
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;

  GemmArgs ga;
  std::memset(&ga, 0, sizeof(ga));
  if (!encode_bf16(&ga.tmA, DX, (int64_t)P * kS * hmp, hkp, kTM) ||
      !encode_bf16(&ga.tmB, DV, (int64_t)P * kS * hnp, hkp, kHalfN))
    return cudaErrorInvalidValue;
  ga.G = G;
  ga.P = P;
  ga.tiles_m = (int)(hmp / kPairM); ga.tiles_n = (int)(hnp / kTN);
  ga.nkb = (int)(hkp / kTK);
  ga.nseg = nseg;
  ga.seg_kb = (int)((ga.nkb + nseg - 1) / nseg);
  ga.h_mp = hmp; ga.h_np = hnp;
  ga.pace = pace;
  const int64_t units = (int64_t)P * ga.tiles_m * ga.tiles_n * ga.nseg;
  const int grid = 2 * (int)std::min<int64_t>(resident_pairs(sms), units);  // whole CTA pairs
  if ((e = cudaMemsetAsync(pace, 0, 2 * sizeof(unsigned), stream)) != cudaSuccess) return e;
  void* gargs[] = {&ga};
  if (stage_events && (e = cudaEventRecord(stage_events[1], stream)) != cudaSuccess) return e;
  e = cudaLaunchKernel((const void*)oz_gemm, dim3(grid), dim3(kThreads), gargs, oz_gemm_smem(), stream);
  if (e != cudaSuccess) return e;
  if (stage_events && (e = cudaEventRecord(stage_events[2], stream)) != cudaSuccess) return e;

  RecombineArgs ra;
  ra.C = C; ra.ldc = ldc; ra.m = m; ra.n = n;
  ra.hm = hm; ra.hn = hn; ra.h_mp = hmp; ra.h_np = hnp;
  ra.levels = levels; ra.P = P; ra.plan_off = kPlanOffset[levels];
  ra.G = G; ra.nseg = nseg; ra.e = ex; ra.f = fx; ra.alpha = alpha;
  // C-update lists per C block, products in table order.
  {
    const int Pn = 1 << levels;
    int n_upd = 0;
    for (int q = 0; q < Pn * Pn; ++q) {
      ra.first[q] = n_upd;
      for (int r = 0; r < P; ++r) {
        const int row = kPlanOffset[levels] + r;
        for (int t = 0; t < kPlanTables.nc[row]; ++t) {
          const uint8_t code = kPlanTables.tc[row][t];
          if (term_bi(code) * Pn + term_bj(code) == q) ra.upd[n_upd++] = (uint16_t)(2 * r + term_neg(code));
        }
      }
    }
    ra.first[Pn * Pn] = n_upd;
  }
  const int threads = 256;
  if (levels <= 2) {
    const int64_t positions = hm * hn;
    const int64_t blocks = std::min<int64_t>((positions + threads - 1) / threads, (int64_t)sms * 32);
    const unsigned grid = (unsigned)std::max<int64_t>(blocks, 1);
    if (levels == 0) oz_recombine_local<1><<<grid, threads, 0, stream>>>(ra);
    else if (levels == 1) oz_recombine_local<4><<<grid, threads, 0, stream>>>(ra);
    else oz_recombine_local<16><<<grid, threads, 0, stream>>>(ra);
  } else {
    const int64_t blocks = std::min<int64_t>(m, (int64_t)sms * 8);
    oz_recombine_scatter<<<(unsigned)std::max<int64_t>(blocks, 1), threads, 0, stream>>>(ra);
  }
  e = cudaGetLastError();
  if (e == cudaSuccess && stage_events) e = cudaEventRecord(stage_events[3], stream);
  return e;
}

}  // namespace sgb
