// FP64-level products on the FP16 tensor cores (tcgen05), exact in integer digit planes.
//
// Used for the batched online phase and its offline preparation: the explicit-inverse
// product x = K^{-1} d (Eq. (4.13) with the solves moved offline), K^{-1} = W^T W itself, the
// d2q product q = Q d (Eq. (4.14)), and the double-FP32 tier's per-frequency products
// d-hat_w = F-hat_w m-hat_w and m-hat_w = F-hat_w^H d-hat_w for batches (Sec. 4).
//
// Take the real product X[b][i] = sum_j A[i][j] D[b][j] (A = K^{-1}, say).  It needs about 48
// significant bits, which no tensor-core input type holds.  Both operands are therefore cut
// into S = 6 planes of balanced base-256 digits, each an integer in [-128, 128] and so exact
// in FP16:
//   A[i][j] = 2^(ea_i - 7) sum_s P_s[i][j] 2^(-8 s),   D[b][j] = 2^(eb_b - 7) sum_t Q_t[b][j] 2^(-8 t)
// with ea_i, eb_b the binary exponents of the row maxima (so the planes hold a 47-bit
// fixed-point image of each row, the rest rounded away).  Then
//   X[b][i] = 2^(ea_i + eb_b - 14) sum_g 2^(-8 g) G_g[i][b],  G_g = sum_{s + t = g} P_s Q_t^T,
// keeping the 21 plane pairs with s + t <= 5 (the dropped ones lie below 2^-48 of the row
// scale).  Every product of two digits is at most 2^14 and group g sums g + 1 plane pairs, so
// over an accumulation period of 192 columns j group g's sum stays below (g + 1) 192 2^14: up
// to group 4 that is below 2^24, and the FP32 accumulators in tensor memory hold it exactly;
// group 5 (6 pairs, 2^-40 of group 0's weight) may exceed 2^24 by a fraction, and its rounding
// stays below 2^-54 of the period's scale.  After each period the epilogue warps read the six
// groups, scale them by 2^(-8 g) (exact) and add them into float-pair accumulators with a
// two-sum, as the double-FP32 kernels do, and convert the result to FP64 with integer
// operations.  The complex spectral products are real GEMMs over
// an interleaved (re, im) K axis, the vectors' rows carrying the complex product's signs.
//
// Layout: a matrix's planes [S][ldk / 64][rows_pad][64] FP16 (rows_pad and ldk multiples of
// 128, zero padding; tiled so each TMA box is contiguous) are formed once; the right-hand-
// side planes [S][ldk / 64][64][64] per call.  In the stream-K kernel a CTA (one per SM)
// walks a contiguous run of (tile, chunk) units, so every SM gets the same number of chunks;
// partial tiles go to an FP64 buffer that a second kernel sums in CTA order.  Warp 0 issues
// the TMA loads (the matrix's planes 128 rows x 64 columns per stage, the six right-hand-side
// planes per 64 columns), warp 1 runs the MMA loop with one elected lane issuing tcgen05.mma
// (M = 128, N = 64 or 32, K = 16) into six TMEM groups, A reused from the tensor core's
// collector across the MMAs of each A plane, and warps 2-9 drain the groups per period (and at
// the end of each tile in the CTA's share).
// Every wait is bounded; on a timeout the kernel sets the error word, stops issuing, lets what
// it issued land and frees its tensor memory.
#include "bti_internal.cuh"

#include <algorithm>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

namespace bti {

namespace {

constexpr int kSl = 6;                 // digit planes per operand
constexpr int kKiRows = 128;           // MMA M: rows of the matrix per tile
constexpr int kKiN = 64;               // MMA N: right-hand-side columns per launch chunk
constexpr int kKiBox = 64;             // FP16 columns per tile of the planes in memory (128 bytes)
constexpr int kKiChunk = 128;          // columns per work chunk (the unit of stream-K and of tile skipping)
constexpr int kDrainK = 12;            // K-steps (16 columns each) per accumulation period: 192 columns
constexpr int kPeriodCols = 204;       // most data columns a period may hold (5 204 2^14 < 2^24)
// FP16 columns per TMA box in the pipeline: two 16-column K-steps (64-byte rows, the 64-byte
// swizzle) in three stages.  One K-step per box (32-byte rows and swizzle, six stages in the same
// shared memory) was measured slower: the adjoint of 64 vectors 0.75 -> 0.94 ms, twice the barrier
// waits, commits and loads per K-step outweighing the finer release of stages.
constexpr int kBx = 32;
constexpr int kKPB = kBx / 16;         // K-steps per box
constexpr int kBoxesPerChunk = kKiChunk / kBx;
constexpr int kBoxesPerTile = kKiBox / kBx;  // boxes per 64-column memory tile
constexpr int kStages = kBx == 32 ? 3 : 6;   // pipeline stages: one box of all six planes of both operands
constexpr int kKiThreads = 320;        // warp 0 TMA, warp 1 MMA, warps 2-9 epilogue
constexpr uint32_t kAPlane = kKiRows * kBx * 2;  // bytes of one A plane in a stage (128 rows x 2 kBx B)
constexpr uint32_t kAStage = kSl * kAPlane;       // 48 KB
constexpr uint32_t kTmemCols = 512;    // six accumulator groups (6 N columns, N <= 64)
constexpr long long kKiSpin = 1ll << 24;              // poll backstop of every wait
constexpr uint64_t kKiWaitNs = 1000000000ull;          // wall-time limit of every wait: 1 s
// shared memory of a kernel whose B operand has NC rows: 1 KB alignment slack and kStages stages
constexpr size_t dig_smem(int NC) { return 1024 + kStages * ((size_t)kAStage + (size_t)kSl * NC * kBx * 2); }

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// K-major operand with rows of 2 kBx bytes swizzled at that width (the layout TMA writes with
// CU_TENSOR_MAP_SWIZZLE_32B or _64B), 8-row groups 16 kBx bytes apart; a K-step of 16 halves
// advances the start by 32 B (descriptor swizzle modes: 6 = 32-byte, 4 = 64-byte)
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)((16 * kBx) >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)(kBx == 32 ? 4 : 6) << 61);
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
               : "=r"(done) : "r"(bar), "r"(parity) : "memory");
  return done != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait: gives up after kKiWaitNs of wall time (checked every 256 polls; a poll of
// try_wait may suspend the thread for microseconds) or kKiSpin polls, whichever comes first,
// or as soon as another thread has flagged an abort.  On giving up it flags the abort.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (long long it = 1; it < kKiSpin; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 255) == 0) {
      if (*abort_flag) return false;
      if (global_ns() - t0 > kKiWaitNs) break;
    }
  }
  *abort_flag = 1;
  return false;
}

__device__ __forceinline__ void two_sum_acc(float& Sh, float& Sl, float p) {
  const float s = Sh + p;
  const float bb = s - Sh;
  Sl += (Sh - (s - bb)) + (p - bb);
  Sh = s;
}

__device__ __forceinline__ void tmem_ld(uint32_t addr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_ld(uint32_t addr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Add one accumulation period's S group sums G_g (TMEM columns NC g + the W columns at taddr,
// this warp's lanes) into the float-pair accumulators: sum_g 2^(-8 g) G_g.  Groups S - 1 .. 3 are
// summed in plain FP32 first: in group 0's units that partial sum is below 0.76 (|G_3| <
// 4 192 2^14), so its rounding, at most 2^-25, stays under 2^-46 of the period's bound
// 192 2^14 on |G_0|; groups 2, 1, 0 and that sum enter by two-sum.
template <int NC, int W, int S>
__device__ __forceinline__ void add_groups(uint32_t taddr, float (&Sh)[W], float (&Sl)[W]) {
  static_assert(S >= 4 && S <= 6, "four to six digit planes");
  uint32_t v[W];
  float low[W];
  tmem_ld(taddr + (S - 1) * NC, v);
  {
    const float sc = __int_as_float((127 - 8 * (S - 1)) << 23);  // 2^(-8 (S - 1)), exact
#pragma unroll
    for (int c = 0; c < W; ++c) low[c] = __uint_as_float(v[c]) * sc;
  }
#pragma unroll
  for (int g = S - 2; g >= 3; --g) {
    tmem_ld(taddr + g * NC, v);
    const float sc = __int_as_float((127 - 8 * g) << 23);
#pragma unroll
    for (int c = 0; c < W; ++c) low[c] = fmaf(__uint_as_float(v[c]), sc, low[c]);
  }
#pragma unroll
  for (int c = 0; c < W; ++c) two_sum_acc(Sh[c], Sl[c], low[c]);
#pragma unroll
  for (int g = 2; g >= 0; --g) {
    tmem_ld(taddr + g * NC, v);
    const float sc = __int_as_float((127 - 8 * g) << 23);  // 2^(-8 g), exact
#pragma unroll
    for (int c = 0; c < W; ++c) two_sum_acc(Sh[c], Sl[c], __uint_as_float(v[c]) * sc);
  }
}

// Integer-only helpers of the slicing kernels (GB300 runs FP64 instructions, conversions and
// scaling included, at a small fraction of its integer rate).  abs_bits: |x| as bits, which order
// like the values for |x| >= 0.  exp_of_bits: the frexp exponent of |x| from those bits (|x| =
// f 2^e, f in [0.5, 1); 0 for zero).  round_scaled: x 2^k rounded to the nearest integer, ties to
// even (as llrint), for |x 2^k| < 2^62: x = m 2^(max(E, 1) - 1075) from its biased exponent E and
// significand m, so x 2^k = m 2^s is a shift of m with the bits shifted out deciding the rounding.
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}
__device__ __forceinline__ int exp_of_bits(unsigned long long mb) {
  if (mb == 0) return 0;
  const int E = (int)(mb >> 52);
  if (E != 0) return E - 1022;
  return 64 - __clzll((long long)mb) - 1074;  // subnormal: m 2^-1074 with its top bit at 63 - clz
}
__device__ __forceinline__ long long round_scaled(double x, int k) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF);
  unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  if (E != 0) m |= 1ull << 52;
  const int sft = (E != 0 ? E : 1) - 1075 + k;
  long long v;
  if (sft >= 0) {
    v = sft < 63 ? (long long)(m << sft) : 0;  // a subnormal x with a large k (m 2^sft < 2^62)
  } else {
    const int r = -sft;
    if (r > 63) {
      v = 0;
    } else {
      const unsigned long long q = m >> r, rem = m & ((1ull << r) - 1), half = 1ull << (r - 1);
      v = (long long)(q + ((rem > half || (rem == half && (q & 1))) ? 1ull : 0ull));
    }
  }
  return (b >> 63) ? -v : v;
}

// Balanced base-256 digits of v (|v| <= 2^47), most significant first: v = sum_s d[s] 256^(5 - s),
// d[s] in [-128, 128] (the lower five in [-128, 127]).
__device__ __forceinline__ void digits6(long long v, int (&d)[kSl]) {
#pragma unroll
  for (int k = 0; k < kSl - 1; ++k) {
    const int dk = (int)(((v & 255) ^ 128) - 128);
    d[kSl - 1 - k] = dk;
    v = (v - dk) >> 8;
  }
  d[0] = (int)v;  // |v| <= 128 here
}

// tcgen05.commit issued by one elected lane of a warp that runs the issuing loop in step.
__device__ __forceinline__ void commit_elect(uint32_t bar) {
  asm volatile(
      "{\n.reg .pred e;\nelect.sync _|e, 0xffffffff;\n"
      "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}\n"
      ::"r"(bar) : "memory");
}
// Whether the accumulation period closes after K-step k (0-based along a K axis of ksteps
// K-steps): at the end of the CTA's share of a tile, and after every kDrainK K-steps, except
// that the axis's last K-step joins the period before it when that period then holds at most
// kPeriodCols data columns (tail_cols: the data columns of the last K-step).
__device__ __forceinline__ bool period_closes(int64_t k, int64_t ksteps, int tail_cols, bool share_last) {
  if (share_last) return true;
  if ((k + 1) % kDrainK != 0) return false;
  return !(k + 2 == ksteps && kDrainK * 16 + tail_cols <= kPeriodCols);
}

// bounded wait taken by a whole warp: true only if every lane saw the phase complete
__device__ __forceinline__ bool mbar_wait_warp(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
  return __all_sync(0xffffffffu, mbar_wait(bar, parity, abort_flag));
}

// One K-step (16 columns) of a stage, as one instruction block under a single elect.sync: the
// S (S + 1) / 2 plane pairs s + t <= S - 1 of the first S planes of each operand (S = 6: all 21),
// group s + t accumulating at TMEM columns NC (s + t), both operands read from shared memory.
// The pairs are issued plane by plane of A, and each A plane slice is read once: the first MMA
// of plane s fills the tensor core's A collector, the next ones reuse it and the last releases
// it (plane S - 1 has one MMA, which reads A directly).  ad, bd: the descriptors of the stage's
// plane 0 of A and of B at this K-step.  first: the K-step opens an accumulation period, so the
// pairs (0, t), issued first, overwrite the groups.  Consecutive planes of a stage are kAPlane
// bytes apart (kAPlane / 16 in the descriptor's 16-byte units) for A and NC kBx 2 bytes for B; the
// shared-memory addresses stay below 2^18, so the offsets add to the descriptors' address field
// without carrying out of it.  Called by a whole warp.
template <int S> struct KStep;
template <> struct KStep<4> {
  template <int NC>
  static __device__ __forceinline__ void issue(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, bool first) {
    constexpr uint64_t bs = (uint64_t)((NC * kBx * 2) >> 4), as = (uint64_t)(kAPlane >> 4);
    asm volatile(
        "{\n"
        ".reg .pred e, pa, pt;\n"
        ".reg .b64 a1, a2, a3, b1, b2, b3;\n"
        ".reg .b32 d1, d2, d3;\n"
        "elect.sync _|e, 0xffffffff;\n"
        "setp.eq.u32 pa, %4, 0;\n"
        "setp.eq.u32 pt, %4, %4;\n"
        "add.u64 a1, %1, %11;\n"
        "add.u64 b1, %2, %5;\n"
        "add.u32 d1, %0, %8;\n"
        "add.u64 a2, %1, %12;\n"
        "add.u64 b2, %2, %6;\n"
        "add.u32 d2, %0, %9;\n"
        "add.u64 a3, %1, %13;\n"
        "add.u64 b3, %2, %7;\n"
        "add.u32 d3, %0, %10;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [%0], %1, %2, %3, pa;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::use [d1], %1, b1, %3, pa;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::use [d2], %1, b2, %3, pa;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [d3], %1, b3, %3, pa;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [d1], a1, %2, %3, pt;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::use [d2], a1, b1, %3, pt;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [d3], a1, b2, %3, pt;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [d2], a2, %2, %3, pt;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [d3], a2, b1, %3, pt;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16 [d3], a3, %2, %3, pt;\n"
        "}\n"
        ::"r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(first ? 1u : 0u), "n"(1 * bs), "n"(2 * bs), "n"(3 * bs),
          "n"(1 * NC), "n"(2 * NC), "n"(3 * NC), "n"(1 * as), "n"(2 * as), "n"(3 * as)
        : "memory");
  }
};
template <> struct KStep<5> {
  template <int NC>
  static __device__ __forceinline__ void issue(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, bool first) {
    constexpr uint64_t bs = (uint64_t)((NC * kBx * 2) >> 4), as = (uint64_t)(kAPlane >> 4);
    asm volatile(
        "{\n"
        ".reg .pred e, pa, pt;\n"
        ".reg .b64 a1, a2, a3, a4, b1, b2, b3, b4;\n"
        ".reg .b32 d1, d2, d3, d4;\n"
        "elect.sync _|e, 0xffffffff;\n"
        "setp.eq.u32 pa, %4, 0;\n"
        "setp.eq.u32 pt, %4, %4;\n"
        "add.u64 a1, %1, %13;\n"
        "add.u64 b1, %2, %5;\n"
        "add.u32 d1, %0, %9;\n"
        "add.u64 a2, %1, %14;\n"
        "add.u64 b2, %2, %6;\n"
        "add.u32 d2, %0, %10;\n"
        "add.u64 a3, %1, %15;\n"
        "add.u64 b3, %2, %7;\n"
        "add.u32 d3, %0, %11;\n"
        "add.u64 a4, %1, %16;\n"
        "add.u64 b4, %2, %8;\n"
        "add.u32 d4, %0, %12;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [%0], %1, %2, %3, pa;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::use [d1], %1, b1, %3, pa;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::use [d2], %1, b2, %3, pa;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::use [d3], %1, b3, %3, pa;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [d4], %1, b4, %3, pa;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [d1], a1, %2, %3, pt;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::use [d2], a1, b1, %3, pt;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::use [d3], a1, b2, %3, pt;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [d4], a1, b3, %3, pt;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [d2], a2, %2, %3, pt;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::use [d3], a2, b1, %3, pt;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [d4], a2, b2, %3, pt;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [d3], a3, %2, %3, pt;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [d4], a3, b1, %3, pt;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16 [d4], a4, %2, %3, pt;\n"
        "}\n"
        ::"r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(first ? 1u : 0u), "n"(1 * bs), "n"(2 * bs), "n"(3 * bs),
          "n"(4 * bs), "n"(1 * NC), "n"(2 * NC), "n"(3 * NC), "n"(4 * NC), "n"(1 * as), "n"(2 * as), "n"(3 * as),
          "n"(4 * as)
        : "memory");
  }
};
template <> struct KStep<6> {
  template <int NC>
  static __device__ __forceinline__ void issue(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, bool first) {
    constexpr uint64_t bs = (uint64_t)((NC * kBx * 2) >> 4), as = (uint64_t)(kAPlane >> 4);
    asm volatile(
        "{\n"
        ".reg .pred e, pa, pt;\n"
        ".reg .b64 a1, a2, a3, a4, a5, b1, b2, b3, b4, b5;\n"
        ".reg .b32 d1, d2, d3, d4, d5;\n"
        "elect.sync _|e, 0xffffffff;\n"
        "setp.eq.u32 pa, %4, 0;\n"
        "setp.eq.u32 pt, %4, %4;\n"
        "add.u64 a1, %1, %15;\n"
        "add.u64 b1, %2, %5;\n"
        "add.u32 d1, %0, %10;\n"
        "add.u64 a2, %1, %16;\n"
        "add.u64 b2, %2, %6;\n"
        "add.u32 d2, %0, %11;\n"
        "add.u64 a3, %1, %17;\n"
        "add.u64 b3, %2, %7;\n"
        "add.u32 d3, %0, %12;\n"
        "add.u64 a4, %1, %18;\n"
        "add.u64 b4, %2, %8;\n"
        "add.u32 d4, %0, %13;\n"
        "add.u64 a5, %1, %19;\n"
        "add.u64 b5, %2, %9;\n"
        "add.u32 d5, %0, %14;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [%0], %1, %2, %3, pa;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::use [d1], %1, b1, %3, pa;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::use [d2], %1, b2, %3, pa;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::use [d3], %1, b3, %3, pa;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::use [d4], %1, b4, %3, pa;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [d5], %1, b5, %3, pa;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [d1], a1, %2, %3, pt;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::use [d2], a1, b1, %3, pt;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::use [d3], a1, b2, %3, pt;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::use [d4], a1, b3, %3, pt;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [d5], a1, b4, %3, pt;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [d2], a2, %2, %3, pt;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::use [d3], a2, b1, %3, pt;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::use [d4], a2, b2, %3, pt;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [d5], a2, b3, %3, pt;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [d3], a3, %2, %3, pt;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::use [d4], a3, b1, %3, pt;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [d5], a3, b2, %3, pt;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [d4], a4, %2, %3, pt;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [d5], a4, b1, %3, pt;\n"
        "@e tcgen05.mma.cta_group::1.kind::f16 [d5], a5, %2, %3, pt;\n"
        "}\n"
        ::"r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(first ? 1u : 0u), "n"(1 * bs), "n"(2 * bs), "n"(3 * bs),
          "n"(4 * bs), "n"(5 * bs), "n"(1 * NC), "n"(2 * NC), "n"(3 * NC), "n"(4 * NC), "n"(5 * NC), "n"(1 * as),
          "n"(2 * as), "n"(3 * as), "n"(4 * as), "n"(5 * as)
        : "memory");
  }
};

// The K-step kk (below kKPB) of a stage whose plane 0 of A and of B sit at a0 and b0.
template <int NC, int S>
__device__ __forceinline__ void issue_kstep(uint32_t tmem, uint32_t a0, uint32_t b0, int kk, uint32_t idesc,
                                            bool first) {
  KStep<S>::template issue<NC>(tmem, sdesc(a0) + 2 * kk, sdesc(b0) + 2 * kk, idesc, first);
}

// (hi + lo) 2^e as an FP64 value with integer operations only (GB300 issues FP64 at 1/64 of
// its FP32 rate, and the epilogue converts every output): the pair is renormalised by a
// two-sum, so |lo| <= ulp(hi) / 2; lo's significand is aligned to hi's in a 64-bit integer
// (together at most 53 bits, so exact up to lo's bits below 2^-29 ulp(hi)), the sum is
// renormalised by one bit if needed, and e is added to the exponent.  0 when hi is 0 or
// below FP32's normal range.
__device__ __forceinline__ double pair_to_double_scaled(float hi, float lo, int e) {
  const float sm = hi + lo;
  const float bb = sm - hi;
  lo = (hi - (sm - bb)) + (lo - bb);
  hi = sm;
  const uint32_t hb = __float_as_uint(hi);
  const int Eh = (int)((hb >> 23) & 255u);
  if (Eh == 0) return 0.0;
  long long X = (long long)((hb & 0x7FFFFFu) | 0x800000u) << 29;  // hi's significand at bit 52
  const uint32_t lb = __float_as_uint(lo);
  const int El = (int)((lb >> 23) & 255u);
  if (El != 0) {
    long long ml = (long long)((lb & 0x7FFFFFu) | 0x800000u);
    const int sh = El - Eh + 29;  // <= 5 since |lo| <= ulp(hi) / 2
    ml = sh >= 0 ? (ml << sh) : (sh > -40 ? (ml >> -sh) : 0);
    X = ((lb ^ hb) >> 31) ? X - ml : X + ml;
  }
  int E = Eh;
  if (X >= (1ll << 53)) {
    X >>= 1;
    ++E;
  } else if (X < (1ll << 52)) {
    X <<= 1;
    --E;
  }
  const long long bits = ((long long)(hb >> 31) << 63) | ((long long)(E - 127 + 1023 + e) << 52) |
                         (X & ((1ll << 52) - 1));
  return __longlong_as_double(bits);
}

// (hi + lo) 2^e as a normalised float pair, the double-FP32 tier's spectral format: a two-sum,
// then both floats times 2^e as two exact power-of-two products (exponents e1 + e2 = e of one
// sign, so no partial product leaves FP32's range unless the result does).  Below FP32's normal
// range the low float, then the high one, lose bits like any FP32 value.  e is clamped to
// [-252, 252], which changes no result that is neither zero nor infinite (|hi + lo| < 2^64).
__device__ __forceinline__ float4 pair_scaled2(float hr, float lr, float hi, float li, int e) {
  e = max(-252, min(252, e));
  const int e1 = e >> 1, e2 = e - e1;  // each in [-126, 126]
  const float p1 = __int_as_float((e1 + 127) << 23), p2 = __int_as_float((e2 + 127) << 23);
  float sr = __fadd_rn(hr, lr), br = __fsub_rn(sr, hr);
  float tr = __fadd_rn(__fsub_rn(hr, __fsub_rn(sr, br)), __fsub_rn(lr, br));
  float si = __fadd_rn(hi, li), bi = __fsub_rn(si, hi);
  float ti = __fadd_rn(__fsub_rn(hi, __fsub_rn(si, bi)), __fsub_rn(li, bi));
  return make_float4(__fmul_rn(__fmul_rn(sr, p1), p2), __fmul_rn(__fmul_rn(tr, p1), p2),
                     __fmul_rn(__fmul_rn(si, p1), p2), __fmul_rn(__fmul_rn(ti, p1), p2));
}

// Digit planes of rows 0 .. rows-1 (columns 0 .. n-1; columns n .. ldk-1 and rows rows ..
// rows_pad-1 are written as zeros), one warp per row: ex[r] = the binary exponent of
// max_j |X[r][j]| (frexp convention, max = f 2^e with f in [0.5, 1); 0 for a zero or padding
// row), then X[r][j] 2^(47 - e) rounded to an integer v (|v| <= 2^47) and split into balanced
// base-256 digits, most significant in plane 0.  Each plane is tiled by 64-column boxes,
// [ldk / 64][rows_pad][64], so that every 128-row TMA box is one contiguous 16 KB block.
__global__ void __launch_bounds__(256)
slice_rows_kernel(const double* __restrict__ X, int64_t ldx, int64_t rows, int64_t n, int* __restrict__ ex,
                  __half* __restrict__ planes, int64_t rows_pad, int64_t ldk) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t plane = rows_pad * ldk;
  for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < rows_pad; r += warps) {
    const double* x = X + r * ldx;
    unsigned long long mb = 0;
    if (r < rows)
      for (int64_t j = lane; j < n; j += 32) mb = max(mb, abs_bits(x[j]));
    for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
    const int e = exp_of_bits(mb);
    if (lane == 0) ex[r] = e;
    __half* out = planes + r * kKiBox;
    for (int64_t j = lane; j < ldk; j += 32) {
      long long v = 0;
      if (r < rows && j < n) v = round_scaled(x[j], 47 - e);
      int d[kSl];
      digits6(v, d);
      const int64_t o = (j / kKiBox) * rows_pad * kKiBox + (j % kKiBox);
#pragma unroll
      for (int sl = 0; sl < kSl; ++sl) out[sl * plane + o] = __int2half_rn(d[sl]);
    }
  }
}

// The same planes for few, long rows (the right-hand sides of a product): CTA (row r, column
// slice of cw), each CTA taking the whole row's maximum itself (the row is read from L2 again by
// the row's other slices) so that a handful of rows still spreads over every SM.
__global__ void __launch_bounds__(256)
slice_rows_wide_kernel(const double* __restrict__ X, int64_t ldx, int64_t rows, int64_t n, int* __restrict__ ex,
                       __half* __restrict__ planes, int64_t rows_pad, int64_t ldk, int64_t cw) {
  __shared__ unsigned long long red[8];
  const int64_t r = blockIdx.x;
  const double* x = X + r * ldx;
  unsigned long long mb = 0;
  if (r < rows)
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) mb = max(mb, abs_bits(x[j]));
  for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mb;
  __syncthreads();
  mb = red[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mb = max(mb, red[w]);
  const int e = exp_of_bits(mb);
  if (blockIdx.y == 0 && threadIdx.x == 0) ex[r] = e;
  const int64_t plane = rows_pad * ldk;
  __half* out = planes + r * kKiBox;
  const int64_t j1 = min(ldk, (int64_t)(blockIdx.y + 1) * cw);
  for (int64_t j = (int64_t)blockIdx.y * cw + threadIdx.x; j < j1; j += blockDim.x) {
    long long v = 0;
    if (r < rows && j < n) v = round_scaled(x[j], 47 - e);
    int d[kSl];
    digits6(v, d);
    const int64_t o = (j / kKiBox) * rows_pad * kKiBox + (j % kKiBox);
#pragma unroll
    for (int sl = 0; sl < kSl; ++sl) out[sl * plane + o] = __int2half_rn(d[sl]);
  }
}

// Column maxima of a rows x cols block of X (row stride ldx) as FP64 bit patterns (|x| >= 0 orders
// like its bits): CTA (column block of 64, row block of 256), four threads per column.
__global__ void __launch_bounds__(256)
col_max_kernel(const double* __restrict__ X, int64_t ldx, int64_t rows, int64_t cols,
               unsigned long long* __restrict__ colmax) {
  __shared__ unsigned long long red[4][64];
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
  const int64_t c = (int64_t)blockIdx.x * 64 + tx;
  const int64_t r0 = (int64_t)blockIdx.y * 256;
  unsigned long long mb = 0;
  if (c < cols)
    for (int64_t r = r0 + ty; r < rows && r < r0 + 256; r += 4) mb = max(mb, abs_bits(X[r * ldx + c]));
  red[ty][tx] = mb;
  __syncthreads();
  if (ty == 0 && c < cols) {
    mb = max(max(red[0][tx], red[1][tx]), max(red[2][tx], red[3][tx]));
    atomicMax(&colmax[c], mb);
  }
}

// Digit planes of the transpose of a rows x cols block of X: row c of X^T (column c of X) is
// planes row c with K index k = row of X, exponent from colmax[c]; the same layout and padding
// as slice_rows_kernel ([6][ldk / 64][rows_pad][64], rows_pad >= cols, ldk >= rows, zeros past
// them).  CTA = (64-value K tile, 64 output rows): the 64 x 64 block of X through shared memory,
// so both its reads (rows of X) and its writes (64 K values of an output row) are contiguous.
__global__ void __launch_bounds__(256)
slice_cols_kernel(const double* __restrict__ X, int64_t ldx, int64_t rows, int64_t cols,
                  const unsigned long long* __restrict__ colmax, int* __restrict__ ex, __half* __restrict__ planes,
                  int64_t rows_pad, int64_t ldk) {
  __shared__ double t[64][65];
  const int64_t k0 = (int64_t)blockIdx.x * 64, c0 = (int64_t)blockIdx.y * 64;
  for (int i = threadIdx.x; i < 64 * 64; i += 256) {
    const int kr = i >> 6, cc = i & 63;
    const int64_t k = k0 + kr, c = c0 + cc;
    t[kr][cc] = (k < rows && c < cols) ? X[k * ldx + c] : 0.0;
  }
  __syncthreads();
  const int cc = threadIdx.x >> 2, kq = (threadIdx.x & 3) * 16;
  const int64_t c = c0 + cc;
  const int e = c < cols ? exp_of_bits(colmax[c]) : 0;
  if (blockIdx.x == 0 && (threadIdx.x & 3) == 0 && c < rows_pad) ex[c] = e;
  const int64_t plane = rows_pad * ldk;
  __half* out = planes + (k0 / kKiBox) * rows_pad * kKiBox + c * kKiBox + kq;
#pragma unroll 4
  for (int j = 0; j < 16; ++j) {
    long long v = 0;
    if (c < cols) v = round_scaled(t[kq + j][cc], 47 - e);
    int d[kSl];
    digits6(v, d);
#pragma unroll
    for (int sl = 0; sl < kSl; ++sl) out[sl * plane + j] = __int2half_rn(d[sl]);
  }
}

// Tile T of the lower trapezoid of 128-row tiles I and 64-column tiles J < JW with J <= 2 I + 1
// (the column tiles that reach row tile I's diagonal): rows I < I0 = JW / 2 hold 2 I + 2 tiles
// (T = I (I + 1) + J), the rows after them JW tiles each.
__device__ __forceinline__ void trap_tile(int64_t T, int64_t JW, int64_t& I, int64_t& J) {
  const int64_t I0 = JW / 2, T0 = I0 * (I0 + 1);
  if (T >= T0) {
    I = I0 + (T - T0) / JW;
    J = (T - T0) % JW;
    return;
  }
  int64_t i = (int64_t)((sqrt(4.0 * (double)T + 1.0) - 1.0) * 0.5);
  while ((i + 1) * (i + 2) <= T) ++i;
  while (i > 0 && i * (i + 1) > T) --i;
  I = i;
  J = T - i * (i + 1);
}

// Which (tile, chunk) work items a CTA takes, in order, and where each tile's result goes.
// Stream-K (tiles == false): units [blockIdx per, + per) of the (tile, chunk) sequence, one FP64
// partial tile per tile touched.  Tile mode (tiles == true): tiles blockIdx, blockIdx + grid, ...
// of a rectangle (T = I JW + J) or of the lower trapezoid (trap_tile), each over its chunk range
// [c0, c1) whole, the result combined into C by op.  The chunk range skips chunks whose A rows
// (row tile I of a lower-triangular A: k < 128 (I + 1)) or B rows (column tile J of the transpose
// of a lower-triangular matrix, or of a triangular inverse: k >= NC J; K-major rows of an upper-
// triangular matrix: k >= 128 I) are known to be zero.
struct TileJob {
  double* C;
  int64_t ldc, mvalid, wvalid;  // C row stride; rows and columns of C written
  int64_t JW, tiles;            // column tiles; tiles in the enumeration
  int trap;                     // 1: lower trapezoid, 0: rectangle
  int lower;                    // 1: write only on and below the diagonal (j <= i)
  int op;                       // 0: C = v, 1: C -= v, 2: C = -v
  int kfirst;                   // first chunk: 0; 1: I; 2: floor(NC J / 128)
  int klast;                    // chunk range end: 0: kpt; 1: I + 1
  int skip_on_err;              // 1: return at once if *err is already set
};

template <bool TILES, int NC>
struct WorkIter {
  int64_t T, c, c1, I, J, u, u1, kpt, wt;
  int side, rg;  // stream-K: NRG CTAs side by side (side = NRG), this CTA's row group; else side = 0
  bool valid;
  __device__ __forceinline__ void tile_range(const TileJob& tj) {
    if (tj.trap) {
      trap_tile(T, tj.JW, I, J);
    } else {
      I = T / tj.JW;
      J = T - I * tj.JW;
    }
    c = tj.kfirst == 1 ? I : (tj.kfirst == 2 ? (J * NC) / kKiChunk : 0);
    c1 = tj.klast == 1 ? I + 1 : kpt;
    if (c1 > kpt) c1 = kpt;
  }
  __device__ __forceinline__ void seek(const TileJob& tj) {  // first nonempty tile from T on
    for (; T < tj.tiles; T += gridDim.x) {
      tile_range(tj);
      if (c < c1) return;
    }
    valid = false;
  }
  __device__ __forceinline__ void locate() {  // stream-K: tile and chunk of unit u
    wt = u / kpt;
    c = u - wt * kpt;
    T = side ? wt * side + rg : wt;
  }
  __device__ __forceinline__ void init(const TileJob& tj, int64_t per, int64_t total, int64_t kpt_, int side_ = 0) {
    kpt = kpt_;
    valid = true;
    if constexpr (TILES) {
      T = blockIdx.x;
      seek(tj);
    } else {
      side = side_;
      rg = side ? (int)(blockIdx.x % side) : 0;
      u = (int64_t)(side ? blockIdx.x / side : blockIdx.x) * per;
      u1 = min(total, u + per);
      valid = u < u1;
      locate();
    }
  }
  __device__ __forceinline__ bool last() const {
    if constexpr (TILES) return c + 1 == c1;
    return u + 1 == u1 || (u + 1) / kpt != wt;
  }
  __device__ __forceinline__ void next(const TileJob& tj) {
    if constexpr (TILES) {
      if (++c < c1) return;
      T += gridDim.x;
      seek(tj);
    } else {
      ++u;
      valid = u < u1;
      locate();
    }
  }
};

// Digit-plane GEMM: D[m][c] = sum_k A[m][k] B[c][k] for tiles of 128 rows m x NC columns c, the
// K axis in exact chunks of 128.  Stream-K form (TILES = false): tile T is (w, rg) = (T / NRG,
// T % NRG) (a problem and a group within it); the 64-column memory tile kbg of tile T sits at
// TMA row (w KB + kbg) a_blk + rg a_rg of the A planes and (w KB + kbg) b_blk + rg b_rg of the B
// planes (KB = 2 kpt); row m's exponent is ea[w ea_w + rg ea_rg + m], column c's
// eb[w eb_w + rg eb_rg + c] (padding rows and columns hold 0); a CTA covers units
// [blockIdx per, + per) and writes one FP64 partial tile [NC][128] per tile it touches.  With
// side = NRG the units are (w, chunk) instead, and CTA b takes row group b % side of units
// [(b / side) per, + per): the NRG CTAs of a group stream the same A planes side by side.  Tile
// form (TILES = true, the Cholesky's updates and the triangular products of the inverse): tile
// (I, J) of tj reads A rows 128 I and B rows NC J (a_blk, b_blk: the planes' padded row counts),
// exponents ea[128 I + m] and eb[NC J + c], and combines its result into tj.C.  Either way the
// pipeline loads each memory tile as two 32-column boxes, and only the first ksteps 16-column
// K-steps hold data (the rest of the last chunk is padding, neither loaded nor multiplied).
template <int NC, bool TILES = false, int S = kSl>
__global__ void __launch_bounds__(kKiThreads, 1)
sk_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
             const int* __restrict__ ea, const int* __restrict__ eb, double* __restrict__ part, int64_t per,
             int64_t total, int64_t kpt, int span, int NRG, int64_t a_blk, int a_rg, int64_t b_blk, int b_rg,
             int ea_w, int ea_rg, int eb_w, int eb_rg, int64_t ksteps, int tail_cols, int side, int drop_stage,
             int* __restrict__ err, const TileJob tj) {
  constexpr uint32_t kBPlane = NC * kBx * 2, kBStage = kSl * kBPlane;
  constexpr int W = NC / 2;             // columns per epilogue thread
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  unsigned char* sA = smem;
  unsigned char* sB = smem + kStages * kAStage;
  __shared__ uint64_t full[kStages], empty[kStages], accf, tfree, mdone;
  __shared__ uint32_t tmem_holder;
  __shared__ int abort_flag;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if constexpr (TILES) {
    if (tj.skip_on_err) {
      // a bounded wait of an earlier product of the same chain gave up: its result is no
      // longer meaningful, so skip the work (read once, so the whole CTA agrees)
      __shared__ int skip;
      if (tid == 0) skip = *(volatile int*)err;
      __syncthreads();
      if (skip) return;
    }
  }
  // stream-K: first tile of the CTA's run, counted in its own sequence of tiles
  const int64_t first_tile = ((int64_t)(side ? blockIdx.x / side : blockIdx.x) * per) / kpt;
  const int KB = (int)(kpt * (kKiChunk / kKiBox));
  // K-steps and 32-column boxes of chunk c (the last chunk may be partly padding)
  auto chunk_ksteps = [&](int64_t c) { return (int)min((int64_t)(kKiChunk / 16), ksteps - c * (kKiChunk / 16)); };

  if (tid == 0) {
    for (int q = 0; q < kStages; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[q])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[q])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&accf)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 8;" ::"r"(smem_u32(&tfree)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mdone)));
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_flag = 0;
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_holder;
  volatile int* abort_v = &abort_flag;

  if (warp == 0) {
    // ---- TMA producer: per 32-column box, the six A planes and the six B planes in one stage
    if (lane == 0) {
      int nbx = 0;
      bool ok = true;
      WorkIter<TILES, NC> it;
      for (it.init(tj, per, total, kpt, side); it.valid && ok; it.next(tj)) {
        const int64_t T = it.T, c = it.c;
        int64_t w, ta, tb;  // problem, and the tile's row offsets in A and in B
        if constexpr (TILES) {
          w = 0;
          ta = it.I * kKiRows;
          tb = it.J * NC;
        } else {
          w = T / NRG;
          const int64_t rg = T - w * NRG;
          ta = rg * a_rg;
          tb = rg * b_rg;
        }
        const int nbox = (chunk_ksteps(c) + kKPB - 1) / kKPB;
        for (int kb = 0; kb < nbox; ++kb, ++nbx) {
          const int64_t gb = c * kBoxesPerChunk + kb;            // box along K
          const int64_t blk = w * KB + gb / kBoxesPerTile;        // (problem, 64-column memory tile)
          const int x = (int)(gb % kBoxesPerTile) * kBx;
          const int arow = (int)(blk * a_blk + ta), brow = (int)(blk * b_blk + tb);
          const int st = nbx % kStages;
          if (nbx >= kStages && !mbar_wait(smem_u32(&empty[st]), ((nbx / kStages) - 1) & 1, abort_v)) {
            ok = false;
            break;
          }
          if (nbx == drop_stage) {  // test hook: this stage never arrives, so the waits run out
            ok = false;
            break;
          }
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&full[st])),
                       "r"((uint32_t)S * (kAPlane + kBPlane)));
          for (int q = 0; q < S; ++q) {
            asm volatile(
                "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
                ::"r"(smem_u32(sA + st * kAStage + q * kAPlane)), "l"(&tmA), "r"(x), "r"(arow), "r"(q),
                "r"(smem_u32(&full[st]))
                : "memory");
            asm volatile(
                "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
                ::"r"(smem_u32(sB + st * kBStage + q * kBPlane)), "l"(&tmB), "r"(x), "r"(brow), "r"(q),
                "r"(smem_u32(&full[st]))
                : "memory");
          }
        }
      }
      // drain: every issued load lands before the CTA may exit (bounded, even after an abort)
      int unused = 0;
      for (int i = (nbx > kStages ? nbx - kStages : 0); i < nbx; ++i)
        mbar_wait(smem_u32(&full[i % kStages]), (i / kStages) & 1, &unused);
    }
  } else if (warp == 1) {
    // ---- MMA issuer (the whole warp, one elected lane issues).  An accumulation period ends
    // after kDrainK K-steps or with the last K-step of the tile's chunks in this CTA's share;
    // the next period starts once the epilogue has drained the groups.
    {
      const uint32_t idesc = (1u << 4) | ((uint32_t)(NC >> 3) << 17) | ((uint32_t)(kKiRows >> 4) << 24);
      int nbx = 0, kp = 0, dc = 0;  // boxes consumed, K-steps in the open period, periods closed
      bool ok = true;
      WorkIter<TILES, NC> it;
      for (it.init(tj, per, total, kpt, side); it.valid && ok; it.next(tj)) {
        const int nks = chunk_ksteps(it.c);
        const bool tile_end = it.last();
        for (int kb = 0; kb < (nks + kKPB - 1) / kKPB && ok; ++kb, ++nbx) {
          const int st = nbx % kStages;
          if (!mbar_wait_warp(smem_u32(&full[st]), (nbx / kStages) & 1, abort_v)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          for (int kk = 0; kk < kKPB && kKPB * kb + kk < nks; ++kk) {
            if (kp == 0 && dc > 0) {
              // the epilogue has drained the previous period's groups
              if (!mbar_wait_warp(smem_u32(&tfree), (dc - 1) & 1, abort_v)) {
                ok = false;
                break;
              }
              asm volatile("tcgen05.fence::after_thread_sync;");
            }
            issue_kstep<NC, S>(tmem, smem_u32(sA + st * kAStage), smem_u32(sB + st * kBStage), kk, idesc, kp == 0);
            ++kp;
            if (period_closes(it.c * (kKiChunk / 16) + kKPB * kb + kk, ksteps, tail_cols,
                              tile_end && kKPB * kb + kk + 1 == nks)) {
              commit_elect(smem_u32(&accf));
              ++dc;
              kp = 0;
            }
          }
          if (!ok) break;
          commit_elect(smem_u32(&empty[st]));
        }
      }
      // completion of every MMA issued above (waited on before the tensor memory is freed)
      commit_elect(smem_u32(&mdone));
    }
  } else {
    // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (rows m of the tile) and
    // columns W h .. + W - 1, h = (w - 2) / 4
    const int q4 = warp & 3, h = (warp - 2) >> 2;
    const int r = q4 * 32 + lane;
    float Sh[W], Sl[W];
#pragma unroll
    for (int c = 0; c < W; ++c) Sh[c] = Sl[c] = 0.f;
    int dc = 0;  // periods drained
    bool ok = true;
    WorkIter<TILES, NC> it;
    for (it.init(tj, per, total, kpt, side); it.valid && ok; it.next(tj)) {
      const int64_t T = it.T;
      const bool tile_end = it.last();
      // periods that close within this chunk (the MMA warp's schedule)
      const int nks = chunk_ksteps(it.c);
      int nd = 0;
      for (int k = 0; k < nks; ++k)
        nd += period_closes(it.c * (kKiChunk / 16) + k, ksteps, tail_cols, tile_end && k + 1 == nks);
      for (int q = 0; q < nd; ++q, ++dc) {
        if (!mbar_wait(smem_u32(&accf), dc & 1, abort_v)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        add_groups<NC, W, S>(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(h * W), Sh, Sl);
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tfree)) : "memory");
      }
      if (!ok || !tile_end) continue;
      // the tile's last chunk in this CTA's share: write the result
      if constexpr (TILES) {
        const int64_t row = it.I * kKiRows + r;
        if (row < tj.mvalid) {
          const int er = ea[row];
          double* Crow = tj.C + row * tj.ldc;
#pragma unroll
          for (int c = 0; c < W; ++c) {
            const int64_t col = it.J * NC + h * W + c;
            if (col < tj.wvalid && (!tj.lower || col <= row)) {
              const double v = pair_to_double_scaled(Sh[c], Sl[c], er + eb[col] - 14);
              Crow[col] = tj.op == 0 ? v : (tj.op == 1 ? Crow[col] - v : -v);
            }
          }
        }
#pragma unroll
        for (int c = 0; c < W; ++c) Sh[c] = Sl[c] = 0.f;
      } else {
        const int64_t w = T / NRG, rg = T - w * NRG;
        const int er = ea[w * ea_w + rg * ea_rg + r];
        const int* ebt = eb + w * eb_w + rg * eb_rg;
        double* P = part + ((blockIdx.x * (int64_t)span + (it.wt - first_tile)) * NC) * kKiRows;
#pragma unroll
        for (int c = 0; c < W; ++c) {
          const int col = h * W + c;
          P[col * kKiRows + r] = pair_to_double_scaled(Sh[c], Sl[c], er + ebt[col] - 14);
          Sh[c] = Sl[c] = 0.f;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 1) {
    // every issued MMA has finished before the tensor memory is released (bounded wait)
    int unused = 0;
    if (lane == 0) mbar_wait(smem_u32(&mdone), 0, &unused);
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
  }
  if (tid == 0 && *abort_v) atomicExch(err, 1);
}

}  // namespace

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

namespace {
// Tensor map of six FP16 digit planes tiled by 64-column memory tiles: dims (64 columns, rows
// tile-major, plane), one plane every plane_elems halves; the pipeline loads boxes of kBx columns
// x box_rows rows swizzled at their row width (x a multiple of kBx within a tile: 16-byte aligned).
bool encode_planes(PFN_cuTensorMapEncodeTiled_v12000 enc, CUtensorMap* tm, const void* planes, int64_t rows,
                   int64_t plane_elems, int box_rows) {
  const cuuint64_t dims[3] = {(cuuint64_t)kKiBox, (cuuint64_t)rows, (cuuint64_t)kSl};
  const cuuint64_t strides[2] = {(cuuint64_t)(kKiBox * 2), (cuuint64_t)(plane_elems * 2)};
  const cuuint32_t box[3] = {(cuuint32_t)kBx, (cuuint32_t)box_rows, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  return enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, const_cast<void*>(planes), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, kBx == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
}  // namespace

void kinv_tc_prepare() {
  static PerDeviceOnce attr;
  attr([] {
    const int s64 = (int)dig_smem(64), s32 = (int)dig_smem(32);
    cudaFuncSetAttribute(sk_tc_kernel<64, false, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, s64);
    cudaFuncSetAttribute(sk_tc_kernel<64, false, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize, s64);
    cudaFuncSetAttribute(sk_tc_kernel<64, false, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize, s64);
    cudaFuncSetAttribute(sk_tc_kernel<32, false, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, s32);
    cudaFuncSetAttribute(sk_tc_kernel<32, false, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize, s32);
    cudaFuncSetAttribute(sk_tc_kernel<32, false, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize, s32);
    cudaFuncSetAttribute(sk_tc_kernel<64, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s64);
  });
}

namespace {
// The stream-K kernel for NC columns and nplanes digit planes (4, 5 or 6; 6 otherwise).
template <int NC>
decltype(&sk_tc_kernel<NC, false, 6>) sk_stream_kernel(int nplanes) {
  return nplanes == 4 ? sk_tc_kernel<NC, false, 4> : (nplanes == 5 ? sk_tc_kernel<NC, false, 5> : sk_tc_kernel<NC, false, 6>);
}
}  // namespace

int64_t kinv_tc_ld(int64_t n) { return (n + kKiChunk - 1) / kKiChunk * kKiChunk; }

bool kinv_tc_supported(int64_t n) {
  const int64_t ld = kinv_tc_ld(n);
  return n > 0 && ld <= INT32_MAX && tensor_map_encoder() != nullptr;
}

size_t kinv_tc_plane_elems(int64_t n) { return (size_t)kSl * kinv_tc_ld(n) * kinv_tc_ld(n); }

namespace {
// data columns of the last 16-column K-step of a K axis of K columns (K > 0)
int tail_cols(int64_t K) { return (int)(K - 16 * ((K + 15) / 16 - 1)); }

int num_sms_tc() {
  static int v = 0;
  if (v == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    if (v <= 0) v = 1;
  }
  return v;
}
}  // namespace

int64_t kinv_tc_slice(const double* X, int64_t ldx, int64_t rows, int64_t n, int* ex, void* planes_v,
                      int64_t rows_pad, cudaStream_t s) {
  if (rows_pad <= 0) return 0;
  const int64_t ldk = kinv_tc_ld(n);
  if (rows_pad < 8 * (int64_t)num_sms_tc()) {  // few rows: split each row over CTAs too
    // at most eight slices per row (each reads the whole row for its maximum), at least 512 wide
    const int64_t cw = std::max<int64_t>(512, (ldk / 8 + 511) / 512 * 512);
    slice_rows_wide_kernel<<<dim3((unsigned)rows_pad, (unsigned)((ldk + cw - 1) / cw)), 256, 0, s>>>(
        X, ldx, rows, n, ex, static_cast<__half*>(planes_v), rows_pad, ldk, cw);
    return 1;
  }
  int64_t blocks = (rows_pad + 7) / 8;  // eight warps (rows) per CTA
  if (blocks > 65535 * 8) blocks = 65535 * 8;
  slice_rows_kernel<<<(unsigned)blocks, 256, 0, s>>>(X, ldx, rows, n, ex, static_cast<__half*>(planes_v), rows_pad,
                                                    ldk);
  return 1;
}

namespace {
struct KiPlan {
  int64_t tiles, kpt, total, per, ctas;
  int span;
};
// M x n matrix (rows padded to Mp, columns to ld, both multiples of 128)
KiPlan ki_plan(int64_t M, int64_t n) {
  KiPlan p;
  p.tiles = kinv_tc_ld(M) / kKiRows;
  p.kpt = kinv_tc_ld(n) / kKiChunk;
  p.total = p.tiles * p.kpt;
  const int64_t slots = num_sms_tc();
  p.per = (p.total + slots - 1) / slots;
  p.ctas = (p.total + p.per - 1) / p.per;
  p.span = (int)((p.per + p.kpt - 1) / p.kpt + 1);
  return p;
}
}  // namespace

size_t rowmat_tc_plane_elems(int64_t M, int64_t n) { return (size_t)kSl * kinv_tc_ld(M) * kinv_tc_ld(n); }

size_t rowmat_tc_work_elems(int64_t M, int64_t n) {
  const int64_t ld = kinv_tc_ld(n);
  const KiPlan p = ki_plan(M, n);
  // right-hand-side planes (FP16, counted in doubles) + exponents + partials
  const size_t planes = ((size_t)kSl * kKiN * ld * 2 + 7) / 8;
  return 32 + planes + kKiN + (size_t)p.ctas * p.span * kKiN * kKiRows;  // 32: alignment slack
}
size_t kinv_tc_work_elems(int64_t n) { return rowmat_tc_work_elems(n, n); }

int kinv_reduce(const double* part, double* X, int64_t ldx, int64_t n, int64_t nb, int BM, int BR, int64_t per,
                int64_t kpt, int span, int64_t tiles, cudaStream_t s);

cudaError_t rowmat_apply_tc(const void* planes, const int* ea, int64_t M, int64_t n, const double* D, int64_t B,
                            double* X, int64_t ldx, double* work, int* err, cudaStream_t s, int64_t* launches,
                            int drop_stage, int nplanes) {
  work = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(work) + 255) & ~(uintptr_t)255);
  *launches = 0;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return cudaErrorNotSupported;
  const int64_t ld = kinv_tc_ld(n), Mp = kinv_tc_ld(M);
  const KiPlan p = ki_plan(M, n);
  __half* bpl = reinterpret_cast<__half*>(work);
  int* eb = reinterpret_cast<int*>(work + ((size_t)kSl * kKiN * ld * 2 + 7) / 8);
  double* part = work + ((size_t)kSl * kKiN * ld * 2 + 7) / 8 + kKiN;
  // tiled planes: (64 columns, tile-major rows kb * Mp + i, plane)
  CUtensorMap tA, tB;
  if (!encode_planes(enc, &tA, planes, ld / kKiBox * Mp, Mp * ld, kKiRows) ||
      !encode_planes(enc, &tB, bpl, ld / kKiBox * kKiN, kKiN * ld, kKiN))
    return cudaErrorInvalidValue;
  kinv_tc_prepare();
  for (int64_t q0 = 0; q0 < B; q0 += kKiN) {
    const int64_t nb = B - q0 < kKiN ? B - q0 : kKiN;
    *launches += kinv_tc_slice(D + q0 * n, n, nb, n, eb, bpl, kKiN, s);
    // tiles: the 128-row tiles of the matrix (one problem); A rows kbg Mp + 128 t, B rows 64 kbg
    sk_stream_kernel<64>(nplanes)<<<(unsigned)p.ctas, kKiThreads, dig_smem(64), s>>>(
        tA, tB, ea, eb, part, p.per, p.total, p.kpt, p.span, (int)p.tiles, Mp, kKiRows, kKiN, 0, 0, kKiRows, 0, 0,
        (n + 15) / 16, tail_cols(n), 0, drop_stage, err, TileJob{});
    *launches += 1;
    *launches += kinv_reduce(part, X + q0 * ldx, ldx, M, nb, kKiRows, kKiN, p.per, p.kpt, p.span, p.tiles, s);
  }
  return cudaGetLastError();
}

cudaError_t kinv_apply_tc(const void* planes, const int* ea, int64_t n, const double* D, int64_t B, double* X,
                          double* work, int* err, cudaStream_t s, int64_t* launches, int drop_stage, int nplanes) {
  return rowmat_apply_tc(planes, ea, n, n, D, B, X, n, work, err, s, launches, drop_stage, nplanes);
}

int64_t kinv_tc_slice_t(const double* X, int64_t ldx, int64_t rows, int64_t cols, int* ex, void* planes,
                        int64_t rows_pad, unsigned long long* colmax, cudaStream_t s) {
  if (rows_pad <= 0) return 0;
  const int64_t ldk = kinv_tc_ld(rows);
  cudaMemsetAsync(colmax, 0, sizeof(unsigned long long) * (size_t)(cols > 0 ? cols : 1), s);
  int64_t nl = 0;
  if (rows > 0 && cols > 0) {
    col_max_kernel<<<dim3((unsigned)((cols + 63) / 64), (unsigned)((rows + 255) / 256)), 256, 0, s>>>(X, ldx, rows,
                                                                                                  cols, colmax);
    ++nl;
  }
  slice_cols_kernel<<<dim3((unsigned)(ldk / 64), (unsigned)(rows_pad / 64)), 256, 0, s>>>(
      X, ldx, rows, cols, colmax, ex, static_cast<__half*>(planes), rows_pad, ldk);
  return nl + 1;
}

// C (op)= A B^T over 128 x 64 tiles (Sec. 4, Phase 2: the Cholesky's updates and the inverse of its
// factor), A and B given by digit planes (rows padded to kinv_tc_ld(M), kinv_tc_ld(N); K columns)
// and row exponents; A and B may be the same planes.  Lower: the lower trapezoid of tiles only,
// written on and below the diagonal (N <= M).  Tiles are dealt round-robin to one CTA per SM.
cudaError_t digit_gemm_tc(const void* pa, const int* ea, const void* pb, const int* eb, const DigitGemm& g, int* err,
                          cudaStream_t s, int64_t* launches, int drop_stage) {
  *launches = 0;
  if (g.M <= 0 || g.N <= 0 || g.K <= 0) return cudaSuccess;
  if (g.lower && g.N > g.M) return cudaErrorInvalidValue;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return cudaErrorNotSupported;
  const int64_t Mp = kinv_tc_ld(g.M), Np = g.Npad > 0 ? g.Npad : kinv_tc_ld(g.N), ld = kinv_tc_ld(g.K);
  const int64_t RT = Mp / kKiRows, JW = (g.N + kKiN - 1) / kKiN, I0 = JW / 2;
  TileJob tj{};
  tj.C = g.C;
  tj.ldc = g.ldc;
  tj.mvalid = g.M;
  tj.wvalid = g.N;
  tj.JW = JW;
  tj.trap = g.lower ? 1 : 0;
  tj.tiles = g.lower ? I0 * (I0 + 1) + (RT - I0) * JW : RT * JW;
  tj.lower = g.lower ? 1 : 0;
  tj.op = g.op;
  tj.kfirst = g.kfirst;
  tj.klast = g.klast;
  tj.skip_on_err = g.skip_on_err ? 1 : 0;
  const int64_t ctas = tj.tiles < num_sms_tc() ? tj.tiles : num_sms_tc();
  CUtensorMap tA, tB;
  if (!encode_planes(enc, &tA, pa, ld / kKiBox * Mp, Mp * ld, kKiRows) ||
      !encode_planes(enc, &tB, pb, ld / kKiBox * Np, Np * ld, kKiN))
    return cudaErrorInvalidValue;
  kinv_tc_prepare();
  sk_tc_kernel<64, true><<<(unsigned)ctas, kKiThreads, dig_smem(64), s>>>(
      tA, tB, ea, eb, nullptr, 0, 0, ld / kKiChunk, 1, 1, Mp, 0, Np, 0, 0, 0, 0, 0, (g.K + 15) / 16, tail_cols(g.K), 0,
      drop_stage, err, tj);
  *launches = 1;
  return cudaGetLastError();
}

// The Cholesky's updates C -= X X[0:w]^T on and below the diagonal, X the m x kdim block whose
// planes kinv_tc_slice formed (rows_pad = kinv_tc_ld(m)), w <= m (w = m: the whole lower
// triangle); B's rows are the first w rows of the same planes.  The epilogue subtracts in place.
cudaError_t syrk_lower_tc(const void* planes, const int* ex, int64_t m, int64_t w, int64_t kdim, double* C,
                          int64_t ldc, int* err, cudaStream_t s, int64_t* launches, int drop_stage) {
  DigitGemm g{};
  g.C = C;
  g.ldc = ldc;
  g.M = m;
  g.N = w;
  g.K = kdim;
  g.Npad = kinv_tc_ld(m);
  g.lower = true;
  g.op = 1;
  g.skip_on_err = true;
  return digit_gemm_tc(planes, ex, planes, ex, g, err, s, launches, drop_stage);
}

// ------------------------------------------------------------------ batched adjoint products
// The double-FP32 tier's adjoint product for batches, m-hat_w[b][j] = sum_i conj(F-hat_w[i][j])
// d-hat_w[b][i] (Sec. 4, the block-diagonalised circulant), by the same exact digit planes.
// Per frequency it is the real GEMM D[j][n] = sum_k A'_w[j][k] B_w[n][k] over k = 2 i + c:
//   A'_w[j][2i] = Re F-hat_w[i][j],  A'_w[j][2i+1] = Im F-hat_w[i][j]           (formed once)
//   B_w[2b][.] = (Re d, Im d),  B_w[2b+1][.] = (Im d, -Re d)  at (2i, 2i+1)      (per call)
// so that D[j][2b] = Re m-hat_w[b][j] and D[j][2b+1] = Im m-hat_w[b][j].  A' has one exponent
// per (w, j) over i and B one per (w, b), so each output's scale factors out of its sum.
// Planes: A' [S][n_f][K_pad / 64][N_m,pad][64], B [S][n_f][K_pad / 64][NB_pad][64] FP16 (tiled
// by 64-column boxes) with K_pad = 2R rounded up to 128, N_m,pad to 128 and NB_pad = 2B to 64.  A unit is (w, 128 rows j, 64 columns n)
// over all of K (chunks of 128 as above); the (w, row tile) units are split evenly over groups of
// NG CTAs (one CTA per SM), the CTAs of a group taking the same units for the NG column groups
// side by side, so a row tile's A' planes come from HBM once and from L2 for the other groups.

namespace {

__global__ void adj_planes_kernel(const float4* __restrict__ hat, int64_t nf, int64_t R, int64_t Nm, int64_t Nmp,
                                  int64_t Kp, __half* __restrict__ planes, int* __restrict__ ex) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // w Nmp + j
  if (idx >= nf * Nmp) return;
  const int64_t w = idx / Nmp, j = idx - w * Nmp;
  const int64_t plane2 = nf * Nmp * Kp / 2;  // one plane in half2 units
  const int64_t KB = Kp / kKiBox;
  // tiled: [w][k / 64][j][64] within a plane
  __half2* row = reinterpret_cast<__half2*>(planes) + (w * KB * Nmp + j) * (kKiBox / 2);
  int e = 0;
  if (j < Nm) {
    double mx = 0.0;
    for (int64_t i = 0; i < R; ++i) {
      const float4 v = hat[(w * R + i) * Nm + j];
      mx = fmax(mx, fmax(fabs((double)v.x + (double)v.y), fabs((double)v.z + (double)v.w)));
    }
    if (mx > 0.0) frexp(mx, &e);
  }
  ex[idx] = e;
  for (int64_t i = 0; i < Kp / 2; ++i) {
    long long vr = 0, vi = 0;
    if (j < Nm && i < R) {
      const float4 v = hat[(w * R + i) * Nm + j];
      vr = __double2ll_rn(scalbn((double)v.x + (double)v.y, 47 - e));
      vi = __double2ll_rn(scalbn((double)v.z + (double)v.w, 47 - e));
    }
    int dr[kSl], di[kSl];
    digits6(vr, dr);
    digits6(vi, di);
#pragma unroll
    for (int s = 0; s < kSl; ++s)
      row[s * plane2 + (i / (kKiBox / 2)) * Nmp * (kKiBox / 2) + (i % (kKiBox / 2))] =
          __halves2half2(__int2half_rn(dr[s]), __int2half_rn(di[s]));
  }
}

// B planes of one call: one CTA per (w, b), b < NBp / 2 (rows past B are zeros).
__global__ void adj_vec_planes_kernel(const float4* __restrict__ dhat, int64_t nf, int64_t R, int64_t B,
                                      int64_t NBp, int64_t Kp, __half* __restrict__ planes, int* __restrict__ eb) {
  const int64_t w = blockIdx.x, b = blockIdx.y;
  const float4* src = dhat + (b * nf + w) * R;  // float-pair spectra, joined in FP64 by integer operations
  unsigned long long mb = 0;
  if (b < B)
    for (int64_t i = threadIdx.x; i < R; i += blockDim.x) {
      const float4 v = src[i];
      mb = max(mb, max(abs_bits(pair_to_double_scaled(v.x, v.y, 0)), abs_bits(pair_to_double_scaled(v.z, v.w, 0))));
    }
  __shared__ unsigned long long red[32];
  __shared__ int es;
  for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mb;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) mb = max(mb, red[k]);
    const int e = exp_of_bits(mb);
    es = e;
    eb[w * NBp + 2 * b] = e;
    eb[w * NBp + 2 * b + 1] = e;
  }
  __syncthreads();
  const int e = es;
  const int64_t plane2 = nf * NBp * Kp / 2;
  const int64_t KB = Kp / kKiBox;
  // tiled: [w][k / 64][n][64] within a plane
  __half2* r0 = reinterpret_cast<__half2*>(planes) + (w * KB * NBp + 2 * b) * (kKiBox / 2);
  __half2* r1 = r0 + kKiBox / 2;
  for (int64_t i = threadIdx.x; i < Kp / 2; i += blockDim.x) {
    long long vr = 0, vi = 0;
    if (b < B && i < R) {
      const float4 v = src[i];
      vr = round_scaled(pair_to_double_scaled(v.x, v.y, 0), 47 - e);
      vi = round_scaled(pair_to_double_scaled(v.z, v.w, 0), 47 - e);
    }
    int dr[kSl], di[kSl];
    digits6(vr, dr);
    digits6(vi, di);
#pragma unroll
    for (int s = 0; s < kSl; ++s) {
      const int64_t o = s * plane2 + (i / (kKiBox / 2)) * NBp * (kKiBox / 2) + (i % (kKiBox / 2));
      r0[o] = __halves2half2(__int2half_rn(dr[s]), __int2half_rn(di[s]));
      r1[o] = __halves2half2(__int2half_rn(di[s]), __int2half_rn(-dr[s]));
    }
  }
}

template <int S>
__global__ void __launch_bounds__(kKiThreads, 1)
adj_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              const int* __restrict__ ea, const int* __restrict__ eb, float4* __restrict__ mhat, int nf,
              int64_t Nm, int64_t Nmp, int64_t NBp, int B, int nchunk, int JT, int NG, int64_t per, int64_t total,
              int ksteps, int tail_cols, int drop_stage, int* __restrict__ err) {
  constexpr uint32_t kBPlane = kKiN * kBx * 2, kBStage = kSl * kBPlane;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  unsigned char* sA = smem;
  unsigned char* sB = smem + kStages * kAStage;
  __shared__ uint64_t full[kStages], empty[kStages], accf, tfree, mdone;
  __shared__ uint32_t tmem_holder;
  __shared__ int abort_flag;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // CTA b takes column group g = b % NG of the (w, row tile) units [q per, (q + 1) per), q = b / NG:
  // the NG CTAs of a row tile stream its planes at about the same time, so all but the first
  // read them from L2
  const int g = (int)(blockIdx.x % NG);
  const int64_t u0 = (int64_t)(blockIdx.x / NG) * per;
  const int64_t u1 = min(total, u0 + per);
  const int nunits = (int)(u1 - u0);
  // K-steps of chunk c (the last chunk may be partly padding, neither loaded nor multiplied)
  auto chunk_ksteps = [&](int c) { return min(kKiChunk / 16, ksteps - c * (kKiChunk / 16)); };

  if (tid == 0) {
    for (int q = 0; q < kStages; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[q])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[q])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&accf)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 8;" ::"r"(smem_u32(&tfree)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mdone)));
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_flag = 0;
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_holder;
  volatile int* abort_v = &abort_flag;

  if (warp == 0) {
    // ---- TMA producer: per 32-column box, the six A' planes and the six B planes in one stage
    if (lane == 0) {
      int nbx = 0;
      bool ok = true;
      for (int u = 0; u < nunits && ok; ++u) {
        const int64_t unit = u0 + u;
        const int jt = (int)(unit % JT);
        const int w = (int)(unit / JT);
        const int KB = nchunk * (kKiChunk / kKiBox);
        for (int c = 0; c < nchunk && ok; ++c) {
          const int nbox = (chunk_ksteps(c) + kKPB - 1) / kKPB;
          for (int kb = 0; kb < nbox; ++kb, ++nbx) {
            const int gb = c * kBoxesPerChunk + kb;  // box along K
            // tiled planes: memory tile gb / kBoxesPerTile of frequency w starts at row (w KB + tile) rows
            const int64_t tile = (int64_t)w * KB + gb / kBoxesPerTile;
            const int arow = (int)(tile * Nmp + (int64_t)jt * kKiRows);
            const int brow = (int)(tile * NBp + (int64_t)g * kKiN);
            const int x = (gb % kBoxesPerTile) * kBx;
            const int st = nbx % kStages;
            if (nbx >= kStages && !mbar_wait(smem_u32(&empty[st]), ((nbx / kStages) - 1) & 1, abort_v)) {
              ok = false;
              break;
            }
            if (nbx == drop_stage) {  // test hook: this stage never arrives, so the waits run out
              ok = false;
              break;
            }
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&full[st])),
                         "r"((uint32_t)S * (kAPlane + kBPlane)));
            for (int q = 0; q < S; ++q) {
              asm volatile(
                  "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
                  ::"r"(smem_u32(sA + st * kAStage + q * kAPlane)), "l"(&tmA), "r"(x), "r"(arow), "r"(q),
                  "r"(smem_u32(&full[st]))
                  : "memory");
              asm volatile(
                  "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
                  ::"r"(smem_u32(sB + st * kBStage + q * kBPlane)), "l"(&tmB), "r"(x), "r"(brow), "r"(q),
                  "r"(smem_u32(&full[st]))
                  : "memory");
            }
          }
        }
      }
      int unused = 0;
      for (int i = (nbx > kStages ? nbx - kStages : 0); i < nbx; ++i)
        mbar_wait(smem_u32(&full[i % kStages]), (i / kStages) & 1, &unused);
    }
  } else if (warp == 1) {
    // ---- MMA issuer (the whole warp, one elected lane issues); accumulation periods of kDrainK
    // K-steps, the last one of each unit closed by the unit's end
    {
      const uint32_t idesc = (1u << 4) | ((uint32_t)(kKiN >> 3) << 17) | ((uint32_t)(kKiRows >> 4) << 24);
      int nbx = 0, kp = 0, dc = 0;  // boxes consumed, K-steps in the open period, periods closed
      bool ok = true;
      for (int u = 0; u < nunits && ok; ++u) {
        for (int c = 0; c < nchunk && ok; ++c) {
          const int nks = chunk_ksteps(c);
          for (int kb = 0; kb < (nks + kKPB - 1) / kKPB && ok; ++kb, ++nbx) {
            const int st = nbx % kStages;
            if (!mbar_wait_warp(smem_u32(&full[st]), (nbx / kStages) & 1, abort_v)) {
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            for (int kk = 0; kk < kKPB && kKPB * kb + kk < nks; ++kk) {
              if (kp == 0 && dc > 0) {
                if (!mbar_wait_warp(smem_u32(&tfree), (dc - 1) & 1, abort_v)) {
                  ok = false;
                  break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
              }
              issue_kstep<kKiN, S>(tmem, smem_u32(sA + st * kAStage), smem_u32(sB + st * kBStage), kk, idesc, kp == 0);
              ++kp;
              if (period_closes(c * (kKiChunk / 16) + kKPB * kb + kk, ksteps, tail_cols,
                                c == nchunk - 1 && kKPB * kb + kk + 1 == nks)) {
                commit_elect(smem_u32(&accf));
                ++dc;
                kp = 0;
              }
            }
            if (!ok) break;
            commit_elect(smem_u32(&empty[st]));
          }
        }
      }
      commit_elect(smem_u32(&mdone));
    }
  } else {
    // ---- epilogue: TMEM lanes 32 (w % 4) .. + 31 = rows j of the tile, columns 32 h .. + 31
    // = vectors 16 h .. + 15 of the group (real, imaginary interleaved)
    const int q4 = warp & 3, h = (warp - 2) >> 2;
    const int r = q4 * 32 + lane;
    float Sh[32], Sl[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) Sh[c] = Sl[c] = 0.f;
    // periods per unit: the MMA warp's schedule over the unit's ksteps K-steps
    int nper = 0;
    for (int k = 0; k < ksteps; ++k) nper += period_closes(k, ksteps, tail_cols, k + 1 == ksteps);
    int dc = 0;
    bool ok = true;
    for (int u = 0; u < nunits && ok; ++u) {
      const int64_t unit = u0 + u;
      const int jt = (int)(unit % JT);
      const int w = (int)(unit / JT);
      for (int q = 0; q < nper; ++q, ++dc) {
        if (!mbar_wait(smem_u32(&accf), dc & 1, abort_v)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        add_groups<kKiN, 32, S>(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(h * 32), Sh, Sl);
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tfree)) : "memory");
      }
      if (!ok) break;
      const int64_t j = (int64_t)jt * kKiRows + r;
      const int ej = ea[w * Nmp + j];
#pragma unroll
      for (int k = 0; k < 32; k += 2) {
        const int n = g * kKiN + h * 32 + k;
        const int b = n >> 1;
        if (j < Nm && b < B) {
          const int sh = ej + eb[w * NBp + n] - 14;
          mhat[((int64_t)b * nf + w) * Nm + j] = pair_scaled2(Sh[k], Sl[k], Sh[k + 1], Sl[k + 1], sh);
        }
      }
#pragma unroll
      for (int k = 0; k < 32; ++k) Sh[k] = Sl[k] = 0.f;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 1) {
    int unused = 0;
    if (lane == 0) mbar_wait(smem_u32(&mdone), 0, &unused);
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
  }
  if (tid == 0 && *abort_v) atomicExch(err, 1);
}

int64_t rup(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

}  // namespace

size_t adj_digits_plane_elems(int64_t nf, int64_t R, int64_t Nm) {
  return (size_t)kSl * nf * rup(Nm, kKiRows) * rup(2 * R, kKiChunk);
}
size_t adj_digits_exp_elems(int64_t nf, int64_t Nm) { return (size_t)nf * rup(Nm, kKiRows); }

bool adj_digits_supported(int64_t nf, int64_t R, int64_t Nm, int64_t B) {
  const int64_t Kp = rup(2 * R, kKiChunk), Nmp = rup(Nm, kKiRows), NBp = rup(2 * B, kKiN);
  return B >= 16 && nf * Nmp <= INT32_MAX && nf * NBp <= INT32_MAX && Kp <= INT32_MAX &&
         tensor_map_encoder() != nullptr;
}

int64_t adj_digits_build(const void* hat, int64_t nf, int64_t R, int64_t Nm, void* planes, int* ex, cudaStream_t s) {
  const int64_t Nmp = rup(Nm, kKiRows), Kp = rup(2 * R, kKiChunk);
  const int64_t total = nf * Nmp;
  adj_planes_kernel<<<(unsigned)((total + 127) / 128), 128, 0, s>>>(static_cast<const float4*>(hat), nf, R, Nm, Nmp,
                                                                    Kp, static_cast<__half*>(planes), ex);
  return 1;
}

size_t adj_digits_work_bytes(int64_t nf, int64_t R, int64_t B) {
  const int64_t Kp = rup(2 * R, kKiChunk), NBp = rup(2 * B, kKiN);
  return 256 + (size_t)kSl * nf * NBp * Kp * 2 + (size_t)nf * NBp * sizeof(int);
}

cudaError_t adj_digits_apply(const void* planes, const int* ea, int64_t nf, int64_t R, int64_t Nm, const void* dhat,
                             void* mhat, int64_t B, void* work, int* err, cudaStream_t s, int* launches,
                             int drop_stage, int nplanes) {
  *launches = 0;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return cudaErrorNotSupported;
  const int64_t Kp = rup(2 * R, kKiChunk), Nmp = rup(Nm, kKiRows), NBp = rup(2 * B, kKiN);
  unsigned char* wb = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(work) + 255) & ~(uintptr_t)255);
  __half* bpl = reinterpret_cast<__half*>(wb);
  int* eb = reinterpret_cast<int*>(wb + (size_t)kSl * nf * NBp * Kp * 2);
  CUtensorMap tA, tB;
  if (!encode_planes(enc, &tA, planes, nf * (Kp / kKiBox) * Nmp, nf * Nmp * Kp, kKiRows) ||
      !encode_planes(enc, &tB, bpl, nf * (Kp / kKiBox) * NBp, nf * NBp * Kp, kKiN))
    return cudaErrorInvalidValue;
  adj_digits_prepare();
  adj_vec_planes_kernel<<<dim3((unsigned)nf, (unsigned)(NBp / 2)), 128, 0, s>>>(
      static_cast<const float4*>(dhat), nf, R, B, NBp, Kp, bpl, eb);
  const int JT = (int)(Nmp / kKiRows), NG = (int)(NBp / kKiN);
  // units (w, row tile), each taken by NG CTAs side by side (one per 64-column group of B)
  const int64_t total = nf * JT;
  const int64_t groups = std::max<int64_t>(1, num_sms_tc() / NG);
  const int64_t per = (total + groups - 1) / groups;
  const int64_t ctas = (total + per - 1) / per * NG;
  auto kern = nplanes == 4 ? adj_tc_kernel<4> : (nplanes == 5 ? adj_tc_kernel<5> : adj_tc_kernel<6>);
  kern<<<(unsigned)ctas, kKiThreads, dig_smem(kKiN), s>>>(
      tA, tB, ea, eb, static_cast<float4*>(mhat), (int)nf, Nm, Nmp, NBp, (int)B, (int)(Kp / kKiChunk), JT, NG, per,
      total, (int)((2 * R + 15) / 16), tail_cols(2 * R), drop_stage, err);
  *launches = 2;
  return cudaGetLastError();
}

void adj_digits_prepare() {
  static PerDeviceOnce attr;
  attr([] {
    const int sm = (int)dig_smem(kKiN);
    cudaFuncSetAttribute(adj_tc_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(adj_tc_kernel<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(adj_tc_kernel<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  });
}


// ------------------------------------------------------------------ batched forward products
// The double-FP32 tier's forward product for batches, d-hat_w[b][i] = sum_j F-hat_w[i][j]
// m-hat_w[b][j], by the same exact digit planes.  Per frequency it is the real GEMM
// D[n][i] = sum_k V_w[n][k] A_w[i][k] over k = 2 j + c with
//   A_w[i][2j] = Re F-hat_w[i][j],  A_w[i][2j+1] = Im F-hat_w[i][j]          (formed once)
//   V_w[2b][.] = (Re m, -Im m),  V_w[2b+1][.] = (Im m, Re m)  at (2j, 2j+1)   (per call)
// so D[2b][i] = Re d-hat_w[b][i] and D[2b+1][i] = Im d-hat_w[b][i]; one exponent per (w, i) for
// A and per (w, b) for V.  The long K axis (2 N_m) runs through the stream-K kernel with tiles
// (w, NC rows i), the 128 vector rows of 64 vectors as the MMA's M, NC = 32 for R <= 32 and
// 64 otherwise; the row groups of a frequency run side by side on neighbouring CTAs.
// Planes: A [S][n_f][K_pad / 64][R_pad][64], V [S][n_f][K_pad / 64][128][64].

namespace {

int fwd_nc(int64_t R) { return R <= 32 ? 32 : 64; }

// A planes: one CTA per (w, i < R_pad)
__global__ void fwd_planes_kernel(const float4* __restrict__ hat, int64_t nf, int64_t R, int64_t Nm, int64_t Rp,
                                  int64_t Kp, __half* __restrict__ planes, int* __restrict__ ex) {
  const int64_t w = blockIdx.x, i = blockIdx.y;
  const int64_t KB = Kp / kKiBox;
  const float4* row = hat + (w * R + i) * Nm;
  double mx = 0.0;
  if (i < R)
    for (int64_t j = threadIdx.x; j < Nm; j += blockDim.x) {
      const float4 v = row[j];
      mx = fmax(mx, fmax(fabs((double)v.x + (double)v.y), fabs((double)v.z + (double)v.w)));
    }
  __shared__ double red[32];
  __shared__ int es;
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) mx = fmax(mx, red[k]);
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);
    es = e;
    ex[w * Rp + i] = e;
  }
  __syncthreads();
  const int e = es;
  const int64_t plane2 = nf * KB * Rp * (kKiBox / 2);
  __half2* out = reinterpret_cast<__half2*>(planes);
  for (int64_t j = threadIdx.x; j < Kp / 2; j += blockDim.x) {
    long long vr = 0, vi = 0;
    if (i < R && j < Nm) {
      const float4 v = row[j];
      vr = __double2ll_rn(scalbn((double)v.x + (double)v.y, 47 - e));
      vi = __double2ll_rn(scalbn((double)v.z + (double)v.w, 47 - e));
    }
    int dr[kSl], di[kSl];
    digits6(vr, dr);
    digits6(vi, di);
    const int64_t o = ((w * KB + j / (kKiBox / 2)) * Rp + i) * (kKiBox / 2) + j % (kKiBox / 2);
#pragma unroll
    for (int s = 0; s < kSl; ++s) out[s * plane2 + o] = __halves2half2(__int2half_rn(dr[s]), __int2half_rn(di[s]));
  }
}

// V planes of one call (vectors b0 .. b0 + nb - 1): one CTA per (w, b < 64); rows past nb zero
__global__ void fwd_vec_planes_kernel(const float4* __restrict__ mhat, int64_t nf, int64_t Nm, int64_t b0, int64_t nb,
                                      int64_t Kp, __half* __restrict__ planes, int* __restrict__ ex) {
  const int64_t w = blockIdx.x, b = blockIdx.y;
  const int64_t KB = Kp / kKiBox;
  const float4* src = mhat + ((b0 + b) * nf + w) * Nm;  // float-pair spectra, joined by integer operations
  unsigned long long mb = 0;
  if (b < nb)
    for (int64_t j = threadIdx.x; j < Nm; j += blockDim.x) {
      const float4 v = src[j];
      mb = max(mb, max(abs_bits(pair_to_double_scaled(v.x, v.y, 0)), abs_bits(pair_to_double_scaled(v.z, v.w, 0))));
    }
  __shared__ unsigned long long red[32];
  __shared__ int es;
  for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mb;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) mb = max(mb, red[k]);
    const int e = exp_of_bits(mb);
    es = e;
    ex[w * kKiRows + 2 * b] = e;
    ex[w * kKiRows + 2 * b + 1] = e;
  }
  __syncthreads();
  const int e = es;
  const int64_t plane2 = nf * KB * kKiRows * (kKiBox / 2);
  __half2* out = reinterpret_cast<__half2*>(planes);
  for (int64_t j = threadIdx.x; j < Kp / 2; j += blockDim.x) {
    long long vr = 0, vi = 0;
    if (b < nb && j < Nm) {
      const float4 v = src[j];
      vr = round_scaled(pair_to_double_scaled(v.x, v.y, 0), 47 - e);
      vi = round_scaled(pair_to_double_scaled(v.z, v.w, 0), 47 - e);
    }
    int dr[kSl], di[kSl];
    digits6(vr, dr);
    digits6(vi, di);
    const int64_t o = ((w * KB + j / (kKiBox / 2)) * kKiRows + 2 * b) * (kKiBox / 2) + j % (kKiBox / 2);
#pragma unroll
    for (int s = 0; s < kSl; ++s) {
      out[s * plane2 + o] = __halves2half2(__int2half_rn(dr[s]), __int2half_rn(-di[s]));
      out[s * plane2 + o + kKiBox / 2] = __halves2half2(__int2half_rn(di[s]), __int2half_rn(dr[s]));
    }
  }
}

// d-hat[b0 + b][w][i] = (D[2b][i], D[2b+1][i]) summed over the CTAs that covered tile (w, i / NC)
__global__ void fwd_reduce_kernel(const double* __restrict__ part, float4* __restrict__ dhat, int64_t nf, int64_t R,
                                  int64_t b0, int64_t nb, int NC, int NRG, int64_t per, int64_t kpt, int span) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nb * nf * R) return;
  const int64_t b = idx / (nf * R), wi = idx - b * nf * R, w = wi / R, i = wi - w * R;
  const int64_t rg = i / NC;
  const int col = (int)(i % NC);
  // the CTA groups whose runs of (w, chunk) units cover frequency w, each through its CTA rg
  const int64_t q0 = (w * kpt) / per, q1 = ((w + 1) * kpt - 1) / per;
  double re = 0.0, im = 0.0;
  for (int64_t q = q0; q <= q1; ++q) {
    const int64_t slot = w - (q * per) / kpt;
    const double* P = part + (((q * NRG + rg) * span + slot) * NC + col) * kKiRows;
    re += P[2 * b];
    im += P[2 * b + 1];
  }
  // stored as float pairs (hi = the sum rounded to FP32, lo = the rest rounded to FP32)
  const float rh = __double2float_rn(re), ih = __double2float_rn(im);
  dhat[((b0 + b) * nf + w) * R + i] =
      make_float4(rh, __double2float_rn(re - (double)rh), ih, __double2float_rn(im - (double)ih));
}

struct FwdPlan {
  int NC, NRG;
  int64_t Rp, Kp, KB, kpt, total, per, ctas;
  int span;
};
FwdPlan fwd_plan(int64_t nf, int64_t R, int64_t Nm) {
  FwdPlan p;
  p.NC = fwd_nc(R);
  p.Rp = rup(R, p.NC);
  p.NRG = (int)(p.Rp / p.NC);
  p.Kp = rup(2 * Nm, kKiChunk);
  p.KB = p.Kp / kKiBox;
  p.kpt = p.Kp / kKiChunk;
  // units (w, chunk), each taken by NRG CTAs side by side (one per row group of F), so that a
  // frequency's vector planes come from HBM once and from L2 for the other row groups
  p.total = nf * p.kpt;
  const int64_t groups = std::max<int64_t>(1, num_sms_tc() / p.NRG);
  p.per = (p.total + groups - 1) / groups;
  p.ctas = (p.total + p.per - 1) / p.per * p.NRG;
  p.span = (int)((p.per + p.kpt - 1) / p.kpt + 1);
  return p;
}

}  // namespace

size_t fwd_digits_plane_elems(int64_t nf, int64_t R, int64_t Nm) {
  const FwdPlan p = fwd_plan(nf, R, Nm);
  return (size_t)kSl * nf * p.KB * p.Rp * kKiBox;
}
size_t fwd_digits_exp_elems(int64_t nf, int64_t R) { return (size_t)nf * rup(R, fwd_nc(R)); }

bool fwd_digits_supported(int64_t nf, int64_t R, int64_t Nm, int64_t B) {
  const int64_t KB = rup(2 * Nm, kKiChunk) / kKiBox;
  const int64_t rows = nf * KB * (rup(R, fwd_nc(R)) > kKiRows ? rup(R, fwd_nc(R)) : kKiRows);
  return B >= 16 && rows <= INT32_MAX && tensor_map_encoder() != nullptr;
}

int64_t fwd_digits_build(const void* hat, int64_t nf, int64_t R, int64_t Nm, void* planes, int* ex, cudaStream_t s) {
  const FwdPlan p = fwd_plan(nf, R, Nm);
  fwd_planes_kernel<<<dim3((unsigned)nf, (unsigned)p.Rp), 256, 0, s>>>(
      static_cast<const float4*>(hat), nf, R, Nm, p.Rp, p.Kp, static_cast<__half*>(planes), ex);
  return 1;
}

size_t fwd_digits_work_bytes(int64_t nf, int64_t R, int64_t Nm) {
  const FwdPlan p = fwd_plan(nf, R, Nm);
  return 512 + (size_t)kSl * nf * p.KB * kKiRows * kKiBox * 2 + (size_t)nf * kKiRows * sizeof(int) +
         (size_t)p.ctas * p.span * p.NC * kKiRows * sizeof(double);
}

cudaError_t fwd_digits_apply(const void* planes, const int* ex, int64_t nf, int64_t R, int64_t Nm, const void* mhat,
                             void* dhat, int64_t B, void* work, int* err, cudaStream_t s, int* launches,
                             int drop_stage, int nplanes) {
  *launches = 0;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return cudaErrorNotSupported;
  const FwdPlan p = fwd_plan(nf, R, Nm);
  unsigned char* wb = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(work) + 255) & ~(uintptr_t)255);
  __half* vpl = reinterpret_cast<__half*>(wb);
  const size_t vbytes = (size_t)kSl * nf * p.KB * kKiRows * kKiBox * 2;
  int* ev = reinterpret_cast<int*>(wb + vbytes);
  double* part = reinterpret_cast<double*>(
      (reinterpret_cast<uintptr_t>(wb + vbytes + (size_t)nf * kKiRows * sizeof(int)) + 255) & ~(uintptr_t)255);
  CUtensorMap tA, tB;
  if (!encode_planes(enc, &tA, vpl, nf * p.KB * kKiRows, nf * p.KB * kKiRows * kKiBox, kKiRows) ||
      !encode_planes(enc, &tB, planes, nf * p.KB * p.Rp, nf * p.KB * p.Rp * kKiBox, p.NC))
    return cudaErrorInvalidValue;
  kinv_tc_prepare();
  for (int64_t b0 = 0; b0 < B; b0 += 64) {
    const int64_t nb = B - b0 < 64 ? B - b0 : 64;
    fwd_vec_planes_kernel<<<dim3((unsigned)nf, 64), 256, 0, s>>>(static_cast<const float4*>(mhat), nf, Nm, b0, nb,
                                                                  p.Kp, vpl, ev);
    // tiles (w, rg): A rows (w KB + kb) 128, B rows (w KB + kb) R_pad + NC rg
    const int64_t ksteps = (2 * Nm + 15) / 16;
    if (p.NC == 32)
      sk_stream_kernel<32>(nplanes)<<<(unsigned)p.ctas, kKiThreads, dig_smem(32), s>>>(
          tA, tB, ev, ex, part, p.per, p.total, p.kpt, p.span, p.NRG, kKiRows, 0, p.Rp, p.NC, kKiRows, 0, (int)p.Rp,
          p.NC, ksteps, tail_cols(2 * Nm), p.NRG, drop_stage, err, TileJob{});
    else
      sk_stream_kernel<64>(nplanes)<<<(unsigned)p.ctas, kKiThreads, dig_smem(64), s>>>(
          tA, tB, ev, ex, part, p.per, p.total, p.kpt, p.span, p.NRG, kKiRows, 0, p.Rp, p.NC, kKiRows, 0, (int)p.Rp,
          p.NC, ksteps, tail_cols(2 * Nm), p.NRG, drop_stage, err, TileJob{});
    const int64_t tot = nb * nf * R;
    fwd_reduce_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(part, static_cast<float4*>(dhat), nf, R, b0, nb,
                                                                   p.NC, p.NRG, p.per, p.kpt, p.span);
    *launches += 3;
  }
  return cudaGetLastError();
}

}  // namespace bti
