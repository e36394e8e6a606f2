// Explicit-inverse product of the online solve on the tensor cores (tcgen05), exact in
// integer slices.
//
// X[b][i] = sum_j Kinv[i][j] D[b][j] (x = K^{-1} d, Eq. (4.13) with the solves moved
// offline) needs about 48 significant bits, which no tensor-core input type holds.  Both
// operands are therefore cut into S = 6 planes of balanced base-256 digits, each digit an
// integer in [-128, 128] and so exact in FP16:
//   Kinv[i][j] = 2^(ea_i - 7) sum_s P_s[i][j] 2^(-8 s),   D[b][j] = 2^(eb_b - 7) sum_t Q_t[b][j] 2^(-8 t)
// with ea_i, eb_b the binary exponents of the row maxima (so the planes hold a 47-bit
// fixed-point image of each row, the rest rounded away).  Then
//   X[b][i] = 2^(ea_i + eb_b - 14) sum_g 2^(-8 g) G_g[i][b],  G_g = sum_{s + t = g} P_s Q_t^T,
// keeping the 21 plane pairs with s + t <= 5 (the dropped ones lie below 2^-48 of the row
// scale).  Every product of two digits is at most 2^14 and each group sums at most six
// plane pairs, so over a chunk of 128 columns j a group's sum stays below 6 * 128 * 2^14
// < 2^24: the FP32 accumulators in tensor memory hold it exactly.  After each chunk the
// epilogue warps read the six groups, scale them by 2^(-8 g) (exact) and add them into
// float-pair accumulators with a two-sum, as the double-FP32 kernels do.
//
// Layout: the K^{-1} planes [S][rows_pad][ldk] FP16 (rows_pad and ldk multiples of 128,
// zero padding) are formed once with the inverse; the right-hand-side planes [S][64][ldk]
// per call.  A CTA (one per SM) walks a contiguous run of (row tile, chunk) units (stream-K,
// as the double-FP32 kernel), so every SM gets the same number of chunks; partial tiles go
// to an FP64 buffer that a second kernel sums in CTA order.  Warp 0 issues the TMA loads
// (K^{-1} planes 128 rows x 64 columns per stage, the six right-hand-side planes per 64
// columns), warp 1 issues tcgen05.mma (M = 128, N = 64, K = 16) into six TMEM groups of 64
// columns, warps 2-9 drain the groups per chunk.  Every wait is bounded; on a timeout the
// kernel sets the error word, stops issuing, lets what it issued land and frees its tensor
// memory.
#include "bti_internal.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

namespace bti {

namespace {

constexpr int kSl = 6;                 // digit planes per operand
constexpr int kKiRows = 128;           // MMA M: rows of K^{-1} per tile
constexpr int kKiN = 64;               // MMA N: right-hand sides per launch chunk
constexpr int kKiBox = 64;             // FP16 columns per TMA box row (128 bytes, the swizzle width)
constexpr int kKiChunk = 128;          // columns per exact accumulation chunk (two boxes)
constexpr int kKiAStages = 4;          // K^{-1} plane stages (16 KB each)
constexpr int kKiBStages = 2;          // right-hand-side stages (six planes, 48 KB each)
constexpr int kKiThreads = 320;        // warp 0 TMA, warp 1 MMA, warps 2-9 epilogue
constexpr uint32_t kKiATile = kKiRows * 128;
constexpr uint32_t kKiBPlane = kKiN * 128;
constexpr uint32_t kKiBTile = kSl * kKiBPlane;
constexpr uint32_t kKiTmemCols = 512;  // six groups of 64 columns (384) rounded to a power of two
constexpr long long kKiSpin = 1ll << 22;
constexpr size_t kKiSmem = 1024 + kKiAStages * (size_t)kKiATile + kKiBStages * (size_t)kKiBTile;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// K-major operand, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
               : "=r"(done) : "r"(bar), "r"(parity) : "memory");
  return done != 0;
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
  for (long long it = 0; it < kKiSpin; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 1023) == 1023 && *abort_flag) return false;
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

// exp[r] = binary exponent of max_j |X[r][j]| (frexp convention: max = f 2^e, f in [0.5, 1);
// 0 for an all-zero row).  One CTA per row.
__global__ void row_exponent_kernel(const double* __restrict__ X, int64_t ldx, int64_t n, int* __restrict__ ex) {
  const int64_t r = blockIdx.x;
  double mx = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) mx = fmax(mx, fabs(X[r * ldx + j]));
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, red[w]);
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);
    ex[r] = e;
  }
}

// Digit planes of rows 0 .. rows-1 (columns 0 .. n-1; columns n .. ldk-1 and rows rows ..
// rows_pad-1 are written as zeros): round X[r][j] 2^(47 - e_r) to an integer v (|v| <= 2^47)
// and peel balanced base-256 digits from the bottom; plane s holds digit 5 - s.
__global__ void slice_digits_kernel(const double* __restrict__ X, int64_t ldx, int64_t rows, int64_t n,
                                    const int* __restrict__ ex, __half* __restrict__ planes, int64_t rows_pad,
                                    int64_t ldk) {
  const int64_t total = rows_pad * ldk;
  const int64_t plane = rows_pad * ldk;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / ldk, j = e - r * ldk;
    long long v = 0;
    if (r < rows && j < n) v = __double2ll_rn(scalbn(X[r * ldx + j], 47 - ex[r]));
    int d[kSl];
#pragma unroll
    for (int k = 0; k < kSl - 1; ++k) {
      const int dk = (int)(((v & 255) ^ 128) - 128);  // in [-128, 127]
      d[k] = dk;
      v = (v - dk) >> 8;
    }
    d[kSl - 1] = (int)v;  // |v| <= 128 here
#pragma unroll
    for (int s = 0; s < kSl; ++s) planes[s * plane + e] = __int2half_rn(d[kSl - 1 - s]);
  }
}

__global__ void __launch_bounds__(kKiThreads, 1)
kinv_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const int* __restrict__ ea, const int* __restrict__ eb, int64_t n, int nb, double* __restrict__ part,
               int64_t per, int64_t total, int64_t kpt, int span, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  unsigned char* sA = smem;
  unsigned char* sB = smem + kKiAStages * kKiATile;
  __shared__ uint64_t fullA[kKiAStages], emptyA[kKiAStages], fullB[kKiBStages], emptyB[kKiBStages], accf, tfree,
      mdone;
  __shared__ uint32_t tmem_holder;
  __shared__ int abort_flag;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t u0 = (int64_t)blockIdx.x * per;
  const int64_t u1 = min(total, u0 + per);
  const int64_t first_tile = u0 / kpt;
  const int nunits = (int)(u1 - u0);

  if (tid == 0) {
    for (int s = 0; s < kKiAStages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&fullA[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&emptyA[s])));
    }
    for (int s = 0; s < kKiBStages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&fullB[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&emptyB[s])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&accf)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 8;" ::"r"(smem_u32(&tfree)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mdone)));
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_flag = 0;
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                 "r"(kKiTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_holder;
  volatile int* abort_v = &abort_flag;

  if (warp == 0) {
    // ---- TMA producer: per 64-column box, the six right-hand-side planes, then the six
    // K^{-1} planes of the unit's row tile
    if (lane == 0) {
      int na = 0, nbx = 0;
      bool ok = true;
      for (int u = 0; u < nunits && ok; ++u) {
        const int64_t unit = u0 + u, t = unit / kpt, c = unit - t * kpt;
        for (int kb = 0; kb < kKiChunk / kKiBox && ok; ++kb, ++nbx) {
          const int k0 = (int)((c * kKiChunk) + kb * kKiBox);
          const int bs = nbx % kKiBStages;
          if (nbx >= kKiBStages && !mbar_wait(smem_u32(&emptyB[bs]), ((nbx / kKiBStages) - 1) & 1, abort_v)) {
            ok = false;
            break;
          }
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&fullB[bs])),
                       "r"(kKiBTile));
          for (int q = 0; q < kSl; ++q)
            asm volatile(
                "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
                ::"r"(smem_u32(sB + bs * kKiBTile + q * kKiBPlane)), "l"(&tmB), "r"(k0), "r"(0), "r"(q),
                "r"(smem_u32(&fullB[bs]))
                : "memory");
          for (int s = 0; s < kSl; ++s, ++na) {
            const int as = na % kKiAStages;
            if (na >= kKiAStages && !mbar_wait(smem_u32(&emptyA[as]), ((na / kKiAStages) - 1) & 1, abort_v)) {
              ok = false;
              break;
            }
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&fullA[as])),
                         "r"(kKiATile));
            asm volatile(
                "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
                ::"r"(smem_u32(sA + as * kKiATile)), "l"(&tmA), "r"(k0), "r"((int)(t * kKiRows)), "r"(s),
                "r"(smem_u32(&fullA[as]))
                : "memory");
          }
        }
      }
      // drain: every issued load lands before the CTA may exit (bounded, even after an abort)
      int unused = 0;
      for (int i = (na > kKiAStages ? na - kKiAStages : 0); i < na; ++i)
        mbar_wait(smem_u32(&fullA[i % kKiAStages]), (i / kKiAStages) & 1, &unused);
      for (int i = (nbx > kKiBStages ? nbx - kKiBStages : 0); i < nbx; ++i)
        mbar_wait(smem_u32(&fullB[i % kKiBStages]), (i / kKiBStages) & 1, &unused);
    }
  } else if (warp == 1) {
    // ---- MMA issuer: group g = s + t accumulates P_s Q_t^T at TMEM columns 64 g
    if (lane == 0) {
      const uint32_t idesc = (1u << 4) | ((uint32_t)(kKiN >> 3) << 17) | ((uint32_t)(kKiRows >> 4) << 24);
      int na = 0, nbx = 0;
      bool ok = true;
      for (int u = 0; u < nunits && ok; ++u) {
        // the epilogue has drained the previous chunk's groups
        if (u > 0 && !mbar_wait(smem_u32(&tfree), (u - 1) & 1, abort_v)) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        for (int kb = 0; kb < kKiChunk / kKiBox && ok; ++kb, ++nbx) {
          const int bs = nbx % kKiBStages;
          if (!mbar_wait(smem_u32(&fullB[bs]), (nbx / kKiBStages) & 1, abort_v)) {
            ok = false;
            break;
          }
          const uint32_t b0 = smem_u32(sB + bs * kKiBTile);
          for (int s = 0; s < kSl; ++s, ++na) {
            const int as = na % kKiAStages;
            if (!mbar_wait(smem_u32(&fullA[as]), (na / kKiAStages) & 1, abort_v)) {
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t a0 = smem_u32(sA + as * kKiATile);
            for (int t = 0; t + s < kSl; ++t) {
#pragma unroll
              for (int kk = 0; kk < kKiBox / 16; ++kk) {
                const uint32_t acc = (kb == 0 && s == 0 && kk == 0) ? 0u : 1u;
                asm volatile(
                    "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                    ::"r"(tmem + (uint32_t)((s + t) * kKiN)), "l"(sdesc(a0 + kk * 32)),
                    "l"(sdesc(b0 + t * kKiBPlane + kk * 32)), "r"(idesc), "r"(acc));
              }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         ::"r"(smem_u32(&emptyA[as])) : "memory");
          }
          if (!ok) break;
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                       ::"r"(smem_u32(&emptyB[bs])) : "memory");
        }
        if (!ok) break;
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     ::"r"(smem_u32(&accf)) : "memory");
      }
      // completion of every MMA issued above (waited on before the tensor memory is freed)
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   ::"r"(smem_u32(&mdone)) : "memory");
    }
  } else {
    // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (rows of the tile) and
    // right-hand sides 32 h .. + 31, h = (w - 2) / 4
    const int q4 = warp & 3, h = (warp - 2) >> 2;
    const int r = q4 * 32 + lane;
    float Sh[32], Sl[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) Sh[c] = Sl[c] = 0.f;
    for (int u = 0; u < nunits; ++u) {
      const int64_t unit = u0 + u, t = unit / kpt;
      if (!mbar_wait(smem_u32(&accf), u & 1, abort_v)) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
      for (int g = 0; g < kSl; ++g) {
        uint32_t v[32];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
              "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
              "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
              "=r"(v[30]), "=r"(v[31])
            : "r"(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(g * kKiN + h * 32)));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const float sc = __int_as_float((127 - 8 * g) << 23);  // 2^(-8 g), exact
#pragma unroll
        for (int c = 0; c < 32; ++c) two_sum_acc(Sh[c], Sl[c], __uint_as_float(v[c]) * sc);
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tfree)) : "memory");
      // last unit of this row tile within the CTA's run: write the partial tile
      if (u == nunits - 1 || (unit + 1) / kpt != t) {
        const int64_t row = t * kKiRows + r;
        const int er = row < n ? ea[row] : 0;
        double* P = part + ((blockIdx.x * (int64_t)span + (t - first_tile)) * kKiN) * kKiRows;
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          const int b = h * 32 + c;
          const double val = (b < nb) ? scalbn((double)Sh[c] + (double)Sl[c], er + eb[b] - 14) : 0.0;
          P[b * kKiRows + r] = val;
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
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kKiTmemCols));
  }
  if (tid == 0 && *abort_v) atomicExch(err, 1);
}

}  // namespace

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

void kinv_tc_prepare() {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(kinv_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kKiSmem);
    attr = true;
  }
}

int64_t kinv_tc_ld(int64_t n) { return (n + kKiChunk - 1) / kKiChunk * kKiChunk; }

bool kinv_tc_supported(int64_t n) {
  const int64_t ld = kinv_tc_ld(n);
  return n > 0 && ld <= INT32_MAX && tensor_map_encoder() != nullptr;
}

size_t kinv_tc_plane_elems(int64_t n) { return (size_t)kSl * kinv_tc_ld(n) * kinv_tc_ld(n); }

int64_t kinv_tc_slice(const double* X, int64_t ldx, int64_t rows, int64_t n, int* ex, void* planes_v,
                      int64_t rows_pad, cudaStream_t s) {
  __half* planes = static_cast<__half*>(planes_v);
  if (rows > 0) row_exponent_kernel<<<(unsigned)rows, 256, 0, s>>>(X, ldx, n, ex);
  const int64_t ldk = kinv_tc_ld(n);
  const int64_t total = rows_pad * ldk;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 65535 * 8) blocks = 65535 * 8;
  slice_digits_kernel<<<(unsigned)blocks, 256, 0, s>>>(X, ldx, rows, n, ex, planes, rows_pad, ldk);
  return rows > 0 ? 2 : 1;
}

namespace {
struct KiPlan {
  int64_t tiles, kpt, total, per, ctas;
  int span;
};
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
KiPlan ki_plan(int64_t n) {
  KiPlan p;
  const int64_t ld = kinv_tc_ld(n);
  p.tiles = ld / kKiRows;
  p.kpt = ld / kKiChunk;
  p.total = p.tiles * p.kpt;
  const int64_t slots = num_sms_tc();
  p.per = (p.total + slots - 1) / slots;
  p.ctas = (p.total + p.per - 1) / p.per;
  p.span = (int)((p.per + p.kpt - 1) / p.kpt + 1);
  return p;
}
}  // namespace

size_t kinv_tc_work_elems(int64_t n) {
  const int64_t ld = kinv_tc_ld(n);
  const KiPlan p = ki_plan(n);
  // right-hand-side planes (FP16, counted in doubles) + exponents + partials
  const size_t planes = ((size_t)kSl * kKiN * ld * 2 + 7) / 8;
  return 32 + planes + kKiN + (size_t)p.ctas * p.span * kKiN * kKiRows;  // 32: alignment slack
}

int kinv_reduce(const double* part, double* X, int64_t ldx, int64_t n, int64_t nb, int BM, int BR, int64_t per,
                int64_t kpt, int span, int64_t tiles, cudaStream_t s);

cudaError_t kinv_apply_tc(const void* planes, const int* ea, int64_t n, const double* D, int64_t B, double* X,
                          double* work, int* err, cudaStream_t s, int64_t* launches) {
  work = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(work) + 255) & ~(uintptr_t)255);
  *launches = 0;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return cudaErrorNotSupported;
  const int64_t ld = kinv_tc_ld(n);
  const KiPlan p = ki_plan(n);
  __half* bpl = reinterpret_cast<__half*>(work);
  int* eb = reinterpret_cast<int*>(work + ((size_t)kSl * kKiN * ld * 2 + 7) / 8);
  double* part = work + ((size_t)kSl * kKiN * ld * 2 + 7) / 8 + kKiN;
  CUtensorMap tA, tB;
  {
    const cuuint64_t dims[3] = {(cuuint64_t)ld, (cuuint64_t)ld, (cuuint64_t)kSl};
    const cuuint64_t strides[2] = {(cuuint64_t)(ld * 2), (cuuint64_t)(ld * ld * 2)};
    const cuuint32_t box[3] = {(cuuint32_t)kKiBox, (cuuint32_t)kKiRows, 1};
    const cuuint32_t es[3] = {1, 1, 1};
    if (enc(&tA, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, const_cast<void*>(planes), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  {
    const cuuint64_t dims[3] = {(cuuint64_t)ld, (cuuint64_t)kKiN, (cuuint64_t)kSl};
    const cuuint64_t strides[2] = {(cuuint64_t)(ld * 2), (cuuint64_t)(kKiN * ld * 2)};
    const cuuint32_t box[3] = {(cuuint32_t)kKiBox, (cuuint32_t)kKiN, 1};
    const cuuint32_t es[3] = {1, 1, 1};
    if (enc(&tB, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, bpl, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  kinv_tc_prepare();
  for (int64_t q0 = 0; q0 < B; q0 += kKiN) {
    const int64_t nb = B - q0 < kKiN ? B - q0 : kKiN;
    *launches += kinv_tc_slice(D + q0 * n, n, nb, n, eb, bpl, kKiN, s);
    kinv_tc_kernel<<<(unsigned)p.ctas, kKiThreads, kKiSmem, s>>>(tA, tB, ea, eb, n, (int)nb, part, p.per, p.total,
                                                                 p.kpt, p.span, err);
    *launches += 1;
    *launches += kinv_reduce(part, X + q0 * n, n, n, nb, kKiRows, kKiN, p.per, p.kpt, p.span, p.tiles, s);
  }
  return cudaGetLastError();
}

}  // namespace bti
