// FP16-tier spectral products on the tensor cores (tcgen05) for batches of right-hand sides.
//
// For B >= 8 vectors the per-frequency product d-hat_w = F-hat_w m-hat_w (Sec. 4, the
// block-diagonalised circulant) is a complex GEMM [R x N_m] x [N_m x B].  It runs as a
// real GEMM whose K axis is the interleaved (real, imaginary) FP16 storage of F-hat
// itself, K = 2 N_m, and whose N axis holds the real and imaginary outputs, N = 2 B_g:
//   D[i][2b]   = sum_j F_r(i,j) m_r(b,j) - F_i(i,j) m_i(b,j)
//   D[i][2b+1] = sum_j F_r(i,j) m_i(b,j) + F_i(i,j) m_r(b,j)
// so row 2b of the B operand is (m_r, -m_i) and row 2b+1 is (m_i, m_r), interleaved
// along K.  F-hat tiles [128 rows x 64 halves] stream in by TMA with the 128-byte
// swizzle; the B tiles are built in shared memory by four warps from the FP32 m-hat
// (scaled by a power of two per vector and chunk, then rounded to FP16); one thread
// issues tcgen05.mma (M = 128, K = 16 per instruction) into an FP32 accumulator in
// tensor memory; the four builder warps read it back (tcgen05.ld), apply the row scale
// of F-hat and the inverse vector scale, and write per-chunk partial sums, which a
// second kernel adds in a fixed order.  Every wait is bounded: on a timeout the kernel
// sets the error word, stops issuing, drains what it issued and frees its tensor memory.
#include "bti_internal.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

namespace bti {

namespace {

constexpr int kTcStages = 4;            // pipeline depth (A + B tiles per stage)
constexpr int kTcRows = 128;            // MMA M: rows of F-hat per CTA
constexpr int kTcKBox = 64;             // halves per TMA box row (128 bytes, the swizzle width)
constexpr int kTcThreads = 192;         // warp 0 TMA, warp 1 MMA, warps 2-5 B tiles + epilogue
constexpr uint32_t kTcATile = kTcRows * 128;  // bytes of one A stage
constexpr long long kTcSpin = 1ll << 24;      // poll backstop of every wait
constexpr uint64_t kTcWaitNs = 1000000000ull;  // wall-time limit of every wait: 1 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1024 B apart
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
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait: false after kTcWaitNs of wall time (checked every 256 polls, since a poll of
// try_wait may suspend the thread for microseconds) or kTcSpin polls, whichever comes first,
// or as soon as another thread has flagged an abort.  On giving up it flags the abort.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (long long it = 1; it < kTcSpin; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 255) == 0) {
      if (*abort_flag) return false;
      if (global_ns() - t0 > kTcWaitNs) break;
    }
  }
  *abort_flag = 1;
  return false;
}

template <int BG>
__global__ void __launch_bounds__(kTcThreads, 1)
prod_fwd_f16_tc_kernel(const __grid_constant__ CUtensorMap tmA, const float* __restrict__ scaleF,
                       const float2* __restrict__ mhat, float2* __restrict__ partial, int nf, int R, int64_t Nm,
                       int B, int Kc, int nchunk, int nrt, int drop_stage, int* __restrict__ err) {
  constexpr int N = 2 * BG;                      // MMA N: real and imaginary output columns
  constexpr uint32_t kBTile = (uint32_t)N * 128;  // bytes of one B stage
  constexpr uint32_t kTmemCols = N < 32 ? 32 : N;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  unsigned char* sA = smem;
  unsigned char* sB = smem + kTcStages * kTcATile;
  __shared__ uint64_t fullA[kTcStages], fullB[kTcStages], empty[kTcStages], accf;
  __shared__ uint32_t tmem_holder;
  __shared__ float inv_scale[BG];
  __shared__ int abort_flag;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ch = blockIdx.x, w = blockIdx.y;
  const int rt = blockIdx.z % nrt, grp = blockIdx.z / nrt;
  const int b0 = grp * BG;
  const int64_t K2 = 2 * Nm;                      // halves per F-hat row
  const int64_t kc0 = (int64_t)ch * Kc;
  const int64_t klen = (K2 - kc0) < Kc ? (K2 - kc0) : Kc;
  const int nst = (int)((klen + kTcKBox - 1) / kTcKBox);

  if (tid == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&fullA[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" ::"r"(smem_u32(&fullB[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[s])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&accf)));
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
    // ---- TMA producer: A stage s holds halves kc0 + 64 s .. + 63 of rows rt*128 .. + 127
    if (lane == 0) {
      int issued = 0;
      for (int s = 0; s < nst; ++s) {
        const int slot = s % kTcStages;
        if (s >= kTcStages && !mbar_wait(smem_u32(&empty[slot]), ((s / kTcStages) - 1) & 1, abort_v)) break;
        if (s == drop_stage) break;  // test hook: this stage never arrives, so the waits run out
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&fullA[slot])),
                     "r"(kTcATile));
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
            ::"r"(smem_u32(sA + slot * kTcATile)), "l"(&tmA), "r"((int)(kc0 + (int64_t)s * kTcKBox)),
            "r"(rt * kTcRows), "r"(w), "r"(smem_u32(&fullA[slot]))
            : "memory");
        ++issued;
      }
      // drain: every issued load lands before the CTA may exit (bounded, even after an abort)
      int unused = 0;
      for (int s = (issued > kTcStages ? issued - kTcStages : 0); s < issued; ++s)
        mbar_wait(smem_u32(&fullA[s % kTcStages]), (s / kTcStages) & 1, &unused);
    }
  } else if (warp == 1) {
    // ---- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);
      for (int s = 0; s < nst; ++s) {
        const int slot = s % kTcStages;
        const uint32_t par = (s / kTcStages) & 1;
        if (!mbar_wait(smem_u32(&fullA[slot]), par, abort_v)) break;
        if (!mbar_wait(smem_u32(&fullB[slot]), par, abort_v)) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t a0 = smem_u32(sA + slot * kTcATile), bb0 = smem_u32(sB + slot * kBTile);
#pragma unroll
        for (int kk = 0; kk < kTcKBox / 16; ++kk) {
          const uint32_t acc = (s > 0 || kk > 0) ? 1u : 0u;
          asm volatile(
              "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
              ::"r"(tmem), "l"(sdesc(a0 + kk * 32)), "l"(sdesc(bb0 + kk * 32)), "r"(idesc), "r"(acc));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     ::"r"(smem_u32(&empty[slot])) : "memory");
      }
      // the accumulator is complete once every MMA issued above has finished
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   ::"r"(smem_u32(&accf)) : "memory");
    }
  } else {
    // ---- B-tile builders (128 threads): vector b = b0 + t / 8 (+16 per round), complex
    // columns 4 (t % 8) .. + 3 of each 32-column stage
    const int t = tid - 64;
    const int g = t & 7;
    constexpr int kRounds = BG / 16;
    const float2* mw = mhat + (int64_t)w * Nm;
    const int64_t jc0 = kc0 / 2;
    const int64_t jlen = klen / 2;
    // pass 1: max |m| per vector over this chunk -> a power-of-two scale into FP16's range.
    // Four 32-byte loads per thread per trip keep enough requests in flight.
#pragma unroll
    for (int rd = 0; rd < kRounds; ++rd) {
      const int bl = t / 8 + 16 * rd, b = b0 + bl;
      float mx = 0.f;
      if (b < B) {
        const float2* mb = mw + (int64_t)b * nf * Nm + jc0;
        for (int64_t j0 = 4 * g; j0 < jlen; j0 += 128) {
          float2 v[16];
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int64_t j = j0 + 32 * u + q;
              v[4 * u + q] = j < jlen ? __ldg(mb + j) : make_float2(0.f, 0.f);
            }
#pragma unroll
          for (int e = 0; e < 16; ++e) mx = fmaxf(mx, fmaxf(fabsf(v[e].x), fabsf(v[e].y)));
        }
      }
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 4));
      if (g == 0) {
        int e = 0;
        if (mx > 0.f) frexpf(mx, &e);  // mx = f 2^e, f in [0.5, 1): mx 2^(14-e) < 2^14
        inv_scale[bl] = ldexpf(1.f, e - 14);
      }
    }
    asm volatile("bar.sync 1, 128;");  // the four builder warps only
    float sc[kRounds];
#pragma unroll
    for (int rd = 0; rd < kRounds; ++rd) sc[rd] = 1.f / inv_scale[t / 8 + 16 * rd];
    // pass 2: B stages.  The m-hat values of stage s + 1 are loaded before the wait for stage
    // s's slot, so their latency overlaps the pipeline instead of adding to it.
    auto load_stage = [&](int st, float2 (&v)[kRounds][4]) {
      const int64_t j = jc0 + (int64_t)st * 32 + 4 * g;  // first of this thread's 4 complex columns
#pragma unroll
      for (int rd = 0; rd < kRounds; ++rd) {
        const int b = b0 + t / 8 + 16 * rd;
#pragma unroll
        for (int q = 0; q < 4; ++q)
          v[rd][q] = (st < nst && b < B && j + q < jc0 + jlen) ? __ldg(mw + (int64_t)b * nf * Nm + j + q)
                                                               : make_float2(0.f, 0.f);
      }
    };
    float2 cur[kRounds][4], nxt[kRounds][4];
    load_stage(0, cur);
    for (int s = 0; s < nst; ++s) {
      load_stage(s + 1, nxt);
      const int slot = s % kTcStages;
      if (s >= kTcStages && !mbar_wait(smem_u32(&empty[slot]), ((s / kTcStages) - 1) & 1, abort_v)) break;
      unsigned char* bt = sB + slot * kBTile;
#pragma unroll
      for (int rd = 0; rd < kRounds; ++rd) {
        const int bl = t / 8 + 16 * rd;
        __half2 re[4], im[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float x = cur[rd][q].x * sc[rd], y = cur[rd][q].y * sc[rd];
          re[q] = __floats2half2_rn(x, -y);  // row 2b:   (m_r, -m_i)
          im[q] = __floats2half2_rn(y, x);   // row 2b+1: (m_i,  m_r)
        }
        const int r0 = 2 * bl, r1 = 2 * bl + 1;
        *reinterpret_cast<uint4*>(bt + r0 * 128 + ((g ^ (r0 & 7)) << 4)) = *reinterpret_cast<uint4*>(re);
        *reinterpret_cast<uint4*>(bt + r1 * 128 + ((g ^ (r1 & 7)) << 4)) = *reinterpret_cast<uint4*>(im);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&fullB[slot])) : "memory");
#pragma unroll
      for (int rd = 0; rd < kRounds; ++rd)
#pragma unroll
        for (int q = 0; q < 4; ++q) cur[rd][q] = nxt[rd][q];
    }
    // ---- epilogue: rows of this warp's lane quarter, all N accumulator columns
    const bool ok = mbar_wait(smem_u32(&accf), 0, abort_v);
    asm volatile("tcgen05.fence::after_thread_sync;");
    const int q4 = warp & 3;
    const int i = rt * kTcRows + q4 * 32 + lane;
    const float fs = (ok && i < R) ? scaleF[(int64_t)w * R + i] : 0.f;
#pragma unroll
    for (int c0 = 0; c0 < N; c0 += 8) {
      uint32_t v[8];
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                   : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                   : "r"(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)c0));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (ok && i < R) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int bl = c0 / 2 + q, b = b0 + bl;
          if (b < B) {
            const float f = fs * inv_scale[bl];
            partial[(((int64_t)b * nf + w) * nchunk + ch) * R + i] =
                make_float2(__uint_as_float(v[2 * q]) * f, __uint_as_float(v[2 * q + 1]) * f);
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 1) {
    // the MMAs have completed if accf fired; otherwise wait for them (bounded) before freeing
    if (*abort_v) {
      int dummy = 0;
      mbar_wait(smem_u32(&accf), 0, &dummy);
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
  }
  if (tid == 0 && *abort_v) atomicExch(err, 1);
}

// Adjoint: m-hat_w[b][j] = sum_i conj(F-hat_w[i][j]) s_F(w, i) d-hat_w[b][i].  Read along
// its interleaved (real, imaginary) axis m' = 2 j + c, the FP16 storage of F-hat is an
// MN-major operand A'[m'][i] (m' contiguous for each row i), so with K = R and B rows
// (d_r s_F, d_i s_F) the MMA gives D'[m'][n] = sum_i A'[m'][i] B[n][i], and
//   Re m-hat(b, j) = D'[2j][2b] + D'[2j+1][2b+1],  Im m-hat(b, j) = D'[2j][2b+1] - D'[2j+1][2b]:
// rows 2j and 2j+1 sit in neighbouring TMEM lanes and are combined with one shuffle.
// A CTA covers one frequency, one vector group and a run of 128-row tiles of m'; the B
// operand (all of K) is built once, and two TMEM accumulators let the epilogue of one
// tile overlap the MMAs of the next.
template <int BG>
__global__ void __launch_bounds__(kTcThreads, 1)
prod_adj_f16_tc_kernel(const __grid_constant__ CUtensorMap tmA, const float* __restrict__ scaleF,
                       const float2* __restrict__ dhat, float2* __restrict__ mhat, int nf, int R, int64_t Nm,
                       int B, int tpc, int ntiles, int* __restrict__ err) {
  constexpr int N = 2 * BG;
  constexpr uint32_t kBTile = (uint32_t)N * 128;  // one 64-row K block of the B operand
  constexpr uint32_t kTmemCols = 2 * N;           // two accumulators
  constexpr uint32_t kHalf = 64 * 128;            // one 64-wide half of an A stage: 64 rows of i x 128 B
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  unsigned char* sA = smem;
  unsigned char* sB = smem + kTcStages * kTcATile;
  __shared__ uint64_t fullA[kTcStages], empty[kTcStages], bfull, accf[2], acce[2], mdone;
  __shared__ uint32_t tmem_holder;
  __shared__ float inv_scale[BG];
  __shared__ int abort_flag;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int w = blockIdx.y, grp = blockIdx.z, b0 = grp * BG;
  const int t0 = blockIdx.x * tpc;
  const int nt = (ntiles - t0) < tpc ? (ntiles - t0) : tpc;
  const int nkb = (R + 63) / 64;
  const int nq = nt * nkb;

  if (tid == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&fullA[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[s])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" ::"r"(smem_u32(&bfull)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mdone)));
    for (int a = 0; a < 2; ++a) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&accf[a])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" ::"r"(smem_u32(&acce[a])));
    }
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
    // ---- TMA producer: stage q = (tile, K block); two boxes of 64 m' x 64 rows of i
    if (lane == 0) {
      int issued = 0;
      for (int q = 0; q < nq; ++q) {
        const int slot = q % kTcStages;
        if (q >= kTcStages && !mbar_wait(smem_u32(&empty[slot]), ((q / kTcStages) - 1) & 1, abort_v)) break;
        const int t = t0 + q / nkb, kb = q % nkb;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&fullA[slot])),
                     "r"(kTcATile));
#pragma unroll
        for (int hh = 0; hh < 2; ++hh)
          asm volatile(
              "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
              ::"r"(smem_u32(sA + slot * kTcATile + hh * kHalf)), "l"(&tmA), "r"(kTcRows * t + 64 * hh), "r"(64 * kb),
              "r"(w), "r"(smem_u32(&fullA[slot]))
              : "memory");
        ++issued;
      }
      // drain: every issued load lands before the CTA may exit (bounded, even after an abort)
      int unused = 0;
      for (int q = (issued > kTcStages ? issued - kTcStages : 0); q < issued; ++q)
        mbar_wait(smem_u32(&fullA[q % kTcStages]), (q / kTcStages) & 1, &unused);
    }
  } else if (warp == 1) {
    // ---- MMA issuer: A MN-major (bit 15), B K-major
    if (lane == 0) {
      const uint32_t idesc =
          (1u << 4) | (1u << 15) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);
      bool ok = mbar_wait(smem_u32(&bfull), 0, abort_v);
      for (int tt = 0; ok && tt < nt; ++tt) {
        const int acc = tt & 1;
        if (tt >= 2 && !mbar_wait(smem_u32(&acce[acc]), ((tt >> 1) - 1) & 1, abort_v)) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        for (int kb = 0; kb < nkb; ++kb) {
          const int q = tt * nkb + kb, slot = q % kTcStages;
          if (!mbar_wait(smem_u32(&fullA[slot]), (q / kTcStages) & 1, abort_v)) { ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t a0 = smem_u32(sA + slot * kTcATile), bb0 = smem_u32(sB + kb * kBTile);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            // A: 16 rows of i per step (2048 B); the two m' halves 8 KB apart (leading byte
            // offset), 8-row groups 1024 B apart (stride byte offset)
            const uint64_t ad = (uint64_t)(((a0 + kk * 2048) >> 4) & 0x3FFF) | ((uint64_t)(kHalf >> 4) << 16) |
                                ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
            const uint32_t accum = (kb > 0 || kk > 0) ? 1u : 0u;
            asm volatile(
                "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                ::"r"(tmem + (uint32_t)(acc * N)), "l"(ad), "l"(sdesc(bb0 + kk * 32)), "r"(idesc), "r"(accum));
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                       ::"r"(smem_u32(&empty[slot])) : "memory");
        }
        if (!ok) break;
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     ::"r"(smem_u32(&accf[acc])) : "memory");
      }
      // completes once every MMA issued above has finished (the teardown waits on it)
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   ::"r"(smem_u32(&mdone)) : "memory");
    }
  } else {
    // ---- B operand builders: vector b = b0 + t / 8 (+16 per round); row chunk g of 8 rows of i
    const int t = tid - 64, g = t & 7;
    constexpr int kRounds = BG / 16;
    const float* sf = scaleF + (int64_t)w * R;
#pragma unroll
    for (int rd = 0; rd < kRounds; ++rd) {
      const int bl = t / 8 + 16 * rd, b = b0 + bl;
      float mx = 0.f;
      if (b < B) {
        const float2* db = dhat + ((int64_t)b * nf + w) * R;
        for (int i = g; i < R; i += 8) {
          const float2 v = db[i];
          const float f = sf[i];
          mx = fmaxf(mx, fmaxf(fabsf(v.x * f), fabsf(v.y * f)));
        }
      }
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 4));
      if (g == 0) {
        int e = 0;
        if (mx > 0.f) frexpf(mx, &e);
        inv_scale[bl] = ldexpf(1.f, e - 14);
      }
    }
    asm volatile("bar.sync 1, 128;");
#pragma unroll
    for (int rd = 0; rd < kRounds; ++rd) {
      const int bl = t / 8 + 16 * rd, b = b0 + bl;
      const float sc = 1.f / inv_scale[bl];
      const float2* db = dhat + ((int64_t)b * nf + w) * R;
      for (int kb = 0; kb < nkb; ++kb) {
        __half re[8], im[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int i = 64 * kb + 8 * g + e;
          float2 v = make_float2(0.f, 0.f);
          if (b < B && i < R) {
            v = db[i];
            const float f = sf[i] * sc;
            v.x *= f;
            v.y *= f;
          }
          re[e] = __float2half_rn(v.x);  // row 2b:   d_r s_F
          im[e] = __float2half_rn(v.y);  // row 2b+1: d_i s_F
        }
        unsigned char* bt = sB + kb * kBTile;
        const int r0 = 2 * bl, r1 = 2 * bl + 1;
        *reinterpret_cast<uint4*>(bt + r0 * 128 + ((g ^ (r0 & 7)) << 4)) = *reinterpret_cast<uint4*>(re);
        *reinterpret_cast<uint4*>(bt + r1 * 128 + ((g ^ (r1 & 7)) << 4)) = *reinterpret_cast<uint4*>(im);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bfull)) : "memory");
    // ---- epilogue per tile
    const int q4 = warp & 3;
    for (int tt = 0; tt < nt; ++tt) {
      const int acc = tt & 1;
      const bool ok = mbar_wait(smem_u32(&accf[acc]), (tt >> 1) & 1, abort_v);
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int64_t mrow = (int64_t)kTcRows * (t0 + tt) + q4 * 32 + lane;  // m' = 2 j + c
      const int64_t j = mrow >> 1;
#pragma unroll
      for (int c0 = 0; c0 < N; c0 += 8) {
        uint32_t v[8];
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                     : "r"(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(acc * N + c0)));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) {
          const float x0 = __uint_as_float(v[2 * qq]), x1 = __uint_as_float(v[2 * qq + 1]);
          const float u0 = __shfl_xor_sync(0xffffffffu, x0, 1), u1 = __shfl_xor_sync(0xffffffffu, x1, 1);
          const int bl = c0 / 2 + qq, b = b0 + bl;
          if (ok && (lane & 1) == 0 && b < B && j < Nm) {
            const float f = inv_scale[bl];
            mhat[((int64_t)b * nf + w) * Nm + j] = make_float2((x0 + u1) * f, (x1 - u0) * f);
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce[acc])) : "memory");
      if (!ok) break;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 1) {
    int dummy = 0;  // every MMA issued has finished before the columns are freed
    mbar_wait(smem_u32(&mdone), 0, &dummy);
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
  }
  if (tid == 0 && *abort_v) atomicExch(err, 1);
}

// dhat[b][w][i] = sum over the nchunk partials, fixed order
__global__ void tc_reduce_kernel(const float2* __restrict__ partial, float2* __restrict__ dhat, int64_t total,
                                 int64_t R, int nchunk) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int64_t bw = idx / R, i = idx - bw * R;
  const float2* p = partial + bw * nchunk * R + i;
  float sr = 0.f, si = 0.f;
  for (int c = 0; c < nchunk; ++c) {
    const float2 v = p[(int64_t)c * R];
    sr += v.x;
    si += v.y;
  }
  dhat[idx] = make_float2(sr, si);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

}  // namespace

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() { return encode_fn(); }

bool tc_fwd_f16_supported(int64_t Nm, int64_t R, int64_t B) {
  // rows of F-hat as FP16 halves must be 16-byte strided for TMA (N_m a multiple of 4), and
  // the row tiles times the vector groups must fit the grid's z extent
  const int64_t BG = B > 16 ? 32 : 16;
  const int64_t tiles = ((R + kTcRows - 1) / kTcRows) * ((B + BG - 1) / BG);
  return B >= 8 && Nm % 4 == 0 && 2 * Nm <= INT32_MAX && tiles <= 65535 && encode_fn() != nullptr;
}

size_t tc_fwd_partial_elems(int64_t nf, int64_t R, int64_t Nm, int64_t B) {
  // at most ceil(2 N_m / 1024) chunks (chunks are at least 1024 halves)
  return (size_t)(B * nf * ((2 * Nm + 1023) / 1024) * R);
}

cudaError_t launch_prod_fwd_f16_tc(const void* Fhat, const float* scale, const float2* mhat, float2* partial,
                                   float2* dhat, int64_t nf, int64_t R, int64_t Nm, int64_t B, int* err,
                                   cudaStream_t s, int* launches, int drop_stage) {
  *launches = 0;
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap tm;
  const cuuint64_t dims[3] = {(cuuint64_t)(2 * Nm), (cuuint64_t)R, (cuuint64_t)nf};
  const cuuint64_t strides[2] = {(cuuint64_t)(2 * Nm * 2), (cuuint64_t)(R * 2 * Nm * 2)};
  const cuuint32_t box[3] = {(cuuint32_t)kTcKBox, (cuuint32_t)kTcRows, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  if (enc(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, const_cast<void*>(Fhat), dims, strides, box, es,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  const int BG = B > 16 ? 32 : 16;
  const int64_t nrt = (R + kTcRows - 1) / kTcRows, ng = (B + BG - 1) / BG;
  // Chunks along K: at least four CTAs per SM in total, and at most 4096 halves per chunk so
  // that a CTA's m-hat chunk (B_g x 2048 complex, 256 KB at B_g = 16) is still in L2 when
  // the B tiles are built right after the scale pass reads it; at least 1024 halves.
  const int64_t tiles = nf * nrt * ng;
  int64_t nchunk = (608 + tiles - 1) / tiles;
  int64_t Kc = ((2 * Nm + nchunk - 1) / nchunk + kTcKBox - 1) / kTcKBox * kTcKBox;
  if (Kc > 4096) Kc = 4096;
  if (Kc < 1024) Kc = 1024;
  nchunk = (2 * Nm + Kc - 1) / Kc;
  if (nf > 65535 || nrt * ng > 65535 || nchunk > INT32_MAX) return cudaErrorInvalidValue;
  dim3 grid((unsigned)nchunk, (unsigned)nf, (unsigned)(nrt * ng));
  const size_t smem = 1024 + kTcStages * (kTcATile + (size_t)2 * BG * 128);
  if (BG == 16) {
    cudaFuncSetAttribute(prod_fwd_f16_tc_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    prod_fwd_f16_tc_kernel<16><<<grid, kTcThreads, smem, s>>>(tm, scale, mhat, partial, (int)nf, (int)R, Nm, (int)B,
                                                              (int)Kc, (int)nchunk, (int)nrt, drop_stage, err);
  } else {
    cudaFuncSetAttribute(prod_fwd_f16_tc_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    prod_fwd_f16_tc_kernel<32><<<grid, kTcThreads, smem, s>>>(tm, scale, mhat, partial, (int)nf, (int)R, Nm, (int)B,
                                                              (int)Kc, (int)nchunk, (int)nrt, drop_stage, err);
  }
  const int64_t total = B * nf * R;
  tc_reduce_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(partial, dhat, total, R, (int)nchunk);
  *launches = 2;
  return cudaGetLastError();
}

bool tc_adj_f16_supported(int64_t Nm, int64_t R, int64_t B) {
  const int64_t BG = B > 16 ? 32 : 16;
  // the whole B operand (R rows of i in 64-row blocks) stays in shared memory
  return B >= 8 && Nm % 4 == 0 && 2 * Nm <= INT32_MAX && ((R + 63) / 64) * 2 * BG * 128 <= 128 * 1024 &&
         (B + BG - 1) / BG <= 65535 && encode_fn() != nullptr;
}

cudaError_t launch_prod_adj_f16_tc(const void* Fhat, const float* scale, const float2* dhat, float2* mhat,
                                   int64_t nf, int64_t R, int64_t Nm, int64_t B, int* err, cudaStream_t s,
                                   int* launches) {
  *launches = 0;
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap tm;
  const cuuint64_t dims[3] = {(cuuint64_t)(2 * Nm), (cuuint64_t)R, (cuuint64_t)nf};
  const cuuint64_t strides[2] = {(cuuint64_t)(2 * Nm * 2), (cuuint64_t)(R * 2 * Nm * 2)};
  const cuuint32_t box[3] = {64, 64, 1};  // 64 m' (128 bytes) x 64 rows of i
  const cuuint32_t es[3] = {1, 1, 1};
  if (enc(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, const_cast<void*>(Fhat), dims, strides, box, es,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  const int BG = B > 16 ? 32 : 16;
  const int64_t ng = (B + BG - 1) / BG, ntiles = (2 * Nm + kTcRows - 1) / kTcRows;
  // runs of tiles per CTA: about eight CTAs per SM in total
  const int64_t work = ntiles * nf * ng;
  int64_t tpc = (work + 1215) / 1216;
  if (tpc < 1) tpc = 1;
  const int64_t nblk = (ntiles + tpc - 1) / tpc;
  if (nf > 65535 || ng > 65535 || nblk > INT32_MAX) return cudaErrorInvalidValue;
  dim3 grid((unsigned)nblk, (unsigned)nf, (unsigned)ng);
  const size_t smem = 1024 + kTcStages * (size_t)kTcATile + (size_t)((R + 63) / 64) * 2 * BG * 128;
  if (BG == 16) {
    cudaFuncSetAttribute(prod_adj_f16_tc_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    prod_adj_f16_tc_kernel<16><<<grid, kTcThreads, smem, s>>>(tm, scale, dhat, mhat, (int)nf, (int)R, Nm, (int)B,
                                                              (int)tpc, (int)ntiles, err);
  } else {
    cudaFuncSetAttribute(prod_adj_f16_tc_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    prod_adj_f16_tc_kernel<32><<<grid, kTcThreads, smem, s>>>(tm, scale, dhat, mhat, (int)nf, (int)R, Nm, (int)B,
                                                              (int)tpc, (int)ntiles, err);
  }
  *launches = 1;
  return cudaGetLastError();
}

}  // namespace bti
