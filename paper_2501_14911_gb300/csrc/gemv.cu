// Products of one (or two) vectors with a dense float-pair matrix: the online solve of the
// real-time case (Sec. 4, Phase 4, one observation vector at a time).
//
// With one or two right-hand sides the explicit-inverse product x = K^{-1} d and the d2q
// product q = Q d (Eq. (4.14)) are matrix-vector products: 0.25 (or 0.5) multiply-adds per
// byte of the matrix, so they are bound by HBM, not by any arithmetic pipe.  Both matrices are
// held as float pairs (hi, lo), 8 bytes per entry like FP64, and the products run in float-pair
// arithmetic on the FP32 pipes (GB300 issues FP64 at 1/64 of the FP32 rate, which would bind
// a single-vector FP64 product below the HBM rate).
//
// K^{-1} is symmetric, so its product reads the lower triangle only: tile (I, J), J <= I, of
// 128 x 128 entries contributes A_IJ x_J to y_I and, below the diagonal, A_IJ^T x_I to y_J.
// The tiles are split evenly over the CTAs in row-panel order; each CTA keeps its rows' partial
// sums in registers across the tiles of a panel and writes one partial per panel it touches,
// and every below-diagonal tile writes its column partial.  A second kernel adds the partials
// of each output block in a fixed order, so the result does not depend on timing.
#include "bti_internal.cuh"

#include <cmath>

namespace bti {

namespace {

constexpr int kSvT = 128;  // tile edge (rows and columns)

__device__ __forceinline__ void pr_mac(float& Sh, float& Sl, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float pe = __fmaf_rn(ah, bh, -p);
  pe = __fmaf_rn(ah, bl, pe);
  pe = __fmaf_rn(al, bh, pe);
  const float s = __fadd_rn(Sh, p);
  const float bb = __fsub_rn(s, Sh);
  const float e = __fadd_rn(__fsub_rn(Sh, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  Sh = s;
  Sl = __fadd_rn(Sl, __fadd_rn(e, pe));
}

// (ah, al) += (bh, bl), renormalised
__device__ __forceinline__ void pr_add(float& ah, float& al, float bh, float bl) {
  const float s = __fadd_rn(ah, bh);
  const float bb = __fsub_rn(s, ah);
  float e = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, bb)), __fsub_rn(bh, bb));
  e = __fadd_rn(e, __fadd_rn(al, bl));
  ah = __fadd_rn(s, e);
  al = __fsub_rn(e, __fsub_rn(ah, s));
}

// sum of a float pair over the 32 lanes of a warp (every lane gets it)
__device__ __forceinline__ void warp_pair_sum(float& h, float& l) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, h, o);
    const float ol = __shfl_xor_sync(0xffffffffu, l, o);
    pr_add(h, l, oh, ol);
  }
}

// tile u of the lower triangle in row-panel order -> (I, J), J <= I
__host__ __device__ inline void tri_tile(int64_t u, int64_t& I, int64_t& J) {
  int64_t i = (int64_t)((std::sqrt(8.0 * (double)u + 1.0) - 1.0) * 0.5);
  while ((i + 1) * (i + 2) / 2 <= u) ++i;
  while (i * (i + 1) / 2 > u) --i;
  I = i;
  J = u - i * (i + 1) / 2;
}

// Writes this lane's row partials of panel I (the warp's 16 rows) to prow after summing them
// over the warp, and clears them.
template <int NB>
__device__ __forceinline__ void flush_rows(float (&rh)[NB][16], float (&rl)[NB][16], double* prow_slot, int warp,
                                           int lane) {
#pragma unroll
  for (int b = 0; b < NB; ++b)
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      float h = rh[b][r], l = rl[b][r];
      warp_pair_sum(h, l);
      if (lane == r) prow_slot[b * kSvT + warp * 16 + r] = (double)h + (double)l;
      rh[b][r] = rl[b][r] = 0.f;
    }
}

// One CTA of 8 warps: tiles [blockIdx.x per, + per) of the lower triangle of the n x n
// float-pair matrix A (row stride lda, a multiple of 16; columns n .. lda-1 hold zeros).  Warp
// w streams rows 16 w .. 16 w + 15 of a tile; lane l holds columns 4 l .. 4 l + 3.  xp: the
// right-hand sides as pairs [NB][ldx] (ldx >= T 128, zeros past n).  prow [ctas][span][NB][128]
// and pcol [tiles][NB][128] receive the row and column partials.
template <int NB>
__global__ void __launch_bounds__(256, 2)
symv_lower_pairs_kernel(const float2* __restrict__ A, int64_t lda, int64_t n, const float2* __restrict__ xp,
                        int64_t ldx, double* __restrict__ prow, double* __restrict__ pcol, int64_t per, int64_t total,
                        int span) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t u0 = (int64_t)blockIdx.x * per;
  const int64_t u1 = min(total, u0 + per);
  if (u0 >= u1) return;
  int64_t I, J;
  tri_tile(u0, I, J);
  const int64_t I0 = I;
  __shared__ float2 xs[NB][kSvT];           // x over row block I
  __shared__ float2 red[8][NB][kSvT];       // per-warp column partials of one tile
  float rh[NB][16], rl[NB][16];
#pragma unroll
  for (int b = 0; b < NB; ++b)
#pragma unroll
    for (int r = 0; r < 16; ++r) rh[b][r] = rl[b][r] = 0.f;
  auto load_xs = [&]() {
    for (int e = tid; e < NB * kSvT; e += 256) {
      const int b = e / kSvT, r = e % kSvT;
      xs[b][r] = xp[b * ldx + I * kSvT + r];
    }
  };
  load_xs();
  __syncthreads();
  for (int64_t u = u0; u < u1; ++u) {
    const int64_t c0 = J * kSvT + 4 * lane;
    const bool col_ok = c0 < lda;
    float2 xj[NB][4];
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
      for (int q = 0; q < 4; ++q) xj[b][q] = xp[b * ldx + J * kSvT + 4 * lane + q];
    const bool below = J < I;
    float ch[NB][4], cl[NB][4];
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
      for (int q = 0; q < 4; ++q) ch[b][q] = cl[b][q] = 0.f;
    constexpr int RB = NB == 1 ? 8 : 4;  // rows per batch of loads in flight (register budget)
#pragma unroll
    for (int rr = 0; rr < 16; rr += RB) {
      float4 va[RB][2];
#pragma unroll
      for (int k = 0; k < RB; ++k) {
        const int64_t row = I * kSvT + warp * 16 + rr + k;
        if (row < n && col_ok) {
          const float4* p = reinterpret_cast<const float4*>(A + row * lda + c0);
          va[k][0] = __ldcs(p);
          va[k][1] = __ldcs(p + 1);
        } else {
          va[k][0] = va[k][1] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
#pragma unroll
      for (int k = 0; k < RB; ++k) {
        const float2 a[4] = {make_float2(va[k][0].x, va[k][0].y), make_float2(va[k][0].z, va[k][0].w),
                             make_float2(va[k][1].x, va[k][1].y), make_float2(va[k][1].z, va[k][1].w)};
#pragma unroll
        for (int b = 0; b < NB; ++b) {
#pragma unroll
          for (int q = 0; q < 4; ++q) pr_mac(rh[b][rr + k], rl[b][rr + k], a[q].x, a[q].y, xj[b][q].x, xj[b][q].y);
          if (below) {
            const float2 xi = xs[b][warp * 16 + rr + k];
#pragma unroll
            for (int q = 0; q < 4; ++q) pr_mac(ch[b][q], cl[b][q], a[q].x, a[q].y, xi.x, xi.y);
          }
        }
      }
    }
    if (below) {
      // column partials: the 8 warps' sums in warp order
#pragma unroll
      for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int q = 0; q < 4; ++q) red[warp][b][4 * lane + q] = make_float2(ch[b][q], cl[b][q]);
      __syncthreads();
      for (int e = tid; e < NB * kSvT; e += 256) {
        const int b = e / kSvT, c = e % kSvT;
        float h = red[0][b][c].x, l = red[0][b][c].y;
#pragma unroll
        for (int w = 1; w < 8; ++w) pr_add(h, l, red[w][b][c].x, red[w][b][c].y);
        pcol[(u * NB + b) * kSvT + c] = (double)h + (double)l;
      }
      __syncthreads();
    }
    if (++J > I) {  // panel I complete within this CTA's run: its row partials go out
      flush_rows<NB>(rh, rl, prow + ((int64_t)blockIdx.x * span + (I - I0)) * NB * kSvT, warp, lane);
      ++I;
      J = 0;
      if (u + 1 < u1) {
        __syncthreads();
        load_xs();
        __syncthreads();
      }
    }
  }
  if (J != 0) flush_rows<NB>(rh, rl, prow + ((int64_t)blockIdx.x * span + (I - I0)) * NB * kSvT, warp, lane);
}

// y[b][i] = the row partials of panel I = i / 128 from the CTAs that covered it, in CTA order,
// plus the column partials of tiles (I', I), I' > I, in order of I'.
template <int NB>
__global__ void symv_reduce_kernel(const double* __restrict__ prow, const double* __restrict__ pcol, double* __restrict__ y,
                                   int64_t ldy, int64_t n, int64_t T, int64_t per, int span) {
  const int64_t I = blockIdx.x;
  const int r = threadIdx.x;
  const int64_t i = I * kSvT + r;
  if (i >= n) return;
  const int64_t s0 = I * (I + 1) / 2, s1 = s0 + I + 1;  // the panel's tiles
  for (int b = 0; b < NB; ++b) {
    double sum = 0.0;
    for (int64_t c = s0 / per; c <= (s1 - 1) / per; ++c) {
      int64_t Ic, Jc;
      tri_tile(c * per, Ic, Jc);
      sum += prow[((c * span + (I - Ic)) * NB + b) * kSvT + r];
    }
    for (int64_t Ip = I + 1; Ip < T; ++Ip) sum += pcol[((Ip * (Ip + 1) / 2 + I) * NB + b) * kSvT + r];
    y[b * ldy + i] = sum;
  }
}

// One warp per row of the rows x cols float-pair matrix A (row stride lda, a multiple of 4):
// y[b][row] = sum_j A[row][j] x[b][j], x as pairs [NB][ldx].  Each lane streams 4 pairs (32 B)
// per step, four steps in flight.
template <int NB>
__global__ void __launch_bounds__(256)
gemv_pairs_kernel(const float2* __restrict__ A, int64_t lda, int64_t rows, int64_t cols,
                  const float2* __restrict__ xp, int64_t ldx, double* __restrict__ y, int64_t ldy) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * 8 + warp;
  if (row >= rows) return;
  const float2* a = A + row * lda;
  float sh[NB], sl[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) sh[b] = sl[b] = 0.f;
  constexpr int kU = 4;
  for (int64_t j0 = 0; j0 < cols; j0 += 128 * kU) {
    float4 va[kU][2];
#pragma unroll
    for (int k = 0; k < kU; ++k) {
      const int64_t j = j0 + 128 * k + 4 * lane;
      if (j < cols) {
        const float4* p = reinterpret_cast<const float4*>(a + j);
        va[k][0] = __ldcs(p);
        va[k][1] = (j + 2 < cols) ? __ldcs(p + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
      } else {
        va[k][0] = va[k][1] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
#pragma unroll
    for (int k = 0; k < kU; ++k) {
      const int64_t j = j0 + 128 * k + 4 * lane;
      if (j >= cols) continue;
      const float2 av[4] = {make_float2(va[k][0].x, va[k][0].y), make_float2(va[k][0].z, va[k][0].w),
                            make_float2(va[k][1].x, va[k][1].y), make_float2(va[k][1].z, va[k][1].w)};
#pragma unroll
      for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (j + q < cols) {
            const float2 xv = xp[b * ldx + j + q];
            pr_mac(sh[b], sl[b], av[q].x, av[q].y, xv.x, xv.y);
          }
    }
  }
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    float h = sh[b], l = sl[b];
    warp_pair_sum(h, l);
    if (lane == 0) y[b * ldy + row] = (double)h + (double)l;
  }
}

struct SymvPlan {
  int64_t T, total, per, ctas;
  int span;
};
SymvPlan symv_plan(int64_t n) {
  SymvPlan p;
  p.T = (n + kSvT - 1) / kSvT;
  p.total = p.T * (p.T + 1) / 2;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t slots = 2 * (int64_t)(sms > 0 ? sms : 1);
  p.per = (p.total + slots - 1) / slots;
  p.ctas = (p.total + p.per - 1) / p.per;
  p.span = 1;
  for (int64_t c = 0; c < p.ctas; ++c) {
    int64_t I0, J0, I1, J1;
    tri_tile(c * p.per, I0, J0);
    tri_tile(std::min(p.total, (c + 1) * p.per) - 1, I1, J1);
    p.span = std::max(p.span, (int)(I1 - I0 + 1));
  }
  return p;
}

}  // namespace

int64_t symv_pairs_ldx(int64_t n) { return (n + kSvT - 1) / kSvT * kSvT; }

size_t symv_pairs_work_elems(int64_t n, int64_t B) {
  if (n <= 0 || B != 1) return 0;
  const SymvPlan p = symv_plan(n);
  // x pairs (one float2 per double of space), row partials, column partials
  return (size_t)B * symv_pairs_ldx(n) + (size_t)p.ctas * p.span * B * kSvT + (size_t)p.total * B * kSvT;
}

int64_t symv_lower_pairs(const float2* A, int64_t lda, int64_t n, const double* D, int64_t B, double* X,
                         double* work, cudaStream_t s) {
  if (B != 1) return 0;
  const SymvPlan p = symv_plan(n);
  const int64_t ldx = symv_pairs_ldx(n);
  float2* xp = reinterpret_cast<float2*>(work);
  double* prow = work + (size_t)ldx;
  double* pcol = prow + (size_t)p.ctas * p.span * kSvT;
  int64_t launches = split_rows_to_pairs_ld(D, n, xp, 1, n, ldx, s);
  symv_lower_pairs_kernel<1><<<(unsigned)p.ctas, 256, 0, s>>>(A, lda, n, xp, ldx, prow, pcol, p.per, p.total, p.span);
  symv_reduce_kernel<1><<<(unsigned)p.T, kSvT, 0, s>>>(prow, pcol, X, n, n, p.T, p.per, p.span);
  return launches + 2;
}

size_t gemv_pairs_work_elems(int64_t cols, int64_t B) { return (size_t)B * ((cols + 3) / 4 * 4); }

int64_t gemv_pairs(const float2* A, int64_t lda, int64_t rows, int64_t cols, const double* D, int64_t B, double* Y,
                   int64_t ldy, double* work, cudaStream_t s) {
  if (B < 1 || B > 2 || rows <= 0) return 0;
  const int64_t ldx = (cols + 3) / 4 * 4;
  float2* xp = reinterpret_cast<float2*>(work);
  int64_t launches = split_rows_to_pairs_ld(D, cols, xp, B, cols, ldx, s);
  const unsigned grid = (unsigned)((rows + 7) / 8);
  if (B == 1)
    gemv_pairs_kernel<1><<<grid, 256, 0, s>>>(A, lda, rows, cols, xp, ldx, Y, ldy);
  else
    gemv_pairs_kernel<2><<<grid, 256, 0, s>>>(A, lda, rows, cols, xp, ldx, Y, ldy);
  return launches + 1;
}

}  // namespace bti
