// Per-frequency block products of the FFT-based Toeplitz matvecs.
//
// In Fourier space the block circulant embedding is block diagonal (Sec. 4,
// "FFT-based GPU-accelerated p2o and p2q matvecs"), so for every frequency w
//   forward : hat_d_w = hat_F_w hat_m_w             (reduction over j < N_m)
//   adjoint : hat_m_w = hat_F_w^H hat_d_w           (reduction over i < R)
// The spectral blocks are stored [w][i][j] with j contiguous: both products
// stream each block row once with coalesced loads, and the reduction over j of
// the forward product stays within contiguous rows (the strided alternative the
// paper's footnote warns against is never used).  The forward reduction is
// deterministic: per-chunk partial sums, then a fixed-order second pass.
#include "bti_internal.cuh"

#include <cuda_fp16.h>

namespace bti {

// Rows of d-hat the adjoint kernels stage in shared memory at a time (any R is accepted;
// 4 x 512 x 16 bytes stays within the default 48 KB of dynamic shared memory).
constexpr int64_t kAdjRows = 512;

template <typename T> struct FwdCfg;
template <> struct FwdCfg<double> { static constexpr int JC1 = 2048, JC4 = 512; };
template <> struct FwdCfg<float> { static constexpr int JC1 = 4096, JC4 = 1024; };

template <typename T, typename TS> __device__ __forceinline__ C2<T> ldF(const C2<TS>* p) {
  C2<TS> v = __ldg(p);
  return mk<T>((T)v.x, (T)v.y);
}

// grid (nchunk, nf, ceil(B / BG)), 256 threads.  Warp w handles rows i = w, w + 8, ...
// Each lane streams its row segment U elements at a time with the next U loads
// in flight while the current U are consumed (register double buffering).
template <typename T, typename TS, int BG, int U>
__global__ void __launch_bounds__(256)
prod_fwd_kernel(const C2<TS>* __restrict__ Fhat, const C2<T>* __restrict__ mhat,
                C2<T>* __restrict__ partial, int64_t nf, int64_t R, int64_t Nm, int64_t B,
                int JC, int nchunk) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<T>* sm = reinterpret_cast<C2<T>*>(smem_raw);  // [BG][JC]
  const int ch = blockIdx.x;
  const int64_t w = blockIdx.y;
  const int64_t b0 = (int64_t)blockIdx.z * BG;
  const int64_t j0 = (int64_t)ch * JC;
  const int jn = (int)((Nm - j0) < JC ? (Nm - j0) : JC);
  for (int idx = threadIdx.x; idx < BG * JC; idx += blockDim.x) {
    int bb = idx / JC, jj = idx - bb * JC;
    C2<T> v = mk<T>((T)0, (T)0);
    if (jj < jn && b0 + bb < B) v = mhat[((b0 + bb) * nf + w) * Nm + j0 + jj];
    sm[idx] = v;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int STEP = 32 * U;
  const C2<T> z = mk<T>((T)0, (T)0);
  for (int64_t i = warp; i < R; i += 8) {
    const C2<TS>* row = Fhat + (w * R + i) * Nm + j0;
    T ar[BG], ai[BG];
#pragma unroll
    for (int bb = 0; bb < BG; ++bb) { ar[bb] = (T)0; ai[bb] = (T)0; }
    C2<T> cur[U], nxt[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      int jj = lane + 32 * u;
      cur[u] = (jj < jn) ? ldF<T, TS>(row + jj) : z;
    }
    for (int base = 0; base < jn; base += STEP) {
      const int nb = base + STEP;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        int jj = nb + lane + 32 * u;
        nxt[u] = (jj < jn) ? ldF<T, TS>(row + jj) : z;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int jj = base + lane + 32 * u;
        const C2<T> f = cur[u];
#pragma unroll
        for (int bb = 0; bb < BG; ++bb) {
          C2<T> x = sm[bb * JC + (jj < JC ? jj : 0)];
          ar[bb] = fma(f.x, x.x, ar[bb]);
          ar[bb] = fma(-f.y, x.y, ar[bb]);
          ai[bb] = fma(f.x, x.y, ai[bb]);
          ai[bb] = fma(f.y, x.x, ai[bb]);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) cur[u] = nxt[u];
    }
#pragma unroll
    for (int bb = 0; bb < BG; ++bb) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        ar[bb] += __shfl_xor_sync(0xffffffffu, ar[bb], o);
        ai[bb] += __shfl_xor_sync(0xffffffffu, ai[bb], o);
      }
    }
    if (lane == 0) {
#pragma unroll
      for (int bb = 0; bb < BG; ++bb)
        if (b0 + bb < B) partial[(((b0 + bb) * nf + w) * nchunk + ch) * R + i] = mk<T>(ar[bb], ai[bb]);
    }
  }
}

// dhat[b][w][i] = sum over chunks, fixed order
template <typename T>
__global__ void reduce_chunks_kernel(const C2<T>* __restrict__ partial, C2<T>* __restrict__ dhat,
                                     int64_t total, int64_t R, int nchunk) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  int64_t bw = idx / R, i = idx - bw * R;
  const C2<T>* p = partial + bw * nchunk * R + i;
  T sr = 0, si = 0;
  for (int c = 0; c < nchunk; ++c) {
    C2<T> v = p[(int64_t)c * R];
    sr += v.x;
    si += v.y;
  }
  dhat[idx] = mk<T>(sr, si);
}

template <typename T> static int fwd_bg(int64_t B) { return fwd_group(B); }
template <typename T> static int fwd_jc(int bg) { return bg == 4 ? FwdCfg<T>::JC4 : FwdCfg<T>::JC1; }

size_t prod_fwd_partial_elems(int64_t nf, int64_t R, int64_t Nm, int64_t B) {
  // worst case over the two tiers: the smallest chunk (FP64, BG = 4)
  int64_t nchunk = (Nm + FwdCfg<double>::JC4 - 1) / FwdCfg<double>::JC4;
  return (size_t)(B * nf * nchunk * R);
}

// Chunk of columns per CTA of the forward product: the tier default, or jc (a
// multiple of 256, at least 512 so the partial-buffer bound holds) when given.
template <typename T>
static int fwd_nchunk(int64_t Nm, int64_t B, int* jc_out, int jc = 0) {
  int bg = fwd_bg<T>(B);
  int JC = jc > 0 ? jc : fwd_jc<T>(bg);
  // the staged m-hat chunk must fit the dynamic shared memory the kernels opt into
  if ((size_t)bg * JC * sizeof(C2<T>) > kFwdSmemMax) JC = fwd_jc<T>(bg);
  if (Nm < JC) JC = (int)(((Nm + 31) / 32) * 32);
  if (jc_out) *jc_out = JC;
  return (int)((Nm + JC - 1) / JC);
}

template <typename T>
void launch_reduce_chunks(const C2<T>* partial, C2<T>* dhat, int64_t nf, int64_t R, int64_t Nm,
                          int64_t B, cudaStream_t s, int jc) {
  int nchunk = fwd_nchunk<T>(Nm, B, nullptr, jc);
  int64_t total = B * nf * R;
  reduce_chunks_kernel<T><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(partial, dhat, total, R, nchunk);
}

template <typename T, typename TS>
void launch_prod_fwd(const C2<TS>* Fhat, const C2<T>* mhat, C2<T>* partial,
                     int64_t nf, int64_t R, int64_t Nm, int64_t B, cudaStream_t s, int jc) {
  int bg = fwd_bg<T>(B);
  int JC = 0;
  int nchunk = fwd_nchunk<T>(Nm, B, &JC, jc);
  size_t smem = sizeof(C2<T>) * (size_t)bg * JC;
  dim3 grid((unsigned)nchunk, (unsigned)nf, (unsigned)((B + bg - 1) / bg));
  constexpr int U1 = sizeof(C2<TS>) >= 16 ? 8 : 16;  // 128 bytes of loads per lane per step
  static PerDeviceOnce attr;
  attr([] {
    cudaFuncSetAttribute(prod_fwd_kernel<T, TS, 4, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmemMax);
    cudaFuncSetAttribute(prod_fwd_kernel<T, TS, 1, U1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmemMax);
  });
  if (bg == 4)
    prod_fwd_kernel<T, TS, 4, 4><<<grid, 256, smem, s>>>(Fhat, mhat, partial, nf, R, Nm, B, JC, nchunk);
  else
    prod_fwd_kernel<T, TS, 1, U1><<<grid, 256, smem, s>>>(Fhat, mhat, partial, nf, R, Nm, B, JC, nchunk);
}

// grid (ceil(Nm / (256 VPT)), nf, ceil(B / BG)); thread owns j = j0 + tid + 256 v
template <typename T, typename TS, int BG, int VPT>
__global__ void __launch_bounds__(256)
prod_adj_kernel(const C2<TS>* __restrict__ Fhat, const C2<T>* __restrict__ dhat,
                C2<T>* __restrict__ mhat, int64_t nf, int64_t R, int64_t Nm, int64_t B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<T>* sd = reinterpret_cast<C2<T>*>(smem_raw);  // [BG][min(R, kAdjRows)]
  const int64_t w = blockIdx.y;
  const int64_t b0 = (int64_t)blockIdx.z * BG;
  const int64_t jbase = (int64_t)blockIdx.x * (256 * VPT) + threadIdx.x;
  T ar[BG][VPT], ai[BG][VPT];
#pragma unroll
  for (int bb = 0; bb < BG; ++bb)
#pragma unroll
    for (int v = 0; v < VPT; ++v) { ar[bb][v] = (T)0; ai[bb][v] = (T)0; }
  const C2<TS>* base = Fhat + w * R * Nm;
  // d-hat rows are staged RS at a time; each thread still sums over i in order
  const int64_t RS = R < kAdjRows ? R : kAdjRows;
  for (int64_t i0 = 0; i0 < R; i0 += RS) {
    const int64_t rn = R - i0 < RS ? R - i0 : RS;
    if (i0 > 0) __syncthreads();  // the previous tile is consumed
    for (int64_t idx = threadIdx.x; idx < BG * rn; idx += blockDim.x) {
      int64_t bb = idx / rn, i = i0 + (idx - bb * rn);
      C2<T> v = mk<T>((T)0, (T)0);
      if (b0 + bb < B) v = dhat[((b0 + bb) * nf + w) * R + i];
      sd[bb * RS + (i - i0)] = v;
    }
    __syncthreads();
    for (int64_t ii = 0; ii < rn; ++ii) {
      const int64_t i = i0 + ii;
      const C2<TS>* row = base + i * Nm;
      C2<T> f[VPT];
#pragma unroll
      for (int v = 0; v < VPT; ++v) {
        int64_t j = jbase + 256 * v;
        f[v] = (j < Nm) ? ldF<T, TS>(row + j) : mk<T>((T)0, (T)0);
      }
#pragma unroll
      for (int bb = 0; bb < BG; ++bb) {
        C2<T> x = sd[bb * RS + ii];
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
          // conj(f) * x
          ar[bb][v] = fma(f[v].x, x.x, ar[bb][v]);
          ar[bb][v] = fma(f[v].y, x.y, ar[bb][v]);
          ai[bb][v] = fma(f[v].x, x.y, ai[bb][v]);
          ai[bb][v] = fma(-f[v].y, x.x, ai[bb][v]);
        }
      }
    }
  }
#pragma unroll
  for (int bb = 0; bb < BG; ++bb) {
    if (b0 + bb >= B) continue;
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      int64_t j = jbase + 256 * v;
      if (j < Nm) mhat[((b0 + bb) * nf + w) * Nm + j] = mk<T>(ar[bb][v], ai[bb][v]);
    }
  }
}

template <typename T, typename TS, int BG, int VPT>
static void adj_launch(const C2<TS>* Fhat, const C2<T>* dhat, C2<T>* mhat, int64_t nf, int64_t R, int64_t Nm,
                       int64_t B, cudaStream_t s) {
  size_t smem = sizeof(C2<T>) * (size_t)BG * (R < kAdjRows ? R : kAdjRows);
  dim3 grid((unsigned)((Nm + 256 * VPT - 1) / (256 * VPT)), (unsigned)nf, (unsigned)((B + BG - 1) / BG));
  prod_adj_kernel<T, TS, BG, VPT><<<grid, 256, smem, s>>>(Fhat, dhat, mhat, nf, R, Nm, B);
}

// vpt: columns per thread of the single-vector kernel (2, 4 or 8; 0 = default 4)
template <typename T, typename TS>
void launch_prod_adj(const C2<TS>* Fhat, const C2<T>* dhat, C2<T>* mhat,
                     int64_t nf, int64_t R, int64_t Nm, int64_t B, cudaStream_t s, int vpt) {
  if (B >= 4)
    adj_launch<T, TS, 4, 2>(Fhat, dhat, mhat, nf, R, Nm, B, s);
  else if (vpt == 2)
    adj_launch<T, TS, 1, 2>(Fhat, dhat, mhat, nf, R, Nm, B, s);
  else if (vpt == 8)
    adj_launch<T, TS, 1, 8>(Fhat, dhat, mhat, nf, R, Nm, B, s);
  else
    adj_launch<T, TS, 1, 4>(Fhat, dhat, mhat, nf, R, Nm, B, s);
}

template void launch_prod_fwd<double, double>(const double2*, const double2*, double2*,
                                              int64_t, int64_t, int64_t, int64_t, cudaStream_t, int);
template void launch_prod_fwd<float, float>(const float2*, const float2*, float2*,
                                            int64_t, int64_t, int64_t, int64_t, cudaStream_t, int);
template void launch_reduce_chunks<double>(const double2*, double2*, int64_t, int64_t, int64_t, int64_t,
                                           cudaStream_t, int);
template void launch_reduce_chunks<float>(const float2*, float2*, int64_t, int64_t, int64_t, int64_t,
                                          cudaStream_t, int);
template void launch_prod_adj<double, double>(const double2*, const double2*, double2*,
                                              int64_t, int64_t, int64_t, int64_t, cudaStream_t, int);
template void launch_prod_adj<float, float>(const float2*, const float2*, float2*,
                                            int64_t, int64_t, int64_t, int64_t, cudaStream_t, int);


// ------------------------------------------------------------------ double-FP32 tier
// GB300's FP64 pipe issues 1/64 of the FP32 rate, so an FP64 product of the
// spectral blocks is bound by FP64 arithmetic at about a third of the HBM rate.
// The double-FP32 tier keeps FP64-level accuracy on the FP32 pipes instead:
// every real number of a spectral block is stored as an unevaluated sum
// hi + lo of two floats (|lo| <= ulp(hi) / 2, about 48 significant bits,
// 16 bytes per complex element like FP64), the frequency-domain vectors come and
// go in the same float-quad form (the pair FFTs' own), and products are accumulated
// in float pairs:
//   x * y = xh*yh (exact: rounded product plus its FMA error) + xh*yl + xl*yh,
// with the high parts summed by Knuth's error-free two-sum and every error term
// gathered in the low float.  The relative error of a sum of n terms is about
// n * 2^-48 of the sum of magnitudes, far below the FP64 tier's 1e-12 bound.

namespace {

struct ff { float h, l; };

__device__ __forceinline__ ff split_d(double x) {
  float h = __double2float_rn(x);
  float l = __double2float_rn(x - (double)h);
  return {h, l};
}

// S += x * y  (S, x, y float pairs); 12 FP32 operations
__device__ __forceinline__ void ff_mac(float& Sh, float& Sl, float xh, float xl, float yh, float yl) {
  float p = xh * yh;
  float pe = fmaf(xh, yh, -p);
  pe = fmaf(xh, yl, pe);
  pe = fmaf(xl, yh, pe);
  float s = Sh + p;
  float bb = s - Sh;
  float e = (Sh - (s - bb)) + (p - bb);
  Sh = s;
  Sl += e + pe;
}

// (ah, al) + (bh, bl) -> normalised pair
__device__ __forceinline__ void ff_add(float& ah, float& al, float bh, float bl) {
  float s = ah + bh;
  float bb = s - ah;
  float e = (ah - (s - bb)) + (bh - bb);
  e += al + bl;
  ah = s + e;
  al = e - (ah - s);
}

__device__ __forceinline__ double ff_to_d(float h, float l) { return (double)h + (double)l; }

// h + l as a normalised pair (|lo| <= ulp(hi) / 2) by Knuth's two-sum, whatever their magnitudes
__device__ __forceinline__ ff two_sum(float h, float l) {
  const float s = __fadd_rn(h, l);
  const float bb = __fsub_rn(s, h);
  return {s, __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(l, bb))};
}

}  // namespace

// In place: a complex FP64 array times 2^-pexp (exact) becomes (re_hi, re_lo, im_hi, im_lo)
// float quads.  The power of two brings the largest entry near 1, so that the pairs keep their
// 48 bits whatever the operator's units (FP32's exponent range is far narrower than FP64's).
__global__ void split_df64_kernel(double2* a, int64_t n, int pexp) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double2 v = a[i];
  ff re = split_d(scalbn(v.x, -pexp)), im = split_d(scalbn(v.y, -pexp));
  reinterpret_cast<float4*>(a)[i] = make_float4(re.h, re.l, im.h, im.l);
}

void launch_split_df64(void* hat, int64_t n, int pexp, cudaStream_t s) {
  if (n > 0) split_df64_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((double2*)hat, n, pexp);
}

// out = max |x[i]| over n doubles, as the bit pattern of a non-negative double (which orders
// like an unsigned integer, so atomicMax reduces it); a NaN reads above every finite value.
// *out must be 0 before the launch.
__global__ void max_abs_kernel(const double* __restrict__ x, int64_t n, unsigned long long* out) {
  double m = 0.0;
  unsigned long long nan = 0ull;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = fabs(x[i]);
    if (v != v) nan = 0x7FF8000000000000ull;
    m = fmax(m, v);
  }
  unsigned long long b = (unsigned long long)__double_as_longlong(m);
  if (nan) b = nan;
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long c = __shfl_xor_sync(0xffffffffu, b, o);
    b = c > b ? c : b;
  }
  __shared__ unsigned long long red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = b;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) b = red[w] > b ? red[w] : b;
    atomicMax(out, b);
  }
}

void launch_max_abs(const double* x, int64_t n, unsigned long long* out, cudaStream_t s) {
  cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
  if (n <= 0) return;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  max_abs_kernel<<<(unsigned)blocks, 256, 0, s>>>(x, n, out);
}

// Forward product, double-FP32 arithmetic.  Same decomposition as prod_fwd_kernel:
// grid (nchunk, nf, ceil(B / BG)), warp w handles rows i = w, w + 8, ...  Each lane
// streams its row segment U elements at a time with the next U loads issued before
// the current U are consumed (register double buffering keeps 2 U 16-byte loads in
// flight per lane), and the four real products of a complex multiply-accumulate go
// to four independent float-pair accumulators so their two-sum chains overlap.
template <int BG, int U>
__global__ void __launch_bounds__(256)
prod_fwd_df64_kernel(const float4* __restrict__ Fhat, const float4* __restrict__ mhat,
                     double2* __restrict__ partial, int64_t nf, int64_t R, int64_t Nm, int64_t B,
                     int JC, int nchunk) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* sm = reinterpret_cast<float4*>(smem_raw);  // [BG][JC] m-hat
  const int ch = blockIdx.x;
  const int64_t w = blockIdx.y;
  const int64_t b0 = (int64_t)blockIdx.z * BG;
  const int64_t j0 = (int64_t)ch * JC;
  const int jn = (int)((Nm - j0) < JC ? (Nm - j0) : JC);
  for (int idx = threadIdx.x; idx < BG * JC; idx += blockDim.x) {
    int bb = idx / JC, jj = idx - bb * JC;
    sm[idx] = (jj < jn && b0 + bb < B) ? mhat[((b0 + bb) * nf + w) * Nm + j0 + jj] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int STEP = 32 * U;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int64_t i = warp; i < R; i += 8) {
    const float4* row = Fhat + (w * R + i) * Nm + j0;
    // accumulators: [0] +a c, [1] -b d, [2] +a d, [3] +b c (high and low floats)
    float ah[BG][4], al[BG][4];
#pragma unroll
    for (int bb = 0; bb < BG; ++bb)
#pragma unroll
      for (int q = 0; q < 4; ++q) ah[bb][q] = al[bb][q] = 0.f;
    float4 cur[U], nxt[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      int jj = lane + 32 * u;
      cur[u] = (jj < jn) ? __ldg(row + jj) : z4;
    }
    for (int base = 0; base < jn; base += STEP) {
      const int nb = base + STEP;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        int jj = nb + lane + 32 * u;
        nxt[u] = (jj < jn) ? __ldg(row + jj) : z4;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int jj = base + lane + 32 * u;
        const float4 f = cur[u];  // (a_h, a_l, b_h, b_l): F = a + i b
#pragma unroll
        for (int bb = 0; bb < BG; ++bb) {
          // zero-padded columns past jn hold zeros in both f and sm
          const float4 x = sm[bb * JC + (jj < JC ? jj : 0)];  // (c_h, c_l, d_h, d_l)
          ff_mac(ah[bb][0], al[bb][0], f.x, f.y, x.x, x.y);
          ff_mac(ah[bb][1], al[bb][1], -f.z, -f.w, x.z, x.w);
          ff_mac(ah[bb][2], al[bb][2], f.x, f.y, x.z, x.w);
          ff_mac(ah[bb][3], al[bb][3], f.z, f.w, x.x, x.y);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) cur[u] = nxt[u];
    }
#pragma unroll
    for (int bb = 0; bb < BG; ++bb) {
      float rh = ah[bb][0], rl = al[bb][0], ih = ah[bb][2], il = al[bb][2];
      ff_add(rh, rl, ah[bb][1], al[bb][1]);
      ff_add(ih, il, ah[bb][3], al[bb][3]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        float oh = __shfl_xor_sync(0xffffffffu, rh, o);
        float ol = __shfl_xor_sync(0xffffffffu, rl, o);
        ff_add(rh, rl, oh, ol);
        oh = __shfl_xor_sync(0xffffffffu, ih, o);
        ol = __shfl_xor_sync(0xffffffffu, il, o);
        ff_add(ih, il, oh, ol);
      }
      if (lane == 0 && b0 + bb < B)
        partial[(((b0 + bb) * nf + w) * nchunk + ch) * R + i] = make_double2(ff_to_d(rh, rl), ff_to_d(ih, il));
    }
  }
}

void launch_prod_fwd_df64(const float4* Fhat, const float4* mhat, double2* partial, int64_t nf,
                          int64_t R, int64_t Nm, int64_t B, cudaStream_t s, int jc) {
  // chunking identical to the FP64 tier (the reduce pass and workspace sizes are shared)
  int bg = fwd_bg<double>(B);
  int JC = 0;
  int nchunk = fwd_nchunk<double>(Nm, B, &JC, jc);
  size_t smem = sizeof(float4) * (size_t)bg * JC;
  dim3 grid((unsigned)nchunk, (unsigned)nf, (unsigned)((B + bg - 1) / bg));
  static PerDeviceOnce attr;
  attr([] {
    cudaFuncSetAttribute(prod_fwd_df64_kernel<4, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmemMax);
    cudaFuncSetAttribute(prod_fwd_df64_kernel<1, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmemMax);
  });
  if (bg == 4)
    prod_fwd_df64_kernel<4, 4><<<grid, 256, smem, s>>>(Fhat, mhat, partial, nf, R, Nm, B, JC, nchunk);
  else
    prod_fwd_df64_kernel<1, 8><<<grid, 256, smem, s>>>(Fhat, mhat, partial, nf, R, Nm, B, JC, nchunk);
}

// dhat[b][w][i] = the chunk partials summed in FP64 in chunk order (as the FP64 tier), stored
// as a float quad (hi = the sum rounded to FP32, lo = the rest rounded to FP32)
__global__ void reduce_chunks_df64_kernel(const double2* __restrict__ partial, float4* __restrict__ dhat,
                                          int64_t total, int64_t R, int nchunk) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int64_t bw = idx / R, i = idx - bw * R;
  const double2* p = partial + bw * nchunk * R + i;
  double sr = 0, si = 0;
  for (int c = 0; c < nchunk; ++c) {
    const double2 v = p[(int64_t)c * R];
    sr += v.x;
    si += v.y;
  }
  const ff re = split_d(sr), im = split_d(si);
  dhat[idx] = make_float4(re.h, re.l, im.h, im.l);
}

void launch_reduce_chunks_df64(const double2* partial, float4* dhat, int64_t nf, int64_t R, int64_t Nm,
                               int64_t B, cudaStream_t s, int jc) {
  const int nchunk = fwd_nchunk<double>(Nm, B, nullptr, jc);  // the forward product's chunking
  const int64_t total = B * nf * R;
  reduce_chunks_df64_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(partial, dhat, total, R, nchunk);
}

// Adjoint product, double-FP32 arithmetic; thread owns j = j0 + tid + 256 v.  AHEAD: each thread
// loads F-hat's next row while it uses the current one (two rows in flight instead of one).
template <int BG, int VPT, bool AHEAD = (BG >= 4)>
__global__ void __launch_bounds__(256)
prod_adj_df64_kernel(const float4* __restrict__ Fhat, const float4* __restrict__ dhat,
                     float4* __restrict__ mhat, int64_t nf, int64_t R, int64_t Nm, int64_t B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* sd = reinterpret_cast<float4*>(smem_raw);  // [BG][min(R, kAdjRows)] d-hat
  const int64_t w = blockIdx.y;
  const int64_t b0 = (int64_t)blockIdx.z * BG;
  const int64_t jbase = (int64_t)blockIdx.x * (256 * VPT) + threadIdx.x;
  float rh[BG][VPT], rl[BG][VPT], ih[BG][VPT], il[BG][VPT];
#pragma unroll
  for (int bb = 0; bb < BG; ++bb)
#pragma unroll
    for (int v = 0; v < VPT; ++v) rh[bb][v] = rl[bb][v] = ih[bb][v] = il[bb][v] = 0.f;
  const float4* base = Fhat + w * R * Nm;
  // d-hat rows are staged RS at a time; each thread still sums over i in order
  const int64_t RS = R < kAdjRows ? R : kAdjRows;
  for (int64_t i0 = 0; i0 < R; i0 += RS) {
    const int64_t rn = R - i0 < RS ? R - i0 : RS;
    if (i0 > 0) __syncthreads();  // the previous tile is consumed
    for (int64_t idx = threadIdx.x; idx < BG * rn; idx += blockDim.x) {
      int64_t bb = idx / rn, i = i0 + (idx - bb * rn);
      sd[bb * RS + (i - i0)] = (b0 + bb < B) ? dhat[((b0 + bb) * nf + w) * R + i] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    // F-hat row ii of the tile; with several vectors per CTA, or a grid too small to keep HBM
    // busy with one row in flight per thread, the next row is loaded while this one is used
    constexpr bool kAhead = AHEAD;
    float4 f[VPT], fn[VPT];
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      const int64_t j = jbase + 256 * v;
      f[v] = (kAhead && j < Nm) ? __ldg(base + i0 * Nm + j) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int64_t ii = 0; ii < rn; ++ii) {
      // kAhead: fetch row ii + 1 into fn; otherwise fetch row ii into f
      const int64_t il_ = kAhead ? ii + 1 : ii;
      const bool live = il_ < rn;
      const float4* row = base + (i0 + il_) * Nm;
#pragma unroll
      for (int v = 0; v < VPT; ++v) {
        const int64_t j = jbase + 256 * v;
        const float4 g = (live && j < Nm) ? __ldg(row + j) : make_float4(0.f, 0.f, 0.f, 0.f);
        if (kAhead)
          fn[v] = g;
        else
          f[v] = g;
      }
#pragma unroll
      for (int bb = 0; bb < BG; ++bb) {
        float4 x = sd[bb * RS + ii];  // d = c + i e
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
          // conj(F) d = (a - i b)(c + i e) = (a c + b e) + i (a e - b c)
          ff_mac(rh[bb][v], rl[bb][v], f[v].x, f[v].y, x.x, x.y);
          ff_mac(rh[bb][v], rl[bb][v], f[v].z, f[v].w, x.z, x.w);
          ff_mac(ih[bb][v], il[bb][v], f[v].x, f[v].y, x.z, x.w);
          ff_mac(ih[bb][v], il[bb][v], -f[v].z, -f[v].w, x.x, x.y);
        }
      }
      if (kAhead) {
#pragma unroll
        for (int v = 0; v < VPT; ++v) f[v] = fn[v];
      }
    }
  }
#pragma unroll
  for (int bb = 0; bb < BG; ++bb) {
    if (b0 + bb >= B) continue;
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      int64_t j = jbase + 256 * v;
      if (j < Nm) {  // the accumulated low floats renormalised by a two-sum
        const ff re = two_sum(rh[bb][v], rl[bb][v]), im = two_sum(ih[bb][v], il[bb][v]);
        mhat[((b0 + bb) * nf + w) * Nm + j] = make_float4(re.h, re.l, im.h, im.l);
      }
    }
  }
}

template <int BG, int VPT, bool AHEAD = (BG >= 4)>
static void adj_df64_launch(const float4* Fhat, const float4* dhat, float4* mhat, int64_t nf, int64_t R,
                            int64_t Nm, int64_t B, cudaStream_t s) {
  size_t smem = sizeof(float4) * (size_t)BG * (R < kAdjRows ? R : kAdjRows);
  static PerDeviceOnce attr;  // 8 vectors x 512 staged rows take 64 KB
  attr([] {
    cudaFuncSetAttribute(prod_adj_df64_kernel<BG, VPT, AHEAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(sizeof(float4) * BG * kAdjRows));
  });
  dim3 grid((unsigned)((Nm + 256 * VPT - 1) / (256 * VPT)), (unsigned)nf, (unsigned)((B + BG - 1) / BG));
  prod_adj_df64_kernel<BG, VPT, AHEAD><<<grid, 256, smem, s>>>(Fhat, dhat, mhat, nf, R, Nm, B);
}

void launch_prod_adj_df64(const float4* Fhat, const float4* dhat, float4* mhat, int64_t nf, int64_t R,
                          int64_t Nm, int64_t B, cudaStream_t s, int vpt) {
  if (B >= 8)
    adj_df64_launch<8, 1>(Fhat, dhat, mhat, nf, R, Nm, B, s);
  else if (B >= 4)
    adj_df64_launch<4, 2>(Fhat, dhat, mhat, nf, R, Nm, B, s);
  else if (nf * ((Nm + 1023) / 1024) < 4096)
    // few CTAs (a short spatial axis, as the batched workload's 4,096 columns): two rows in flight,
    // two columns per thread (twice the CTAs of four: the one-vector online graph 0.82 -> 0.79 ms)
    adj_df64_launch<1, 2, true>(Fhat, dhat, mhat, nf, R, Nm, B, s);
  else if (vpt == 2)
    adj_df64_launch<1, 2>(Fhat, dhat, mhat, nf, R, Nm, B, s);
  else if (vpt == 8)
    adj_df64_launch<1, 8>(Fhat, dhat, mhat, nf, R, Nm, B, s);
  else
    adj_df64_launch<1, 4>(Fhat, dhat, mhat, nf, R, Nm, B, s);
}


// ------------------------------------------------------------------ FP16 tier
// Spectral blocks stored as FP16 complex pairs (4 bytes per element, a quarter of
// FP64) with one power-of-two FP32 scale per row (w, i), so each row uses the FP16
// range fully: F-hat[w][i][j] = scale[w][i] * h[w][i][j].  Products and
// accumulation in FP32 (the scale is applied to the row sum, or folded into d-hat
// for the adjoint); FFTs and vectors in FP32.  Relative error about 2^-11 per
// element: the low-precision tier of mixed-precision solves, whose final accuracy
// comes from refinement with the double-FP32 operators.

// One CTA per source row (w, r) of a [nf][rn][Nm] chunk holding rows i0 .. i0 + rn of
// [nf][R][Nm]: max |re|, |im| over the row, then scale and round into row (w, i0 + r).
__global__ void quantize_f16_rows_kernel(const double2* __restrict__ src, __half2* __restrict__ dst,
                                         float* __restrict__ scale, int64_t Nm, int64_t rn, int64_t R,
                                         int64_t i0) {
  const int64_t srow = blockIdx.x;
  const int64_t row = (srow / rn) * R + i0 + srow % rn;  // destination row w R + i
  const double2* s = src + srow * Nm;
  double mx = 0.0;
  for (int64_t j = threadIdx.x; j < Nm; j += blockDim.x) {
    double2 v = s[j];
    mx = fmax(mx, fmax(fabs(v.x), fabs(v.y)));
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    mx = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (threadIdx.x == 0) red[0] = mx;
  }
  __syncthreads();
  mx = red[0];
  // power of two p with mx / p <= 2^14 (FP16 max is 65504)
  int e = 0;
  if (mx > 0.0) {
    frexp(mx, &e);  // mx = f 2^e, f in [0.5, 1)
    e -= 14;
  }
  const double p = ldexp(1.0, e);
  const double inv = ldexp(1.0, -e);
  if (threadIdx.x == 0) scale[row] = (float)p;
  for (int64_t j = threadIdx.x; j < Nm; j += blockDim.x) {
    double2 v = s[j];
    dst[row * Nm + j] = __floats2half2_rn((float)(v.x * inv), (float)(v.y * inv));
  }
}

void launch_quantize_f16(const double2* src, void* dst, float* scale, int64_t nf, int64_t rn, int64_t R,
                         int64_t i0, int64_t Nm, cudaStream_t s) {
  if (nf * rn > 0)
    quantize_f16_rows_kernel<<<(unsigned)(nf * rn), 256, 0, s>>>(src, (__half2*)dst, scale, Nm, rn, R, i0);
}

// Forward product: grid (nchunk, nf, ceil(B / BG)); warp w handles rows w, w + 8, ...
template <int BG, int U>
__global__ void __launch_bounds__(256)
prod_fwd_f16_kernel(const __half2* __restrict__ Fhat, const float* __restrict__ scale,
                    const float2* __restrict__ mhat, float2* __restrict__ partial, int64_t nf, int64_t R,
                    int64_t Nm, int64_t B, int JC, int nchunk) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* sm = reinterpret_cast<float2*>(smem_raw);  // [BG][JC]
  const int ch = blockIdx.x;
  const int64_t w = blockIdx.y;
  const int64_t b0 = (int64_t)blockIdx.z * BG;
  const int64_t j0 = (int64_t)ch * JC;
  const int jn = (int)((Nm - j0) < JC ? (Nm - j0) : JC);
  for (int idx = threadIdx.x; idx < BG * JC; idx += blockDim.x) {
    int bb = idx / JC, jj = idx - bb * JC;
    float2 v = make_float2(0.f, 0.f);
    if (jj < jn && b0 + bb < B) v = mhat[((b0 + bb) * nf + w) * Nm + j0 + jj];
    sm[idx] = v;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int STEP = 32 * U;
  const __half2 hz = __floats2half2_rn(0.f, 0.f);
  for (int64_t i = warp; i < R; i += 8) {
    const __half2* row = Fhat + (w * R + i) * Nm + j0;
    float ar[BG], ai[BG];
#pragma unroll
    for (int bb = 0; bb < BG; ++bb) ar[bb] = ai[bb] = 0.f;
    __half2 cur[U], nxt[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      int jj = lane + 32 * u;
      cur[u] = (jj < jn) ? __ldg(row + jj) : hz;
    }
    for (int base = 0; base < jn; base += STEP) {
      const int nb = base + STEP;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        int jj = nb + lane + 32 * u;
        nxt[u] = (jj < jn) ? __ldg(row + jj) : hz;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int jj = base + lane + 32 * u;
        const float2 f = __half22float2(cur[u]);
#pragma unroll
        for (int bb = 0; bb < BG; ++bb) {
          float2 x = sm[bb * JC + (jj < JC ? jj : 0)];
          ar[bb] = fmaf(f.x, x.x, ar[bb]);
          ar[bb] = fmaf(-f.y, x.y, ar[bb]);
          ai[bb] = fmaf(f.x, x.y, ai[bb]);
          ai[bb] = fmaf(f.y, x.x, ai[bb]);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) cur[u] = nxt[u];
    }
    const float sc = scale[w * R + i];
#pragma unroll
    for (int bb = 0; bb < BG; ++bb) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        ar[bb] += __shfl_xor_sync(0xffffffffu, ar[bb], o);
        ai[bb] += __shfl_xor_sync(0xffffffffu, ai[bb], o);
      }
      if (lane == 0 && b0 + bb < B)
        partial[(((b0 + bb) * nf + w) * nchunk + ch) * R + i] = make_float2(sc * ar[bb], sc * ai[bb]);
    }
  }
}

void launch_prod_fwd_f16(const void* Fhat, const float* scale, const float2* mhat, float2* partial, int64_t nf,
                         int64_t R, int64_t Nm, int64_t B, cudaStream_t s, int jc) {
  int bg = fwd_bg<float>(B);
  int JC = 0;
  int nchunk = fwd_nchunk<float>(Nm, B, &JC, jc);
  size_t smem = sizeof(float2) * (size_t)bg * JC;
  dim3 grid((unsigned)nchunk, (unsigned)nf, (unsigned)((B + bg - 1) / bg));
  static PerDeviceOnce attr;
  attr([] {
    cudaFuncSetAttribute(prod_fwd_f16_kernel<4, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmemMax);
    cudaFuncSetAttribute(prod_fwd_f16_kernel<1, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmemMax);
  });
  if (bg == 4)
    prod_fwd_f16_kernel<4, 8><<<grid, 256, smem, s>>>((const __half2*)Fhat, scale, mhat, partial, nf, R, Nm, B,
                                                      JC, nchunk);
  else
    prod_fwd_f16_kernel<1, 32><<<grid, 256, smem, s>>>((const __half2*)Fhat, scale, mhat, partial, nf, R, Nm, B,
                                                       JC, nchunk);
}

// Adjoint product; the row scale is folded into d-hat as it is staged.
template <int BG, int VPT>
__global__ void __launch_bounds__(256)
prod_adj_f16_kernel(const __half2* __restrict__ Fhat, const float* __restrict__ scale,
                    const float2* __restrict__ dhat, float2* __restrict__ mhat, int64_t nf, int64_t R, int64_t Nm,
                    int64_t B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* sd = reinterpret_cast<float2*>(smem_raw);  // [BG][min(R, kAdjRows)]
  const int64_t w = blockIdx.y;
  const int64_t b0 = (int64_t)blockIdx.z * BG;
  const int64_t jbase = (int64_t)blockIdx.x * (256 * VPT) + threadIdx.x;
  float ar[BG][VPT], ai[BG][VPT];
#pragma unroll
  for (int bb = 0; bb < BG; ++bb)
#pragma unroll
    for (int v = 0; v < VPT; ++v) ar[bb][v] = ai[bb][v] = 0.f;
  const __half2* base = Fhat + w * R * Nm;
  const __half2 hz = __floats2half2_rn(0.f, 0.f);
  // d-hat rows are staged RS at a time; each thread still sums over i in order
  const int64_t RS = R < kAdjRows ? R : kAdjRows;
  for (int64_t i0 = 0; i0 < R; i0 += RS) {
    const int64_t rn = R - i0 < RS ? R - i0 : RS;
    if (i0 > 0) __syncthreads();  // the previous tile is consumed
    for (int64_t idx = threadIdx.x; idx < BG * rn; idx += blockDim.x) {
      int64_t bb = idx / rn, i = i0 + (idx - bb * rn);
      float2 v = make_float2(0.f, 0.f);
      if (b0 + bb < B) {
        v = dhat[((b0 + bb) * nf + w) * R + i];
        float sc = scale[w * R + i];
        v.x *= sc;
        v.y *= sc;
      }
      sd[bb * RS + (i - i0)] = v;
    }
    __syncthreads();
    for (int64_t ii = 0; ii < rn; ++ii) {
      const int64_t i = i0 + ii;
      const __half2* row = base + i * Nm;
      float2 f[VPT];
#pragma unroll
      for (int v = 0; v < VPT; ++v) {
        int64_t j = jbase + 256 * v;
        f[v] = __half22float2((j < Nm) ? __ldg(row + j) : hz);
      }
#pragma unroll
      for (int bb = 0; bb < BG; ++bb) {
        float2 x = sd[bb * RS + ii];
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
          ar[bb][v] = fmaf(f[v].x, x.x, ar[bb][v]);
          ar[bb][v] = fmaf(f[v].y, x.y, ar[bb][v]);
          ai[bb][v] = fmaf(f[v].x, x.y, ai[bb][v]);
          ai[bb][v] = fmaf(-f[v].y, x.x, ai[bb][v]);
        }
      }
    }
  }
#pragma unroll
  for (int bb = 0; bb < BG; ++bb) {
    if (b0 + bb >= B) continue;
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      int64_t j = jbase + 256 * v;
      if (j < Nm) mhat[((b0 + bb) * nf + w) * Nm + j] = make_float2(ar[bb][v], ai[bb][v]);
    }
  }
}

template <int BG, int VPT>
static void adj_f16_launch(const void* Fhat, const float* scale, const float2* dhat, float2* mhat, int64_t nf,
                           int64_t R, int64_t Nm, int64_t B, cudaStream_t s) {
  size_t smem = sizeof(float2) * (size_t)BG * (R < kAdjRows ? R : kAdjRows);
  dim3 grid((unsigned)((Nm + 256 * VPT - 1) / (256 * VPT)), (unsigned)nf, (unsigned)((B + BG - 1) / BG));
  prod_adj_f16_kernel<BG, VPT><<<grid, 256, smem, s>>>((const __half2*)Fhat, scale, dhat, mhat, nf, R, Nm, B);
}

void launch_prod_adj_f16(const void* Fhat, const float* scale, const float2* dhat, float2* mhat, int64_t nf,
                         int64_t R, int64_t Nm, int64_t B, cudaStream_t s, int vpt) {
  if (B >= 4)
    adj_f16_launch<4, 4>(Fhat, scale, dhat, mhat, nf, R, Nm, B, s);
  else if (vpt == 2)
    adj_f16_launch<1, 2>(Fhat, scale, dhat, mhat, nf, R, Nm, B, s);
  else if (vpt == 4)
    adj_f16_launch<1, 4>(Fhat, scale, dhat, mhat, nf, R, Nm, B, s);
  else
    adj_f16_launch<1, 8>(Fhat, scale, dhat, mhat, nf, R, Nm, B, s);
}

}  // namespace bti
