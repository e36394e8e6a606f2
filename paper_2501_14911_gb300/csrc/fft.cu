// Batched zero-padded real FFTs along time for many spatial columns.
//
// Sec. 4 ("FFT-based GPU-accelerated p2o and p2q matvecs") embeds the block
// Toeplitz map in a block circulant of length L and diagonalises it with the
// DFT.  With L = 2 N_t the circulant product reproduces the truncated causal
// convolution exactly, so every transform here is:
//   forward : X[w] = sum_{t < N_t} x[t] e^{-2 pi i w t / L},  w = 0..N_t
//             (real input, second half zero, Hermitian half spectrum kept)
//   inverse : y[t] = scale * sum_{w < L} Y[w] e^{+2 pi i w t / L}, t < N_t only,
//             with Y extended by Hermitian symmetry from w = 0..N_t.
// A "column" is one spatial index; time runs along the strided axis and
// columns are contiguous, so every global access is a coalesced row segment.
//
// Each CTA transforms 2P real columns as P complex transforms (column 2p in the
// real part, 2p+1 in the imaginary part), in shared memory with a mixed-radix
// (8, 4, 2, 7, 5, 3) Stockham pass sequence; twiddles e^{-2 pi i n / L} come from
// a table computed in FP64 on the host with std::cos / std::sin.  The arithmetic
// type T is float, double, or the double-FP32 pair (ffloat), which carries FP64-
// level accuracy on the FP32 pipes (GB300 issues FP64 at 1/64 of the FP32 rate).
// The pair transforms take and give their spectra as float pairs (re_hi, re_lo, im_hi,
// im_lo): converting FP64 spectra to pairs on load and back on store kept the FP64 pipe
// 62 % busy and cost 28-36 % of the transforms' time.
#include "bti_internal.cuh"

#include <cmath>
#include <type_traits>
#include <vector>

namespace bti {

struct FftDesc {
  int L;
  int npass;
  int P;
  int radix[kMaxPasses];
};

void fft_plan_free(FftPlan& p) {
  cudaFree(p.tw64);
  cudaFree(p.tw32);
  cudaFree(p.twff);
  p.tw64 = nullptr;
  p.tw32 = nullptr;
  p.twff = nullptr;
}

bool fft_plan_make(FftPlan& p, int L) {
  if (L < 2 || L > kMaxL) return false;
  int n = L, np = 0;
  const int order[6] = {8, 4, 2, 7, 5, 3};
  for (int oi = 0; oi < 6; ++oi) {
    int r = order[oi];
    while (n % r == 0) {
      if (np >= kMaxPasses) return false;
      p.radix[np++] = r;
      n /= r;
    }
  }
  if (n != 1) return false;
  p.L = L;
  p.npass = np;
  int P = kMaxL / L;  // P L <= kMaxL complex elements per CTA (two buffers)
  if (P > 16) P = 16;
  if (P < 1) P = 1;
  p.P = P;
  std::vector<double2> t64(L);
  std::vector<float2> t32(L);
  const double two_pi = 6.283185307179586476925286766559;
  for (int k = 0; k < L; ++k) {
    double a = two_pi * (double)k / (double)L;
    t64[k] = make_double2(std::cos(a), -std::sin(a));
    t32[k] = make_float2((float)t64[k].x, (float)t64[k].y);
  }
  std::vector<ffc> tff(L);
  for (int k = 0; k < L; ++k) {
    tff[k].x = ffloat(t64[k].x);
    tff[k].y = ffloat(t64[k].y);
  }
  if (cudaMalloc(&p.tw64, sizeof(double2) * L) != cudaSuccess || cudaMalloc(&p.tw32, sizeof(float2) * L) != cudaSuccess ||
      cudaMalloc(&p.twff, sizeof(ffc) * L) != cudaSuccess) {
    fft_plan_free(p);  // no table outlives a failed plan
    return false;
  }
  cudaMemcpy(p.tw64, t64.data(), sizeof(double2) * L, cudaMemcpyHostToDevice);
  cudaMemcpy(p.tw32, t32.data(), sizeof(float2) * L, cudaMemcpyHostToDevice);
  cudaMemcpy(p.twff, tff.data(), sizeof(ffc) * L, cudaMemcpyHostToDevice);
  return true;
}

bool fft_plan_factor(FftPlan& p, int L) {
  if (L < 2 || L > kMaxL) return false;
  int n = L, np = 0;
  const int order[6] = {8, 4, 2, 7, 5, 3};
  for (int oi = 0; oi < 6; ++oi) {
    int r = order[oi];
    while (n % r == 0) {
      if (np >= kMaxPasses) return false;
      p.radix[np++] = r;
      n /= r;
    }
  }
  if (n != 1) return false;
  p.L = L;
  p.npass = np;
  int P = kMaxL / L;  // P L <= kMaxL complex elements per CTA (two buffers)
  if (P > 16) P = 16;
  if (P < 1) P = 1;
  p.P = P;
  p.tw64 = nullptr;
  p.tw32 = nullptr;
  p.twff = nullptr;
  return true;
}

struct TwTabs {
  const double2* t64;
  const float2* t32;
  const ffc* tff;
};
template <typename T> __device__ __forceinline__ const C2<T>* twtab(const TwTabs& t);
template <> __device__ __forceinline__ const double2* twtab<double>(const TwTabs& t) { return t.t64; }
template <> __device__ __forceinline__ const float2* twtab<float>(const TwTabs& t) { return t.t32; }
template <> __device__ __forceinline__ const ffc* twtab<ffloat>(const TwTabs& t) { return t.tff; }

template <typename T> __device__ __forceinline__ C2<T> tw_load(const C2<T>* __restrict__ tw, int n) {
  return __ldg(&tw[n]);
}
template <> __device__ __forceinline__ ffc tw_load<ffloat>(const ffc* __restrict__ tw, int n) {
  float4 v = __ldg(reinterpret_cast<const float4*>(tw) + n);
  ffc z;
  z.x = ffloat(v.x, v.y);
  z.y = ffloat(v.z, v.w);
  return z;
}

template <typename T, bool INV>
__device__ __forceinline__ C2<T> tw_get(const C2<T>* __restrict__ tw, int n) {
  C2<T> w = tw_load<T>(tw, n);
  if (INV) w.y = -w.y;
  return w;
}

// The butterflies' arithmetic.  For float pairs the sums and products inside a butterfly are
// left unnormalised: the high parts are still summed by an exact two-sum and the products'
// errors kept by FMA, but the low float is not folded back to |lo| <= ulp(hi) / 2 after every
// operation (8 FP32 operations per sum instead of 11, 4 per product instead of 7, 16 per
// complex-product part instead of 19).  Rounding the low floats costs about 2^-48 of the
// operands' magnitude either way; each butterfly output is renormalised once, as it is stored.
template <typename T> __device__ __forceinline__ C2<T> badd(C2<T> a, C2<T> b) { return cadd<T>(a, b); }
template <typename T> __device__ __forceinline__ C2<T> bsub(C2<T> a, C2<T> b) { return csub<T>(a, b); }
template <typename T> __device__ __forceinline__ C2<T> bmul(C2<T> a, C2<T> b) { return cmul<T>(a, b); }
template <typename T> __device__ __forceinline__ C2<T> bscale(T c, C2<T> a) { return mk<T>(c * a.x, c * a.y); }
template <typename T> __device__ __forceinline__ C2<T> bnorm(C2<T> a) { return a; }

__device__ __forceinline__ ffloat ff_add_u(ffloat a, ffloat b) {
  const float s = __fadd_rn(a.h, b.h);
  const float bb = __fsub_rn(s, a.h);
  const float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
  return ffloat(s, __fadd_rn(e, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ ffloat ff_mul_u(ffloat a, ffloat b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return ffloat(p, e);
}
// x1 y1 - x2 y2 (sub) or x1 y1 + x2 y2: both high products exact, summed by two-sum
__device__ __forceinline__ ffloat ff_dot2_u(ffloat x1, ffloat y1, ffloat x2, ffloat y2, bool sub) {
  const float sg = sub ? -1.f : 1.f;
  const float p1 = __fmul_rn(x1.h, y1.h);
  const float p2 = __fmul_rn(sg * x2.h, y2.h);
  float lo = __fmaf_rn(x1.h, y1.h, -p1);
  lo = __fadd_rn(lo, __fmaf_rn(sg * x2.h, y2.h, -p2));
  const float s = __fadd_rn(p1, p2);
  const float bb = __fsub_rn(s, p1);
  lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(p1, __fsub_rn(s, bb)), __fsub_rn(p2, bb)));
  lo = __fmaf_rn(x1.h, y1.l, lo);
  lo = __fmaf_rn(x1.l, y1.h, lo);
  lo = __fmaf_rn(sg * x2.h, y2.l, lo);
  lo = __fmaf_rn(sg * x2.l, y2.h, lo);
  return ffloat(s, lo);
}
__device__ __forceinline__ ffloat ff_norm(ffloat a) {
  const float h = __fadd_rn(a.h, a.l);
  return ffloat(h, __fsub_rn(a.l, __fsub_rn(h, a.h)));
}
template <> __device__ __forceinline__ ffc badd<ffloat>(ffc a, ffc b) {
  return mk<ffloat>(ff_add_u(a.x, b.x), ff_add_u(a.y, b.y));
}
template <> __device__ __forceinline__ ffc bsub<ffloat>(ffc a, ffc b) {
  return mk<ffloat>(ff_add_u(a.x, -b.x), ff_add_u(a.y, -b.y));
}
template <> __device__ __forceinline__ ffc bmul<ffloat>(ffc a, ffc b) {
  return mk<ffloat>(ff_dot2_u(a.x, b.x, a.y, b.y, true), ff_dot2_u(a.x, b.y, a.y, b.x, false));
}
template <> __device__ __forceinline__ ffc bscale<ffloat>(ffloat c, ffc a) {
  return mk<ffloat>(ff_mul_u(c, a.x), ff_mul_u(c, a.y));
}
template <> __device__ __forceinline__ ffc bnorm<ffloat>(ffc a) { return mk<ffloat>(ff_norm(a.x), ff_norm(a.y)); }

// multiply by -i (forward) or +i (inverse)
template <typename T, bool INV>
__device__ __forceinline__ C2<T> rot90(C2<T> a) {
  return INV ? mk<T>(-a.y, a.x) : mk<T>(a.y, -a.x);
}

// Shared-memory slot of element n of one transform: one padding slot after every 8
// elements, so the stride-8 stores of a first radix-8 pass (and the column staging)
// spread over all 32 banks instead of serialising on four of them.
__device__ __forceinline__ int sp(int n) { return n + (n >> 3); }

template <typename T, bool INV>
__device__ __forceinline__ void dft4(C2<T>& a0, C2<T>& a1, C2<T>& a2, C2<T>& a3) {
  C2<T> t0 = badd<T>(a0, a2), t1 = bsub<T>(a0, a2);
  C2<T> t2 = badd<T>(a1, a3), t3 = rot90<T, INV>(bsub<T>(a1, a3));
  a0 = badd<T>(t0, t2);
  a2 = bsub<T>(t0, t2);
  a1 = badd<T>(t1, t3);
  a3 = bsub<T>(t1, t3);
}

// One radix-R Stockham butterfly: inputs element i0 + q Lr of src, q < R; outputs element
// o0 + m Ns of dst, m < R (elements at their padded slots).
template <int R, typename T, bool INV>
__device__ __forceinline__ void butterfly(const C2<T>* src, int i0, int Lr, C2<T>* dst, int o0, int Ns,
                                          const C2<T>* __restrict__ tw, int twstep, int L) {
  C2<T> a[R];
#pragma unroll
  for (int q = 0; q < R; ++q) a[q] = src[sp(i0 + q * Lr)];
  if (twstep != 0) {
#pragma unroll
    for (int q = 1; q < R; ++q) a[q] = bmul<T>(a[q], tw_get<T, INV>(tw, q * twstep));
  }
  if (R == 2) {
    C2<T> b0 = badd<T>(a[0], a[1]), b1 = bsub<T>(a[0], a[1]);
    a[0] = b0;
    a[1] = b1;
  } else if (R == 4) {
    dft4<T, INV>(a[0], a[1], a[2], a[3]);
  } else if (R == 8) {
    // even / odd radix-4 halves, combined with powers of w8 = e^{-+ i pi / 4}
    C2<T> e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
    C2<T> o0 = a[1], o1 = a[3], o2 = a[5], o3 = a[7];
    dft4<T, INV>(e0, e1, e2, e3);
    dft4<T, INV>(o0, o1, o2, o3);
    const T h = (T)0.70710678118654752440084436210485;  // sqrt(1/2)
    C2<T> w1 = INV ? mk<T>(h, h) : mk<T>(h, -h);
    C2<T> w3 = INV ? mk<T>(-h, h) : mk<T>(-h, -h);
    o1 = bmul<T>(o1, w1);
    o2 = rot90<T, INV>(o2);
    o3 = bmul<T>(o3, w3);
    a[0] = badd<T>(e0, o0);
    a[4] = bsub<T>(e0, o0);
    a[1] = badd<T>(e1, o1);
    a[5] = bsub<T>(e1, o1);
    a[2] = badd<T>(e2, o2);
    a[6] = bsub<T>(e2, o2);
    a[3] = badd<T>(e3, o3);
    a[7] = bsub<T>(e3, o3);
  } else if (R == 5) {
    // radix 5 with constant twiddles: with t1 = a1 + a4, t2 = a2 + a3, t3 = a1 - a4,
    // t4 = a2 - a3, c_k = cos(2 pi k / 5) and s_k = sin(2 pi k / 5) (k = 1, 2), the outputs are
    // b0 = a0 + t1 + t2, b1,4 = u1 -+ i v1, b2,3 = u2 -+ i v2 (signs of i flipped for the
    // inverse) with u1 = a0 + c1 t1 + c2 t2, u2 = a0 + c2 t1 + c1 t2, v1 = s1 t3 + s2 t4 and
    // v2 = s2 t3 - s1 t4, since w^4 = conj(w) and w^3 = conj(w^2) for w = e^{-2 pi i / 5}
    const T c1 = (T)0.30901699437494742410229341718282, c2 = (T)-0.80901699437494742410229341718282;
    const T s1 = (T)0.95105651629515357211643933337938, s2 = (T)0.58778525229247312916870595463907;
    const C2<T> t1 = badd<T>(a[1], a[4]), t2 = badd<T>(a[2], a[3]);
    const C2<T> t3 = bsub<T>(a[1], a[4]), t4 = bsub<T>(a[2], a[3]);
    const C2<T> u1 = badd<T>(a[0], badd<T>(bscale<T>(c1, t1), bscale<T>(c2, t2)));
    const C2<T> u2 = badd<T>(a[0], badd<T>(bscale<T>(c2, t1), bscale<T>(c1, t2)));
    const C2<T> v1 = rot90<T, INV>(badd<T>(bscale<T>(s1, t3), bscale<T>(s2, t4)));
    const C2<T> v2 = rot90<T, INV>(bsub<T>(bscale<T>(s2, t3), bscale<T>(s1, t4)));
    a[0] = badd<T>(a[0], badd<T>(t1, t2));
    a[1] = badd<T>(u1, v1);
    a[4] = bsub<T>(u1, v1);
    a[2] = badd<T>(u2, v2);
    a[3] = bsub<T>(u2, v2);
  } else {
    // generic small DFT (R = 3, 7): b_m = sum_q a_q w_R^{q m}, w_R^n = tw[(n mod R) L / R]
    C2<T> b[R];
    const int LR = L / R;
#pragma unroll
    for (int m = 0; m < R; ++m) {
      C2<T> acc = a[0];
#pragma unroll
      for (int q = 1; q < R; ++q) {
        int e = (q * m) % R;
        C2<T> w = tw_get<T, INV>(tw, e * LR);
        acc = badd<T>(acc, bmul<T>(a[q], w));
      }
      b[m] = acc;
    }
#pragma unroll
    for (int m = 0; m < R; ++m) a[m] = b[m];
  }
#pragma unroll
  for (int m = 0; m < R; ++m) dst[sp(o0 + m * Ns)] = bnorm<T>(a[m]);
}

// First radix-8 pass of a forward transform whose second half is zero padding
// (L = 2 N_t, so inputs q = 4..7 of every first-pass butterfly vanish; the pass has
// no twiddles since Ns = 1): the two radix-4 halves reduce to two additions each.
template <typename T>
__device__ __forceinline__ void butterfly8_half_zero(const C2<T>* src, int i0, int Lr, C2<T>* dst, int o0) {
  const C2<T> a0 = src[sp(i0)], a1 = src[sp(i0 + Lr)], a2 = src[sp(i0 + 2 * Lr)], a3 = src[sp(i0 + 3 * Lr)];
  // even half: DFT4(a0, a2, 0, 0); odd half: DFT4(a1, a3, 0, 0)
  const C2<T> r2 = rot90<T, false>(a2), r3 = rot90<T, false>(a3);
  C2<T> e0 = badd<T>(a0, a2), e2 = bsub<T>(a0, a2), e1 = badd<T>(a0, r2), e3 = bsub<T>(a0, r2);
  C2<T> o0v = badd<T>(a1, a3), o2 = bsub<T>(a1, a3), o1 = badd<T>(a1, r3), o3 = bsub<T>(a1, r3);
  const T h = (T)0.70710678118654752440084436210485;  // sqrt(1/2)
  o1 = bmul<T>(o1, mk<T>(h, -h));
  o2 = rot90<T, false>(o2);
  o3 = bmul<T>(o3, mk<T>(-h, -h));
  dst[sp(o0)] = bnorm<T>(badd<T>(e0, o0v));
  dst[sp(o0 + 4)] = bnorm<T>(bsub<T>(e0, o0v));
  dst[sp(o0 + 1)] = bnorm<T>(badd<T>(e1, o1));
  dst[sp(o0 + 5)] = bnorm<T>(bsub<T>(e1, o1));
  dst[sp(o0 + 2)] = bnorm<T>(badd<T>(e2, o2));
  dst[sp(o0 + 6)] = bnorm<T>(bsub<T>(e2, o2));
  dst[sp(o0 + 3)] = bnorm<T>(badd<T>(e3, o3));
  dst[sp(o0 + 7)] = bnorm<T>(bsub<T>(e3, o3));
}

// The radix sequence of a length L in fft_plan_make's order (8, 4, 2, 7, 5, 3), at compile time
// for the kernels specialised on L.
__host__ __device__ constexpr int ct_radix(int L, int i) {
  const int order[6] = {8, 4, 2, 7, 5, 3};
  int n = L, k = 0;
  for (int oi = 0; oi < 6; ++oi)
    while (n % order[oi] == 0) {
      if (k == i) return order[oi];
      n /= order[oi];
      ++k;
    }
  return 1;
}
__host__ __device__ constexpr int ct_npass(int L) {
  int k = 0;
  while (ct_radix(L, k) != 1) ++k;
  return k;
}

// Radix sets compiled into a kernel: fewer butterflies compiled in means fewer registers,
// and the restricted sets fit 3 CTAs per SM instead of 2.
enum { kRadixAll = 0, kRadixPow2 = 1, kRadix25 = 2 };  // (8, 4, 2, 7, 5, 3); (8, 4, 2); (8, 4, 2, 5)

// One Stockham pass of radix r over the CTA's P transforms (src -> dst, padded slots).
template <typename T, bool INV, int RS>
__device__ __forceinline__ void one_pass(const C2<T>* src, C2<T>* dst, const C2<T>* __restrict__ tw, int r, int L,
                                         int Ns, int P, int LP) {
  const int Lr = L / r;
  const int nbf = P * Lr;
  for (int bi = threadIdx.x; bi < nbf; bi += blockDim.x) {
    int p = bi / Lr;
    int j = bi - p * Lr;
    int k = j % Ns;
    const C2<T>* s = src + p * LP;
    C2<T>* d = dst + p * LP;
    const int o0 = (j - k) * r + k;
    int twstep = k * (L / (Ns * r));
    if (RS == kRadixPow2) {
      if (r == 8) butterfly<8, T, INV>(s, j, Lr, d, o0, Ns, tw, twstep, L);
      else if (r == 4) butterfly<4, T, INV>(s, j, Lr, d, o0, Ns, tw, twstep, L);
      else butterfly<2, T, INV>(s, j, Lr, d, o0, Ns, tw, twstep, L);
    } else if (RS == kRadix25) {
      if (r == 8) butterfly<8, T, INV>(s, j, Lr, d, o0, Ns, tw, twstep, L);
      else if (r == 4) butterfly<4, T, INV>(s, j, Lr, d, o0, Ns, tw, twstep, L);
      else if (r == 2) butterfly<2, T, INV>(s, j, Lr, d, o0, Ns, tw, twstep, L);
      else butterfly<5, T, INV>(s, j, Lr, d, o0, Ns, tw, twstep, L);
    } else {
      switch (r) {
        case 8: butterfly<8, T, INV>(s, j, Lr, d, o0, Ns, tw, twstep, L); break;
        case 4: butterfly<4, T, INV>(s, j, Lr, d, o0, Ns, tw, twstep, L); break;
        case 2: butterfly<2, T, INV>(s, j, Lr, d, o0, Ns, tw, twstep, L); break;
        case 7: butterfly<7, T, INV>(s, j, Lr, d, o0, Ns, tw, twstep, L); break;
        case 5: butterfly<5, T, INV>(s, j, Lr, d, o0, Ns, tw, twstep, L); break;
        default: butterfly<3, T, INV>(s, j, Lr, d, o0, Ns, tw, twstep, L); break;
      }
    }
  }
}

// The first radix-8 pass of a forward transform whose second half is zero padding.
template <typename T>
__device__ __forceinline__ void first_pass_half_zero(const C2<T>* src, C2<T>* dst, int L, int P, int LP) {
  const int Lr = L / 8;
  const int nbf = P * Lr;
  for (int bi = threadIdx.x; bi < nbf; bi += blockDim.x) {
    int p = bi / Lr, j = bi - p * Lr;
    butterfly8_half_zero<T>(src + p * LP, j, Lr, dst + p * LP, j * 8);
  }
}

// All passes; data starts in buf0, result pointer returned (buf0 or buf1); transform p
// of the CTA occupies LP slots from p LP.  With half_zero, the first pass is radix 8 and
// only the first half of each input is nonzero.  RS selects the compiled radix set.  CL > 0:
// the length is CL at compile time (D.L must equal it): the radix sequence, every index
// divisor and twiddle stride are constants and the pass loop is unrolled; for a forward
// transform half_zero must then hold (L = 2 N_t).
template <typename T, bool INV, int RS, int CL = 0>
__device__ C2<T>* run_passes(const FftDesc& D, C2<T>* buf0, C2<T>* buf1, const C2<T>* __restrict__ tw,
                             int LP, bool half_zero = false) {
  C2<T>* src = buf0;
  C2<T>* dst = buf1;
  if constexpr (CL > 0) {
    constexpr bool hz = !INV && ct_radix(CL, 0) == 8;  // the zero-padded first pass (forward)
    if constexpr (hz) {
      first_pass_half_zero<T>(src, dst, CL, D.P, LP);
      __syncthreads();
      C2<T>* tmp = src;
      src = dst;
      dst = tmp;
    }
    int Ns = hz ? 8 : 1;
#pragma unroll
    for (int ps = hz ? 1 : 0; ps < ct_npass(CL); ++ps) {
      const int r = ct_radix(CL, ps);
      one_pass<T, INV, RS>(src, dst, tw, r, CL, Ns, D.P, LP);
      __syncthreads();
      C2<T>* tmp = src;
      src = dst;
      dst = tmp;
      Ns *= r;
    }
  } else {
    const int L = D.L;
    int Ns = 1;
    int ps0 = 0;
    if (!INV && half_zero && D.npass > 0 && D.radix[0] == 8) {
      first_pass_half_zero<T>(src, dst, L, D.P, LP);
      __syncthreads();
      C2<T>* tmp = src;
      src = dst;
      dst = tmp;
      Ns = 8;
      ps0 = 1;
    }
    for (int ps = ps0; ps < D.npass; ++ps) {
      const int r = D.radix[ps];
      one_pass<T, INV, RS>(src, dst, tw, r, L, Ns, D.P, LP);
      __syncthreads();
      C2<T>* tmp = src;
      src = dst;
      dst = tmp;
      Ns *= r;
    }
  }
  return src;
}

template <typename TO, typename T> __device__ __forceinline__ C2<TO> cvt2(C2<T> z) {
  return mk<TO>((TO)z.x, (TO)z.y);
}
template <typename T> __device__ __forceinline__ C2<T> czero() { return mk<T>((T)0, (T)0); }

template <typename T, typename TI, typename TO, int RS, int CL = 0>
__global__ void __launch_bounds__(256, RS == kRadixAll ? 2 : 3)  // restricted radix sets fit 3 CTAs per SM
rfft_cols_kernel(FftDesc D, int Nt, const TI* __restrict__ x, int64_t ld, int64_t xbs,
                 C2<TO>* __restrict__ X, int64_t Xbs, int64_t ncols, TwTabs tabs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = CL ? CL : D.L, P = D.P, W2 = 2 * P, LP = fft_slots(L);
  C2<T>* buf0 = reinterpret_cast<C2<T>*>(smem_raw);
  C2<T>* buf1 = buf0 + P * LP;
  const C2<T>* tw = twtab<T>(tabs);
  const int64_t col0 = (int64_t)blockIdx.x * W2;
  const TI* xb = x + (int64_t)blockIdx.y * xbs;
  C2<TO>* Xb = X + (int64_t)blockIdx.y * Xbs;

  // stage the 2P columns (time along rows): eight loads per thread in flight before the
  // shared-memory stores
  const int total = Nt * W2;
  for (int base = 0; base < total; base += 8 * blockDim.x) {
    T v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = base + u * blockDim.x + threadIdx.x;
      const int t = idx / W2, c = idx - t * W2;
      const int64_t col = col0 + c;
      v[u] = (idx < total && col < ncols) ? (T)xb[(int64_t)t * ld + col] : (T)0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = base + u * blockDim.x + threadIdx.x;
      if (idx < total) {
        const int t = idx / W2, c = idx - t * W2;
        reinterpret_cast<T*>(&buf0[(c >> 1) * LP + sp(t)])[c & 1] = v[u];
      }
    }
  }
  const int pad = L - Nt;
  for (int idx = threadIdx.x; idx < P * pad; idx += blockDim.x) {
    int p = idx / pad, t = Nt + (idx - p * pad);
    buf0[p * LP + sp(t)] = czero<T>();
  }
  __syncthreads();
  C2<T>* Z = run_passes<T, false, RS, CL>(D, buf0, buf1, tw, LP, 2 * Nt == L);
  // unpack the two real spectra of each pair and store bins 0..N_t
  const int nf = Nt + 1;
  for (int idx = threadIdx.x; idx < nf * W2; idx += blockDim.x) {
    int k = idx / W2, c = idx - k * W2;
    int64_t col = col0 + c;
    if (col >= ncols) continue;
    int p = c >> 1;
    C2<T> z = Z[p * LP + sp(k)];
    C2<T> zc = Z[p * LP + sp(k == 0 ? 0 : L - k)];
    C2<T> out;
    const T half = (T)0.5;
    if ((c & 1) == 0) {
      out = mk<T>(half * (z.x + zc.x), half * (z.y - zc.y));   // (Z + conj Zc) / 2
    } else {
      out = mk<T>(half * (z.y + zc.y), half * (zc.x - z.x));   // (Z - conj Zc) / 2i
    }
    Xb[(int64_t)k * ncols + col] = cvt2<TO, T>(out);
  }
}

template <typename T, typename TYI, typename TO, int RS, int CL = 0>
__global__ void __launch_bounds__(256, RS == kRadixAll ? 2 : 3)
irfft_cols_kernel(FftDesc D, int Nt, const C2<TYI>* __restrict__ Y, int64_t ld, int64_t Ybs,
                  TO* __restrict__ y, int64_t ybs, int64_t ncols, double scale_d, TwTabs tabs, int ostride) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = CL ? CL : D.L, P = D.P, W2 = 2 * P, LP = fft_slots(L);
  C2<T>* buf0 = reinterpret_cast<C2<T>*>(smem_raw);
  C2<T>* buf1 = buf0 + P * LP;
  const C2<T>* tw = twtab<T>(tabs);
  const T scale = (T)scale_d;
  const int64_t col0 = (int64_t)blockIdx.x * W2;
  const C2<TYI>* Yb = Y + (int64_t)blockIdx.y * Ybs;
  TO* yb = y + (int64_t)blockIdx.y * ybs;
  const int nf = Nt + 1;
  // Stage the two spectra of each column pair straight into the complex input of one
  // transform: Z[k] = A[k] + i B[k] for k <= N_t and Z[L-k] = conj(A[k]) + i conj(B[k]).
  // Bins 0 and N_t of a real signal's spectrum are real: their imaginary parts are dropped.
  // Each thread reads the pair's two neighbouring columns of one row.
  for (int idx = threadIdx.x; idx < nf * P; idx += blockDim.x) {
    const int k = idx / P, p = idx - k * P;
    const int64_t c0 = col0 + 2 * p;
    const C2<TYI>* row = Yb + (int64_t)k * ld;
    const C2<T> a = (c0 < ncols) ? cvt2<T, TYI>(row[c0]) : czero<T>();
    const C2<T> b = (c0 + 1 < ncols) ? cvt2<T, TYI>(row[c0 + 1]) : czero<T>();
    if (k == 0 || k == Nt) {
      buf0[p * LP + sp(k)] = mk<T>(a.x, b.x);
    } else {
      buf0[p * LP + sp(k)] = mk<T>(a.x - b.y, a.y + b.x);
      buf0[p * LP + sp(L - k)] = mk<T>(a.x + b.y, b.x - a.y);
    }
  }
  __syncthreads();
  C2<T>* Z = run_passes<T, true, RS, CL>(D, buf0, buf1, tw, LP);
  // rows t = ostride (k + 1) - 1 only (every row when ostride == 1), stored as row k
  const int nout = Nt / ostride;
  for (int idx = threadIdx.x; idx < nout * W2; idx += blockDim.x) {
    int k = idx / W2, c = idx - k * W2;
    int64_t col = col0 + c;
    if (col >= ncols) continue;
    const int t = ostride * (k + 1) - 1;
    C2<T> z = Z[(c >> 1) * LP + sp(t)];
    T v = ((c & 1) ? z.y : z.x) * scale;
    yb[(int64_t)k * ld + col] = (TO)v;
  }
}

static FftDesc desc_of(const FftPlan& p) {
  FftDesc d;
  d.L = p.L;
  d.npass = p.npass;
  d.P = p.P;
  for (int i = 0; i < kMaxPasses; ++i) d.radix[i] = (i < p.npass) ? p.radix[i] : 1;
  return d;
}

static TwTabs tabs_of(const FftPlan& p) { return TwTabs{p.tw64, p.tw32, p.twff}; }

// the smallest compiled radix set that covers the plan's passes
static int radix_set(const FftPlan& p) {
  bool only2 = true, only25 = true;
  for (int i = 0; i < p.npass; ++i) {
    const int r = p.radix[i];
    if (r != 8 && r != 4 && r != 2) only2 = false;
    if (r != 8 && r != 4 && r != 2 && r != 5) only25 = false;
  }
  return only2 ? kRadixPow2 : (only25 ? kRadix25 : kRadixAll);
}

template <typename T, typename TI, typename TO>
void launch_rfft_cols(const FftPlan& p, int Nt, const TI* x, int64_t ld, int64_t x_bstride,
                      C2<TO>* X, int64_t X_bstride, int64_t ncols, int64_t B, cudaStream_t s) {
  if (ncols <= 0 || B <= 0) return;
  FftDesc D = desc_of(p);
  size_t smem = 2 * sizeof(C2<T>) * (size_t)p.P * fft_slots(p.L);
  static PerDeviceOnce attr;
  attr([] {
    cudaFuncSetAttribute(rfft_cols_kernel<T, TI, TO, kRadixPow2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    cudaFuncSetAttribute(rfft_cols_kernel<T, TI, TO, kRadix25>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    cudaFuncSetAttribute(rfft_cols_kernel<T, TI, TO, kRadixAll>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
  });
  const int rs = radix_set(p);
  // the float-pair lengths of the headline sweep (512) and the batched workload (400) run
  // kernels compiled for their length (L = 2 N_t, so the first pass is the zero-padded one)
  constexpr bool ff = std::is_same<T, ffloat>::value;
  const int cl = (ff && 2 * Nt == p.L && (p.L == 400 || p.L == 512)) ? p.L : 0;
  if constexpr (ff) {
    static PerDeviceOnce attr_cl;
    attr_cl([] {
      cudaFuncSetAttribute(rfft_cols_kernel<T, TI, TO, kRadix25, 400>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           200 * 1024);
      cudaFuncSetAttribute(rfft_cols_kernel<T, TI, TO, kRadixPow2, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           200 * 1024);
    });
  }
  int64_t gx = (ncols + 2 * p.P - 1) / (2 * p.P);
  for (int64_t b0 = 0; b0 < B; b0 += 65535) {
    int64_t nb = B - b0 < 65535 ? B - b0 : 65535;
    dim3 grid((unsigned)gx, (unsigned)nb);
    const TI* xb = x + b0 * x_bstride;
    C2<TO>* Xb = X + b0 * X_bstride;
    if constexpr (ff) {
      if (cl == 400) {
        rfft_cols_kernel<T, TI, TO, kRadix25, 400><<<grid, 256, smem, s>>>(D, Nt, xb, ld, x_bstride, Xb, X_bstride,
                                                                           ncols, tabs_of(p));
        continue;
      }
      if (cl == 512) {
        rfft_cols_kernel<T, TI, TO, kRadixPow2, 512><<<grid, 256, smem, s>>>(D, Nt, xb, ld, x_bstride, Xb,
                                                                             X_bstride, ncols, tabs_of(p));
        continue;
      }
    }
    if (rs == kRadixPow2)
      rfft_cols_kernel<T, TI, TO, kRadixPow2><<<grid, 256, smem, s>>>(D, Nt, xb, ld, x_bstride, Xb, X_bstride, ncols,
                                                                      tabs_of(p));
    else if (rs == kRadix25)
      rfft_cols_kernel<T, TI, TO, kRadix25><<<grid, 256, smem, s>>>(D, Nt, xb, ld, x_bstride, Xb, X_bstride, ncols,
                                                                    tabs_of(p));
    else
      rfft_cols_kernel<T, TI, TO, kRadixAll><<<grid, 256, smem, s>>>(D, Nt, xb, ld, x_bstride, Xb, X_bstride, ncols,
                                                                     tabs_of(p));
  }
}

template <typename T, typename TYI, typename TO>
void launch_irfft_cols(const FftPlan& p, int Nt, const C2<TYI>* X, int64_t ld, int64_t X_bstride,
                       TO* y, int64_t y_bstride, int64_t ncols, int64_t B, double scale, cudaStream_t s,
                       int ostride) {
  if (ncols <= 0 || B <= 0) return;
  FftDesc D = desc_of(p);
  size_t smem = 2 * sizeof(C2<T>) * (size_t)p.P * fft_slots(p.L);
  static PerDeviceOnce attr;
  attr([] {
    cudaFuncSetAttribute(irfft_cols_kernel<T, TYI, TO, kRadixPow2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    cudaFuncSetAttribute(irfft_cols_kernel<T, TYI, TO, kRadix25>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    cudaFuncSetAttribute(irfft_cols_kernel<T, TYI, TO, kRadixAll>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
  });
  const int rs = radix_set(p);
  const int os = ostride < 1 ? 1 : ostride;
  // compile-time lengths, as in launch_rfft_cols
  constexpr bool ff = std::is_same<T, ffloat>::value;
  const int cl = (ff && (p.L == 400 || p.L == 512)) ? p.L : 0;
  if constexpr (ff) {
    static PerDeviceOnce attr_cl;
    attr_cl([] {
      cudaFuncSetAttribute(irfft_cols_kernel<T, TYI, TO, kRadix25, 400>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      cudaFuncSetAttribute(irfft_cols_kernel<T, TYI, TO, kRadixPow2, 512>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    });
  }
  int64_t gx = (ncols + 2 * p.P - 1) / (2 * p.P);
  for (int64_t b0 = 0; b0 < B; b0 += 65535) {
    int64_t nb = B - b0 < 65535 ? B - b0 : 65535;
    dim3 grid((unsigned)gx, (unsigned)nb);
    const C2<TYI>* Xb = X + b0 * X_bstride;
    TO* yb = y + b0 * y_bstride;
    if constexpr (ff) {
      if (cl == 400) {
        irfft_cols_kernel<T, TYI, TO, kRadix25, 400><<<grid, 256, smem, s>>>(D, Nt, Xb, ld, X_bstride, yb,
                                                                              y_bstride, ncols, scale, tabs_of(p), os);
        continue;
      }
      if (cl == 512) {
        irfft_cols_kernel<T, TYI, TO, kRadixPow2, 512><<<grid, 256, smem, s>>>(D, Nt, Xb, ld, X_bstride, yb,
                                                                                y_bstride, ncols, scale, tabs_of(p),
                                                                                os);
        continue;
      }
    }
    if (rs == kRadixPow2)
      irfft_cols_kernel<T, TYI, TO, kRadixPow2><<<grid, 256, smem, s>>>(D, Nt, Xb, ld, X_bstride, yb, y_bstride,
                                                                        ncols, scale, tabs_of(p), os);
    else if (rs == kRadix25)
      irfft_cols_kernel<T, TYI, TO, kRadix25><<<grid, 256, smem, s>>>(D, Nt, Xb, ld, X_bstride, yb, y_bstride,
                                                                      ncols, scale, tabs_of(p), os);
    else
      irfft_cols_kernel<T, TYI, TO, kRadixAll><<<grid, 256, smem, s>>>(D, Nt, Xb, ld, X_bstride, yb, y_bstride,
                                                                       ncols, scale, tabs_of(p), os);
  }
}

#define INST_R(T, TI, TO)                                                                    \
  template void launch_rfft_cols<T, TI, TO>(const FftPlan&, int, const TI*, int64_t, int64_t, \
                                            C2<TO>*, int64_t, int64_t, int64_t, cudaStream_t);
INST_R(double, double, double)
INST_R(double, double, float)
INST_R(double, float, double)
INST_R(float, float, float)
INST_R(float, double, float)
INST_R(ffloat, double, ffloat)
INST_R(ffloat, float, ffloat)
#define INST_I(T, TYI, TO)                                                                             \
  template void launch_irfft_cols<T, TYI, TO>(const FftPlan&, int, const C2<TYI>*, int64_t, int64_t, TO*, \
                                              int64_t, int64_t, int64_t, double, cudaStream_t, int);
INST_I(double, double, double)
INST_I(double, double, float)
INST_I(float, float, float)
INST_I(float, float, double)
INST_I(ffloat, ffloat, double)
INST_I(ffloat, ffloat, float)

}  // namespace bti
