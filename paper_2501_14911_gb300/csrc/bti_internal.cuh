// Internal declarations shared by the libbti translation units.
#pragma once

#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>
#include <string>

#include "../../include/bti.h"

namespace bti {

// Runs a set-up step once for each CUDA device of the process.  Kernel attributes such as the
// dynamic shared-memory limit belong to the device the module is loaded on, so a step done
// once per process would leave the other devices of a multi-device process without them.
struct PerDeviceOnce {
  std::atomic<unsigned long long> done{0};
  template <typename Fn> void operator()(Fn fn) {
    int dev = 0;
    cudaGetDevice(&dev);
    const unsigned long long bit = 1ull << (dev & 63);
    if (done.load(std::memory_order_acquire) & bit) return;
    fn();
    done.fetch_or(bit, std::memory_order_acq_rel);
  }
};

// ----------------------------------------------------------------- complex helpers
template <typename T> struct cplx;
template <> struct cplx<double> { using type = double2; };
template <> struct cplx<float> { using type = float2; };
struct ffloat;
struct ffc;
template <> struct cplx<ffloat> { using type = ffc; };
template <typename T> using C2 = typename cplx<T>::type;

template <typename T> __host__ __device__ __forceinline__ C2<T> mk(T re, T im) {
  C2<T> z; z.x = re; z.y = im; return z;
}
template <typename T> __device__ __forceinline__ C2<T> cadd(C2<T> a, C2<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ C2<T> csub(C2<T> a, C2<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ C2<T> cmul(C2<T> a, C2<T> b) {
  return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * b where b is conjugated when CONJ
template <typename T> __device__ __forceinline__ C2<T> cmulc(C2<T> a, C2<T> b) {
  return mk<T>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);  // a * conj(b)
}

// ----------------------------------------------------------------- double-FP32 scalar
// An unevaluated sum h + l of two floats (|l| <= ulp(h)/2): about 48 significant
// bits carried on the FP32 pipes.  Addition uses Knuth's error-free two-sum and
// multiplication the FMA-exact product; both renormalise.  The intrinsics keep
// the compiler from contracting or reassociating the error terms away.
struct ffloat {
  float h, l;
  ffloat() = default;
  __host__ __device__ constexpr ffloat(float hh, float ll) : h(hh), l(ll) {}
  __host__ __device__ constexpr explicit ffloat(double x) : h((float)x), l((float)(x - (double)(float)x)) {}
  __host__ __device__ constexpr explicit ffloat(float x) : h(x), l(0.f) {}
  __host__ __device__ constexpr explicit ffloat(int x) : h((float)x), l(0.f) {}
  __host__ __device__ explicit operator double() const { return (double)h + (double)l; }
  __host__ __device__ explicit operator float() const { return h + l; }
};
__device__ __forceinline__ ffloat operator+(ffloat a, ffloat b) {
  float s = __fadd_rn(a.h, b.h);
  float bb = __fsub_rn(s, a.h);
  float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  float h = __fadd_rn(s, e);
  return ffloat(h, __fsub_rn(e, __fsub_rn(h, s)));
}
__device__ __forceinline__ ffloat operator-(ffloat a) { return ffloat(-a.h, -a.l); }
__device__ __forceinline__ ffloat operator-(ffloat a, ffloat b) { return a + (-b); }
__device__ __forceinline__ ffloat operator*(ffloat a, ffloat b) {
  float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  float h = __fadd_rn(p, e);
  return ffloat(h, __fsub_rn(e, __fsub_rn(h, p)));
}
struct __align__(16) ffc {
  ffloat x, y;
};

// One real part of a float-pair complex product: x1*y1 - x2*y2 (sub) or x1*y1 + x2*y2,
// with both high products exact (FMA errors), their sum by two-sum, the cross terms
// and errors gathered in the low float, then one renormalisation (19 FP32 operations).
__device__ __forceinline__ ffloat ff_dot2(ffloat x1, ffloat y1, ffloat x2, ffloat y2, bool sub) {
  const float sg = sub ? -1.f : 1.f;
  float p1 = __fmul_rn(x1.h, y1.h);
  float p2 = __fmul_rn(sg * x2.h, y2.h);
  float lo = __fmaf_rn(x1.h, y1.h, -p1);
  lo = __fadd_rn(lo, __fmaf_rn(sg * x2.h, y2.h, -p2));
  float s = __fadd_rn(p1, p2);
  float bb = __fsub_rn(s, p1);
  float e = __fadd_rn(__fsub_rn(p1, __fsub_rn(s, bb)), __fsub_rn(p2, bb));
  lo = __fadd_rn(lo, e);
  lo = __fmaf_rn(x1.h, y1.l, lo);
  lo = __fmaf_rn(x1.l, y1.h, lo);
  lo = __fmaf_rn(sg * x2.h, y2.l, lo);
  lo = __fmaf_rn(sg * x2.l, y2.h, lo);
  float hh = __fadd_rn(s, lo);
  return ffloat(hh, __fsub_rn(lo, __fsub_rn(hh, s)));
}

template <> __device__ __forceinline__ ffc cmul<ffloat>(ffc a, ffc b) {
  ffc z;
  z.x = ff_dot2(a.x, b.x, a.y, b.y, true);
  z.y = ff_dot2(a.x, b.y, a.y, b.x, false);
  return z;
}

// ----------------------------------------------------------------- FFT plan
constexpr int kMaxPasses = 12;
constexpr int kMaxL = 2048;  // longest transform (N_t <= 1024); also the per-CTA FFT size

// Shared-memory slots per transform in the FFT kernels: element n sits at slot n + n / 8
// (a padding slot after every 8 elements), and the count is 1 modulo 8 so that the
// transforms of one CTA start in different banks.
__host__ __device__ constexpr int fft_slots(int L) {
  return (L + (L >> 3) + 1) + ((9 - ((L + (L >> 3) + 1) & 7)) & 7);
}

struct FftPlan {
  int L = 0;              // transform length (2 N_t)
  int npass = 0;
  int radix[kMaxPasses];  // radices in pass order (8, 4, 2, 7, 5, 3)
  int P = 1;              // complex transforms per CTA (2 P real columns)
  double2* tw64 = nullptr;  // e^{-2 pi i n / L}, n < L (device)
  float2* tw32 = nullptr;
  ffc* twff = nullptr;      // the same table as double-FP32 pairs
};

bool fft_plan_make(FftPlan& p, int L);   // host: factor L, choose P; false if unsupported
void fft_plan_free(FftPlan& p);          // host: release the twiddle tables (null entries are skipped)
// The same factorisation without the twiddle tables (tw64 / tw32 left null for the caller to set).
bool fft_plan_factor(FftPlan& p, int L);

// Kernel launchers (fft.cu).  All act on "columns".  Forward: element (t, c) of the
// real input sits at x[t * ld + c] and spectrum element (w, c) is written to
// X[w * ncols + c].  Inverse: spectrum element (w, c) at X[w * ld + c], output
// element (t, c) at y[t * ld + c].  Batch b offsets by the b-strides.
template <typename T, typename TI, typename TO>
void launch_rfft_cols(const FftPlan& p, int Nt, const TI* x, int64_t ld, int64_t x_bstride,
                      C2<TO>* X, int64_t X_bstride, int64_t ncols, int64_t B, cudaStream_t s);
// Inverse: spectrum stored as C2<TYI>, arithmetic in T, output TO.
// ostride > 1 keeps only rows t = ostride (k + 1) - 1, written as row k (N_t / ostride rows).
template <typename T, typename TYI, typename TO>
void launch_irfft_cols(const FftPlan& p, int Nt, const C2<TYI>* X, int64_t ld, int64_t X_bstride,
                       TO* y, int64_t y_bstride, int64_t ncols, int64_t B, double scale, cudaStream_t s,
                       int ostride = 1);

// Spectral block products (spectral.cu).
// Forward: dhat[b][w][i] = sum_j Fhat[w][i][j] mhat[b][w][j]  (T compute, TS storage)
// jc: columns per CTA (0 = tier default; else a multiple of 256, >= 512), the tuning knob.
// A CTA takes fwd_group(B) right-hand sides and stages their m-hat chunk in shared memory;
// a jc whose chunk would exceed kFwdSmemMax falls back to the tier default.
inline int fwd_group(int64_t B) { return B >= 4 ? 4 : 1; }
constexpr size_t kFwdSmemMax = 96 * 1024;
template <typename T, typename TS>
void launch_prod_fwd(const C2<TS>* Fhat, const C2<T>* mhat, C2<T>* partial,
                     int64_t nf, int64_t R, int64_t Nm, int64_t B, cudaStream_t s, int jc = 0);
// dhat[b][w][i] = sum over the forward product's chunk partials (fixed order); jc as above
template <typename T>
void launch_reduce_chunks(const C2<T>* partial, C2<T>* dhat, int64_t nf, int64_t R, int64_t Nm,
                          int64_t B, cudaStream_t s, int jc = 0);
size_t prod_fwd_partial_elems(int64_t nf, int64_t R, int64_t Nm, int64_t B);
// Double-FP32 tier: spectral blocks as (re_hi, re_lo, im_hi, im_lo) float quads.
// in place, from complex FP64 scaled by 2^-pexp
void launch_split_df64(void* hat, int64_t n, int pexp, cudaStream_t s);
// *out = bit pattern of max |x[i]| (a non-negative double; a NaN input reads as a NaN)
void launch_max_abs(const double* x, int64_t n, unsigned long long* out, cudaStream_t s);
// The tier's vector spectra are float quads too (the pair FFTs' format): mhat and dhat below.
// Forward partials stay complex FP64, summed in FP64 by launch_reduce_chunks_df64, which stores
// each sum as a float quad.
void launch_prod_fwd_df64(const float4* Fhat, const float4* mhat, double2* partial, int64_t nf,
                          int64_t R, int64_t Nm, int64_t B, cudaStream_t s, int jc = 0);
void launch_reduce_chunks_df64(const double2* partial, float4* dhat, int64_t nf, int64_t R, int64_t Nm,
                               int64_t B, cudaStream_t s, int jc = 0);
void launch_prod_adj_df64(const float4* Fhat, const float4* dhat, float4* mhat, int64_t nf, int64_t R,
                          int64_t Nm, int64_t B, cudaStream_t s, int vpt = 0);
// FP16 tier: spectral blocks as FP16 complex pairs with one FP32 power-of-two scale per row.
// src [nf][rn][Nm] FP64 spectrum of rows i0 .. i0 + rn -> rows (w, i0 + r) of dst [nf][R][Nm]
void launch_quantize_f16(const double2* src, void* dst, float* scale, int64_t nf, int64_t rn, int64_t R,
                         int64_t i0, int64_t Nm, cudaStream_t s);
void launch_prod_fwd_f16(const void* Fhat, const float* scale, const float2* mhat, float2* partial, int64_t nf,
                         int64_t R, int64_t Nm, int64_t B, cudaStream_t s, int jc = 0);
void launch_prod_adj_f16(const void* Fhat, const float* scale, const float2* dhat, float2* mhat, int64_t nf,
                         int64_t R, int64_t Nm, int64_t B, cudaStream_t s, int vpt = 0);
// Adjoint: mhat[b][w][j] = sum_i conj(Fhat[w][i][j]) dhat[b][w][i]
// vpt: columns per thread for single-vector calls (2, 4, 8; 0 = default)
template <typename T, typename TS>
void launch_prod_adj(const C2<TS>* Fhat, const C2<T>* dhat, C2<T>* mhat,
                     int64_t nf, int64_t R, int64_t Nm, int64_t B, cudaStream_t s, int vpt = 0);

// Dense FP64 (dense.cu)
// C[b] = alpha * A[b] * op(B[b]) + beta * C[b]; A is M x K (lda), op(B) is K x N:
// TRANSB=false: B stored K x N (ldb); TRANSB=true: B stored N x K (ldb).
// lower_only: skip output tiles strictly above the diagonal (row tile < col tile).
// Each dense launcher returns the number of kernels it launched.
int gemm_f64(bool transB, int64_t M, int64_t N, int64_t K, double alpha, const double* A,
             int64_t lda, int64_t sA, const double* Bm, int64_t ldb, int64_t sB, double beta,
             double* C, int64_t ldc, int64_t sC, int64_t batch, bool lower_only, cudaStream_t s);
// Same contract as gemm_f64, computed in double-FP32 arithmetic on the FP32 pipes.
int gemm_df64(bool transB, int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t lda,
              int64_t sA, const double* Bm, int64_t ldb, int64_t sB, double beta, double* C, int64_t ldc,
              int64_t sC, int64_t batch, bool lower_only, cudaStream_t s);
// X[r][e] *= W[e] for nrows rows of ne entries (the elliptic prior's spectral weights)
int scale_blocks(double* X, const double* W, int64_t ne, int64_t nrows, cudaStream_t s);
int k_diag_cumsum(double* WK, int64_t Nt, int64_t R, double sigma2, const double* diag,
                  cudaStream_t s);
// Blocked Cholesky, lower, in place; Linv receives the inverses of the diagonal blocks
// ([nblk][nb][nb]); status receives the first failing 1-based pivot (0 if none).
// dd: run the panel and trailing-update GEMMs in double-FP32 arithmetic (FP32 pipes)
int64_t cholesky_f64(double* A, int64_t n, double* Linv, double* work, int* status, cudaStream_t s,
                     bool dd = false);
constexpr int kCholNB = 64;
// X [B][n] rows: X := L^{-1} X (forward) then L^{-T} X (backward), in place.
int64_t trsm_lower_f64(const double* Lm, const double* Linv, int64_t n, double* X, int64_t B,
                       double* work, const int* status, cudaStream_t s, bool dd = false);
size_t trsm_work_elems(int64_t n, int64_t B);
// Explicit inverse for the online solve: Kinv [n][kinv_ld(n)] float pairs (hi, lo) of K^{-1}
// (zero padding); X [B][n] = rows K^{-1} D[b] for D [B][n] (X != D); work of
// kinv_apply_work_elems(n, B) doubles.  split_to_pairs: FP64 X [n][n] -> pairs Y [n][ldk].
int64_t kinv_ld(int64_t n);
size_t kinv_apply_work_elems(int64_t n, int64_t B);
int64_t kinv_apply(const float2* Kinv, int64_t n, const double* D, int64_t B, double* X, double* work,
                   cudaStream_t s);
int split_to_pairs(const double* X, float2* Y, int64_t n, int64_t ldk, cudaStream_t s);
// rows x n FP64 (row stride ldx) -> float pairs [rows][ldk], zeros in columns n .. ldk-1
int split_rows_to_pairs_ld(const double* X, int64_t ldx, float2* Y, int64_t rows, int64_t n, int64_t ldk,
                           cudaStream_t s);
// Few right-hand sides (gemv.cu), float-pair arithmetic, HBM-bound:
// symv_lower_pairs: X [1][n] = A D for the symmetric n x n float-pair matrix A (row stride lda,
// a multiple of 16, zeros past column n) reading its lower triangle only (B = 1; returns 0
// launches otherwise); work of symv_pairs_work_elems(n, 1) doubles.  gemv_pairs: Y [B][ldy] =
// A D[b] for a rows x cols float-pair matrix (row stride lda, a multiple of 4, zeros past column
// cols), B = 1 or 2 (0 launches otherwise); work of gemv_pairs_work_elems(cols, B) doubles.
int64_t symv_pairs_ldx(int64_t n);
size_t symv_pairs_work_elems(int64_t n, int64_t B);
int64_t symv_lower_pairs(const float2* A, int64_t lda, int64_t n, const double* D, int64_t B, double* X,
                         double* work, cudaStream_t s);
size_t gemv_pairs_work_elems(int64_t cols, int64_t B);
int64_t gemv_pairs(const float2* A, int64_t lda, int64_t rows, int64_t cols, const double* D, int64_t B, double* Y,
                   int64_t ldy, double* work, cudaStream_t s);
// the same sum with partial tiles of BM rows x BR right-hand sides (both kinv paths)
int kinv_reduce(const double* part, double* X, int64_t ldx, int64_t n, int64_t nb, int BM, int BR, int64_t per,
                int64_t kpt, int span, int64_t tiles, cudaStream_t s);
// Tensor-core form (tc_digits.cu): K^{-1} as six FP16 planes of base-256 digits
// [6][kinv_tc_ld(n)]^2 with row exponents ex [kinv_tc_ld(n)] (kinv_tc_slice of the FP64 inverse),
// applied exactly per 128-column chunk.  work: kinv_tc_work_elems(n) doubles; err: the
// handle's wait-timeout word.
// one-time kernel attributes and occupancy queries, kept out of graph captures
void kinv_prepare();
void kinv_tc_prepare();
int64_t kinv_tc_ld(int64_t n);
bool kinv_tc_supported(int64_t n);
size_t kinv_tc_plane_elems(int64_t n);
size_t kinv_tc_work_elems(int64_t n);
int64_t kinv_tc_slice(const double* X, int64_t ldx, int64_t rows, int64_t n, int* ex, void* planes,
                      int64_t rows_pad, cudaStream_t s);
// planes (4 to 6, every product here): how many of the six digit planes of each operand the
// product uses, most significant first (8 planes - 1 bits); 6 keeps the 47-bit image.
cudaError_t kinv_apply_tc(const void* planes, const int* ea, int64_t n, const double* D, int64_t B, double* X,
                          double* work, int* err, cudaStream_t s, int64_t* launches, int drop_stage = -1,
                          int nplanes = 6);
// The same for any row-major M x n matrix (planes of kinv_tc_slice with rows_pad =
// kinv_tc_ld(M)): X [B][ldx] rows = matrix D[b] (the d2q map Q of Eq. (4.14)).
size_t rowmat_tc_plane_elems(int64_t M, int64_t n);
size_t rowmat_tc_work_elems(int64_t M, int64_t n);
cudaError_t rowmat_apply_tc(const void* planes, const int* ea, int64_t M, int64_t n, const double* D, int64_t B,
                            double* X, int64_t ldx, double* work, int* err, cudaStream_t s, int64_t* launches,
                            int drop_stage = -1, int nplanes = 6);
// C -= X X[0:w]^T on and below the diagonal (C row stride ldc, the first w <= m columns), X
// m x kdim given by its planes (kinv_tc_slice, rows_pad = kinv_tc_ld(m)) and row exponents ex:
// the tensor-core updates of cholesky_tc.
cudaError_t syrk_lower_tc(const void* planes, const int* ex, int64_t m, int64_t w, int64_t kdim, double* C,
                          int64_t ldc, int* err, cudaStream_t s, int64_t* launches, int drop_stage = -1);
// Digit planes of the transpose of a rows x cols block of X (row stride ldx): planes row c = column
// c of X, K = rows; rows_pad >= kinv_tc_ld(cols); colmax: cols scratch words.  Three launches.
int64_t kinv_tc_slice_t(const double* X, int64_t ldx, int64_t rows, int64_t cols, int* ex, void* planes,
                        int64_t rows_pad, unsigned long long* colmax, cudaStream_t s);
// C (op)= A B^T for A (M x K) and B (N x K) given by digit planes and row exponents, over tiles
// of 128 rows x 64 columns; lower: only the tiles and entries on and below the diagonal (N <= M).
// op: 0 C = v, 1 C -= v, 2 C = -v.  kfirst / klast skip chunks of 128 along K that triangular
// operands make zero: kfirst 1 starts row tile I at chunk I (A K-major upper triangular, row i
// zero for k < i), 2 starts column tile J at chunk floor(64 J / 128) (B K-major upper
// triangular); klast 1 ends row tile I at chunk I (A lower triangular, row i zero for k > i).
// skip_on_err: do nothing if *err is already set (a chain of products after a timeout).  Npad:
// B's padded row count if its planes were formed for more rows than N (0: kinv_tc_ld(N)).
struct DigitGemm {
  double* C;
  int64_t ldc, M, N, K;
  int64_t Npad;
  bool lower;
  int op, kfirst, klast;
  bool skip_on_err;
};
cudaError_t digit_gemm_tc(const void* pa, const int* ea, const void* pb, const int* eb, const DigitGemm& g, int* err,
                          cudaStream_t s, int64_t* launches, int drop_stage = -1);
// W = L^{-1} for the n x n lower-triangular factor L (row stride n; the inverses of its 64 x 64
// diagonal blocks in Linv), on the tensor cores by recursive halves (cholesky_tc's planes).
// W: n x n, zero above the diagonal.  Work: T (h x h doubles), planes pa / pb (each
// lower_inverse_tc_plane_elems(n) halves), exponents ea / eb and colmax (kinv_tc_ld(h) each),
// h = lower_inverse_tc_half(n).
int64_t lower_inverse_tc_half(int64_t n);
size_t lower_inverse_tc_plane_elems(int64_t n);
int64_t lower_inverse_tc(const double* L, const double* Linv, int64_t n, double* W, double* T, void* pa, int* ea,
                         void* pb, int* eb, unsigned long long* colmax, int* err, cudaStream_t s, cudaError_t* cerr,
                         int drop_stage = -1);
// Mirror the lower triangle of the n x n matrix X (row stride n) into its upper triangle.
int symmetrize_lower(double* X, int64_t n, cudaStream_t s);
// Blocked Cholesky with panels of P columns (a multiple of 64), each panel factored
// recursively: its left half, then the update of its right half on the tensor cores, then the
// right half; 64-column leaves take the FP64 diagonal block and the double-FP32 solve of the
// rows below it.  The trailing update of each panel runs on the tensor cores too
// (syrk_lower_tc).  Same outputs as cholesky_f64 (L in place, Linv of the 64 x 64 diagonal
// blocks, status).  work: n x 64 doubles; planes / ex: cholesky_tc_plane_elems(n, P) halves
// and kinv_tc_ld(n) ints.
size_t cholesky_tc_plane_elems(int64_t n, int64_t P);
int64_t cholesky_tc(double* A, int64_t n, int64_t P, double* Linv, double* work, void* planes, int* ex,
                    int* status, int* err, cudaStream_t s, cudaError_t* cerr, int drop_stage = -1);
// Double-FP32 tier's adjoint product for B >= 16 on the tensor cores (tc_digits.cu): digit
// planes of conj(F-hat)^T, K-major over (i, re/im), one exponent per (w, j); built once from
// the float-quad blocks.  adj_digits_apply: dhat [B][nf][R], mhat [B][nf][N_m] float-quad
// spectra; work of adj_digits_work_bytes bytes.
size_t adj_digits_plane_elems(int64_t nf, int64_t R, int64_t Nm);
size_t adj_digits_exp_elems(int64_t nf, int64_t Nm);
bool adj_digits_supported(int64_t nf, int64_t R, int64_t Nm, int64_t B);
void adj_digits_prepare();
int64_t adj_digits_build(const void* hat, int64_t nf, int64_t R, int64_t Nm, void* planes, int* ex, cudaStream_t s);
size_t adj_digits_work_bytes(int64_t nf, int64_t R, int64_t B);
// Forward products of the same tier for B >= 16 (tc_digits.cu): planes of F-hat K-major over
// (j, re/im), one exponent per (w, i); mhat [B][nf][N_m] -> dhat [B][nf][R] float-quad spectra.
size_t fwd_digits_plane_elems(int64_t nf, int64_t R, int64_t Nm);
size_t fwd_digits_exp_elems(int64_t nf, int64_t R);
bool fwd_digits_supported(int64_t nf, int64_t R, int64_t Nm, int64_t B);
int64_t fwd_digits_build(const void* hat, int64_t nf, int64_t R, int64_t Nm, void* planes, int* ex, cudaStream_t s);
size_t fwd_digits_work_bytes(int64_t nf, int64_t R, int64_t Nm);
cudaError_t fwd_digits_apply(const void* planes, const int* ex, int64_t nf, int64_t R, int64_t Nm, const void* mhat,
                             void* dhat, int64_t B, void* work, int* err, cudaStream_t s, int* launches,
                             int drop_stage = -1, int nplanes = 6);
cudaError_t adj_digits_apply(const void* planes, const int* ea, int64_t nf, int64_t R, int64_t Nm, const void* dhat,
                             void* mhat, int64_t B, void* work, int* err, cudaStream_t s, int* launches,
                             int drop_stage = -1, int nplanes = 6);
int axpby_f64(double* y, const double* x, double a, double b, int64_t n, cudaStream_t s);
// FP32 Gram product W = A B^T into an FP64 matrix (lower tiles) and the FP64 -> FP32 copy
int sgemm_nt_lower_to_f64(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda, const float* Bm,
                          int64_t ldb, double* C, int64_t ldc, cudaStream_t s);
int convert_f64_to_f32(const double* x, float* y, int64_t n, cudaStream_t s);
// out = (alpha1 I - alpha2 Delta_h) m for nblocks grids of gx x gy (5-point, Neumann)
int elliptic_apply(const double* m, double* out, int gx, int gy, double a1, double a2, int64_t nblocks,
                   cudaStream_t s);
// out[k1 R + i][k2 R + j] = in[(s (k1+1) - 1) R + i][(s (k2+1) - 1) R + j]: rows and columns at
// every s-th time block of an (Nt R)^2 matrix (ld Nt R); out is (Nt/s R)^2.
int select_time_blocks_sq(const double* in, double* out, int64_t Nt, int64_t R, int s, cudaStream_t st);
// Block-diagonal prefix sums on both sides of the diagonal (block-Toeplitz product A B^*).
int block_diag_cumsum_all(double* X, int64_t Nt, int64_t R1, int64_t R2, cudaStream_t s);
int noise_residual_f64(double* r, const double* x, const double* diag, int64_t n, int64_t B,
                       cudaStream_t s);

// Tensor-core FP16-tier forward product (tc_f16.cu): for B >= 8 right-hand sides and N_m a
// multiple of 4.  Writes per-chunk partials into `partial` (tc_fwd_partial_elems elements)
// and their fixed-order sum into dhat [B][nf][R]; err is set when a bounded device wait
// gave up.  *launches receives the number of kernels launched.
bool tc_fwd_f16_supported(int64_t Nm, int64_t R, int64_t B);
size_t tc_fwd_partial_elems(int64_t nf, int64_t R, int64_t Nm, int64_t B);
// drop_stage >= 0 (test hook): the producer withholds that stage's tile, so the kernel's bounded
// waits run out and it reports through err.
cudaError_t launch_prod_fwd_f16_tc(const void* Fhat, const float* scale, const float2* mhat, float2* partial,
                                   float2* dhat, int64_t nf, int64_t R, int64_t Nm, int64_t B, int* err,
                                   cudaStream_t s, int* launches, int drop_stage = -1);
// Adjoint: mhat [B][nf][N_m] = F-hat^H (scale-folded dhat) for B >= 8 and N_d up to 2048 (16
// vectors per group) or 1024 (32 per group); no partials.
bool tc_adj_f16_supported(int64_t Nm, int64_t R, int64_t B);
cudaError_t launch_prod_adj_f16_tc(const void* Fhat, const float* scale, const float2* dhat, float2* mhat,
                                   int64_t nf, int64_t R, int64_t Nm, int64_t B, int* err, cudaStream_t s,
                                   int* launches);

// Probe estimate of pointwise variances (krylov.cu): num/den accumulate sum_k V[k] U[k] and
// sum_k V[k]^2 elementwise over nb probes [nb][n]; out = num / den (0 where den = 0).
int probe_accumulate(const double* V, const double* U, int64_t nb, int64_t n, double* num, double* den,
                     cudaStream_t s);
int probe_finish(const double* num, const double* den, double* out, int64_t n, cudaStream_t s);
// Krylov vector kernels (krylov.cu); vectors [B][n], per-vector scalars on the device.
// out[b] = x[b] . y[b] in FP64 with a fixed reduction order; part holds
// dot_workspace_elems(B) doubles.
size_t dot_workspace_elems(int64_t B);
template <typename T>
int dot_batched(const T* x, const T* y, int64_t n, int64_t B, double* part, double* out, cudaStream_t s);
// x += (rr / pq) p and r -= (rr / pq) q per vector (no step where pq <= 0 or rr <= 0)
template <typename T>
int cg_update_xr(T* x, T* r, const T* p, const T* q, const double* rr, const double* pq, int64_t n, int64_t B,
                 cudaStream_t s);
// p = r + (rr_new / rr_old) p per vector
template <typename T>
int cg_update_p(T* p, const T* r, const double* rr_new, const double* rr_old, int64_t n, int64_t B, cudaStream_t s);
// q = y + Gamma_noise p (diag[i] per datum, else sigma2); q may alias y
template <typename T>
int add_noise(T* q, const T* y, const T* p, const double* diag, double sigma2, int64_t n, int64_t B, cudaStream_t s);
// out = float(x / sqrt(nrm2)) and x += sqrt(nrm2) * d (the scaled hand-over between an FP64
// refinement loop and an FP32 inner solve)
int normalize_to_f32(const double* x, const double* nrm2, float* out, int64_t n, int64_t B, cudaStream_t s);
int add_scaled_f32(double* x, const float* d, const double* nrm2, int64_t n, int64_t B, cudaStream_t s);
// z [B][N_t][R] = blockdiag(P[t]) r with P [N_t][R][R] (FP64), r and z in T (float or double)
template <typename T>
int block_precond_apply(const double* P, const T* r, T* z, int64_t Nt, int64_t R, int64_t B, cudaStream_t s);
int convert_f32_f64(const float* x, double* y, int64_t n, cudaStream_t s);
int convert_f64_f32(const double* x, float* y, int64_t n, cudaStream_t s);
// Time-diagonal blocks of K for the block-Jacobi preconditioner (dense.cu): W [Nt][R][R] holds
// F_k G_k^T on entry and Gamma_noise(t) + sum_{k <= t} F_k G_k^T on exit; identity fill.
int diag_block_cumsum(double* W, int64_t Nt, int64_t R, double sigma2, const double* diag, cudaStream_t s);
int identity_blocks(double* X, int64_t nb, int64_t R, cudaStream_t s);

}  // namespace bti
