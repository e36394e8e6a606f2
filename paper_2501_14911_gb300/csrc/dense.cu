// Dense FP64 kernels of the data-space solve: the Gram product and block-
// diagonal accumulation that assemble K = Gamma_noise + F G^* (Sec. 4,
// Phase 2), the blocked Cholesky factorisation of K, the triangular solves of
// the online phase (Eq. (4.13)), and the separable SE prior used to form the
// G blocks.
#include "bti_internal.cuh"

#include <algorithm>

namespace bti {

// 0: choose the GEMM tile by grid size; 16 / 32 / 64: force that tile (tuning hook).
int g_gemm_tile_override = 0;

static int num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

// ------------------------------------------------------------------ GEMM (FP64)
// BM x BN output tile per CTA, k-step 16, 256 threads each owning a TM x TN
// sub-tile at rows ty + (BM/TM) a and columns tx + (BN/TN) b (conflict-free smem
// reads).  Three shapes: 64x64 (4x4 per thread) for large products, 32x32 (2x2)
// and 16x16 (1x1) so that small outputs still spread over many SMs.
constexpr int GBK = 16;

template <bool TRANSB, int BM, int BN>
__global__ void __launch_bounds__(256)
gemm_f64_kernel(int64_t M, int64_t N, int64_t K, double alpha, const double* __restrict__ A,
                int64_t lda, int64_t sA, const double* __restrict__ Bm, int64_t ldb, int64_t sB,
                double beta, double* __restrict__ C, int64_t ldc, int64_t sC, int64_t batch,
                bool lower_only) {
  constexpr int TM = BM / 16, TN = BN / 16;
  __shared__ double As[GBK][BM + 1];
  __shared__ double Bs[GBK][BN + 1];
  const int64_t m0 = (int64_t)blockIdx.x * BM;
  const int64_t n0 = (int64_t)blockIdx.y * BN;
  if (lower_only && m0 + BM - 1 < n0) return;  // tile strictly above the diagonal
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int64_t bz = blockIdx.z; bz < batch; bz += gridDim.z) {
    const double* Ab = A + bz * sA;
    const double* Bb = Bm + bz * sB;
    double* Cb = C + bz * sC;
    double acc[TM][TN];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TN; ++b) acc[a][b] = 0.0;
    for (int64_t k0 = 0; k0 < K; k0 += GBK) {
      // A tile: BM rows x 16 k, element (r, c) at A[m0 + r][k0 + c]
#pragma unroll
      for (int e = 0; e < (BM * GBK) / 256; ++e) {
        int idx = threadIdx.x + 256 * e;
        int r = idx >> 4, c = idx & 15;
        int64_t gm = m0 + r, gk = k0 + c;
        As[c][r] = (gm < M && gk < K) ? Ab[gm * lda + gk] : 0.0;
      }
      if (TRANSB) {
#pragma unroll
        for (int e = 0; e < (BN * GBK) / 256; ++e) {
          int idx = threadIdx.x + 256 * e;
          int r = idx >> 4, c = idx & 15;
          int64_t gn = n0 + r, gk = k0 + c;
          Bs[c][r] = (gn < N && gk < K) ? Bb[gn * ldb + gk] : 0.0;
        }
      } else {
#pragma unroll
        for (int e = 0; e < (BN * GBK) / 256; ++e) {
          int idx = threadIdx.x + 256 * e;
          int r = idx / BN, c = idx % BN;
          int64_t gk = k0 + r, gn = n0 + c;
          Bs[r][c] = (gn < N && gk < K) ? Bb[gk * ldb + gn] : 0.0;
        }
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < GBK; ++kk) {
        double av[TM], bv[TN];
#pragma unroll
        for (int a = 0; a < TM; ++a) av[a] = As[kk][ty + 16 * a];
#pragma unroll
        for (int b = 0; b < TN; ++b) bv[b] = Bs[kk][tx + 16 * b];
#pragma unroll
        for (int a = 0; a < TM; ++a)
#pragma unroll
          for (int b = 0; b < TN; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < TM; ++a) {
      int64_t gm = m0 + ty + 16 * a;
      if (gm >= M) continue;
#pragma unroll
      for (int b = 0; b < TN; ++b) {
        int64_t gn = n0 + tx + 16 * b;
        if (gn >= N) continue;
        double* cp = Cb + gm * ldc + gn;
        double v = alpha * acc[a][b];
        if (beta != 0.0) v = fma(beta, *cp, v);
        *cp = v;
      }
    }
  }
}

// ------------------------------------------------------------------ GEMM (double-FP32)
// Same interface and tiling as gemm_f64_kernel, for GB300 where FP64 issues at 1/64
// of the FP32 rate: operand tiles are split on load into float pairs hi + lo (one
// FP64 subtraction per loaded element, reused BM or BN times), products are formed
// exactly in float pairs (FMA error of hi*hi plus the two cross terms) and summed
// with Knuth's two-sum, and the epilogue applies alpha and beta in FP64.  About 48
// significant bits per operation: FP64-level results for the Gram product, the
// Cholesky updates and the triangular solves.
namespace {
__device__ __forceinline__ void dd_split(double x, float& h, float& l) {
  h = __double2float_rn(x);
  l = __double2float_rn(x - (double)h);
}
__device__ __forceinline__ void dd_mac(float& Sh, float& Sl, float ah, float al, float bh, float bl) {
  float p = __fmul_rn(ah, bh);
  float pe = __fmaf_rn(ah, bh, -p);
  pe = __fmaf_rn(ah, bl, pe);
  pe = __fmaf_rn(al, bh, pe);
  float s = __fadd_rn(Sh, p);
  float bb = __fsub_rn(s, Sh);
  float e = __fadd_rn(__fsub_rn(Sh, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  Sh = s;
  Sl = __fadd_rn(Sl, __fadd_rn(e, pe));
}
}  // namespace

template <bool TRANSB, int BM, int BN>
__global__ void __launch_bounds__(256)
gemm_df64_kernel(int64_t M, int64_t N, int64_t K, double alpha, const double* __restrict__ A,
                 int64_t lda, int64_t sA, const double* __restrict__ Bm, int64_t ldb, int64_t sB,
                 double beta, double* __restrict__ C, int64_t ldc, int64_t sC, int64_t batch,
                 bool lower_only) {
  constexpr int TM = BM / 16, TN = BN / 16;
  __shared__ float2 As[GBK][BM + 1];  // (hi, lo)
  __shared__ float2 Bs[GBK][BN + 1];
  const int64_t m0 = (int64_t)blockIdx.x * BM;
  const int64_t n0 = (int64_t)blockIdx.y * BN;
  if (lower_only && m0 + BM - 1 < n0) return;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int64_t bz = blockIdx.z; bz < batch; bz += gridDim.z) {
    const double* Ab = A + bz * sA;
    const double* Bb = Bm + bz * sB;
    double* Cb = C + bz * sC;
    float ah_[TM][TN], al_[TM][TN];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TN; ++b) ah_[a][b] = al_[a][b] = 0.f;
    for (int64_t k0 = 0; k0 < K; k0 += GBK) {
#pragma unroll
      for (int e = 0; e < (BM * GBK) / 256; ++e) {
        int idx = threadIdx.x + 256 * e;
        int r = idx >> 4, c = idx & 15;
        int64_t gm = m0 + r, gk = k0 + c;
        double v = (gm < M && gk < K) ? Ab[gm * lda + gk] : 0.0;
        float h, l;
        dd_split(v, h, l);
        As[c][r] = make_float2(h, l);
      }
      if (TRANSB) {
#pragma unroll
        for (int e = 0; e < (BN * GBK) / 256; ++e) {
          int idx = threadIdx.x + 256 * e;
          int r = idx >> 4, c = idx & 15;
          int64_t gn = n0 + r, gk = k0 + c;
          double v = (gn < N && gk < K) ? Bb[gn * ldb + gk] : 0.0;
          float h, l;
          dd_split(v, h, l);
          Bs[c][r] = make_float2(h, l);
        }
      } else {
#pragma unroll
        for (int e = 0; e < (BN * GBK) / 256; ++e) {
          int idx = threadIdx.x + 256 * e;
          int r = idx / BN, c = idx % BN;
          int64_t gk = k0 + r, gn = n0 + c;
          double v = (gn < N && gk < K) ? Bb[gk * ldb + gn] : 0.0;
          float h, l;
          dd_split(v, h, l);
          Bs[r][c] = make_float2(h, l);
        }
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < GBK; ++kk) {
        float2 av[TM], bv[TN];
#pragma unroll
        for (int a = 0; a < TM; ++a) av[a] = As[kk][ty + 16 * a];
#pragma unroll
        for (int b = 0; b < TN; ++b) bv[b] = Bs[kk][tx + 16 * b];
#pragma unroll
        for (int a = 0; a < TM; ++a)
#pragma unroll
          for (int b = 0; b < TN; ++b) dd_mac(ah_[a][b], al_[a][b], av[a].x, av[a].y, bv[b].x, bv[b].y);
      }
      __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < TM; ++a) {
      int64_t gm = m0 + ty + 16 * a;
      if (gm >= M) continue;
#pragma unroll
      for (int b = 0; b < TN; ++b) {
        int64_t gn = n0 + tx + 16 * b;
        if (gn >= N) continue;
        double* cp = Cb + gm * ldc + gn;
        double v = alpha * ((double)ah_[a][b] + (double)al_[a][b]);
        if (beta != 0.0) v = fma(beta, *cp, v);
        *cp = v;
      }
    }
  }
}

int gemm_df64(bool transB, int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t lda,
              int64_t sA, const double* Bm, int64_t ldb, int64_t sB, double beta, double* C, int64_t ldc,
              int64_t sC, int64_t batch, bool lower_only, cudaStream_t s) {
  if (M <= 0 || N <= 0 || batch <= 0) return 0;
  int tile = 16;
  {
    const int64_t want = 2 * (int64_t)num_sms();
    for (int t : {64, 32}) {
      if (((M + t - 1) / t) * ((N + t - 1) / t) * std::min<int64_t>(batch, 65535) >= want) {
        tile = t;
        break;
      }
    }
  }
  const unsigned gz = (unsigned)std::min<int64_t>(batch, 65535);
#define BTI_DF_LAUNCH(T_)                                                                                    \
  {                                                                                                          \
    dim3 grid((unsigned)((M + T_ - 1) / T_), (unsigned)((N + T_ - 1) / T_), gz);                            \
    if (transB)                                                                                              \
      gemm_df64_kernel<true, T_, T_><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, sA, Bm, ldb, sB, beta, C,  \
                                                           ldc, sC, batch, lower_only);                      \
    else                                                                                                     \
      gemm_df64_kernel<false, T_, T_><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, sA, Bm, ldb, sB, beta, C, \
                                                            ldc, sC, batch, lower_only);                     \
  }
  if (tile == 64)
    BTI_DF_LAUNCH(64)
  else if (tile == 32)
    BTI_DF_LAUNCH(32)
  else
    BTI_DF_LAUNCH(16)
#undef BTI_DF_LAUNCH
  return 1;
}

// Small-M products (M <= 8 rows, e.g. a handful of right-hand sides).
// NN: C[m][n] (+)= alpha sum_k A[m][k] B[k][n]; one thread per column n.
template <int MM>
__global__ void __launch_bounds__(256)
gemm_smallm_nn_kernel(int64_t M, int64_t N, int64_t K, double alpha, const double* __restrict__ A,
                      int64_t lda, const double* __restrict__ Bm, int64_t ldb, double beta,
                      double* __restrict__ C, int64_t ldc) {
  __shared__ double As[MM][64];
  const int64_t n = (int64_t)blockIdx.x * 256 + threadIdx.x;
  double acc[MM];
#pragma unroll
  for (int m = 0; m < MM; ++m) acc[m] = 0.0;
  for (int64_t k0 = 0; k0 < K; k0 += 64) {
    for (int idx = threadIdx.x; idx < MM * 64; idx += 256) {
      int m = idx >> 6, c = idx & 63;
      As[m][c] = (m < M && k0 + c < K) ? A[m * lda + k0 + c] : 0.0;
    }
    __syncthreads();
    if (n < N) {
      int kn = (int)std::min<int64_t>(64, K - k0);
      for (int c = 0; c < kn; ++c) {
        double b = Bm[(k0 + c) * ldb + n];
#pragma unroll
        for (int m = 0; m < MM; ++m) acc[m] = fma(As[m][c], b, acc[m]);
      }
    }
    __syncthreads();
  }
  if (n < N) {
#pragma unroll
    for (int m = 0; m < MM; ++m) {
      if (m >= M) break;
      double* cp = C + m * ldc + n;
      double v = alpha * acc[m];
      if (beta != 0.0) v = fma(beta, *cp, v);
      *cp = v;
    }
  }
}

// NT: C[m][n] (+)= alpha sum_k A[m][k] B[n][k]; one warp per column n.
template <int MM>
__global__ void __launch_bounds__(256)
gemm_smallm_nt_kernel(int64_t M, int64_t N, int64_t K, double alpha, const double* __restrict__ A,
                      int64_t lda, const double* __restrict__ Bm, int64_t ldb, double beta,
                      double* __restrict__ C, int64_t ldc) {
  const int lane = threadIdx.x & 31;
  const int64_t n = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (n >= N) return;
  double acc[MM];
#pragma unroll
  for (int m = 0; m < MM; ++m) acc[m] = 0.0;
  const double* brow = Bm + n * ldb;
  for (int64_t k = lane; k < K; k += 32) {
    double b = brow[k];
#pragma unroll
    for (int m = 0; m < MM; ++m)
      if (m < M) acc[m] = fma(A[m * lda + k], b, acc[m]);
  }
#pragma unroll
  for (int m = 0; m < MM; ++m)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[m] += __shfl_xor_sync(0xffffffffu, acc[m], o);
  if (lane == 0) {
#pragma unroll
    for (int m = 0; m < MM; ++m) {
      if (m >= M) break;
      double* cp = C + m * ldc + n;
      double v = alpha * acc[m];
      if (beta != 0.0) v = fma(beta, *cp, v);
      *cp = v;
    }
  }
}

int gemm_f64(bool transB, int64_t M, int64_t N, int64_t K, double alpha, const double* A,
             int64_t lda, int64_t sA, const double* Bm, int64_t ldb, int64_t sB, double beta,
             double* C, int64_t ldc, int64_t sC, int64_t batch, bool lower_only, cudaStream_t s) {
  if (M <= 0 || N <= 0 || batch <= 0) return 0;
  if (M <= 8 && batch == 1 && !lower_only && K > 0) {
    if (transB) {
      unsigned g = (unsigned)((N + 7) / 8);
      if (M <= 1) gemm_smallm_nt_kernel<1><<<g, 256, 0, s>>>(M, N, K, alpha, A, lda, Bm, ldb, beta, C, ldc);
      else gemm_smallm_nt_kernel<8><<<g, 256, 0, s>>>(M, N, K, alpha, A, lda, Bm, ldb, beta, C, ldc);
    } else {
      unsigned g = (unsigned)((N + 255) / 256);
      if (M <= 1) gemm_smallm_nn_kernel<1><<<g, 256, 0, s>>>(M, N, K, alpha, A, lda, Bm, ldb, beta, C, ldc);
      else gemm_smallm_nn_kernel<8><<<g, 256, 0, s>>>(M, N, K, alpha, A, lda, Bm, ldb, beta, C, ldc);
    }
    return 1;
  }
  // tile shape: the largest whose grid still gives every SM work, unless overridden
  int tile = g_gemm_tile_override;
  if (tile == 0) {
    const int64_t want = 2 * (int64_t)num_sms();
    tile = 16;
    for (int t : {64, 32}) {
      if (((M + t - 1) / t) * ((N + t - 1) / t) * std::min<int64_t>(batch, 65535) >= want) {
        tile = t;
        break;
      }
    }
  }
  const unsigned gz = (unsigned)std::min<int64_t>(batch, 65535);
#define BTI_GEMM_LAUNCH(T_)                                                                                  \
  {                                                                                                          \
    dim3 grid((unsigned)((M + T_ - 1) / T_), (unsigned)((N + T_ - 1) / T_), gz);                            \
    if (transB)                                                                                              \
      gemm_f64_kernel<true, T_, T_><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, sA, Bm, ldb, sB, beta, C,   \
                                                          ldc, sC, batch, lower_only);                       \
    else                                                                                                     \
      gemm_f64_kernel<false, T_, T_><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, sA, Bm, ldb, sB, beta, C,  \
                                                           ldc, sC, batch, lower_only);                      \
  }
  if (tile == 64)
    BTI_GEMM_LAUNCH(64)
  else if (tile == 32)
    BTI_GEMM_LAUNCH(32)
  else
    BTI_GEMM_LAUNCH(16)
#undef BTI_GEMM_LAUNCH
  return 1;
}

// ------------------------------------------------------------------ prior, spectral weights
// X[r][e] *= W[e] for rows r < nrows of ne entries (the elliptic prior's DCT-domain weights)
__global__ void scale_blocks_kernel(double* X, const double* __restrict__ W, int64_t ne, int64_t total) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < total) X[i] *= W[i % ne];
}
int scale_blocks(double* X, const double* W, int64_t ne, int64_t nrows, cudaStream_t s) {
  const int64_t total = ne * nrows;
  if (total <= 0) return 0;
  scale_blocks_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(X, W, ne, total);
  return 1;
}

// ------------------------------------------------------------------ K from the Gram matrix
// On entry WK holds (at least the lower triangle of) W = F_stack G_stack^T,
// W[(k,i),(k',i')] = F_k[i,:] . G_k'[i',:].  Block (t, t') of F G^* is
// sum_{u=0}^{min(t,t')} W(t-u, t'-u), so along each block diagonal
// delta = t - t' >= 0 the blocks are prefix sums of W's blocks.  One thread per
// (delta, i, i') walks its diagonal and overwrites W with K, adding the noise
// variance on the main diagonal.
__global__ void k_diag_cumsum_kernel(double* WK, int64_t Nt, int64_t R, double sigma2,
                                     const double* __restrict__ diag) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t RR = R * R;
  if (idx >= Nt * RR) return;
  int64_t delta = idx / RR;
  int64_t rem = idx - delta * RR;
  int64_t i = rem / R, ip = rem - i * R;
  if (delta == 0 && ip > i) return;  // strict upper triangle of a diagonal block: unused
  const int64_t n = Nt * R;
  double acc = 0.0;
  for (int64_t u = 0; u + delta < Nt; ++u) {
    int64_t row = (u + delta) * R + i, col = u * R + ip;
    double* p = WK + row * n + col;
    acc += *p;
    double v = acc;
    if (delta == 0 && i == ip) v += diag ? diag[u * R + i] : sigma2;
    *p = v;
  }
}
int k_diag_cumsum(double* WK, int64_t Nt, int64_t R, double sigma2, const double* diag,
                  cudaStream_t s) {
  int64_t total = Nt * R * R;
  k_diag_cumsum_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(WK, Nt, R, sigma2, diag);
  return 1;
}

// K(t,t) for the time-diagonal blocks only: W [Nt][R][R] holds F_k G_k^T; afterwards W[t] =
// Gamma_noise(t) + sum_{k <= t} W[k] (the diagonal blocks of K, full R x R).
__global__ void diag_block_cumsum_kernel(double* W, int64_t Nt, int64_t R, double sigma2,
                                         const double* __restrict__ diag) {
  const int64_t RR = R * R;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= RR) return;
  const int64_t i = e / R, j = e - i * R;
  double acc = 0.0;
  for (int64_t t = 0; t < Nt; ++t) {
    acc += W[t * RR + e];
    W[t * RR + e] = acc + (i == j ? (diag ? diag[t * R + i] : sigma2) : 0.0);
  }
}
int diag_block_cumsum(double* W, int64_t Nt, int64_t R, double sigma2, const double* diag, cudaStream_t s) {
  const int64_t RR = R * R;
  if (RR <= 0 || Nt <= 0) return 0;
  diag_block_cumsum_kernel<<<(unsigned)((RR + 255) / 256), 256, 0, s>>>(W, Nt, R, sigma2, diag);
  return 1;
}

// X [nb][R][R] = identity in every block
__global__ void identity_blocks_kernel(double* X, int64_t total, int64_t R) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const int64_t r = e % (R * R);
  X[e] = (r / R == r % R) ? 1.0 : 0.0;
}
int identity_blocks(double* X, int64_t nb, int64_t R, cudaStream_t s) {
  const int64_t total = nb * R * R;
  if (total <= 0) return 0;
  identity_blocks_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(X, total, R);
  return 1;
}

// ------------------------------------------------------------------ Cholesky
// Factor the kb x kb diagonal block (kb <= 64) in shared memory, write L back, and write its
// inverse (lower, zeros elsewhere) to Linv (ld 64).  All in FP64; GB300 runs FP64 at about
// two FMAs per clock per SM, so the kernel keeps every step in shared memory and every thread
// busy: 64 groups of 4 threads, group g owning row g in the factorisation and column g in the
// inversion.
//
// Factorisation, right-looking, two barriers per column j: (a) column j of L goes to the
// upper triangle, S[j][i] = S[i][j] / sqrt(d_j) (i > j), where the trailing update reads it
// row-wise; (b) row i's group updates S[i][c] -= L[i][j] L[c][j] for j < c <= i, and the lane
// that updates the next diagonal entry takes its pivot d_{j+1}: sqrt into the diagonal, the
// reciprocal into rinv.  Inversion, X = L^{-1} by columns (no barriers: column c of X depends
// only on itself): X[c][c] = 1 / L[c][c], X[r][c] = -(sum_{l=c}^{r-1} L[r][l] X[l][c]) / L[r][r],
// the four lanes of a group splitting the sum; X overwrites the lower triangle.
__global__ void __launch_bounds__(256)
potrf_diag_kernel(double* A, int64_t lda, int kb, double* Linv, int* status, int64_t k0) {
  __shared__ double S[kCholNB][kCholNB + 1];
  __shared__ double rinv[kCholNB];
  __shared__ int failed;
  if (*status != 0) return;  // an earlier block already failed
  const int tid = threadIdx.x, g = tid >> 2, q = tid & 3;
  if (tid == 0) failed = 0;
  for (int idx = tid; idx < kb * kb; idx += blockDim.x) {
    const int r = idx / kb, c = idx - r * kb;
    if (c <= r) S[r][c] = A[r * lda + c];
  }
  __syncthreads();
  // The pivot d_i's square root and its reciprocal are on the critical path of every column,
  // and GB300's FP64 square root and division take long chains of FP64 instructions.  Instead:
  // d = f 4^k with f in [0.5, 2) (exact exponent arithmetic), y = 1 / sqrt(f) by the Newton-
  // Raphson iteration for the reciprocal square root, y <- y + y (1 - f y^2) / 2, seeded with
  // FP32 rsqrtf (about 23 bits) and taken twice in FP64 (the error squares each time: about
  // 2^-46, then below FP64 rounding); then 1 / sqrt(d) = y 2^-k and sqrt(d) = f y 2^k.
  auto pivot = [&](int i) {
    const double d = S[i][i];
    if (!(d > 0.0) || !isfinite(d)) {
      failed = 1;
      atomicCAS(status, 0, (int)(k0 + i + 1));
    } else {
      int e = 0;
      double f = frexp(d, &e);  // d = f 2^e, f in [0.5, 1)
      if (e & 1) {
        f *= 2.0;
        e -= 1;
      }
      double y = (double)rsqrtf((float)f);
      y = fma(0.5 * y, fma(-f * y, y, 1.0), y);
      y = fma(0.5 * y, fma(-f * y, y, 1.0), y);
      S[i][i] = ldexp(f * y, e / 2);
      rinv[i] = ldexp(y, -e / 2);
    }
  };
  if (tid == 0 && kb > 0) pivot(0);
  __syncthreads();
  for (int j = 0; j < kb; ++j) {
    if (failed) return;  // set before the last barrier: uniform
    const double rj = rinv[j];
    for (int i = j + 1 + tid; i < kb; i += blockDim.x) S[j][i] = S[i][j] * rj;
    __syncthreads();
    if (g > j && g < kb) {
      const double li = S[j][g];
      for (int c = j + 1 + q; c <= g; c += 4) S[g][c] = fma(-li, S[j][c], S[g][c]);
      if (q == 0 && g == j + 1) pivot(g);  // this lane just updated S[g][g] (c = j + 1)
    }
    __syncthreads();
  }
  // L back to memory: the diagonal, and the columns from the upper triangle
  for (int idx = tid; idx < kb * kb; idx += blockDim.x) {
    const int r = idx / kb, c = idx - r * kb;
    if (c <= r) A[r * lda + c] = (c == r) ? S[r][r] : S[c][r];
  }
  __syncthreads();
  if (g < kb) {
    const unsigned mask = 0xFu << (threadIdx.x & 28);  // the group's four lanes
    const int c = g;
    if (q == 0) S[c][c] = rinv[c];
    __syncwarp(mask);
    for (int r = c + 1; r < kb; ++r) {
      double part = 0.0;
      for (int l = c + q; l < r; l += 4) part = fma(S[l][r], S[l][c], part);
      part += __shfl_xor_sync(mask, part, 1);
      part += __shfl_xor_sync(mask, part, 2);
      if (q == 0) S[r][c] = -rinv[r] * part;
      __syncwarp(mask);
    }
  }
  __syncthreads();
  for (int idx = tid; idx < kCholNB * kCholNB; idx += blockDim.x) {
    const int r = idx / kCholNB, c = idx - r * kCholNB;
    Linv[idx] = (c <= r && r < kb) ? S[r][c] : 0.0;
  }
}

// GEMM used by the blocked factorisation and solves: FP64, or double-FP32 for products
// with more than 8 rows when dd is set (tiny ones stay on the FP64 small-M kernels).
static int gemm_sel(bool dd, bool transB, int64_t M, int64_t N, int64_t K, double alpha, const double* A,
                    int64_t lda, const double* Bm, int64_t ldb, double beta, double* C, int64_t ldc, bool lower_only,
                    cudaStream_t s) {
  if (dd && M > 8)
    return gemm_df64(transB, M, N, K, alpha, A, lda, 0, Bm, ldb, 0, beta, C, ldc, 0, 1, lower_only, s);
  return gemm_f64(transB, M, N, K, alpha, A, lda, 0, Bm, ldb, 0, beta, C, ldc, 0, 1, lower_only, s);
}

int64_t cholesky_f64(double* A, int64_t n, double* Linv, double* work, int* status, cudaStream_t s, bool dd) {
  const int nb = kCholNB;
  int64_t launches = 0;
  for (int64_t k = 0; k < n; k += nb) {
    int kb = (int)std::min<int64_t>(nb, n - k);
    double* Lk = Linv + (k / nb) * nb * nb;
    potrf_diag_kernel<<<1, 256, 0, s>>>(A + k * n + k, n, kb, Lk, status, k);
    launches += 1;
    int64_t m = n - k - kb;
    if (m <= 0) continue;
    // panel: P = A[k+kb:, k:k+kb] L_kk^{-T}
    launches += gemm_sel(dd, true, m, kb, kb, 1.0, A + (k + kb) * n + k, n, Lk, nb, 0.0, work, kb, false, s);
    cudaMemcpy2DAsync(A + (k + kb) * n + k, n * sizeof(double), work, kb * sizeof(double),
                      kb * sizeof(double), m, cudaMemcpyDeviceToDevice, s);
    // trailing update of the lower triangle: A22 -= P P^T
    launches += gemm_sel(dd, true, m, m, kb, -1.0, work, kb, work, kb, 1.0, A + (k + kb) * n + (k + kb), n, true,
                         s);
  }
  return launches;
}

// The same factorisation with wide panels, so that nearly all of its n^3 / 3 flop runs on the
// tensor cores.  Panel K0 .. K0 + P - 1 (all rows below K0) is factored recursively: its left
// half, then the update of its right half by the left half's columns, then its right half.  The
// 64-column leaves are the steps above (the FP64 diagonal block, the double-FP32 solve of the
// rows below it); every update is a digit-plane product on the tensor cores, lower trapezoid
// only, subtracted in place (syrk_lower_tc): within a panel, then the trailing matrix's
// A22 -= L21 L21^T once per panel.  The planes are 47-bit images of the rows of L.
namespace {
struct CholTc {
  double* A;
  int64_t n;
  double* Linv;
  double* work;
  void* planes;
  int* ex;
  int* status;
  int* err;
  cudaStream_t s;
  int drop_stage;
  int64_t launches = 0;
  cudaError_t cerr = cudaSuccess;
};

// C = A[r0:n, r0:r0 + w] -= X X[0:w]^T (lower), X = A[r0:n, c0:r0] (m = n - r0 rows)
void chol_update_tc(CholTc& c, int64_t c0, int64_t r0, int64_t w) {
  const int64_t m = c.n - r0, kdim = r0 - c0;
  if (m <= 0 || w <= 0 || c.cerr != cudaSuccess) return;
  c.launches += kinv_tc_slice(c.A + r0 * c.n + c0, c.n, m, kdim, c.ex, c.planes, kinv_tc_ld(m), c.s);
  int64_t tl = 0;
  c.cerr = syrk_lower_tc(c.planes, c.ex, m, w, kdim, c.A + r0 * c.n + r0, c.n, c.err, c.s, &tl, c.drop_stage);
  c.launches += tl;
}

// columns c0 .. c0 + width - 1 for rows c0 .. n - 1, those columns up to date
void chol_panel_tc(CholTc& c, int64_t c0, int64_t width) {
  if (c.cerr != cudaSuccess) return;
  const int nb = kCholNB;
  if (width <= nb) {
    const int kb = (int)width;
    double* Lk = c.Linv + (c0 / nb) * nb * nb;
    potrf_diag_kernel<<<1, 256, 0, c.s>>>(c.A + c0 * c.n + c0, c.n, kb, Lk, c.status, c0);
    c.launches += 1;
    const int64_t m = c.n - c0 - kb;
    if (m <= 0) return;
    // rows below the diagonal block: A[c0+kb:, c0:c0+kb] L_kk^{-T}
    c.launches += gemm_sel(true, true, m, kb, kb, 1.0, c.A + (c0 + kb) * c.n + c0, c.n, Lk, nb, 0.0, c.work, kb,
                           false, c.s);
    cudaMemcpy2DAsync(c.A + (c0 + kb) * c.n + c0, c.n * sizeof(double), c.work, kb * sizeof(double),
                      kb * sizeof(double), m, cudaMemcpyDeviceToDevice, c.s);
    return;
  }
  const int64_t h = (width / 2 + nb - 1) / nb * nb;  // a multiple of 64 below width
  chol_panel_tc(c, c0, h);
  chol_update_tc(c, c0, c0 + h, width - h);
  chol_panel_tc(c, c0 + h, width - h);
}
}  // namespace

size_t cholesky_tc_plane_elems(int64_t n, int64_t P) {
  const int64_t w = P < n ? P : n;
  return (size_t)6 * kinv_tc_ld(n) * kinv_tc_ld(w);
}

int64_t cholesky_tc(double* A, int64_t n, int64_t P, double* Linv, double* work, void* planes, int* ex,
                    int* status, int* err, cudaStream_t s, cudaError_t* cerr, int drop_stage) {
  CholTc c{A, n, Linv, work, planes, ex, status, err, s, drop_stage};
  for (int64_t K0 = 0; K0 < n && c.cerr == cudaSuccess; K0 += P) {
    const int64_t pend = std::min<int64_t>(K0 + P, n);
    chol_panel_tc(c, K0, pend - K0);
    chol_update_tc(c, K0, pend, n - pend);  // the trailing matrix, whole lower triangle
  }
  *cerr = c.cerr;
  return c.launches;
}

// ------------------------------------------------------------------ inverse of the factor
// W = L^{-1} on the tensor cores, for the explicit inverse K^{-1} = W^T W of the online phase
// (Eq. (4.13) with both triangular solves moved offline).  Recursively by halves: with
// L = [L11 0; L21 L22] and W11 = L11^{-1}, W22 = L22^{-1} known, W21 = -W22 (L21 W11).  Both
// products are digit-plane GEMMs (digit_gemm_tc) of K-major operands: T = L21 W11 takes L21's
// rows and W11's columns (the rows of W11^T, zero before the diagonal, so column tile J starts at
// chunk J / 2); W21 = -W22 T takes W22's rows (zero past the diagonal: row tile I ends at chunk
// I) and T's columns.  The 64 x 64 diagonal blocks are the factorisation's FP64 inverses.
namespace {
// W's diagonal 64 x 64 blocks from Linv ([nblk][64][64]); the rest of W is zero beforehand
__global__ void diag_blocks_kernel(const double* __restrict__ Linv, int64_t n, double* __restrict__ W) {
  const int64_t b = blockIdx.x;
  for (int i = threadIdx.x; i < kCholNB * kCholNB; i += blockDim.x) {
    const int r = i / kCholNB, c = i - r * kCholNB;
    const int64_t gr = b * kCholNB + r, gc = b * kCholNB + c;
    if (gr < n && gc < n) W[gr * n + gc] = Linv[b * kCholNB * kCholNB + i];
  }
}

// X[c][r] = X[r][c] for r > c, by 32 x 32 tiles through shared memory (tile (R, C), C < R, is
// read by rows and written transposed into tile (C, R); diagonal tiles mirror in place)
__global__ void __launch_bounds__(256) symmetrize_kernel(double* X, int64_t n) {
  __shared__ double t[32][33];
  const int64_t R = blockIdx.y, C = blockIdx.x;
  if (C > R) return;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int j = ty; j < 32; j += 8) {
    const int64_t r = R * 32 + j, c = C * 32 + tx;
    t[j][tx] = (r < n && c < n) ? X[r * n + c] : 0.0;
  }
  __syncthreads();
  for (int j = ty; j < 32; j += 8) {
    const int64_t r = C * 32 + j, c = R * 32 + tx;  // upper entry (r, c) = lower entry (c, r)
    if (r < n && c < n && c > r) X[r * n + c] = t[tx][j];
  }
}

struct InvTc {
  const double* L;
  int64_t n;
  double* W;
  double* T;
  void* pa;
  int* ea;
  void* pb;
  int* eb;
  unsigned long long* colmax;
  int* err;
  cudaStream_t s;
  int drop_stage;
  int64_t launches = 0;
  cudaError_t cerr = cudaSuccess;
};

void inv_gemm(InvTc& v, const DigitGemm& g) {
  if (v.cerr != cudaSuccess) return;
  int64_t tl = 0;
  v.cerr = digit_gemm_tc(v.pa, v.ea, v.pb, v.eb, g, v.err, v.s, &tl, v.drop_stage);
  v.launches += tl;
}

// W[c0:c0+w, c0:c0+w] = L[c0:c0+w, c0:c0+w]^{-1}
void inv_rec(InvTc& v, int64_t c0, int64_t w) {
  if (w <= kCholNB || v.cerr != cudaSuccess) return;
  const int64_t h = (w / 2 + kCholNB - 1) / kCholNB * kCholNB, m2 = w - h, n = v.n;
  inv_rec(v, c0, h);
  inv_rec(v, c0 + h, m2);
  // T = L21 W11 (m2 x h, row stride h)
  v.launches += kinv_tc_slice(v.L + (c0 + h) * n + c0, n, m2, h, v.ea, v.pa, kinv_tc_ld(m2), v.s);
  v.launches += kinv_tc_slice_t(v.W + c0 * n + c0, n, h, h, v.eb, v.pb, kinv_tc_ld(h), v.colmax, v.s);
  DigitGemm g{};
  g.C = v.T;
  g.ldc = h;
  g.M = m2;
  g.N = h;
  g.K = h;
  g.op = 0;
  g.kfirst = 2;
  g.skip_on_err = true;
  inv_gemm(v, g);
  // W21 = -W22 T (m2 x h, into W)
  v.launches += kinv_tc_slice(v.W + (c0 + h) * n + (c0 + h), n, m2, m2, v.ea, v.pa, kinv_tc_ld(m2), v.s);
  v.launches += kinv_tc_slice_t(v.T, h, m2, h, v.eb, v.pb, kinv_tc_ld(h), v.colmax, v.s);
  g = DigitGemm{};
  g.C = v.W + (c0 + h) * n + c0;
  g.ldc = n;
  g.M = m2;
  g.N = h;
  g.K = m2;
  g.op = 2;
  g.klast = 1;
  g.skip_on_err = true;
  inv_gemm(v, g);
}
}  // namespace

int64_t lower_inverse_tc_half(int64_t n) { return (n / 2 + kCholNB - 1) / kCholNB * kCholNB; }

size_t lower_inverse_tc_plane_elems(int64_t n) {
  const int64_t h = kinv_tc_ld(lower_inverse_tc_half(n));
  return (size_t)6 * h * h;
}

int64_t lower_inverse_tc(const double* L, const double* Linv, int64_t n, double* W, double* T, void* pa, int* ea,
                         void* pb, int* eb, unsigned long long* colmax, int* err, cudaStream_t s, cudaError_t* cerr,
                         int drop_stage) {
  InvTc v{L, n, W, T, pa, ea, pb, eb, colmax, err, s, drop_stage};
  cudaMemsetAsync(W, 0, sizeof(double) * (size_t)n * n, s);
  const int64_t nblk = (n + kCholNB - 1) / kCholNB;
  diag_blocks_kernel<<<(unsigned)nblk, 256, 0, s>>>(Linv, n, W);
  v.launches = 1;
  inv_rec(v, 0, n);
  *cerr = v.cerr;
  return v.launches;
}

int symmetrize_lower(double* X, int64_t n, cudaStream_t s) {
  if (n <= 0) return 0;
  const unsigned t = (unsigned)((n + 31) / 32);
  symmetrize_kernel<<<dim3(t, t), 256, 0, s>>>(X, n);
  return 1;
}

// ------------------------------------------------------------------ triangular solves
size_t trsm_work_elems(int64_t n, int64_t B) { return (size_t)B * kCholNB; }

// Right-hand sides are the rows of X ([B][n]).  Forward: L Y = X, then
// backward: L^T Z = Y; both blocked by the factor's diagonal blocks, whose
// inverses Linv come from the factorisation.
int64_t trsm_lower_f64(const double* Lm, const double* Linv, int64_t n, double* X, int64_t B,
                       double* work, const int* status, cudaStream_t s, bool dd) {
  (void)status;
  const int nb = kCholNB;
  int64_t launches = 0;
  for (int64_t k = 0; k < n; k += nb) {
    int kb = (int)std::min<int64_t>(nb, n - k);
    const double* Lk = Linv + (k / nb) * nb * nb;
    // Y_k = X_k L_kk^{-T}
    launches += gemm_sel(dd, true, B, kb, kb, 1.0, X + k, n, Lk, nb, 0.0, work, kb, false, s);
    cudaMemcpy2DAsync(X + k, n * sizeof(double), work, kb * sizeof(double), kb * sizeof(double), B,
                      cudaMemcpyDeviceToDevice, s);
    int64_t m = n - k - kb;
    if (m > 0)  // X[:, k+kb:] -= Y_k L[k+kb:, k:k+kb]^T
      launches += gemm_sel(dd, true, B, m, kb, -1.0, X + k, n, Lm + (k + kb) * n + k, n, 1.0, X + k + kb, n, false,
                           s);
  }
  int64_t last = ((n - 1) / nb) * nb;
  for (int64_t k = last; k >= 0; k -= nb) {
    int kb = (int)std::min<int64_t>(nb, n - k);
    const double* Lk = Linv + (k / nb) * nb * nb;
    // Z_k = X_k L_kk^{-1}
    launches += gemm_sel(dd, false, B, kb, kb, 1.0, X + k, n, Lk, nb, 0.0, work, kb, false, s);
    cudaMemcpy2DAsync(X + k, n * sizeof(double), work, kb * sizeof(double), kb * sizeof(double), B,
                      cudaMemcpyDeviceToDevice, s);
    if (k > 0)  // X[:, 0:k] -= Z_k L[k:k+kb, 0:k]
      launches += gemm_sel(dd, false, B, k, kb, -1.0, X + k, n, Lm + k * n, n, 1.0, X, n, false, s);
  }
  return launches;
}

// ------------------------------------------------------------------ explicit inverse of K
// The online solve x = K^{-1} d as one dense product with a precomputed K^{-1} (Eq. (4.13)
// with the two triangular solves folded offline into the inverse): the blocked solves
// above walk the factor's n / 64 diagonal blocks in sequence, each step a thin GEMM;
// this product has no sequential dependence and keeps every SM busy.
//
// Kinv: [n][ldk] float pairs (hi, lo), ldk a multiple of 16 with zero padding, so every
// 16-wide k-step reads whole 16-byte vectors.  D, X: FP64 [nb][n] (rows = right-hand
// sides).  Products in double-FP32 arithmetic on the FP32 pipes (as gemm_df64).  Stream-K
// partition: the (row tile, k-step) iterations are split evenly over a grid sized to the
// resident CTAs, each CTA writes one FP64 partial tile per row tile it touches, and
// kinv_reduce_kernel sums a tile's partials in CTA order (deterministic).
constexpr int KIBK = 16;

__global__ void split_pairs_kernel(const double* __restrict__ X, int64_t ldx, float2* __restrict__ Y, int64_t rows,
                                   int64_t n, int64_t ldk) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * ldk) return;
  const int64_t i = e / ldk, j = e - i * ldk;
  float h = 0.f, l = 0.f;
  if (j < n) dd_split(X[i * ldx + j], h, l);
  Y[e] = make_float2(h, l);
}
static int split_rows_to_pairs(const double* X, int64_t ldx, float2* Y, int64_t rows, int64_t n, int64_t ldk,
                               cudaStream_t s) {
  const int64_t total = rows * ldk;
  if (total <= 0) return 0;
  split_pairs_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(X, ldx, Y, rows, n, ldk);
  return 1;
}
int split_rows_to_pairs_ld(const double* X, int64_t ldx, float2* Y, int64_t rows, int64_t n, int64_t ldk,
                           cudaStream_t s) {
  return split_rows_to_pairs(X, ldx, Y, rows, n, ldk, s);
}
int split_to_pairs(const double* X, float2* Y, int64_t n, int64_t ldk, cudaStream_t s) {
  return split_rows_to_pairs(X, n, Y, n, n, ldk, s);
}

// One CTA: BM rows of K^{-1} x BR right-hand sides; thread (tx, ty) owns rows ty + YG a
// (a < TM) and right-hand sides tx + RG b (b < TR).  Dp: the right-hand sides as float
// pairs [BR][ldk] (rows >= nb read as zeros).
template <int BM, int BR, int TM, int TR>
__global__ void __launch_bounds__(256)
kinv_apply_kernel(const float2* __restrict__ Kinv, int64_t ldk, int64_t n, const float2* __restrict__ Dp,
                  int64_t nb, double* __restrict__ part, int64_t per, int64_t total, int64_t kpt, int span) {
  constexpr int RG = BR / TR, YG = BM / TM;
  static_assert(RG * YG == 256, "256 threads: rhs groups x row groups");
  constexpr int NA = BM * KIBK / 2 / 256;            // float4 (two k) of K^{-1} per thread per k-step
  constexpr int ND = (BR * KIBK / 2 + 255) / 256;    // float4 of the right-hand sides per thread
  extern __shared__ float2 kinv_smem[];  // As [2][KIBK][BM + 1], then Ds [2][KIBK][BR + 1]
  float2(*As)[KIBK][BM + 1] = reinterpret_cast<float2(*)[KIBK][BM + 1]>(kinv_smem);
  float2(*Ds)[KIBK][BR + 1] = reinterpret_cast<float2(*)[KIBK][BR + 1]>(kinv_smem + 2 * KIBK * (BM + 1));
  const int tid = threadIdx.x;
  const int tx = tid % RG, ty = tid / RG;
  int64_t it = (int64_t)blockIdx.x * per;
  const int64_t end = min(total, it + per);
  const int64_t first_tile = it / kpt;
  float4 ra[NA], rd[ND];
  while (it < end) {
    const int64_t t = it / kpt;
    const int64_t kb = it - t * kpt;
    const int64_t ke = min(kpt, kb + (end - it));
    const int64_t m0 = t * BM;
    auto load = [&](int64_t ks) {
      const int64_t k0 = ks * KIBK;
#pragma unroll
      for (int e = 0; e < NA; ++e) {
        const int idx = e * 256 + tid;
        const int r = idx >> 3, q = idx & 7;
        const int64_t row = m0 + r;
        ra[e] = row < n ? __ldg(reinterpret_cast<const float4*>(Kinv + row * ldk + k0 + 2 * q))
                        : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int e = 0; e < ND; ++e) {
        const int idx = e * 256 + tid;
        const int b = idx >> 3, q = idx & 7;
        rd[e] = (idx < BR * KIBK / 2 && b < nb)
                    ? __ldg(reinterpret_cast<const float4*>(Dp + b * ldk + k0 + 2 * q))
                    : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    };
    auto store = [&](int buf) {
#pragma unroll
      for (int e = 0; e < NA; ++e) {
        const int idx = e * 256 + tid;
        const int r = idx >> 3, q = idx & 7;
        As[buf][2 * q][r] = make_float2(ra[e].x, ra[e].y);
        As[buf][2 * q + 1][r] = make_float2(ra[e].z, ra[e].w);
      }
#pragma unroll
      for (int e = 0; e < ND; ++e) {
        const int idx = e * 256 + tid;
        if (idx < BR * KIBK / 2) {
          const int b = idx >> 3, q = idx & 7;
          Ds[buf][2 * q][b] = make_float2(rd[e].x, rd[e].y);
          Ds[buf][2 * q + 1][b] = make_float2(rd[e].z, rd[e].w);
        }
      }
    };
    float sh[TM][TR], sl[TM][TR];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TR; ++b) sh[a][b] = sl[a][b] = 0.f;
    load(kb);
    store(0);
    __syncthreads();
    for (int64_t ks = kb; ks < ke; ++ks) {
      const int buf = (int)((ks - kb) & 1);
      const bool more = ks + 1 < ke;
      if (more) load(ks + 1);
#pragma unroll
      for (int kk = 0; kk < KIBK; ++kk) {
        float2 av[TM], bv[TR];
#pragma unroll
        for (int a = 0; a < TM; ++a) av[a] = As[buf][kk][ty + YG * a];
#pragma unroll
        for (int b = 0; b < TR; ++b) bv[b] = Ds[buf][kk][tx + RG * b];
#pragma unroll
        for (int a = 0; a < TM; ++a)
#pragma unroll
          for (int b = 0; b < TR; ++b) dd_mac(sh[a][b], sl[a][b], av[a].x, av[a].y, bv[b].x, bv[b].y);
      }
      if (more) store(buf ^ 1);
      __syncthreads();
    }
    double* P = part + ((blockIdx.x * (int64_t)span + (t - first_tile)) * BR) * BM;
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TR; ++b) P[(tx + RG * b) * BM + ty + YG * a] = (double)sh[a][b] + (double)sl[a][b];
    it += ke - kb;
  }
}

// X[q][row] = sum over the CTAs that covered row tile t of their partials (CTA order).
__global__ void kinv_reduce_kernel(const double* __restrict__ part, double* __restrict__ X, int64_t ldx,
                                   int64_t n, int64_t nb, int BM, int BR, int64_t per, int64_t kpt, int span) {
  const int64_t t = blockIdx.x;
  const int q = blockIdx.y;
  const int64_t row = t * BM + threadIdx.x;
  if (threadIdx.x >= BM || row >= n || q >= nb) return;
  const int64_t c0 = (t * kpt) / per, c1 = ((t + 1) * kpt - 1) / per;
  double sum = 0.0;
  for (int64_t c = c0; c <= c1; ++c) {
    const int64_t slot = t - (c * per) / kpt;
    sum += part[((c * span + slot) * BR + q) * BM + threadIdx.x];
  }
  X[q * ldx + row] = sum;
}

int kinv_reduce(const double* part, double* X, int64_t ldx, int64_t n, int64_t nb, int BM, int BR, int64_t per,
                int64_t kpt, int span, int64_t tiles, cudaStream_t s) {
  kinv_reduce_kernel<<<dim3((unsigned)tiles, (unsigned)nb), 128, 0, s>>>(part, X, ldx, n, nb, BM, BR, per, kpt, span);
  return 1;
}

namespace {
// Tile shapes (rows x right-hand sides, per-thread rows x right-hand sides): 64 x 64 (4 x 4),
// 128 x 16 (8 x 1) and 128 x 4 (2 x 1), chosen by the number of right-hand sides.
struct KinvShape {
  int BM, BR;
};
KinvShape kinv_shape(int64_t nb) {
  if (nb > 16) return {64, 64};
  if (nb > 4) return {128, 16};
  return {128, 4};
}
constexpr size_t kinv_smem_bytes(int BM, int BR) { return sizeof(float2) * 2 * KIBK * ((BM + 1) + (BR + 1)); }
// CTAs of kinv_apply_kernel<BM, BR, TM, TR> resident per SM (the first call also lifts the
// kernel's dynamic shared-memory limit)
template <int BM, int BR, int TM, int TR>
int kinv_resident() {
  static PerDeviceOnce attr;
  static std::atomic<int> occ{1};
  attr([] {
    cudaFuncSetAttribute(kinv_apply_kernel<BM, BR, TM, TR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kinv_smem_bytes(BM, BR));
    int o = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kinv_apply_kernel<BM, BR, TM, TR>, 256, kinv_smem_bytes(BM, BR));
    occ.store(o > 0 ? o : 1);
  });
  return occ.load();
}
struct KinvPlan {
  int BM, BR;
  int64_t tiles, kpt, total, per, ctas;
  int span;
};
KinvPlan kinv_plan(int64_t n, int64_t ldk, int64_t nb) {
  KinvPlan p;
  const KinvShape sh = kinv_shape(nb);
  p.BM = sh.BM;
  p.BR = sh.BR;
  const int occ = p.BR == 64 ? kinv_resident<64, 64, 4, 4>()
                             : (p.BR == 16 ? kinv_resident<128, 16, 8, 1>() : kinv_resident<128, 4, 2, 1>());
  p.tiles = (n + p.BM - 1) / p.BM;
  p.kpt = ldk / KIBK;
  p.total = p.tiles * p.kpt;
  const int64_t slots = (int64_t)num_sms() * occ;
  p.per = (p.total + slots - 1) / slots;
  p.ctas = (p.total + p.per - 1) / p.per;
  p.span = (int)((p.per + p.kpt - 1) / p.kpt + 1);
  return p;
}
}  // namespace

int64_t kinv_ld(int64_t n) { return (n + KIBK - 1) / KIBK * KIBK; }

void kinv_prepare() {
  kinv_resident<64, 64, 4, 4>();
  kinv_resident<128, 16, 8, 1>();
  kinv_resident<128, 4, 2, 1>();
}

size_t kinv_apply_work_elems(int64_t n, int64_t B) {
  if (n <= 0 || B <= 0) return 0;
  const int64_t ldk = kinv_ld(n);
  size_t most = 0;
  for (int64_t nb : {B < 64 ? B : (int64_t)64, B % 64}) {
    if (nb <= 0) continue;
    const KinvPlan p = kinv_plan(n, ldk, nb);
    // right-hand-side pairs (one float2 = one double of space), then the partials
    size_t w = (size_t)nb * ldk + (size_t)p.ctas * p.span * p.BR * p.BM;
    if (w > most) most = w;
  }
  return most;
}

int64_t kinv_apply(const float2* Kinv, int64_t n, const double* D, int64_t B, double* X, double* work,
                   cudaStream_t s) {
  const int64_t ldk = kinv_ld(n);
  int64_t launches = 0;
  for (int64_t q0 = 0; q0 < B; q0 += 64) {
    const int64_t nb = B - q0 < 64 ? B - q0 : 64;
    const KinvPlan p = kinv_plan(n, ldk, nb);
    float2* Dp = reinterpret_cast<float2*>(work);
    double* part = work + nb * ldk;
    launches += split_rows_to_pairs(D + q0 * n, n, Dp, nb, n, ldk, s);
    const size_t sm = kinv_smem_bytes(p.BM, p.BR);
    if (p.BR == 64)
      kinv_apply_kernel<64, 64, 4, 4><<<(unsigned)p.ctas, 256, sm, s>>>(Kinv, ldk, n, Dp, nb, part, p.per, p.total,
                                                                      p.kpt, p.span);
    else if (p.BR == 16)
      kinv_apply_kernel<128, 16, 8, 1><<<(unsigned)p.ctas, 256, sm, s>>>(Kinv, ldk, n, Dp, nb, part, p.per,
                                                                       p.total, p.kpt, p.span);
    else
      kinv_apply_kernel<128, 4, 2, 1><<<(unsigned)p.ctas, 256, sm, s>>>(Kinv, ldk, n, Dp, nb, part, p.per,
                                                                      p.total, p.kpt, p.span);
    launches += 1 + kinv_reduce(part, X + q0 * n, n, n, nb, p.BM, p.BR, p.per, p.kpt, p.span, p.tiles, s);
  }
  return launches;
}

__global__ void axpby_kernel(double* y, const double* x, double a, double b, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = fma(a, x[i], b * y[i]);
}
int axpby_f64(double* y, const double* x, double a, double b, int64_t n, cudaStream_t s) {
  if (n <= 0) return 0;
  axpby_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(y, x, a, b, n);
  return 1;
}

// r[b][i] -= diag[i] x[b][i] for B rows of length n (diagonal noise term of K x)
__global__ void noise_residual_kernel(double* r, const double* x, const double* diag, int64_t n,
                                      int64_t total) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < total) r[i] = fma(-diag[i % n], x[i], r[i]);
}
int noise_residual_f64(double* r, const double* x, const double* diag, int64_t n, int64_t B,
                       cudaStream_t s) {
  int64_t total = n * B;
  if (total <= 0) return 0;
  noise_residual_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(r, x, diag, n, total);
  return 1;
}

}  // namespace bti

namespace bti {

// ------------------------------------------------------------------ FP32 Gram product
// W = A B^T (A: M x K, B: N x K, both row-major FP32), FP32 accumulation, written to
// an FP64 matrix C (ldc), lower tiles only.  128 x 128 tile per CTA, k-step 8, 256
// threads each owning an 8 x 8 sub-tile; the low-precision assembly of K for
// mixed-precision solves (FP32 issues 64x the FP64 rate on GB300).
constexpr int SBM = 128, SBN = 128, SBK = 8;

__global__ void __launch_bounds__(256)
sgemm_nt_lower_kernel(int64_t M, int64_t N, int64_t K, const float* __restrict__ A, int64_t lda,
                      const float* __restrict__ Bm, int64_t ldb, double* __restrict__ C, int64_t ldc) {
  __shared__ float As[SBK][SBM + 4];
  __shared__ float Bs[SBK][SBN + 4];
  const int64_t m0 = (int64_t)blockIdx.x * SBM;
  const int64_t n0 = (int64_t)blockIdx.y * SBN;
  if (m0 + SBM - 1 < n0) return;  // strictly above the diagonal
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
  for (int64_t k0 = 0; k0 < K; k0 += SBK) {
    // 128 rows x 8 k of A and of B: 1024 elements each, 4 per thread
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      int idx = threadIdx.x + 256 * e;
      int r = idx >> 3, c = idx & 7;
      int64_t gk = k0 + c;
      int64_t gm = m0 + r, gn = n0 + r;
      As[c][r] = (gm < M && gk < K) ? A[gm * lda + gk] : 0.f;
      Bs[c][r] = (gn < N && gk < K) ? Bm[gn * ldb + gk] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < SBK; ++kk) {
      float av[8], bv[8];
#pragma unroll
      for (int a = 0; a < 8; ++a) av[a] = As[kk][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 8; ++b) bv[b] = Bs[kk][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    int64_t gm = m0 + ty + 16 * a;
    if (gm >= M) continue;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      int64_t gn = n0 + tx + 16 * b;
      if (gn < N) C[gm * ldc + gn] = (double)acc[a][b];
    }
  }
}

int sgemm_nt_lower_to_f64(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda, const float* Bm,
                          int64_t ldb, double* C, int64_t ldc, cudaStream_t s) {
  if (M <= 0 || N <= 0) return 0;
  dim3 grid((unsigned)((M + SBM - 1) / SBM), (unsigned)((N + SBN - 1) / SBN));
  sgemm_nt_lower_kernel<<<grid, 256, 0, s>>>(M, N, K, A, lda, Bm, ldb, C, ldc);
  return 1;
}

__global__ void f64_to_f32_kernel(const double* __restrict__ x, float* __restrict__ y, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = (float)x[i];
}
int convert_f64_to_f32(const double* x, float* y, int64_t n, cudaStream_t s) {
  if (n <= 0) return 0;
  f64_to_f32_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, y, n);
  return 1;
}

}  // namespace bti

namespace bti {

// ------------------------------------------------------------------ elliptic prior operator
// out = A_s m per time block, A_s = alpha1 I - alpha2 Delta_h on the gx x gy grid
// (node ix * gy + iy), Delta_h the 5-point graph Laplacian with homogeneous Neumann
// boundaries: (A_s u)_p = (alpha1 + alpha2 deg(p)) u_p - alpha2 sum_{q ~ p} u_q.
// Eq. (5.1) uses A_s^{-2} as the prior covariance, so 0.5 ||A_s m_t||^2 is the prior
// term of the negative log-posterior for each time block.
__global__ void elliptic_apply_kernel(const double* __restrict__ m, double* __restrict__ out, int gx, int gy,
                                      double a1, double a2, int64_t nblocks) {
  const int64_t Nm = (int64_t)gx * gy;
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nblocks * Nm) return;
  const int64_t blk = idx / Nm;
  const int p = (int)(idx - blk * Nm);
  const int ix = p / gy, iy = p - ix * gy;
  const double* u = m + blk * Nm;
  double nb = 0.0;
  int deg = 0;
  if (ix > 0) { nb += u[p - gy]; ++deg; }
  if (ix + 1 < gx) { nb += u[p + gy]; ++deg; }
  if (iy > 0) { nb += u[p - 1]; ++deg; }
  if (iy + 1 < gy) { nb += u[p + 1]; ++deg; }
  out[idx] = fma(a1 + a2 * deg, u[p], -a2 * nb);
}

int elliptic_apply(const double* m, double* out, int gx, int gy, double a1, double a2, int64_t nblocks,
                   cudaStream_t s) {
  int64_t total = nblocks * gx * gy;
  if (total <= 0) return 0;
  elliptic_apply_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(m, out, gx, gy, a1, a2, nblocks);
  return 1;
}

}  // namespace bti

namespace bti {

// ------------------------------------------------------------------ two-sided block-diagonal accumulation
// X (Nt R1 x Nt R2, ld = Nt R2) holds W(k, k') = A_k B_{k'}^T block by block on entry;
// on exit block (t, t') = sum_{u=0}^{min(t,t')} W(t-u, t'-u), i.e. prefix sums along every
// block diagonal delta = t - t' (negative and positive): the block-Toeplitz product
// A B^* of two causal maps (e.g. F_q G^*).  One thread per (delta, i, i').
__global__ void block_diag_cumsum_all_kernel(double* X, int64_t Nt, int64_t R1, int64_t R2) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t RR = R1 * R2;
  if (idx >= (2 * Nt - 1) * RR) return;
  const int64_t dd = idx / RR;
  const int64_t rem = idx - dd * RR;
  const int64_t i = rem / R2, ip = rem - i * R2;
  const int64_t delta = dd - (Nt - 1);
  const int64_t t0 = delta > 0 ? delta : 0, tp0 = delta < 0 ? -delta : 0;
  const int64_t len = Nt - (delta > 0 ? delta : -delta);
  const int64_t ld = Nt * R2;
  double acc = 0.0;
  for (int64_t u = 0; u < len; ++u) {
    double* p = X + ((t0 + u) * R1 + i) * ld + (tp0 + u) * R2 + ip;
    acc += *p;
    *p = acc;
  }
}

int block_diag_cumsum_all(double* X, int64_t Nt, int64_t R1, int64_t R2, cudaStream_t s) {
  int64_t total = (2 * Nt - 1) * R1 * R2;
  if (total <= 0) return 0;
  block_diag_cumsum_all_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(X, Nt, R1, R2);
  return 1;
}

}  // namespace bti

namespace bti {

__global__ void select_time_blocks_sq_kernel(const double* __restrict__ in, double* __restrict__ out, int64_t Nt,
                                             int64_t R, int s) {
  const int64_t nc = (Nt / s) * R;
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nc * nc) return;
  const int64_t r = idx / nc, c = idx - r * nc;
  const int64_t tr = s * (r / R + 1) - 1, tc = s * (c / R + 1) - 1;
  out[idx] = in[(tr * R + r % R) * (Nt * R) + tc * R + c % R];
}

int select_time_blocks_sq(const double* in, double* out, int64_t Nt, int64_t R, int s, cudaStream_t st) {
  const int64_t nc = (Nt / s) * R;
  if (nc <= 0) return 0;
  select_time_blocks_sq_kernel<<<(unsigned)((nc * nc + 255) / 256), 256, 0, st>>>(in, out, Nt, R, s);
  return 1;
}

}  // namespace bti
