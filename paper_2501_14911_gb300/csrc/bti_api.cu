// C ABI of libbti: handle, state checks, buffer ownership and orchestration of
// the kernels in fft.cu, spectral.cu and dense.cu.  See include/bti.h for the
// contract of every entry point.
#include "bti_internal.cuh"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <utility>
#include <algorithm>
#include <vector>

using namespace bti;

static constexpr int kProfPairs = 4096;

namespace {

struct OpStore {
  bool set = false;
  bti_prec prec = BTI_P_F64;
  int64_t R = 0;
  void* hat = nullptr;     // [nf][R][Nm] complex, storage tier
  float* scale = nullptr;  // [nf][R] row scales of the FP16 tier
  double* time = nullptr;  // [Nt][R][Nm] FP64 time-domain copy (F and G only)
  void* dig = nullptr;     // adjoint digit planes of the double-FP32 tier (bti_set_digit_planes)
  int* dig_ex = nullptr;   // their exponents, one per (w, j)
  void* dig_f = nullptr;   // forward digit planes
  int* dig_f_ex = nullptr; // their exponents, one per (w, i)
  int pexp = 0;            // double-FP32 tier: hat holds F-hat 2^-pexp; outputs are scaled back
};

}  // namespace

// Launch shapes chosen by bti_autotune (0 = library default), per storage tier.
struct Tune {
  int fft_p = 0;  // column pairs per FFT CTA
  int jc[2] = {0, 0};  // columns per CTA of the forward product: single vectors, groups of 4
  int vpt = 0;    // columns per thread of the adjoint product
};

struct bti_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int64_t Nm = 0, Nd = 0, Nq = 0, Nt = 0, L = 0, nf = 0;
  FftPlan plan;
  OpStore op[3];
  OpStore shadow[3];  // lower-tier copies for the inner iteration of bti_solve_matfree
  double* pinv = nullptr;  // block-Jacobi preconditioner: [N_t][N_d][N_d] inverses of K's diagonal blocks
  Tune tune[4];  // indexed by bti_prec
  bool tc_enabled = true;  // tensor-core FP16 products for B >= 8 (bti_set_tensor_cores)
  int tc_drop_stage = -1;  // failure-handling test hook (bti_test_withhold_tc_stage)
  bti_prec dense_prec = BTI_P_F64;  // arithmetic of K assembly, Cholesky and solves
  int64_t factor_panel = 4096;      // panel width of the tensor-core Cholesky (bti_set_factor_panel)
  bool noise_set = false;
  double sigma2 = 0.0;
  double* noise_diag = nullptr;  // [Nt][Nd] or null
  bool prior_set = false;        // prior of bti_set_prior_se_grid / _elliptic_grid (also applied to F_q)
  bool g_from_prior = false;     // the G blocks were formed from F's by that prior (not bti_set_blocks)
  int prior_kind = 0;            // 0: squared exponential C_x (x) C_y; 1: elliptic (A_s^2)^{-1} by DCT
  int prior_gx = 0, prior_gy = 0;
  double prior_ell = 0.0, prior_sigma = 0.0;
  double* prior_axes = nullptr;  // C_x [gx][gx] then C_y [gy][gy]
  double* Q = nullptr;           // [N_q N_t][N_d N_t] d2q map
  double* covq = nullptr;        // [N_q N_t][N_q N_t] posterior covariance of the QoI
  bool Q_built = false, covq_built = false;
  int64_t Q_gen = 0;             // incremented by every successful build_Q
  void* Q_planes = nullptr;      // Q as FP16 digit planes for the tensor cores (bti_set_online_qoi)
  int* Q_ea = nullptr;           // their row exponents
  int64_t Qp_gen = -1;           // Q_gen the planes were formed from
  float2* Q_pairs = nullptr;     // Q as float pairs [nq][kQpairLd(n)] for one or two vectors per call
  int64_t Qpr_gen = -1;          // Q_gen the pairs were formed from
  bool online_via_Q = false;     // bti_online takes q_map = Q d_obs (Eq. (4.14))
  int online_prec = BTI_P_DF64;  // bti_set_online_precision: BTI_P_DF64 or BTI_P_F32
  // digit planes the tensor-core products use (6: all); fewer only while bti_online captures the
  // graph of the FP32-level online form
  int planes_kinv = 6, planes_op = 6;
  int qstride = 1;               // QoI time grid: every qstride-th step (N_t^q = N_t / qstride)
  double* K = nullptr;           // [n][n], lower triangle: K, then L after factor_K
  double* Linv = nullptr;        // inverses of the factor's diagonal blocks
  bool K_built = false, K_factored = false;
  int64_t factor_gen = 0;        // incremented by every successful factor_K
  float2* Kinv = nullptr;        // explicit K^{-1} as float pairs [n][kinv_ld(n)] (bti_invert_K)
  void* kinv_planes = nullptr;   // and as six FP16 digit planes for the tensor cores
  int* kinv_ea = nullptr;        // their row exponents
  int64_t kinv_gen = -1;         // factor_gen it was formed from
  int* status = nullptr;  // device status word
  void* ws = nullptr;     // spectral workspace
  size_t ws_bytes = 0;
  double* wsolve = nullptr;  // dense-solve workspace
  size_t wsolve_bytes = 0;
  // online phase captured as a CUDA graph (bti_online)
  cudaGraphExec_t online_exec = nullptr;
  const void* og_d = nullptr;
  void* og_m = nullptr;
  void* og_q = nullptr;
  int64_t og_B = -1;
  int og_refine = -1;
  int og_prec = -1;
  cudaStream_t og_stream = nullptr;
  // measurement hook (bti_profile_enable / bti_profile_read)
  bool prof_on = false;
  std::vector<cudaEvent_t> prof_ev;          // pool of 2 * kProfPairs events
  std::vector<std::pair<int, int>> prof_rec;  // (class, first event index)
  int64_t prof_count[BTI_K_NCLASS] = {0};
  int64_t prof_untimed = 0;
  std::string err;
};

namespace {

bti_status fail(bti_ctx* h, bti_status st, const std::string& msg) {
  if (h) h->err = msg;
  return st;
}

bti_status cuda_check(bti_ctx* h, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return BTI_OK;
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return fail(h, BTI_ERR_OOM, std::string(what) + ": " + cudaGetErrorString(e));
  }
  return fail(h, BTI_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

bti_status launched(bti_ctx* h, const char* what) {
  return cuda_check(h, cudaGetLastError(), what);
}

// Count one launch of class cls; with profiling on, bracket it with an event pair.
struct ProfScope {
  bti_ctx* h;
  int cls;
  int ev = -1;
  ProfScope(bti_ctx* hh, int c) : h(hh), cls(c) {
    h->prof_count[cls] += 1;
    if (h->prof_on && cls != BTI_K_DENSE) {
      int used = (int)h->prof_rec.size();
      if (used < kProfPairs) {
        ev = 2 * used;
        cudaEventRecord(h->prof_ev[ev], h->stream);
      } else {
        h->prof_untimed += 1;
      }
    }
  }
  ~ProfScope() {
    if (ev >= 0) {
      cudaEventRecord(h->prof_ev[ev + 1], h->stream);
      h->prof_rec.emplace_back(cls, ev);
    }
  }
};
#define PROF(h, cls, call) \
  do {                     \
    ProfScope ps_(h, cls); \
    call;                  \
  } while (0)

void count_dense(bti_ctx* h, int64_t launches) { h->prof_count[BTI_K_DENSE] += launches; }

bti_status dev_alloc(bti_ctx* h, void** p, size_t bytes, const char* what) {
  *p = nullptr;
  if (bytes == 0) return BTI_OK;
  return cuda_check(h, cudaMalloc(p, bytes), what);
}

void dev_free(void*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}
template <typename P> void dev_freep(P*& p) {
  void* v = p;
  dev_free(v);
  p = nullptr;
}

bti_status ensure(bti_ctx* h, void** buf, size_t* have, size_t need, const char* what) {
  if (need <= *have) return BTI_OK;
  cudaStreamSynchronize(h->stream);
  dev_free(*buf);
  *have = 0;
  bti_status st = dev_alloc(h, buf, need, what);
  if (st == BTI_OK) *have = need;
  return st;
}

size_t celem_size(bti_prec p) { return p == BTI_P_F32 ? 8 : (p == BTI_P_F16 ? 4 : 16); }
bool prec_ok(int p) { return p == BTI_P_F64 || p == BTI_P_F32 || p == BTI_P_DF64 || p == BTI_P_F16; }
bool double_path(bti_prec p) { return p == BTI_P_F64 || p == BTI_P_DF64; }  // FP64 FFTs and spectra
bool io_ok(int p) { return p == BTI_P_F64 || p == BTI_P_F32; }

int64_t rows_of(bti_ctx* h, bti_op op) { return op == BTI_OP_FQ ? h->Nq : h->Nd; }

bti_status check_handle(bti_ctx* h) {
  if (!h) return BTI_ERR_ARG;
  cudaError_t e = cudaSetDevice(h->device);
  return cuda_check(h, e, "cudaSetDevice");
}

// spectral blocks of an op from FP64 time-domain blocks [Nt][R][Nm] (device)
bti_status make_spectral(bti_ctx* h, OpStore& o, const double* time_blocks) {
  const int64_t cols = o.R * h->Nm;
  if (o.prec == BTI_P_F16) {
    // FP64 spectrum of a few rows at a time in a temporary (at most ~2 GB), then per-row
    // scaled FP16
    const int64_t row_bytes = h->nf * h->Nm * (int64_t)sizeof(double2);
    int64_t ri = ((int64_t)2 << 30) / row_bytes;
    ri = ri < 1 ? 1 : (ri > o.R ? o.R : ri);
    double2* tmp = nullptr;
    bti_status st = dev_alloc(h, (void**)&tmp, (size_t)(ri * row_bytes), "spectral temporary");
    if (st != BTI_OK) return st;
    st = dev_alloc(h, (void**)&o.scale, sizeof(float) * (size_t)h->nf * o.R, "row scales");
    if (st != BTI_OK) { dev_freep(tmp); return st; }
    for (int64_t i0 = 0; i0 < o.R; i0 += ri) {
      const int64_t rn = o.R - i0 < ri ? o.R - i0 : ri;
      PROF(h, BTI_K_RFFT, (launch_rfft_cols<double, double, double>(h->plan, (int)h->Nt, time_blocks + i0 * h->Nm,
                                                                     cols, 0, tmp, 0, rn * h->Nm, 1, h->stream)));
      PROF(h, BTI_K_RFFT, launch_quantize_f16(tmp, o.hat, o.scale, h->nf, rn, o.R, i0, h->Nm, h->stream));
    }
    cudaStreamSynchronize(h->stream);
    dev_freep(tmp);
    return launched(h, "spectral blocks");
  }
  if (o.prec != BTI_P_F32)
    PROF(h, BTI_K_RFFT, (launch_rfft_cols<double, double, double>(h->plan, (int)h->Nt, time_blocks, cols, 0,
                                                                   (double2*)o.hat, 0, cols, 1, h->stream)));
  else
    PROF(h, BTI_K_RFFT, (launch_rfft_cols<double, double, float>(h->plan, (int)h->Nt, time_blocks, cols, 0,
                                                                  (float2*)o.hat, 0, cols, 1, h->stream)));
  o.pexp = 0;
  if (o.prec == BTI_P_DF64) {
    // each FP64 complex becomes a (hi, lo) float pair per part, in place, after an exact
    // power-of-two scaling that puts the largest entry in [1/2, 1): float pairs have FP32's
    // exponent range, and operators in physical units may sit far outside it
    unsigned long long* mx = nullptr;
    bti_status st = dev_alloc(h, (void**)&mx, sizeof(unsigned long long), "alloc max word");
    if (st != BTI_OK) return st;
    PROF(h, BTI_K_RFFT, launch_max_abs((const double*)o.hat, 2 * h->nf * cols, mx, h->stream));
    unsigned long long bits = 0;
    st = cuda_check(h, cudaMemcpyAsync(&bits, mx, sizeof bits, cudaMemcpyDeviceToHost, h->stream),
                    "read block maximum");
    if (st == BTI_OK) st = cuda_check(h, cudaStreamSynchronize(h->stream), "read block maximum");
    dev_freep(mx);
    if (st != BTI_OK) return st;
    double m;
    std::memcpy(&m, &bits, sizeof m);
    if (!std::isfinite(m)) return fail(h, BTI_ERR_ARG, "set_blocks: the blocks hold a non-finite value");
    if (m > 0.0) std::frexp(m, &o.pexp);
    PROF(h, BTI_K_RFFT, launch_split_df64(o.hat, h->nf * cols, o.pexp, h->stream));
  }
  return launched(h, "spectral blocks");
}

void drop_store(OpStore& o) {
  dev_free(o.hat);
  dev_freep(o.time);
  dev_freep(o.scale);
  dev_free(o.dig);
  dev_freep(o.dig_ex);
  dev_free(o.dig_f);
  dev_freep(o.dig_f_ex);
  o.hat = nullptr;
  o.pexp = 0;
  o.set = false;
}

void drop_online_graph_any(bti_ctx* h) {
  if (h->online_exec) cudaGraphExecDestroy(h->online_exec);
  h->online_exec = nullptr;
  h->og_B = -1;
}

bti_status store_op(bti_ctx* h, bti_op opi, const double* blocks, bti_prec store, bool keep_time) {
  drop_online_graph_any(h);
  OpStore& o = h->op[opi];
  const int64_t R = rows_of(h, opi);
  if (R <= 0) return fail(h, BTI_ERR_SHAPE, "operator has zero rows (N_q = 0?)");
  drop_store(h->shadow[opi]);  // a shadow copy describes the blocks being replaced
  if (opi != BTI_OP_FQ) dev_freep(h->pinv);
  drop_store(o);  // the old blocks' spectra, time copy, scales and digit planes
  if (opi == BTI_OP_F && h->g_from_prior) {  // G = F Gamma_prior was formed from the old F
    drop_store(h->op[BTI_OP_G]);
    drop_store(h->shadow[BTI_OP_G]);
  }
  if (opi != BTI_OP_FQ) h->g_from_prior = false;
  h->Q_built = h->covq_built = false;  // Q = F_q G^* K^{-1} involves every operator
  o.R = R;
  o.prec = store;
  size_t hat_bytes = (size_t)h->nf * R * h->Nm * celem_size(store);
  bti_status st = dev_alloc(h, &o.hat, hat_bytes, "alloc spectral blocks");
  if (st != BTI_OK) return st;
  const double* src = blocks;
  if (keep_time) {
    size_t tb = (size_t)h->Nt * R * h->Nm * sizeof(double);
    st = dev_alloc(h, (void**)&o.time, tb, "alloc time-domain blocks");
    if (st != BTI_OK) return st;
    if (blocks != o.time) {
      st = cuda_check(h, cudaMemcpyAsync(o.time, blocks, tb, cudaMemcpyDeviceToDevice, h->stream),
                      "copy blocks");
      if (st != BTI_OK) return st;
    }
    src = o.time;
  }
  st = make_spectral(h, o, src);
  if (st != BTI_OK) return st;
  o.set = true;
  if (opi != BTI_OP_FQ) {
    h->K_built = false;
    h->K_factored = false;
  }
  return BTI_OK;
}

// Forward FFT of B input vectors (io element type) into a spectrum of C2<T> elements.
// The double-FP32 tier transforms in float pairs (FP64 accuracy on the FP32 pipes);
// its spectra stay float pairs (ffc: re_hi, re_lo, im_hi, im_lo) between its kernels.
FftPlan tuned_plan(bti_ctx* h, const OpStore& o) {
  FftPlan p = h->plan;
  if (h->tune[o.prec].fft_p > 0 && h->tune[o.prec].fft_p <= p.P) p.P = h->tune[o.prec].fft_p;
  return p;
}

template <typename T>
void rfft_in(bti_ctx* h, const OpStore& o, const void* in, int64_t ld, int64_t bstride, C2<T>* X,
             int64_t Xbstride, int64_t ncols, int64_t B, bti_prec io) {
  const int Nt = (int)h->Nt;
  cudaStream_t s = h->stream;
  const FftPlan plan = tuned_plan(h, o);
  if (o.prec == BTI_P_DF64) {  // spectra as float pairs (ffc), the double-FP32 tier's own format
    if (io == BTI_P_F64)
      PROF(h, BTI_K_RFFT, (launch_rfft_cols<ffloat, double, ffloat>(plan, Nt, (const double*)in, ld, bstride,
                                                                     (ffc*)X, Xbstride, ncols, B, s)));
    else
      PROF(h, BTI_K_RFFT, (launch_rfft_cols<ffloat, float, ffloat>(plan, Nt, (const float*)in, ld, bstride,
                                                                    (ffc*)X, Xbstride, ncols, B, s)));
  } else if (io == BTI_P_F64) {
    PROF(h, BTI_K_RFFT, (launch_rfft_cols<T, double, T>(plan, Nt, (const double*)in, ld, bstride, X, Xbstride,
                                                         ncols, B, s)));
  } else {
    PROF(h, BTI_K_RFFT, (launch_rfft_cols<T, float, T>(plan, Nt, (const float*)in, ld, bstride, X, Xbstride,
                                                        ncols, B, s)));
  }
}

// Inverse FFT with truncation to N_t steps and the 1/L scale, output in the io type.
template <typename T>
void irfft_out(bti_ctx* h, const OpStore& o, const C2<T>* Y, int64_t ld, int64_t Ybstride, void* out,
               int64_t obstride, int64_t ncols, int64_t B, bti_prec io, int os = 1) {
  const int Nt = (int)h->Nt;
  cudaStream_t s = h->stream;
  const FftPlan plan = tuned_plan(h, o);
  // 1/L, times the power of two the stored double-FP32 blocks were divided by (exact)
  const double scale = std::ldexp(1.0 / (double)h->L, o.pexp);
  if (o.prec == BTI_P_DF64) {  // float-pair spectra in
    if (io == BTI_P_F64)
      PROF(h, BTI_K_IRFFT, (launch_irfft_cols<ffloat, ffloat, double>(plan, Nt, (const ffc*)Y, ld, Ybstride,
                                                                       (double*)out, obstride, ncols, B, scale, s, os)));
    else
      PROF(h, BTI_K_IRFFT, (launch_irfft_cols<ffloat, ffloat, float>(plan, Nt, (const ffc*)Y, ld, Ybstride,
                                                                      (float*)out, obstride, ncols, B, scale, s, os)));
  } else if (io == BTI_P_F64) {
    PROF(h, BTI_K_IRFFT, (launch_irfft_cols<T, T, double>(plan, Nt, Y, ld, Ybstride, (double*)out, obstride,
                                                           ncols, B, scale, s, os)));
  } else {
    PROF(h, BTI_K_IRFFT, (launch_irfft_cols<T, T, float>(plan, Nt, Y, ld, Ybstride, (float*)out, obstride,
                                                          ncols, B, scale, s, os)));
  }
}

// forward-type product: out[b] = T(op) in[b]; in [B][Nt][Nm] (io) -> out [B][Nt][R] (io)
template <typename T>
bti_status apply_fwd_t(bti_ctx* h, const OpStore& o, const void* in, void* out, int64_t B, bti_prec io) {
  const int64_t nf = h->nf, Nm = h->Nm, R = o.R, Nt = h->Nt;
  size_t n_mhat = (size_t)B * nf * Nm;
  // FP16 blocks with B >= 8 vectors: the tensor-core product (its own chunking)
  const bool tc = o.prec == BTI_P_F16 && h->tc_enabled && tc_fwd_f16_supported(Nm, R, B);
  // double-FP32 blocks with digit planes and B >= 16: exact digit-plane product on the tensor cores
  const bool dig = o.prec == BTI_P_DF64 && o.dig_f && h->tc_enabled && fwd_digits_supported(nf, R, Nm, B);
  size_t n_part = prod_fwd_partial_elems(nf, R, Nm, B);
  if (tc && tc_fwd_partial_elems(nf, R, Nm, B) > n_part) n_part = tc_fwd_partial_elems(nf, R, Nm, B);
  size_t n_dhat = (size_t)B * nf * R;
  const size_t base = sizeof(C2<T>) * (n_mhat + n_part + n_dhat);
  bti_status st = ensure(h, &h->ws, &h->ws_bytes, base + (dig ? fwd_digits_work_bytes(nf, R, Nm) : 0), "workspace");
  if (st != BTI_OK) return st;
  C2<T>* mhat = (C2<T>*)h->ws;
  C2<T>* part = mhat + n_mhat;
  C2<T>* dhat = part + n_part;
  cudaStream_t s = h->stream;
  rfft_in<T>(h, o, in, Nm, Nt * Nm, mhat, nf * Nm, Nm, B, io);
  const int jc = h->tune[o.prec].jc[fwd_group(B) == 4];
  if (tc) {
    int nl = 0;
    cudaError_t e;
    {
      ProfScope ps(h, BTI_K_PROD_FWD);  // the MMA kernel and its fixed-order chunk sum
      e = launch_prod_fwd_f16_tc(o.hat, o.scale, (const float2*)mhat, (float2*)part, (float2*)dhat, nf, R, Nm, B,
                                 h->status + 1, s, &nl, h->tc_drop_stage);
    }
    h->prof_count[BTI_K_PROD_FWD] += nl - 1;
    if (e != cudaSuccess) return cuda_check(h, e, "tensor-core forward product");
  } else if (dig) {
    int nl = 0;
    cudaError_t e;
    {
      ProfScope ps(h, BTI_K_PROD_FWD);  // vector planes, the MMA kernel and its fixed-order sum
      e = fwd_digits_apply(o.dig_f, o.dig_f_ex, nf, R, Nm, mhat, dhat, B, (char*)h->ws + base, h->status + 1, s, &nl,
                           h->tc_drop_stage, h->planes_op);
    }
    h->prof_count[BTI_K_PROD_FWD] += nl - 1;
    if (e != cudaSuccess) return cuda_check(h, e, "tensor-core forward product (digit planes)");
  } else if (o.prec == BTI_P_DF64)
    PROF(h, BTI_K_PROD_FWD, launch_prod_fwd_df64((const float4*)o.hat, (const float4*)mhat, (double2*)part, nf,
                                                 R, Nm, B, s, jc));
  else if (o.prec == BTI_P_F16)
    PROF(h, BTI_K_PROD_FWD, launch_prod_fwd_f16(o.hat, o.scale, (const float2*)mhat, (float2*)part, nf, R, Nm, B,
                                                s, jc));
  else
    PROF(h, BTI_K_PROD_FWD, (launch_prod_fwd<T, T>((const C2<T>*)o.hat, mhat, part, nf, R, Nm, B, s,
                                                   jc)));
  if (!tc && !dig) {
    if (o.prec == BTI_P_DF64)  // FP64 sums of the chunks, stored as float pairs for the inverse FFT
      PROF(h, BTI_K_REDUCE, launch_reduce_chunks_df64((const double2*)part, (float4*)dhat, nf, R, Nm, B, s, jc));
    else
      PROF(h, BTI_K_REDUCE, (launch_reduce_chunks<T>(part, dhat, nf, R, Nm, B, s, jc)));
  }
  // the QoI map writes every qstride-th time step only (N_t / qstride rows per vector)
  const int os = (&o == &h->op[BTI_OP_FQ]) ? h->qstride : 1;
  irfft_out<T>(h, o, dhat, R, nf * R, out, (Nt / os) * R, R, B, io, os);
  return launched(h, "forward Toeplitz product");
}

// adjoint-type product: out[b] = T(op)^T in[b]; in [B][Nt][R] -> out [B][Nt][Nm]
template <typename T>
bti_status apply_adj_t(bti_ctx* h, const OpStore& o, const void* in, void* out, int64_t B, bti_prec io) {
  const int64_t nf = h->nf, Nm = h->Nm, R = o.R, Nt = h->Nt;
  size_t n_dhat = (size_t)B * nf * R;
  size_t n_mhat = (size_t)B * nf * Nm;
  // exact digit-plane product on the tensor cores: its per-call planes follow the spectra
  const bool dig = o.prec == BTI_P_DF64 && o.dig && h->tc_enabled && adj_digits_supported(nf, R, Nm, B);
  const size_t base = sizeof(C2<T>) * (n_mhat + n_dhat);
  bti_status st = ensure(h, &h->ws, &h->ws_bytes, base + (dig ? adj_digits_work_bytes(nf, R, B) : 0), "workspace");
  if (st != BTI_OK) return st;
  C2<T>* dhat = (C2<T>*)h->ws;
  C2<T>* mhat = dhat + n_dhat;
  cudaStream_t s = h->stream;
  rfft_in<T>(h, o, in, R, Nt * R, dhat, nf * R, R, B, io);
  if (o.prec == BTI_P_F16 && h->tc_enabled && tc_adj_f16_supported(Nm, R, B)) {
    int nl = 0;
    cudaError_t e;
    {
      ProfScope ps(h, BTI_K_PROD_ADJ);
      e = launch_prod_adj_f16_tc(o.hat, o.scale, (const float2*)dhat, (float2*)mhat, nf, R, Nm, B, h->status + 1, s,
                                 &nl);
    }
    h->prof_count[BTI_K_PROD_ADJ] += nl - 1;
    if (e != cudaSuccess) return cuda_check(h, e, "tensor-core adjoint product");
  } else if (dig) {
    int nl = 0;
    cudaError_t e;
    {
      ProfScope ps(h, BTI_K_PROD_ADJ);
      e = adj_digits_apply(o.dig, o.dig_ex, nf, R, Nm, dhat, mhat, B, (char*)h->ws + base, h->status + 1, s, &nl,
                           h->tc_drop_stage, h->planes_op);
    }
    h->prof_count[BTI_K_PROD_ADJ] += nl - 1;
    if (e != cudaSuccess) return cuda_check(h, e, "tensor-core adjoint product (digit planes)");
  } else if (o.prec == BTI_P_DF64)
    PROF(h, BTI_K_PROD_ADJ, launch_prod_adj_df64((const float4*)o.hat, (const float4*)dhat, (float4*)mhat, nf,
                                                 R, Nm, B, s, h->tune[o.prec].vpt));
  else if (o.prec == BTI_P_F16)
    PROF(h, BTI_K_PROD_ADJ, launch_prod_adj_f16(o.hat, o.scale, (const float2*)dhat, (float2*)mhat, nf, R, Nm, B,
                                                s, h->tune[o.prec].vpt));
  else
    PROF(h, BTI_K_PROD_ADJ, (launch_prod_adj<T, T>((const C2<T>*)o.hat, dhat, mhat, nf, R, Nm, B, s,
                                                   h->tune[o.prec].vpt)));
  irfft_out<T>(h, o, mhat, Nm, nf * Nm, out, Nt * Nm, Nm, B, io);
  return launched(h, "adjoint Toeplitz product");
}

// out = op(in) with an explicit store (an operator or its shadow copy); no argument checks
bti_status apply_store(bti_ctx* h, const OpStore& o, bool adjoint, const void* in, void* out, int64_t B,
                       bti_prec io) {
  if (double_path(o.prec))  // FP64 and double-FP32 tiers: 16-byte spectra (FP64 complex, float-pair complex)
    return adjoint ? apply_adj_t<double>(h, o, in, out, B, io) : apply_fwd_t<double>(h, o, in, out, B, io);
  return adjoint ? apply_adj_t<float>(h, o, in, out, B, io) : apply_fwd_t<float>(h, o, in, out, B, io);
}

bti_status apply_op(bti_ctx* h, bti_op opi, bool adjoint, const void* in, void* out, int64_t B,
                    bti_prec io, const char* name) {
  bti_status st = check_handle(h);
  if (st != BTI_OK) return st;
  if (!io_ok(io)) return fail(h, BTI_ERR_ARG, std::string(name) + ": bad io precision");
  if (B < 0) return fail(h, BTI_ERR_ARG, std::string(name) + ": B < 0");
  const OpStore& o = h->op[opi];
  if (!o.set) return fail(h, BTI_ERR_STATE, std::string(name) + ": operator blocks not set");
  if (B == 0) return BTI_OK;
  if (!in || !out) return fail(h, BTI_ERR_ARG, std::string(name) + ": null pointer");
  return apply_store(h, o, adjoint, in, out, B, io);
}

// out = Gamma_prior applied to `rows` grid-shaped rows (row r viewed as X_r [gx][gy]), the
// time-invariant prior applied block by block.  U is a caller-provided temporary of
// rows * N_m doubles; in and out must not alias.  Stream-ordered, no sync.
//  - squared exponential: C_s = C_x (x) C_y, so X_r -> C_x X_r C_y (the axis matrices are
//    symmetric);
//  - elliptic, Eq. (5.1): Gamma_prior = (alpha1 I - alpha2 Delta_h)^{-2}.  The Neumann
//    grid Laplacian is diagonalised by the orthonormal DCT-II on each axis (D_x, D_y), so
//    X_r -> D_x^T [ (D_x X_r D_y^T) o W ] D_y with W[k][l] = (alpha1 + alpha2 (lx_k + ly_l))^{-2}.
bti_status se_rows_into(bti_ctx* h, const double* in, double* out, int64_t rows, double* U) {
  const int gx = h->prior_gx, gy = h->prior_gy;
  const int64_t gg = (int64_t)gx * gy;
  cudaStream_t s = h->stream;
  int64_t nl = 0;
  if (h->prior_kind == 0) {
    const double* Cx = h->prior_axes;
    const double* Cy = Cx + (size_t)gx * gx;
    nl += gemm_f64(false, rows * gx, gy, gy, 1.0, in, gy, 0, Cy, gy, 0, 0.0, U, gy, 0, 1, false, s);
    nl += gemm_f64(false, gx, gy, gx, 1.0, Cx, gx, 0, U, gy, gg, 0.0, out, gy, gg, rows, false, s);
  } else {
    const double* Dx = h->prior_axes;
    const double* DxT = Dx + (size_t)gx * gx;
    const double* Dy = DxT + (size_t)gx * gx;
    const double* W = Dy + (size_t)gy * gy;
    nl += gemm_f64(true, rows * gx, gy, gy, 1.0, in, gy, 0, Dy, gy, 0, 0.0, U, gy, 0, 1, false, s);     // X D_y^T
    nl += gemm_f64(false, gx, gy, gx, 1.0, Dx, gx, 0, U, gy, gg, 0.0, out, gy, gg, rows, false, s);    // D_x (.)
    nl += scale_blocks(out, W, gg, rows, s);                                                             // o W
    nl += gemm_f64(false, rows * gx, gy, gy, 1.0, out, gy, 0, Dy, gy, 0, 0.0, U, gy, 0, 1, false, s);  // (.) D_y
    nl += gemm_f64(false, gx, gy, gx, 1.0, DxT, gx, 0, U, gy, gg, 0.0, out, gy, gg, rows, false, s);   // D_x^T (.)
  }
  count_dense(h, nl);
  return launched(h, "prior");
}

}  // namespace

namespace {

// Median device time (ms) of `reps` runs of fn on the handle's stream, after one warm-up.
template <typename Fn>
float time_ms(bti_ctx* h, Fn fn, int reps) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fn();
  float t[8];
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(e0, h->stream);
    fn();
    cudaEventRecord(e1, h->stream);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&t[r], e0, e1);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (int i = 0; i < reps; ++i)
    for (int j = i + 1; j < reps; ++j)
      if (t[j] < t[i]) { float x = t[i]; t[i] = t[j]; t[j] = x; }
  return t[reps / 2];
}

}  // namespace

extern "C" {

const char* bti_version(void) { return "libbti 0.1 (sm_103a)"; }

bti_status bti_create(int64_t Nm, int64_t Nd, int64_t Nq, int64_t Nt, int device, void* cuda_stream,
                      bti_handle* out) {
  if (!out) return BTI_ERR_ARG;
  *out = nullptr;
  if (Nm <= 0 || Nd <= 0 || Nq < 0 || Nt <= 0) return BTI_ERR_ARG;
  if (2 * Nt > kMaxL) return BTI_ERR_ARG;
  if (Nm > ((int64_t)1 << 40) || Nd > (1 << 20) || Nq > (1 << 20)) return BTI_ERR_ARG;
  {  // L = 2 N_t must factor into 2, 3, 5, 7 (checked before touching the device)
    int64_t n = 2 * Nt;
    const int r[4] = {2, 3, 5, 7};
    for (int i = 0; i < 4; ++i)
      while (n % r[i] == 0) n /= r[i];
    if (n != 1) return BTI_ERR_ARG;
  }
  bti_ctx* h = new (std::nothrow) bti_ctx();
  if (!h) return BTI_ERR_OOM;
  h->device = device;
  h->stream = (cudaStream_t)cuda_stream;
  h->Nm = Nm;
  h->Nd = Nd;
  h->Nq = Nq;
  h->Nt = Nt;
  h->L = 2 * Nt;
  h->nf = Nt + 1;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return BTI_ERR_CUDA;
  }
  if (!fft_plan_make(h->plan, (int)h->L)) {
    cudaGetLastError();
    delete h;
    return BTI_ERR_OOM;
  }
  // status[0]: first bad Cholesky pivot; status[1]: a bounded device wait gave up
  if (cudaMalloc(&h->status, 2 * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    fft_plan_free(h->plan);
    delete h;
    return BTI_ERR_OOM;
  }
  cudaMemset(h->status, 0, 2 * sizeof(int));
  *out = h;
  return BTI_OK;
}

bti_status bti_destroy(bti_handle h) {
  if (!h) return BTI_ERR_ARG;
  cudaSetDevice(h->device);
  cudaStreamSynchronize(h->stream);
  for (auto* set : {h->op, h->shadow})
    for (int i = 0; i < 3; ++i) drop_store(set[i]);  // spectral blocks, time copies, scales, digit planes
  dev_freep(h->prior_axes);
  dev_freep(h->pinv);
  dev_freep(h->noise_diag);
  dev_freep(h->K);
  dev_freep(h->Q);
  dev_free(h->Q_planes);
  dev_freep(h->Q_ea);
  dev_freep(h->Q_pairs);
  dev_freep(h->covq);
  dev_freep(h->Linv);
  dev_freep(h->Kinv);
  dev_free(h->kinv_planes);
  dev_freep(h->kinv_ea);
  dev_freep(h->status);
  dev_free(h->ws);
  dev_freep(h->wsolve);
  drop_online_graph_any(h);
  fft_plan_free(h->plan);
  for (cudaEvent_t e : h->prof_ev) cudaEventDestroy(e);
  delete h;
  return BTI_OK;
}

bti_status bti_profile_enable(bti_handle h, int enable) {
  bti_status st = check_handle(h);
  if (st != BTI_OK) return st;
  if (enable && h->prof_ev.empty()) {
    h->prof_ev.resize(2 * kProfPairs);
    for (auto& e : h->prof_ev) {
      st = cuda_check(h, cudaEventCreate(&e), "profile events");
      if (st != BTI_OK) return st;
    }
  }
  h->prof_on = enable != 0;
  return BTI_OK;
}

bti_status bti_profile_read(bti_handle h, double* ms, int64_t* launches, int* timed_all) {
  bti_status st = check_handle(h);
  if (st != BTI_OK) return st;
  st = cuda_check(h, cudaStreamSynchronize(h->stream), "profile sync");
  if (st != BTI_OK) return st;
  double acc[BTI_K_NCLASS] = {0};
  for (auto& r : h->prof_rec) {
    float t = 0.f;
    st = cuda_check(h, cudaEventElapsedTime(&t, h->prof_ev[r.second], h->prof_ev[r.second + 1]), "profile elapsed");
    if (st != BTI_OK) return st;
    acc[r.first] += t;
  }
  for (int c = 0; c < BTI_K_NCLASS; ++c) {
    if (ms) ms[c] = acc[c];
    if (launches) launches[c] = h->prof_count[c];
    h->prof_count[c] = 0;
  }
  if (timed_all) *timed_all = h->prof_untimed == 0;
  h->prof_untimed = 0;
  h->prof_rec.clear();
  return BTI_OK;
}

bti_status bti_set_stream(bti_handle h, void* cuda_stream) {
  if (!h) return BTI_ERR_ARG;
  h->stream = (cudaStream_t)cuda_stream;
  return BTI_OK;
}

bti_status bti_set_blocks(bti_handle h, bti_op op, const double* blocks, bti_prec store) {
  bti_status st = check_handle(h);
  if (st != BTI_OK) return st;
  if (op < BTI_OP_F || op > BTI_OP_FQ) return fail(h, BTI_ERR_ARG, "set_blocks: bad op");
  if (!prec_ok(store)) return fail(h, BTI_ERR_ARG, "set_blocks: bad precision");
  if (!blocks) return fail(h, BTI_ERR_ARG, "set_blocks: null blocks");
  return store_op(h, op, blocks, store, true);
}

}  // extern "C"

namespace {

// Shared part of the two prior set-ups: the axis tables (host, `tables` doubles) go to the
// device, G_k = F_k Gamma_prior is formed from F's time-domain blocks, and its spectral
// blocks are made in tier `store`.
bti_status set_prior_common(bti_ctx* h, int gx, int gy, int kind, const std::vector<double>& tables,
                            bti_prec store, const char* name) {
  OpStore& F = h->op[BTI_OP_F];
  if (!F.set || !F.time) return fail(h, BTI_ERR_STATE, std::string(name) + ": F blocks not set");
  const int64_t rows = h->Nt * h->Nd;
  double* U = nullptr;
  double* G = nullptr;
  drop_online_graph_any(h);
  dev_freep(h->prior_axes);
  h->prior_set = false;
  h->g_from_prior = false;
  // the previous G (and its shadow copy) goes first, so the peak holds one set of G blocks
  drop_store(h->op[BTI_OP_G]);
  drop_store(h->shadow[BTI_OP_G]);
  dev_freep(h->pinv);
  h->K_built = h->K_factored = false;
  h->Q_built = h->covq_built = false;
  bti_status st = dev_alloc(h, (void**)&h->prior_axes, sizeof(double) * tables.size(), "alloc prior tables");
  if (st != BTI_OK) return st;
  cudaStream_t s = h->stream;
  st = cuda_check(h, cudaMemcpyAsync(h->prior_axes, tables.data(), sizeof(double) * tables.size(),
                                     cudaMemcpyHostToDevice, s), "prior tables");
  if (st == BTI_OK) st = cuda_check(h, cudaStreamSynchronize(s), "prior tables");  // host vector goes away
  if (st != BTI_OK) return st;
  st = dev_alloc(h, (void**)&U, sizeof(double) * (size_t)rows * h->Nm, "alloc prior temp");
  if (st != BTI_OK) return st;
  st = dev_alloc(h, (void**)&G, sizeof(double) * (size_t)rows * h->Nm, "alloc G blocks");
  if (st != BTI_OK) { dev_freep(U); return st; }
  h->prior_set = true;
  h->prior_kind = kind;
  h->prior_gx = gx;
  h->prior_gy = gy;
  // row r of the blocks viewed as X_r [gx][gy]: G_r = Gamma_prior applied to X_r
  st = se_rows_into(h, F.time, G, rows, U);
  cudaStreamSynchronize(s);
  dev_freep(U);  // before the spectral blocks are made
  if (st == BTI_OK) {
    OpStore& o = h->op[BTI_OP_G];
    o.R = h->Nd;
    o.prec = store;
    o.time = G;
    G = nullptr;
    st = dev_alloc(h, &o.hat, (size_t)h->nf * o.R * h->Nm * celem_size(store), "alloc spectral blocks");
    if (st == BTI_OK) st = make_spectral(h, o, o.time);
    if (st == BTI_OK) {
      o.set = true;
      h->g_from_prior = true;
      h->K_built = false;
      h->K_factored = false;
    }
  }
  cudaStreamSynchronize(s);
  dev_freep(G);
  return st;
}

// Squared-exponential axis matrix C[a][b] = scale exp(-(a - b)^2 / (2 ell^2)) (host copy of the
// device table builder's definition)
void se_axis_host(std::vector<double>& out, int n, double ell, double scale) {
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) out.push_back(scale * std::exp(-0.5 * (double)(a - b) * (a - b) / (ell * ell)));
}

// Orthonormal DCT-II matrix D[k][j] = s_k cos(pi k (2 j + 1) / (2 n)): the eigenvectors of the
// path-graph (Neumann) Laplacian, whose eigenvalues are 2 - 2 cos(pi k / n)
void dct2_host(std::vector<double>& out, int n, bool transpose) {
  const double pi = 3.14159265358979323846264338327950288;
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) {
      const int k = transpose ? c : r, j = transpose ? r : c;
      const double sk = k == 0 ? std::sqrt(1.0 / n) : std::sqrt(2.0 / n);
      out.push_back(sk * std::cos(pi * k * (2.0 * j + 1.0) / (2.0 * n)));
    }
}

}  // namespace

extern "C" {

bti_status bti_set_prior_se_grid(bti_handle h, int gx, int gy, double ell, double sigma, bti_prec store) {
  bti_status st = check_handle(h);
  if (st != BTI_OK) return st;
  if (gx <= 0 || gy <= 0 || !(ell > 0.0) || !(sigma > 0.0) || !prec_ok(store))
    return fail(h, BTI_ERR_ARG, "set_prior_se_grid: bad argument");
  if ((int64_t)gx * gy != h->Nm) return fail(h, BTI_ERR_SHAPE, "set_prior_se_grid: gx * gy != N_m");
  // C_s = C_x (x) C_y with sigma on each axis, node index ix * gy + iy
  std::vector<double> tables;
  tables.reserve((size_t)gx * gx + (size_t)gy * gy);
  se_axis_host(tables, gx, ell, sigma);
  se_axis_host(tables, gy, ell, sigma);
  h->prior_ell = ell;
  h->prior_sigma = sigma;
  return set_prior_common(h, gx, gy, 0, tables, store, "set_prior_se_grid");
}

bti_status bti_set_prior_elliptic_grid(bti_handle h, int gx, int gy, double alpha1, double alpha2, bti_prec store) {
  bti_status st = check_handle(h);
  if (st != BTI_OK) return st;
  if (gx <= 0 || gy <= 0 || !(alpha1 > 0.0) || !(alpha2 >= 0.0) || !prec_ok(store))
    return fail(h, BTI_ERR_ARG, "set_prior_elliptic_grid: bad argument");
  if ((int64_t)gx * gy != h->Nm) return fail(h, BTI_ERR_SHAPE, "set_prior_elliptic_grid: gx * gy != N_m");
  // tables: D_x, D_x^T, D_y, then W[k][l] = (alpha1 + alpha2 (lx_k + ly_l))^{-2}
  std::vector<double> tables;
  tables.reserve(2 * (size_t)gx * gx + (size_t)gy * gy + (size_t)gx * gy);
  dct2_host(tables, gx, false);
  dct2_host(tables, gx, true);
  dct2_host(tables, gy, false);
  const double pi = 3.14159265358979323846264338327950288;
  for (int k = 0; k < gx; ++k)
    for (int l = 0; l < gy; ++l) {
      const double lam = (2.0 - 2.0 * std::cos(pi * k / gx)) + (2.0 - 2.0 * std::cos(pi * l / gy));
      const double mu = alpha1 + alpha2 * lam;
      tables.push_back(1.0 / (mu * mu));
    }
  return set_prior_common(h, gx, gy, 1, tables, store, "set_prior_elliptic_grid");
}

bti_status bti_set_dense_precision(bti_handle h, bti_prec arith) {
  bti_status st = check_handle(h);
  if (st != BTI_OK) return st;
  if (arith != BTI_P_F64 && arith != BTI_P_DF64)
    return fail(h, BTI_ERR_ARG, "set_dense_precision: BTI_P_F64 or BTI_P_DF64 only");
  if (arith != h->dense_prec) drop_online_graph_any(h);
  h->dense_prec = arith;
  return BTI_OK;
}

bti_status bti_set_noise(bti_handle h, double sigma2, const double* diag) {
  bti_status st = check_handle(h);
  if (st != BTI_OK) return st;
  if (!diag && !(sigma2 > 0.0)) return fail(h, BTI_ERR_ARG, "set_noise: sigma2 must be > 0");
  // everything derived from the old noise goes first, so that a failure below leaves no K,
  // factor, Q or preconditioner built with a noise the handle no longer holds
  drop_online_graph_any(h);
  h->noise_set = false;
  h->K_built = false;
  h->K_factored = false;
  h->Q_built = h->covq_built = false;
  dev_freep(h->pinv);
  double* nd = nullptr;
  if (diag) {
    size_t bytes = sizeof(double) * (size_t)h->Nt * h->Nd;
    st = dev_alloc(h, (void**)&nd, bytes, "alloc noise");
    if (st == BTI_OK)
      st = cuda_check(h, cudaMemcpyAsync(nd, diag, bytes, cudaMemcpyDeviceToDevice, h->stream), "copy noise");
    if (st != BTI_OK) {
      dev_freep(nd);
      return st;
    }
  }
  // the new noise replaces the old one only once it is complete
  dev_freep(h->noise_diag);
  h->noise_diag = nd;
  h->sigma2 = sigma2;
  h->noise_set = true;
  return BTI_OK;
}

bti_status bti_apply_F(bti_handle h, const void* m, void* d, int64_t B, bti_prec io) {
  return apply_op(h, BTI_OP_F, false, m, d, B, io, "apply_F");
}
bti_status bti_apply_FT(bti_handle h, const void* d, void* m, int64_t B, bti_prec io) {
  return apply_op(h, BTI_OP_F, true, d, m, B, io, "apply_FT");
}
bti_status bti_apply_Fq(bti_handle h, const void* m, void* q, int64_t B, bti_prec io) {
  return apply_op(h, BTI_OP_FQ, false, m, q, B, io, "apply_Fq");
}
bti_status bti_apply_Gstar(bti_handle h, const void* d, void* m, int64_t B, bti_prec io) {
  return apply_op(h, BTI_OP_G, true, d, m, B, io, "apply_Gstar");
}

static bti_status build_K_impl(bti_handle h, int64_t col_block, bti_prec assembly);

bti_status bti_build_K(bti_handle h, int64_t col_block) { return build_K_impl(h, col_block, BTI_P_F64); }

bti_status bti_build_K_prec(bti_handle h, int64_t col_block, bti_prec assembly) {
  if (h && assembly != BTI_P_F64 && assembly != BTI_P_F32)
    return fail(h, BTI_ERR_ARG, "build_K_prec: assembly precision must be BTI_P_F64 or BTI_P_F32");
  return build_K_impl(h, col_block, assembly);
}

static bti_status build_K_impl(bti_handle h, int64_t col_block, bti_prec assembly) {
  bti_status st = check_handle(h);
  if (st != BTI_OK) return st;
  if (col_block < 0) return fail(h, BTI_ERR_ARG, "build_K: col_block < 0");
  if (col_block == 0) col_block = 512;
  drop_online_graph_any(h);
  const OpStore& F = h->op[BTI_OP_F];
  const OpStore& G = h->op[BTI_OP_G];
  if (!F.set || !G.set || !F.time || !G.time) return fail(h, BTI_ERR_STATE, "build_K: F and G blocks required");
  if (!h->noise_set) return fail(h, BTI_ERR_STATE, "build_K: noise not set");
  const int64_t n = h->Nt * h->Nd;
  if (!h->K) {
    st = dev_alloc(h, (void**)&h->K, sizeof(double) * (size_t)n * n, "alloc K");
    if (st != BTI_OK) return st;
  }
  cudaStream_t s = h->stream;
  if (assembly == BTI_P_F32) {
    // low-precision assembly: W in FP32 from FP32 copies of the blocks (K stays FP64)
    float* Ff = nullptr;
    float* Gf = nullptr;
    const size_t ne = (size_t)n * h->Nm;
    st = dev_alloc(h, (void**)&Ff, sizeof(float) * 2 * ne, "FP32 blocks");
    if (st != BTI_OK) return st;
    Gf = Ff + ne;
    int64_t nl = convert_f64_to_f32(F.time, Ff, (int64_t)ne, s);
    nl += convert_f64_to_f32(G.time, Gf, (int64_t)ne, s);
    nl += sgemm_nt_lower_to_f64(n, n, h->Nm, Ff, h->Nm, Gf, h->Nm, h->K, n, s);
    count_dense(h, nl);
    cudaStreamSynchronize(s);
    dev_freep(Ff);
  } else if (h->dense_prec == BTI_P_DF64 && h->tc_enabled && kinv_tc_supported(n) && kinv_tc_supported(h->Nm)) {
    // W = F_stack G_stack^T on the tensor cores in exact digit planes, lower triangle only (the
    // block-diagonal prefix sums read nothing else): one tile product with F_stack's rows as A
    // and G_stack's rows as B, W[b][i] = sum_j F[b][j] G[i][j] for i <= b
    const int64_t Nm = h->Nm, Mp = kinv_tc_ld(n);
    void* planes = nullptr;
    int* ex = nullptr;
    st = dev_alloc(h, &planes, sizeof(uint16_t) * 2 * rowmat_tc_plane_elems(n, Nm), "Gram planes");
    if (st == BTI_OK) st = dev_alloc(h, (void**)&ex, sizeof(int) * (size_t)(2 * Mp), "Gram exponents");
    if (st != BTI_OK) {
      dev_free(planes);
      dev_freep(ex);
      return st;
    }
    void* gplanes = static_cast<uint16_t*>(planes) + rowmat_tc_plane_elems(n, Nm);
    kinv_tc_prepare();
    int64_t nl = kinv_tc_slice(F.time, Nm, n, Nm, ex, planes, Mp, s);
    nl += kinv_tc_slice(G.time, Nm, n, Nm, ex + Mp, gplanes, Mp, s);
    DigitGemm g{};
    g.C = h->K;
    g.ldc = n;
    g.M = n;
    g.N = n;
    g.K = Nm;
    g.lower = true;
    g.op = 0;
    int64_t tl = 0;
    cudaError_t e = digit_gemm_tc(planes, ex, gplanes, ex + Mp, g, h->status + 1, s, &tl, h->tc_drop_stage);
    count_dense(h, nl + tl);
    cudaStreamSynchronize(s);
    dev_free(planes);
    dev_freep(ex);
    if (e != cudaSuccess) return cuda_check(h, e, "build_K (tensor-core Gram)");
  } else {
    // W = F_stack G_stack^T (lower block triangle), by column panels
    const bool dd = h->dense_prec == BTI_P_DF64;
    for (int64_t c0 = 0; c0 < n; c0 += col_block) {
      int64_t nc = (n - c0) < col_block ? (n - c0) : col_block;
      count_dense(h, (dd ? gemm_df64 : gemm_f64)(true, n - c0, nc, h->Nm, 1.0, F.time + c0 * h->Nm, h->Nm, 0,
                                                 G.time + c0 * h->Nm, h->Nm, 0, 0.0, h->K + c0 * n + c0, n, 0, 1,
                                                 true, s));
    }
  }
  count_dense(h, k_diag_cumsum(h->K, h->Nt, h->Nd, h->sigma2, h->noise_diag, s));
  st = launched(h, "build_K");
  if (st != BTI_OK) return st;
  h->K_built = true;
  h->K_factored = false;
  h->Q_built = h->covq_built = false;
  return BTI_OK;
}

bti_status bti_factor_K(bti_handle h) {
  bti_status st = check_handle(h);
  if (st != BTI_OK) return st;
  if (!h->K_built) return fail(h, BTI_ERR_STATE, "factor_K: K not built");
  if (h->K_factored) return BTI_OK;
  const int64_t n = h->Nt * h->Nd;
  const int64_t nblk = (n + kCholNB - 1) / kCholNB;
  if (!h->Linv) {
    st = dev_alloc(h, (void**)&h->Linv, sizeof(double) * (size_t)nblk * kCholNB * kCholNB, "alloc Linv");
    if (st != BTI_OK) return st;
  }
  st = ensure(h, (void**)&h->wsolve, &h->wsolve_bytes, sizeof(double) * (size_t)n * kCholNB, "solve workspace");
  if (st != BTI_OK) return st;
  cudaMemsetAsync(h->status, 0, 2 * sizeof(int), h->stream);
  const int64_t P = h->factor_panel;
  const bool tc = h->dense_prec == BTI_P_DF64 && h->tc_enabled && n > kCholNB && kinv_tc_supported(n);
  if (tc) {
    // wide panels, trailing updates on the tensor cores in digit planes
    void* planes = nullptr;
    int* ex = nullptr;
    st = dev_alloc(h, &planes, sizeof(uint16_t) * cholesky_tc_plane_elems(n, P), "Cholesky planes");
    if (st == BTI_OK) st = dev_alloc(h, (void**)&ex, sizeof(int) * (size_t)kinv_tc_ld(n), "Cholesky exponents");
    if (st != BTI_OK) {
      dev_free(planes);
      return st;
    }
    kinv_tc_prepare();
    cudaError_t ce = cudaSuccess;
    count_dense(h, cholesky_tc(h->K, n, P, h->Linv, h->wsolve, planes, ex, h->status, h->status + 1, h->stream, &ce,
                               h->tc_drop_stage));
    cudaStreamSynchronize(h->stream);
    dev_free(planes);
    dev_freep(ex);
    if (ce != cudaSuccess) {
      h->K_built = false;
      return cuda_check(h, ce, "factor_K (tensor-core trailing update)");
    }
  } else {
    count_dense(h, cholesky_f64(h->K, n, h->Linv, h->wsolve, h->status, h->stream, h->dense_prec == BTI_P_DF64));
  }
  st = launched(h, "factor_K");
  if (st != BTI_OK) return st;
  int stat2[2] = {0, 0};
  st = cuda_check(h, cudaMemcpyAsync(stat2, h->status, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->stream),
                  "status");
  if (st != BTI_OK) return st;
  st = cuda_check(h, cudaStreamSynchronize(h->stream), "factor_K sync");
  if (st != BTI_OK) return st;
  const int stat = stat2[0];
  if (stat2[1] != 0) {
    h->K_built = false;  // K was partly overwritten
    cudaMemsetAsync(h->status, 0, 2 * sizeof(int), h->stream);
    cudaStreamSynchronize(h->stream);
    return fail(h, BTI_ERR_TIMEOUT, "factor_K: a bounded wait in the tensor-core trailing update gave up");
  }
  if (stat != 0) {
    h->K_built = false;  // K was overwritten
    char buf[128];
    snprintf(buf, sizeof buf, "factor_K: K is not positive definite (pivot %d)", stat);
    return fail(h, BTI_ERR_NOT_SPD, buf);
  }
  h->K_factored = true;
  ++h->factor_gen;
  return BTI_OK;
}

static bool kinv_ready(const bti_ctx* h) { return h->Kinv && h->K_factored && h->kinv_gen == h->factor_gen; }

bti_status bti_invert_K(bti_handle h, int enable) {
  bti_status st = check_handle(h);
  if (st != BTI_OK) return st;
  drop_online_graph_any(h);
  auto release = [&]() {
    dev_freep(h->Kinv);
    dev_free(h->kinv_planes);
    dev_freep(h->kinv_ea);
    h->kinv_gen = -1;
  };
  if (!enable) {
    cudaStreamSynchronize(h->stream);
    release();
    return BTI_OK;
  }
  if (!h->K_factored) return fail(h, BTI_ERR_STATE, "invert_K: K not factored");
  if (kinv_ready(h)) return BTI_OK;
  const int64_t n = h->Nt * h->Nd;
  const int64_t ldk = kinv_ld(n);
  cudaStream_t s = h->stream;
  const bool tc = kinv_tc_supported(n);
  const int64_t ldt = kinv_tc_ld(n);
  kinv_prepare();
  if (tc) kinv_tc_prepare();
  if (!h->Kinv) st = dev_alloc(h, (void**)&h->Kinv, sizeof(float2) * (size_t)n * ldk, "alloc K inverse");
  if (st == BTI_OK && tc && !h->kinv_planes)
    st = dev_alloc(h, &h->kinv_planes, sizeof(uint16_t) * kinv_tc_plane_elems(n), "alloc K inverse planes");
  if (st == BTI_OK && tc && !h->kinv_ea)
    st = dev_alloc(h, (void**)&h->kinv_ea, sizeof(int) * (size_t)ldt, "alloc K inverse exponents");
  if (st == BTI_OK)
    st = ensure(h, (void**)&h->wsolve, &h->wsolve_bytes, sizeof(double) * trsm_work_elems(n, n), "solve workspace");
  double* X = nullptr;
  if (st == BTI_OK) st = dev_alloc(h, (void**)&X, sizeof(double) * (size_t)n * n, "K inverse temporary");
  if (st != BTI_OK) {
    release();
    return st;
  }
  int64_t nl = 0;
  if (tc && h->tc_enabled) {
    // W = L^{-1} on the tensor cores by recursive halves, then K^{-1} = W^T W: the rows of W^T
    // (the columns of W, zero before the diagonal, so row tile I starts at chunk I) are both
    // operands of one lower-triangle digit-plane product, mirrored into the upper triangle.
    // W^T's planes use the buffer that K^{-1}'s planes take afterwards.
    const int64_t hh = lower_inverse_tc_half(n), ldh = kinv_tc_ld(hh);
    double* W = nullptr;
    double* T = nullptr;
    void* pa = nullptr;
    void* pb = nullptr;
    int* eab = nullptr;
    unsigned long long* colmax = nullptr;
    st = dev_alloc(h, (void**)&W, sizeof(double) * (size_t)n * n, "inverse factor");
    if (st == BTI_OK) st = dev_alloc(h, (void**)&T, sizeof(double) * (size_t)hh * hh, "inverse temporary");
    if (st == BTI_OK) st = dev_alloc(h, &pa, sizeof(uint16_t) * lower_inverse_tc_plane_elems(n), "inverse planes");
    if (st == BTI_OK) st = dev_alloc(h, &pb, sizeof(uint16_t) * lower_inverse_tc_plane_elems(n), "inverse planes");
    if (st == BTI_OK) st = dev_alloc(h, (void**)&eab, sizeof(int) * (size_t)(2 * ldh), "inverse exponents");
    if (st == BTI_OK)
      st = dev_alloc(h, (void**)&colmax, sizeof(unsigned long long) * (size_t)(ldt > ldh ? ldt : ldh),
                     "column maxima");
    cudaError_t e = cudaSuccess;
    if (st == BTI_OK) {
      kinv_tc_prepare();
      nl += lower_inverse_tc(h->K, h->Linv, n, W, T, pa, eab, pb, eab + ldh, colmax, h->status + 1, s, &e,
                             h->tc_drop_stage);
    }
    if (st == BTI_OK && e == cudaSuccess) {
      nl += kinv_tc_slice_t(W, n, n, n, h->kinv_ea, h->kinv_planes, ldt, colmax, s);
      DigitGemm g{};
      g.C = X;
      g.ldc = n;
      g.M = n;
      g.N = n;
      g.K = n;
      g.lower = true;
      g.op = 0;
      g.kfirst = 1;
      g.skip_on_err = true;
      int64_t tl = 0;
      e = digit_gemm_tc(h->kinv_planes, h->kinv_ea, h->kinv_planes, h->kinv_ea, g, h->status + 1, s, &tl,
                        h->tc_drop_stage);
      nl += tl;
      nl += symmetrize_lower(X, n, s);
    }
    cudaStreamSynchronize(s);
    dev_freep(W);
    dev_freep(T);
    dev_free(pa);
    dev_free(pb);
    dev_freep(eab);
    dev_freep(colmax);
    if (st == BTI_OK && e != cudaSuccess) st = cuda_check(h, e, "invert_K (tensor-core inverse)");
    if (st != BTI_OK) {
      dev_freep(X);
      release();
      return st;
    }
  } else {
    // rows of X: K^{-1} e_b (= row b of the symmetric K^{-1}), by both triangular solves
    nl += identity_blocks(X, 1, n, s);
    nl += trsm_lower_f64(h->K, h->Linv, n, X, n, h->wsolve, h->status, s, true);
  }
  nl += split_to_pairs(X, h->Kinv, n, ldk, s);
  if (tc) nl += kinv_tc_slice(X, n, n, n, h->kinv_ea, h->kinv_planes, ldt, s);
  count_dense(h, nl);
  st = launched(h, "invert_K");
  int stat2[2] = {0, 0};
  bti_status sy = cuda_check(h, cudaMemcpyAsync(stat2, h->status, 2 * sizeof(int), cudaMemcpyDeviceToHost, s),
                             "status");
  if (sy == BTI_OK) sy = cuda_check(h, cudaStreamSynchronize(s), "invert_K sync");
  dev_freep(X);
  if (st == BTI_OK) st = sy;
  if (st == BTI_OK && stat2[1] != 0) {
    cudaMemsetAsync(h->status + 1, 0, sizeof(int), s);
    cudaStreamSynchronize(s);
    st = fail(h, BTI_ERR_TIMEOUT, "invert_K: a bounded wait in a tensor-core product gave up");
  }
  if (st != BTI_OK) {
    release();
    return st;
  }
  h->kinv_gen = h->factor_gen;
  return BTI_OK;
}

bti_status bti_copy_K(bti_handle h, double* dst) {
  bti_status st = check_handle(h);
  if (st != BTI_OK) return st;
  if (!dst) return fail(h, BTI_ERR_ARG, "copy_K: null pointer");
  if (!h->K || !(h->K_built || h->K_factored)) return fail(h, BTI_ERR_STATE, "copy_K: K not built");
  const int64_t n = h->Nt * h->Nd;
  return cuda_check(h, cudaMemcpyAsync(dst, h->K, sizeof(double) * (size_t)n * n, cudaMemcpyDeviceToDevice,
                                       h->stream), "copy_K");
}

// Dense-solve workspace of infer_map for B vectors: x and r ([B][n] each), then either the
// blocked solves' work or the explicit inverse's correction [B][n] and partials; at least
// the Cholesky panel work.
static bti_status reserve_solve(bti_ctx* h, int64_t B) {
  const int64_t n = h->Nt * h->Nd;
  size_t tail = trsm_work_elems(n, B);
  if (kinv_ready(h))
    tail = std::max(tail, (size_t)B * n + std::max(std::max(kinv_apply_work_elems(n, B), symv_pairs_work_elems(n, B)),
                                                   h->kinv_planes ? kinv_tc_work_elems(n) : (size_t)0));
  size_t need = sizeof(double) * ((size_t)2 * B * n + tail);
  size_t chol = sizeof(double) * (size_t)n * kCholNB;
  return ensure(h, (void**)&h->wsolve, &h->wsolve_bytes, need > chol ? need : chol, "solve workspace");
}

static bti_status infer_map_impl(bti_handle h, const double* d_obs, double* m_map, int64_t B, int refine_iters) {
  bti_status st = check_handle(h);
  if (st != BTI_OK) return st;
  if (B < 0 || refine_iters < 0) return fail(h, BTI_ERR_ARG, "infer_map: bad B or refine_iters");
  if (!h->K_factored) return fail(h, BTI_ERR_STATE, "infer_map: K not factored");
  if (!h->op[BTI_OP_G].set) return fail(h, BTI_ERR_STATE, "infer_map: G blocks not set");
  if (B == 0) return BTI_OK;
  if (!d_obs || !m_map) return fail(h, BTI_ERR_ARG, "infer_map: null pointer");
  const int64_t n = h->Nt * h->Nd;
  st = reserve_solve(h, B);
  if (st != BTI_OK) return st;
  // solve workspace: x [B][n], r [B][n], then the explicit-inverse correction [B][n] and
  // its partials, or the blocked solves' work
  double* x = h->wsolve;
  double* r = x + (size_t)B * n;
  double* work = r + (size_t)B * n;
  cudaStream_t s = h->stream;
  const bool inv = kinv_ready(h);
  // x = K^{-1} v (v != x), by the explicit inverse or the blocked triangular solves
  // tensor-core form of the explicit inverse when the planes exist, tensor cores are on and
  // the batch fills its 64-column tiles enough (B >= 16, as for the spectral products); fewer
  // vectors take the memory-bound double-FP32 kernel
  const bool inv_tc = inv && h->kinv_planes && h->tc_enabled && B >= 16;
  cudaError_t tc_err = cudaSuccess;
  auto solve_into = [&](const double* v, double* xo) -> int64_t {
    if (inv_tc) {
      int64_t nl = 0;
      cudaError_t e = kinv_apply_tc(h->kinv_planes, h->kinv_ea, n, v, B, xo, work + (size_t)B * n, h->status + 1, s,
                                    &nl, h->tc_drop_stage, h->planes_kinv);
      if (e != cudaSuccess) tc_err = e;
      return nl;
    }
    // one vector: the symmetric product reads K^{-1}'s lower triangle only
    if (inv && B == 1) return symv_lower_pairs(h->Kinv, kinv_ld(n), n, v, 1, xo, work + (size_t)B * n, s);
    if (inv) return kinv_apply(h->Kinv, n, v, B, xo, work + (size_t)B * n, s);
    if (v != xo) cudaMemcpyAsync(xo, v, sizeof(double) * B * n, cudaMemcpyDeviceToDevice, s);
    return trsm_lower_f64(h->K, h->Linv, n, xo, B, work, h->status, s, h->dense_prec == BTI_P_DF64);
  };
  count_dense(h, solve_into(d_obs, x));
  if (tc_err != cudaSuccess) return cuda_check(h, tc_err, "tensor-core inverse product");
  st = launched(h, "triangular solves");
  if (st != BTI_OK) return st;
  for (int it = 0; it < refine_iters; ++it) {
    // r = d - (Gamma_n x + F (G^* x)), evaluated with the spectral operators;
    // m_map serves as the parameter-space temporary.
    st = apply_op(h, BTI_OP_G, true, x, m_map, B, BTI_P_F64, "refine G*");
    if (st != BTI_OK) return st;
    st = apply_op(h, BTI_OP_F, false, m_map, r, B, BTI_P_F64, "refine F");
    if (st != BTI_OK) return st;
    // r = d - r - Gamma_n x
    int64_t nl = axpby_f64(r, d_obs, 1.0, -1.0, B * n, s);
    if (h->noise_diag)
      nl += noise_residual_f64(r, x, h->noise_diag, n, B, s);
    else
      nl += axpby_f64(r, x, -h->sigma2, 1.0, B * n, s);
    if (inv) {
      nl += solve_into(r, work);
      nl += axpby_f64(x, work, 1.0, 1.0, B * n, s);
    } else {
      nl += solve_into(r, r);
      nl += axpby_f64(x, r, 1.0, 1.0, B * n, s);
    }
    count_dense(h, nl);
    if (tc_err != cudaSuccess) return cuda_check(h, tc_err, "tensor-core inverse product");
    st = launched(h, "refinement");
    if (st != BTI_OK) return st;
  }
  return apply_op(h, BTI_OP_G, true, x, m_map, B, BTI_P_F64, "infer_map G*");
}

bti_status bti_infer_map(bti_handle h, const double* d_obs, double* m_map, int64_t B, int refine_iters) {
  return infer_map_impl(h, d_obs, m_map, B, refine_iters);
}

// out = in C_s for `rows` grid-shaped rows (row r viewed as X_r [gx][gy]: C_x X_r C_y),
// with the stored SE prior: the time-invariant Gamma_prior applied block by block.
static bti_status apply_se_rows(bti_ctx* h, const double* in, double* out, int64_t rows) {
  double* U = nullptr;
  bti_status st = dev_alloc(h, (void**)&U, sizeof(double) * (size_t)rows * h->Nm, "prior temp");
  if (st != BTI_OK) return st;
  st = se_rows_into(h, in, out, rows, U);
  cudaStreamSynchronize(h->stream);
  dev_freep(U);
  return st;
}

// G_q = F_q C_s from F_q's time-domain blocks.
static bti_status prior_apply_fq(bti_ctx* h, double* out) {
  return apply_se_rows(h, h->op[BTI_OP_FQ].time, out, h->Nt * h->Nq);
}

// Digit planes (and row exponents) of a rows x cols FP64 matrix, allocated here: for the
// tensor-core tile products of bti_build_Q.  rows_pad = kinv_tc_ld(rows).
struct Planes {
  void* p = nullptr;
  int* ex = nullptr;
};
static bti_status make_planes(bti_ctx* h, const double* X, int64_t ldx, int64_t rows, int64_t cols, Planes& out,
                              int64_t* nl, const char* what) {
  const int64_t rp = kinv_tc_ld(rows);
  bti_status st = dev_alloc(h, &out.p, sizeof(uint16_t) * (size_t)6 * rp * kinv_tc_ld(cols), what);
  if (st == BTI_OK) st = dev_alloc(h, (void**)&out.ex, sizeof(int) * (size_t)rp, what);
  if (st != BTI_OK) return st;
  *nl += kinv_tc_slice(X, ldx, rows, cols, out.ex, out.p, rp, h->stream);
  return BTI_OK;
}
static void free_planes(Planes& q) {
  dev_free(q.p);
  dev_freep(q.ex);
}
// C (op)= A B^T on the tensor cores for planes A (M x K) and B (N x K)
static cudaError_t tile_product(bti_ctx* h, const Planes& A, const Planes& B, double* C, int64_t ldc, int64_t M,
                                int64_t N, int64_t K, int op, int64_t* nl) {
  DigitGemm g{};
  g.C = C;
  g.ldc = ldc;
  g.M = M;
  g.N = N;
  g.K = K;
  g.op = op;
  int64_t tl = 0;
  const cudaError_t e = digit_gemm_tc(A.p, A.ex, B.p, B.ex, g, h->status + 1, h->stream, &tl, h->tc_drop_stage);
  *nl += tl;
  return e;
}

bti_status bti_build_Q(bti_handle h, int with_covariance) {
  bti_status st = check_handle(h);
  if (st != BTI_OK) return st;
  const OpStore& Fq = h->op[BTI_OP_FQ];
  const OpStore& G = h->op[BTI_OP_G];
  if (!h->K_factored) return fail(h, BTI_ERR_STATE, "build_Q: K not factored");
  if (!Fq.set || !Fq.time) return fail(h, BTI_ERR_STATE, "build_Q: F_q blocks not set");
  if (!G.set || !G.time) return fail(h, BTI_ERR_STATE, "build_Q: G blocks not set");
  if (with_covariance && !h->prior_set)
    return fail(h, BTI_ERR_STATE, "build_Q: the covariance needs the SE prior (bti_set_prior_se_grid)");
  const int64_t n = h->Nt * h->Nd, nqf = h->Nt * h->Nq, Nm = h->Nm;
  const int qs = h->qstride;
  const int64_t nq = (h->Nt / qs) * h->Nq;  // rows of Q on the QoI time grid
  const bool dd = h->dense_prec == BTI_P_DF64;
  // dense products on the tensor cores in digit planes under double-FP32 dense arithmetic
  const bool tcg = dd && h->tc_enabled && kinv_tc_supported(n) && kinv_tc_supported(Nm) && kinv_tc_supported(nqf);
  auto gemm = dd ? gemm_df64 : gemm_f64;
  cudaStream_t s = h->stream;
  drop_online_graph_any(h);  // a captured online graph may read Q (bti_set_online_qoi)
  dev_freep(h->Q);  // the QoI grid may have changed since the last build
  dev_freep(h->covq);
  st = dev_alloc(h, (void**)&h->Q, sizeof(double) * (size_t)nq * n, "alloc Q");
  if (st != BTI_OK) return st;
  h->Q_built = h->covq_built = false;
  Planes pFq, pG, pX;
  auto done = [&](bti_status r) {
    cudaStreamSynchronize(s);
    free_planes(pFq);
    free_planes(pG);
    free_planes(pX);
    return r;
  };
  cudaError_t e = cudaSuccess;
  // X = F_q G^*: Gram of the stacked blocks, then block-diagonal prefix sums (fine time grid);
  // the rows at QoI times t = qs (k + 1) - 1 form Q's right-hand sides
  double* Xf = h->Q;
  if (qs > 1) {
    st = dev_alloc(h, (void**)&Xf, sizeof(double) * (size_t)nqf * n, "F_q G* (fine)");
    if (st != BTI_OK) return st;
  }
  int64_t nl = 0;
  if (tcg) {
    kinv_tc_prepare();
    st = make_planes(h, Fq.time, Nm, nqf, Nm, pFq, &nl, "F_q planes");
    if (st == BTI_OK) st = make_planes(h, G.time, Nm, n, Nm, pG, &nl, "G planes");
    if (st == BTI_OK) e = tile_product(h, pFq, pG, Xf, n, nqf, n, Nm, 0, &nl);
    if (st == BTI_OK && e != cudaSuccess) st = cuda_check(h, e, "build_Q (tensor-core Gram)");
    free_planes(pG);
    if (st != BTI_OK) {
      if (qs > 1) dev_freep(Xf);
      return done(st);
    }
  } else {
    nl += gemm(true, nqf, n, Nm, 1.0, Fq.time, Nm, 0, G.time, Nm, 0, 0.0, Xf, n, 0, 1, false, s);
  }
  nl += block_diag_cumsum_all(Xf, h->Nt, h->Nq, h->Nd, s);
  if (qs > 1) {
    const size_t blk = sizeof(double) * (size_t)h->Nq * n;  // one time block of rows
    cudaMemcpy2DAsync(h->Q, blk, (const char*)Xf + (qs - 1) * blk, qs * blk, blk, h->Nt / qs,
                      cudaMemcpyDeviceToDevice, s);
    cudaStreamSynchronize(s);
    dev_freep(Xf);
  }
  // Q = X K^{-1}: every row of X is a right-hand side of the two triangular solves, or the rows of
  // X against the explicit inverse's planes in one tile product on the tensor cores when
  // bti_invert_K formed it (K^{-1} is symmetric: its rows are its columns)
  const bool inv_tc = kinv_ready(h) && h->kinv_planes && h->tc_enabled;
  double* X = nullptr;  // X on the QoI grid (the covariance subtracts Q X^T)
  if (with_covariance && !tcg) {
    st = dev_alloc(h, (void**)&X, sizeof(double) * (size_t)nq * n, "F_q G* copy");
    if (st != BTI_OK) return done(st);
    cudaMemcpyAsync(X, h->Q, sizeof(double) * (size_t)nq * n, cudaMemcpyDeviceToDevice, s);
  }
  if (inv_tc || (with_covariance && tcg)) {
    st = make_planes(h, h->Q, n, nq, n, pX, &nl, "X planes");
    if (st != BTI_OK) return done(st);
  }
  if (inv_tc) {
    double* Qn = nullptr;
    st = dev_alloc(h, (void**)&Qn, sizeof(double) * (size_t)nq * n, "alloc Q");
    if (st != BTI_OK) return done(st);
    Planes pK;
    pK.p = h->kinv_planes;
    pK.ex = h->kinv_ea;
    e = tile_product(h, pX, pK, Qn, n, nq, n, n, 0, &nl);
    cudaStreamSynchronize(s);
    dev_freep(h->Q);
    h->Q = Qn;
    if (e != cudaSuccess) return done(cuda_check(h, e, "build_Q (tensor-core K^{-1})"));
  } else {
    st = ensure(h, (void**)&h->wsolve, &h->wsolve_bytes,
                sizeof(double) * std::max(trsm_work_elems(n, nq), (size_t)n * kCholNB), "solve workspace");
    if (st != BTI_OK) {
      dev_freep(X);
      return done(st);
    }
    nl += trsm_lower_f64(h->K, h->Linv, n, h->Q, nq, h->wsolve, h->status, s, dd);
  }
  if (with_covariance) {
    double* Gq = nullptr;
    double* Cf = nullptr;
    st = dev_alloc(h, (void**)&Gq, sizeof(double) * (size_t)nqf * Nm, "G_q blocks");
    if (st == BTI_OK) st = prior_apply_fq(h, Gq);
    if (st == BTI_OK) st = dev_alloc(h, (void**)&h->covq, sizeof(double) * (size_t)nq * nq, "alloc cov");
    if (st == BTI_OK && qs > 1) st = dev_alloc(h, (void**)&Cf, sizeof(double) * (size_t)nqf * nqf, "cov (fine)");
    if (st != BTI_OK) {
      dev_freep(X);
      dev_freep(Gq);
      dev_freep(Cf);
      return done(st);
    }
    // Gamma_post(q) = F_q Gamma_prior F_q^T - Q X^T  (Eq. (4.10) with F G_q^* = X^T), on the QoI grid
    double* C0 = qs > 1 ? Cf : h->covq;
    if (tcg) {
      Planes pGq, pQ;
      st = make_planes(h, Gq, Nm, nqf, Nm, pGq, &nl, "G_q planes");
      if (st == BTI_OK) e = tile_product(h, pFq, pGq, C0, nqf, nqf, nqf, Nm, 0, &nl);
      if (st == BTI_OK && e == cudaSuccess) {
        nl += block_diag_cumsum_all(C0, h->Nt, h->Nq, h->Nq, s);
        if (qs > 1) nl += select_time_blocks_sq(Cf, h->covq, h->Nt, h->Nq, qs, s);
        st = make_planes(h, h->Q, n, nq, n, pQ, &nl, "Q planes");
        if (st == BTI_OK) e = tile_product(h, pQ, pX, h->covq, nq, nq, nq, n, 1, &nl);
      }
      cudaStreamSynchronize(s);
      free_planes(pGq);
      free_planes(pQ);
      if (st == BTI_OK && e != cudaSuccess) st = cuda_check(h, e, "build_Q (tensor-core covariance)");
    } else {
      nl += gemm(true, nqf, nqf, Nm, 1.0, Fq.time, Nm, 0, Gq, Nm, 0, 0.0, C0, nqf, 0, 1, false, s);
      nl += block_diag_cumsum_all(C0, h->Nt, h->Nq, h->Nq, s);
      if (qs > 1) nl += select_time_blocks_sq(Cf, h->covq, h->Nt, h->Nq, qs, s);
      nl += gemm(true, nq, nq, n, -1.0, h->Q, n, 0, X, n, 0, 1.0, h->covq, nq, 0, 1, false, s);
    }
    cudaStreamSynchronize(s);
    dev_freep(Gq);
    dev_freep(Cf);
    if (st != BTI_OK) {
      dev_freep(X);
      return done(st);
    }
  }
  dev_freep(X);
  count_dense(h, nl);
  st = launched(h, "build_Q");
  if (st != BTI_OK) return done(st);
  done(BTI_OK);
  h->Q_built = true;
  ++h->Q_gen;
  h->covq_built = with_covariance != 0;
  return BTI_OK;
}

static bool Q_planes_ready(const bti_ctx* h) { return h->Q_planes && h->Q_built && h->Qp_gen == h->Q_gen; }
static bool Q_pairs_ready(const bti_ctx* h) { return h->Q_pairs && h->Q_built && h->Qpr_gen == h->Q_gen; }
// row stride of Q's float pairs (16-byte rows for the vector loads)
static int64_t qpair_ld(int64_t n) { return (n + 3) / 4 * 4; }

// Workspace of apply_Q's tensor-core form (in the dense-solve workspace, after x and r of
// infer_map so that the online graph can run both).
static size_t apply_Q_work_elems(const bti_ctx* h, int64_t B) {
  const int64_t n = h->Nt * h->Nd, nq = (h->Nt / h->qstride) * h->Nq;
  return (size_t)2 * B * n + rowmat_tc_work_elems(nq, n);
}

// q[b] = Q d[b] (Eq. (4.14)): by the digit-plane product on the tensor cores when Q's planes
// are current and B >= 16, else as one dense GEMM (double-FP32 for B > 8 with dense_prec DF64,
// else FP64)
static bti_status apply_Q_impl(bti_ctx* h, const double* d_obs, double* q_map, int64_t B) {
  const int64_t n = h->Nt * h->Nd, nq = (h->Nt / h->qstride) * h->Nq;
  if (Q_planes_ready(h) && h->tc_enabled && B >= 16) {
    bti_status st = ensure(h, (void**)&h->wsolve, &h->wsolve_bytes, sizeof(double) * apply_Q_work_elems(h, B),
                           "solve workspace");
    if (st != BTI_OK) return st;
    int64_t nl = 0;
    cudaError_t e = rowmat_apply_tc(h->Q_planes, h->Q_ea, nq, n, d_obs, B, q_map, nq, h->wsolve + (size_t)2 * B * n,
                                    h->status + 1, h->stream, &nl, h->tc_drop_stage, h->planes_op);
    count_dense(h, nl);
    if (e != cudaSuccess) return cuda_check(h, e, "tensor-core Q product");
    return launched(h, "apply_Q");
  }
  if (Q_pairs_ready(h) && B <= 2) {
    // one or two vectors: a matrix-vector product over Q's float pairs, HBM-bound
    bti_status st = ensure(h, (void**)&h->wsolve, &h->wsolve_bytes,
                           sizeof(double) * ((size_t)2 * B * n + gemv_pairs_work_elems(n, B)), "solve workspace");
    if (st != BTI_OK) return st;
    count_dense(h, gemv_pairs(h->Q_pairs, qpair_ld(n), nq, n, d_obs, B, q_map, nq, h->wsolve + (size_t)2 * B * n,
                              h->stream));
    return launched(h, "apply_Q");
  }
  const bool dd = h->dense_prec == BTI_P_DF64 && B > 8;
  count_dense(h, (dd ? gemm_df64 : gemm_f64)(true, B, nq, n, 1.0, d_obs, n, 0, h->Q, n, 0, 0.0, q_map, nq, 0, 1,
                                             false, h->stream));
  return launched(h, "apply_Q");
}

bti_status bti_set_online_precision(bti_handle h, bti_prec prec) {
  bti_status st = check_handle(h);
  if (st != BTI_OK) return st;
  if (prec != BTI_P_DF64 && prec != BTI_P_F32)
    return fail(h, BTI_ERR_ARG, "set_online_precision: BTI_P_DF64 or BTI_P_F32");
  if (prec != h->online_prec) drop_online_graph_any(h);
  h->online_prec = prec;
  return BTI_OK;
}

bti_status bti_set_online_qoi(bti_handle h, int via_Q) {
  bti_status st = check_handle(h);
  if (st != BTI_OK) return st;
  if (via_Q != 0 && via_Q != 1) return fail(h, BTI_ERR_ARG, "set_online_qoi: via_Q must be 0 or 1");
  drop_online_graph_any(h);
  cudaStreamSynchronize(h->stream);
  dev_free(h->Q_planes);
  dev_freep(h->Q_ea);
  dev_freep(h->Q_pairs);
  h->Qp_gen = h->Qpr_gen = -1;
  h->online_via_Q = false;
  if (!via_Q) return BTI_OK;
  if (!h->Q_built) return fail(h, BTI_ERR_STATE, "set_online_qoi: Q not built");
  const int64_t n = h->Nt * h->Nd, nq = (h->Nt / h->qstride) * h->Nq;
  // Q as float pairs: the one- and two-vector products read it at the HBM rate
  st = dev_alloc(h, (void**)&h->Q_pairs, sizeof(float2) * (size_t)nq * qpair_ld(n), "alloc Q pairs");
  if (st != BTI_OK) return st;
  count_dense(h, split_rows_to_pairs_ld(h->Q, n, h->Q_pairs, nq, n, qpair_ld(n), h->stream));
  h->Qpr_gen = h->Q_gen;
  if (kinv_tc_supported(n) && kinv_tc_supported(nq)) {
    st = dev_alloc(h, &h->Q_planes, sizeof(uint16_t) * rowmat_tc_plane_elems(nq, n), "alloc Q planes");
    if (st == BTI_OK) st = dev_alloc(h, (void**)&h->Q_ea, sizeof(int) * (size_t)kinv_tc_ld(nq), "alloc Q exponents");
    if (st == BTI_OK) {
      kinv_prepare();
      kinv_tc_prepare();
      count_dense(h, kinv_tc_slice(h->Q, n, nq, n, h->Q_ea, h->Q_planes, kinv_tc_ld(nq), h->stream));
      st = launched(h, "set_online_qoi");
      if (st == BTI_OK) st = cuda_check(h, cudaStreamSynchronize(h->stream), "set_online_qoi sync");
    }
    if (st != BTI_OK) {
      dev_free(h->Q_planes);
      dev_freep(h->Q_ea);
      return st;
    }
    h->Qp_gen = h->Q_gen;
  }
  h->online_via_Q = true;
  return BTI_OK;
}

bti_status bti_apply_Q(bti_handle h, const double* d_obs, double* q_map, int64_t B) {
  bti_status st = check_handle(h);
  if (st != BTI_OK) return st;
  if (B < 0) return fail(h, BTI_ERR_ARG, "apply_Q: B < 0");
  if (!h->Q_built) return fail(h, BTI_ERR_STATE, "apply_Q: Q not built");
  if (B == 0) return BTI_OK;
  if (!d_obs || !q_map) return fail(h, BTI_ERR_ARG, "apply_Q: null pointer");
  return apply_Q_impl(h, d_obs, q_map, B);
}

bti_status bti_copy_Q(bti_handle h, double* Q_out, double* cov_out) {
  bti_status st = check_handle(h);
  if (st != BTI_OK) return st;
  if (!h->Q_built) return fail(h, BTI_ERR_STATE, "copy_Q: Q not built");
  if (cov_out && !h->covq_built) return fail(h, BTI_ERR_STATE, "copy_Q: covariance not built");
  const size_t nq = (size_t)(h->Nt / h->qstride) * h->Nq, n = (size_t)h->Nt * h->Nd;
  if (Q_out) {
    st = cuda_check(h, cudaMemcpyAsync(Q_out, h->Q, sizeof(double) * nq * n, cudaMemcpyDeviceToDevice, h->stream),
                    "copy Q");
    if (st != BTI_OK) return st;
  }
  if (cov_out)
    st = cuda_check(h, cudaMemcpyAsync(cov_out, h->covq, sizeof(double) * nq * nq, cudaMemcpyDeviceToDevice,
                                       h->stream), "copy covariance");
  return st;
}

bti_status bti_set_matfree_precond(bti_handle h, int kind) {
  bti_status st = check_handle(h);
  if (st != BTI_OK) return st;
  if (kind != 0 && kind != 1) return fail(h, BTI_ERR_ARG, "set_matfree_precond: kind must be 0 or 1");
  dev_freep(h->pinv);
  if (kind == 0) return BTI_OK;
  const OpStore& F = h->op[BTI_OP_F];
  const OpStore& G = h->op[BTI_OP_G];
  if (!F.set || !F.time || !G.set || !G.time) return fail(h, BTI_ERR_STATE, "set_matfree_precond: F or G not set");
  if (!h->noise_set) return fail(h, BTI_ERR_STATE, "set_matfree_precond: noise not set");
  const int64_t R = h->Nd, RR = R * R, Nt = h->Nt, Nm = h->Nm;
  const int64_t nblk = (R + kCholNB - 1) / kCholNB;
  const size_t nwork = std::max((size_t)R * kCholNB, trsm_work_elems(R, R));
  double *W = nullptr, *P = nullptr, *Linv = nullptr, *work = nullptr;
  st = dev_alloc(h, (void**)&W, sizeof(double) * (size_t)(Nt * RR), "preconditioner blocks");
  if (st == BTI_OK) st = dev_alloc(h, (void**)&P, sizeof(double) * (size_t)(Nt * RR), "preconditioner");
  if (st == BTI_OK) st = dev_alloc(h, (void**)&Linv, sizeof(double) * (size_t)(nblk * kCholNB * kCholNB), "Linv");
  if (st == BTI_OK) st = dev_alloc(h, (void**)&work, sizeof(double) * nwork, "preconditioner work");
  cudaStream_t s = h->stream;
  if (st == BTI_OK) {
    // K(t,t) = Gamma_noise(t) + sum_{k <= t} F_k G_k^T, the Gram blocks in double-FP32 arithmetic
    int64_t nl = gemm_df64(true, R, R, Nm, 1.0, F.time, Nm, R * Nm, G.time, Nm, R * Nm, 0.0, W, R, RR, Nt, false, s);
    nl += diag_block_cumsum(W, Nt, R, h->sigma2, h->noise_diag, s);
    nl += identity_blocks(P, Nt, R, s);
    cudaMemsetAsync(h->status, 0, sizeof(int), s);
    for (int64_t t = 0; t < Nt; ++t) {  // P[t] = K(t,t)^{-1} from its Cholesky factor
      nl += cholesky_f64(W + t * RR, R, Linv, work, h->status, s, true);
      nl += trsm_lower_f64(W + t * RR, Linv, R, P + t * RR, R, work, h->status, s, true);
    }
    count_dense(h, nl);
    st = launched(h, "block-Jacobi preconditioner");
    int stat = 0;
    if (st == BTI_OK)
      st = cuda_check(h, cudaMemcpyAsync(&stat, h->status, sizeof(int), cudaMemcpyDeviceToHost, s), "status");
    if (st == BTI_OK) st = cuda_check(h, cudaStreamSynchronize(s), "preconditioner sync");
    if (st == BTI_OK && stat != 0) {
      cudaMemsetAsync(h->status, 0, sizeof(int), s);
      st = fail(h, BTI_ERR_NOT_SPD, "set_matfree_precond: a diagonal block of K is not SPD");
    }
  }
  cudaStreamSynchronize(s);
  dev_freep(W);
  dev_freep(Linv);
  dev_freep(work);
  if (st != BTI_OK) {
    dev_freep(P);
    return st;
  }
  h->pinv = P;
  return BTI_OK;
}

bti_status bti_set_digit_planes(bti_handle h, bti_op op, int enable) {
  bti_status st = check_handle(h);
  if (st != BTI_OK) return st;
  if (op < BTI_OP_F || op > BTI_OP_FQ || (enable != 0 && enable != 1))
    return fail(h, BTI_ERR_ARG, "set_digit_planes: bad op or enable");
  OpStore& o = h->op[op];
  drop_online_graph_any(h);
  cudaStreamSynchronize(h->stream);
  auto release = [&]() {
    dev_free(o.dig);
    dev_freep(o.dig_ex);
    dev_free(o.dig_f);
    dev_freep(o.dig_f_ex);
  };
  release();
  if (!enable) return BTI_OK;
  if (!o.set || o.prec != BTI_P_DF64)
    return fail(h, BTI_ERR_STATE, "set_digit_planes: the operator's blocks must be set in the BTI_P_DF64 tier");
  const int64_t nf = h->nf, R = o.R, Nm = h->Nm;
  st = dev_alloc(h, &o.dig, sizeof(uint16_t) * adj_digits_plane_elems(nf, R, Nm), "alloc digit planes");
  if (st == BTI_OK) st = dev_alloc(h, (void**)&o.dig_ex, sizeof(int) * adj_digits_exp_elems(nf, Nm), "alloc exps");
  if (st == BTI_OK) st = dev_alloc(h, &o.dig_f, sizeof(uint16_t) * fwd_digits_plane_elems(nf, R, Nm), "alloc planes");
  if (st == BTI_OK) st = dev_alloc(h, (void**)&o.dig_f_ex, sizeof(int) * fwd_digits_exp_elems(nf, R), "alloc exps");
  if (st == BTI_OK) {
    adj_digits_prepare();
    kinv_tc_prepare();
    int64_t nl = adj_digits_build(o.hat, nf, R, Nm, o.dig, o.dig_ex, h->stream);
    nl += fwd_digits_build(o.hat, nf, R, Nm, o.dig_f, o.dig_f_ex, h->stream);
    count_dense(h, nl);
    st = launched(h, "set_digit_planes");
    if (st == BTI_OK) st = cuda_check(h, cudaStreamSynchronize(h->stream), "set_digit_planes sync");
  }
  if (st != BTI_OK) release();
  return st;
}

bti_status bti_set_tensor_cores(bti_handle h, int on) {
  bti_status st = check_handle(h);
  if (st != BTI_OK) return st;
  if (on != 0 && on != 1) return fail(h, BTI_ERR_ARG, "set_tensor_cores: on must be 0 or 1");
  if (h->tc_enabled != (on == 1)) drop_online_graph_any(h);
  h->tc_enabled = on == 1;
  return BTI_OK;
}

bti_status bti_set_factor_panel(bti_handle h, int64_t width) {
  bti_status st = check_handle(h);
  if (st != BTI_OK) return st;
  if (width == 0) width = 4096;
  if (width < kCholNB || width % kCholNB != 0 || width > (int64_t)1 << 30)
    return fail(h, BTI_ERR_ARG, "set_factor_panel: width must be 0 or a positive multiple of 64");
  h->factor_panel = width;
  return BTI_OK;
}

bti_status bti_test_withhold_tc_stage(bti_handle h, int stage) {
  bti_status st = check_handle(h);
  if (st != BTI_OK) return st;
  if (stage < -1) return fail(h, BTI_ERR_ARG, "test_withhold_tc_stage: stage must be >= -1");
  drop_online_graph_any(h);
  h->tc_drop_stage = stage;
  return BTI_OK;
}

bti_status bti_set_shadow(bti_handle h, bti_op op, bti_prec store) {
  bti_status st = check_handle(h);
  if (st != BTI_OK) return st;
  if (op != BTI_OP_F && op != BTI_OP_G) return fail(h, BTI_ERR_ARG, "set_shadow: op must be F or G");
  if (!prec_ok(store)) return fail(h, BTI_ERR_ARG, "set_shadow: bad precision");
  const OpStore& o = h->op[op];
  if (!o.set || !o.time) return fail(h, BTI_ERR_STATE, "set_shadow: operator blocks not set");
  OpStore& sh = h->shadow[op];
  drop_store(sh);
  sh.R = o.R;
  sh.prec = store;
  st = dev_alloc(h, &sh.hat, (size_t)h->nf * sh.R * h->Nm * celem_size(store), "alloc shadow blocks");
  if (st == BTI_OK) st = make_spectral(h, sh, o.time);
  if (st == BTI_OK) st = cuda_check(h, cudaStreamSynchronize(h->stream), "set_shadow sync");
  if (st != BTI_OK) {
    drop_store(sh);
    return st;
  }
  sh.set = true;
  return BTI_OK;
}

}  // extern "C"

namespace {

// Buffers of one matrix-free solve for B right-hand sides (n = N_t N_d data, np = N_t N_m
// parameters per vector).
struct MatfreeWork {
  double *x, *r, *y, *p, *q, *ro, *w1, *w2, *U;  // FP64 vectors and FP64 operator temporaries
  float *dlt, *rt, *pt, *qt, *wf;                 // FP32 inner-iteration vectors
  double *part, *dn2, *rn2, *rr, *rr2, *pq;       // dot workspace and per-vector scalars
  double *rz, *zr, *zro, *num;                    // scalars of the flexible outer iteration
  double* z;                                      // preconditioned residual
  float* zt;                                      // preconditioned inner residual
};

// z = P^{-1} r with the block-Jacobi inverses: z_t = K(t,t)^{-1} r_t for every time block
template <typename T>
int apply_block_precond(bti_ctx* h, const T* r, T* z, int64_t B) {
  return block_precond_apply<T>(h->pinv, r, z, h->Nt, h->Nd, B, h->stream);
}

// y = K x = Gamma_noise x + F (G^* x) with FP64-accurate operators: the F store (FP64 or
// double-FP32) and G^* from the G store when that is FP64-accurate, else Gamma_prior F^T.
bti_status apply_K_accurate(bti_ctx* h, const double* x, double* y, int64_t B, MatfreeWork& w) {
  const int64_t n = h->Nt * h->Nd;
  bti_status st;
  if (double_path(h->op[BTI_OP_G].prec)) {
    st = apply_store(h, h->op[BTI_OP_G], true, x, w.w2, B, BTI_P_F64);
  } else {
    st = apply_store(h, h->op[BTI_OP_F], true, x, w.w1, B, BTI_P_F64);
    if (st == BTI_OK) st = se_rows_into(h, w.w1, w.w2, B * h->Nt, w.U);
  }
  if (st == BTI_OK) st = apply_store(h, h->op[BTI_OP_F], false, w.w2, y, B, BTI_P_F64);
  if (st != BTI_OK) return st;
  count_dense(h, add_noise<double>(y, y, x, h->noise_diag, h->sigma2, n, B, h->stream));
  return launched(h, "K x");
}

// m = G^* x with the FP64-accurate operators (as apply_K_accurate)
bti_status apply_Gstar_accurate(bti_ctx* h, const double* x, double* m, int64_t B, MatfreeWork& w) {
  if (double_path(h->op[BTI_OP_G].prec)) return apply_store(h, h->op[BTI_OP_G], true, x, m, B, BTI_P_F64);
  bti_status st = apply_store(h, h->op[BTI_OP_F], true, x, w.w1, B, BTI_P_F64);
  if (st == BTI_OK) st = se_rows_into(h, w.w1, m, B * h->Nt, w.U);
  return st;
}

// q = K~ p with the inner (shadow where set) operators in FP32 vectors
bti_status apply_K_inner(bti_ctx* h, const float* p, float* q, int64_t B, MatfreeWork& w) {
  const OpStore& G = h->shadow[BTI_OP_G].set ? h->shadow[BTI_OP_G] : h->op[BTI_OP_G];
  const OpStore& F = h->shadow[BTI_OP_F].set ? h->shadow[BTI_OP_F] : h->op[BTI_OP_F];
  bti_status st = apply_store(h, G, true, p, w.wf, B, BTI_P_F32);
  if (st == BTI_OK) st = apply_store(h, F, false, w.wf, q, B, BTI_P_F32);
  if (st != BTI_OK) return st;
  count_dense(h, add_noise<float>(q, q, p, h->noise_diag, h->sigma2, h->Nt * h->Nd, B, h->stream));
  return launched(h, "inner K x");
}

// the per-vector scalars v[0..B) on the host (synchronises the stream)
bti_status fetch(bti_ctx* h, const double* v, std::vector<double>& out, int64_t B) {
  out.resize((size_t)B);
  cudaError_t e = cudaMemcpyAsync(out.data(), v, sizeof(double) * B, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return cuda_check(h, e, "solver scalars");
}

// max over the batch of sqrt(a / b) (0 where b == 0); NaN propagates
double max_ratio(const std::vector<double>& a, const std::vector<double>& b) {
  double m = 0.0;
  for (size_t i = 0; i < a.size(); ++i) {
    const double v = b[i] > 0.0 ? std::sqrt(a[i] / b[i]) : (a[i] > 0.0 ? INFINITY : 0.0);
    if (!(v <= m)) m = v;  // NaN wins
  }
  return m;
}

}  // namespace

extern "C" {

bti_status bti_solve_matfree(bti_handle h, const double* d_obs, double* m_map, double* x_out, int64_t B, int refine,
                             double tol, int max_outer, int max_inner, double inner_tol, bti_solve_info* info) {
  bti_status st = check_handle(h);
  if (st != BTI_OK) return st;
  if (info) *info = bti_solve_info{0, 0, 0.0};
  if (B < 0 || refine < 0 || refine > 2 || !(tol > 0.0) || max_inner < 1 || max_outer < 0 ||
      (refine != 0 && !(inner_tol > 0.0 && inner_tol < 1.0)))
    return fail(h, BTI_ERR_ARG, "solve_matfree: bad B, refine, tolerance or iteration limit");
  if (!h->op[BTI_OP_F].set || !double_path(h->op[BTI_OP_F].prec))
    return fail(h, BTI_ERR_STATE, "solve_matfree: F must be stored in FP64 or double-FP32");
  if (!h->prior_set || !h->op[BTI_OP_G].set) return fail(h, BTI_ERR_STATE, "solve_matfree: no prior set");
  if (!h->noise_set) return fail(h, BTI_ERR_STATE, "solve_matfree: noise not set");
  if (B == 0) return BTI_OK;
  if (!d_obs || !m_map) return fail(h, BTI_ERR_ARG, "solve_matfree: null pointer");
  const int64_t n = h->Nt * h->Nd, np = h->Nt * h->Nm;
  const size_t Bn = (size_t)B * n, Bp = (size_t)B * np;
  cudaStream_t s = h->stream;
  // one allocation: 7 FP64 data vectors, 3 FP64 parameter temporaries, 5 FP32 data and
  // 1 FP32 parameter vector, the dot workspace and 9 scalar rows
  const size_t nd = 7 * Bn + 3 * Bp + dot_workspace_elems(B) + 9 * (size_t)B;
  const size_t nfl = 5 * Bn + Bp;
  void* buf = nullptr;
  st = dev_alloc(h, &buf, sizeof(double) * nd + sizeof(float) * nfl, "solver workspace");
  if (st != BTI_OK) return st;
  MatfreeWork w;
  double* dp = (double*)buf;
  w.x = dp; dp += Bn;
  w.r = dp; dp += Bn;
  w.y = dp; dp += Bn;
  w.p = dp; dp += Bn;
  w.q = dp; dp += Bn;
  w.ro = dp; dp += Bn;
  w.z = dp; dp += Bn;
  w.w1 = dp; dp += Bp;
  w.w2 = dp; dp += Bp;
  w.U = dp; dp += Bp;
  w.part = dp; dp += dot_workspace_elems(B);
  w.dn2 = dp; dp += B;
  w.rn2 = dp; dp += B;
  w.rr = dp; dp += B;
  w.rr2 = dp; dp += B;
  w.pq = dp; dp += B;
  w.rz = dp; dp += B;
  w.zr = dp; dp += B;
  w.zro = dp; dp += B;
  w.num = dp; dp += B;
  float* fp = (float*)dp;
  w.dlt = fp; fp += Bn;
  w.rt = fp; fp += Bn;
  w.pt = fp; fp += Bn;
  w.qt = fp; fp += Bn;
  w.zt = fp; fp += Bn;
  w.wf = fp;
  std::vector<double> hd, hr;
  int outer = 0, inner = 0;
  double rel = 0.0;
  bool converged = false;
  auto dot = [&](auto* a, auto* b, double* out) { count_dense(h, dot_batched(a, b, n, B, w.part, out, s)); };
  const bool pc = h->pinv != nullptr;  // block-Jacobi preconditioning of every CG iteration
  auto precond_d = [&](const double* r, double* z) { count_dense(h, apply_block_precond<double>(h, r, z, B)); };
  auto precond_f = [&](const float* r, float* z) { count_dense(h, apply_block_precond<float>(h, r, z, B)); };
  // r = d - K x with the FP64-accurate operator, rn2 = r . r, and the max relative residual
  auto true_residual = [&](double& out_rel) -> bti_status {
    bti_status sr = apply_K_accurate(h, w.x, w.y, B, w);
    if (sr != BTI_OK) return sr;
    cudaMemcpyAsync(w.r, d_obs, sizeof(double) * Bn, cudaMemcpyDeviceToDevice, s);
    count_dense(h, axpby_f64(w.r, w.y, -1.0, 1.0, (int64_t)Bn, s));
    dot(w.r, w.r, w.rn2);
    sr = fetch(h, w.rn2, hr, B);
    if (sr == BTI_OK) out_rel = max_ratio(hr, hd);
    return sr;
  };
  // The recursive residual of CG drifts from the true one by about the operator's rounding
  // floor; when it meets tol, the true residual decides, and otherwise replaces it and the
  // iteration restarts from there (at most kReplace times).
  constexpr int kReplace = 4;
  int replaced = 0;
  do {
    st = cuda_check(h, cudaMemsetAsync(w.x, 0, sizeof(double) * Bn, s), "solver init");
    if (st != BTI_OK) break;
    st = cuda_check(h, cudaMemcpyAsync(w.r, d_obs, sizeof(double) * Bn, cudaMemcpyDeviceToDevice, s), "solver init");
    if (st != BTI_OK) break;
    dot(w.r, w.r, w.dn2);
    st = fetch(h, w.dn2, hd, B);
    if (st != BTI_OK) break;
    if (refine == 0) {
      // conjugate gradients on K with the FP64-accurate operators (preconditioned when a
      // block-Jacobi preconditioner is set: rr then holds r . z)
      auto restart = [&]() {
        if (pc) {
          precond_d(w.r, w.z);
          cudaMemcpyAsync(w.p, w.z, sizeof(double) * Bn, cudaMemcpyDeviceToDevice, s);
          dot(w.r, w.z, w.rr);
        } else {
          cudaMemcpyAsync(w.p, w.r, sizeof(double) * Bn, cudaMemcpyDeviceToDevice, s);
          dot(w.r, w.r, w.rr);
        }
      };
      restart();
      for (int it = 0; it < max_inner; ++it) {
        st = apply_K_accurate(h, w.p, w.q, B, w);
        if (st != BTI_OK) break;
        dot(w.p, w.q, w.pq);
        count_dense(h, cg_update_xr(w.x, w.r, w.p, w.q, w.rr, w.pq, n, B, s));
        dot(w.r, w.r, w.rr2);
        ++inner;
        st = fetch(h, w.rr2, hr, B);
        if (st != BTI_OK) break;
        rel = max_ratio(hr, hd);
        if (rel <= tol) {
          st = true_residual(rel);
          if (st != BTI_OK || rel <= tol || !(rel == rel) || replaced == kReplace) break;
          ++replaced;  // restart from the true residual
          restart();
          continue;
        }
        if (pc) {
          precond_d(w.r, w.z);
          dot(w.r, w.z, w.num);
          count_dense(h, cg_update_p(w.p, w.z, w.num, w.rr, n, B, s));
          std::swap(w.rr, w.num);
        } else {
          count_dense(h, cg_update_p(w.p, w.r, w.rr2, w.rr, n, B, s));
          std::swap(w.rr, w.rr2);
        }
      }
    } else {
      // z = ||r|| delta with K~ delta = r / ||r|| solved by FP32 conjugate gradients with the
      // inner operators until the inner residual drops by inner_tol (rn2 = r . r on the device)
      auto inner_solve = [&](const double* rv, const double* rn2, double* z) -> bti_status {
        count_dense(h, normalize_to_f32(rv, rn2, w.rt, n, B, s));
        cudaMemsetAsync(w.dlt, 0, sizeof(float) * Bn, s);
        dot(w.rt, w.rt, w.rr2);
        std::vector<double> h0, hi;
        bti_status si = fetch(h, w.rr2, h0, B);
        if (pc) {  // rr holds r . z for the preconditioned iteration
          precond_f(w.rt, w.zt);
          cudaMemcpyAsync(w.pt, w.zt, sizeof(float) * Bn, cudaMemcpyDeviceToDevice, s);
          dot(w.rt, w.zt, w.rr);
        } else {
          cudaMemcpyAsync(w.pt, w.rt, sizeof(float) * Bn, cudaMemcpyDeviceToDevice, s);
          cudaMemcpyAsync(w.rr, w.rr2, sizeof(double) * B, cudaMemcpyDeviceToDevice, s);
        }
        for (int it = 0; si == BTI_OK && it < max_inner; ++it) {
          si = apply_K_inner(h, w.pt, w.qt, B, w);
          if (si != BTI_OK) break;
          dot(w.pt, w.qt, w.pq);
          count_dense(h, cg_update_xr(w.dlt, w.rt, w.pt, w.qt, w.rr, w.pq, n, B, s));
          dot(w.rt, w.rt, w.rr2);
          ++inner;
          si = fetch(h, w.rr2, hi, B);
          if (si != BTI_OK) break;
          const double ri = max_ratio(hi, h0);
          if (ri <= inner_tol || !(ri == ri)) break;
          if (pc) {
            precond_f(w.rt, w.zt);
            dot(w.rt, w.zt, w.num);
            count_dense(h, cg_update_p(w.pt, w.zt, w.num, w.rr, n, B, s));
            std::swap(w.rr, w.num);
          } else {
            count_dense(h, cg_update_p(w.pt, w.rt, w.rr2, w.rr, n, B, s));
            std::swap(w.rr, w.rr2);
          }
        }
        if (si != BTI_OK) return si;
        cudaMemsetAsync(z, 0, sizeof(double) * Bn, s);
        count_dense(h, add_scaled_f32(z, w.dlt, rn2, n, B, s));
        return launched(h, "inner solve");
      };
      if (refine == 1) {
        // FP64 iterative refinement: x += z with z from the inner solve of the residual
        for (;;) {
          dot(w.r, w.r, w.rn2);
          st = fetch(h, w.rn2, hr, B);
          if (st != BTI_OK) break;
          rel = max_ratio(hr, hd);
          if (rel <= tol || outer == max_outer || !(rel == rel)) break;
          ++outer;
          st = inner_solve(w.r, w.rn2, w.p);
          if (st != BTI_OK) break;
          count_dense(h, axpby_f64(w.x, w.p, 1.0, 1.0, (int64_t)Bn, s));
          // r = d - K x with the FP64-accurate operators
          st = apply_K_accurate(h, w.x, w.y, B, w);
          if (st != BTI_OK) break;
          cudaMemcpyAsync(w.r, d_obs, sizeof(double) * Bn, cudaMemcpyDeviceToDevice, s);
          count_dense(h, axpby_f64(w.r, w.y, -1.0, 1.0, (int64_t)Bn, s));
        }
      } else {
        // refinement accelerated by flexible conjugate gradients in FP64 (the CG analogue
        // of GMRES-based refinement): the inner solve is a variable preconditioner, so
        // beta takes the Polak-Ribiere form z_new . (r_new - r_old) / (z_old . r_old).
        // y holds z; ro the previous residual.
        dot(w.r, w.r, w.rn2);
        st = inner_solve(w.r, w.rn2, w.y);
        if (st != BTI_OK) break;
        cudaMemcpyAsync(w.p, w.y, sizeof(double) * Bn, cudaMemcpyDeviceToDevice, s);
        dot(w.r, w.y, w.rz);
        for (;;) {
          if (outer == max_outer) break;
          ++outer;
          st = apply_K_accurate(h, w.p, w.q, B, w);
          if (st != BTI_OK) break;
          dot(w.p, w.q, w.pq);
          cudaMemcpyAsync(w.ro, w.r, sizeof(double) * Bn, cudaMemcpyDeviceToDevice, s);
          count_dense(h, cg_update_xr(w.x, w.r, w.p, w.q, w.rz, w.pq, n, B, s));
          dot(w.r, w.r, w.rn2);
          st = fetch(h, w.rn2, hr, B);
          if (st != BTI_OK) break;
          rel = max_ratio(hr, hd);
          if (!(rel == rel)) break;
          if (rel <= tol) {
            st = true_residual(rel);
            if (st != BTI_OK || rel <= tol || !(rel == rel) || replaced == kReplace) break;
            ++replaced;  // restart the flexible iteration from the true residual
            st = inner_solve(w.r, w.rn2, w.y);
            if (st != BTI_OK) break;
            cudaMemcpyAsync(w.p, w.y, sizeof(double) * Bn, cudaMemcpyDeviceToDevice, s);
            dot(w.r, w.y, w.rz);
            continue;
          }
          st = inner_solve(w.r, w.rn2, w.y);
          if (st != BTI_OK) break;
          dot(w.y, w.r, w.zr);    // z_new . r_new
          dot(w.y, w.ro, w.zro);  // z_new . r_old
          cudaMemcpyAsync(w.num, w.zr, sizeof(double) * B, cudaMemcpyDeviceToDevice, s);
          count_dense(h, axpby_f64(w.num, w.zro, -1.0, 1.0, B, s));
          count_dense(h, cg_update_p(w.p, w.y, w.num, w.rz, n, B, s));
          std::swap(w.rz, w.zr);
        }
      }
    }
    if (st != BTI_OK) break;
    if (refine != 1) {  // the recursive CG residual drifts: report the true one
      st = true_residual(rel);
      if (st != BTI_OK) break;
    }
    converged = rel <= tol;
    st = apply_Gstar_accurate(h, w.x, m_map, B, w);
    if (st != BTI_OK) break;
    if (x_out) cudaMemcpyAsync(x_out, w.x, sizeof(double) * Bn, cudaMemcpyDeviceToDevice, s);
    st = launched(h, "solve_matfree");
    if (st == BTI_OK) st = cuda_check(h, cudaStreamSynchronize(s), "solve_matfree sync");
  } while (false);
  cudaStreamSynchronize(s);
  dev_free(buf);
  if (info) *info = bti_solve_info{outer, inner, rel};
  if (st == BTI_OK && !converged) {
    char msg[160];
    snprintf(msg, sizeof msg, "solve_matfree: relative residual %.3e above tol %.3e after %d outer, %d inner iterations",
             rel, tol, outer, inner);
    return fail(h, BTI_ERR_NO_CONVERGENCE, msg);
  }
  return st;
}

bti_status bti_set_qoi_stride(bti_handle h, int stride) {
  bti_status st = check_handle(h);
  if (st != BTI_OK) return st;
  if (stride < 1 || h->Nt % stride != 0) return fail(h, BTI_ERR_ARG, "set_qoi_stride: stride must divide N_t");
  if (stride != h->qstride) {
    drop_online_graph_any(h);
    h->Q_built = h->covq_built = false;
  }
  h->qstride = stride;
  return BTI_OK;
}

bti_status bti_apply_prior(bti_handle h, const double* v, double* out, int64_t B) {
  bti_status st = check_handle(h);
  if (st != BTI_OK) return st;
  if (B < 0) return fail(h, BTI_ERR_ARG, "apply_prior: B < 0");
  if (!h->prior_set) return fail(h, BTI_ERR_STATE, "apply_prior: no prior set");
  if (B == 0) return BTI_OK;
  if (!v || !out || v == out) return fail(h, BTI_ERR_ARG, "apply_prior: null or aliased pointers");
  return apply_se_rows(h, v, out, B * h->Nt);
}

bti_status bti_apply_postcov(bti_handle h, const double* v, double* out, int64_t B) {
  bti_status st = check_handle(h);
  if (st != BTI_OK) return st;
  if (B < 0) return fail(h, BTI_ERR_ARG, "apply_postcov: B < 0");
  if (!h->prior_set) return fail(h, BTI_ERR_STATE, "apply_postcov: no prior set");
  if (!h->K_factored || !h->op[BTI_OP_G].set) return fail(h, BTI_ERR_STATE, "apply_postcov: K not factored");
  if (B == 0) return BTI_OK;
  if (!v || !out || v == out) return fail(h, BTI_ERR_ARG, "apply_postcov: null or aliased pointers");
  const int64_t n = h->Nt * h->Nd, npar = h->Nt * h->Nm;
  // Eq. (4.7): out = w - G^* K^{-1} F w with w = Gamma_prior v
  st = apply_se_rows(h, v, out, B * h->Nt);
  if (st != BTI_OK) return st;
  double* z = nullptr;
  st = dev_alloc(h, (void**)&z, sizeof(double) * ((size_t)B * npar + (size_t)B * n), "postcov temporaries");
  if (st != BTI_OK) return st;
  double* y = z + (size_t)B * npar;
  st = apply_op(h, BTI_OP_F, false, out, y, B, BTI_P_F64, "postcov F");
  if (st == BTI_OK) st = infer_map_impl(h, y, z, B, 0);  // z = G^* K^{-1} y
  if (st == BTI_OK) {
    count_dense(h, axpby_f64(out, z, -1.0, 1.0, B * npar, h->stream));
    st = launched(h, "apply_postcov");
  }
  cudaStreamSynchronize(h->stream);
  dev_freep(z);
  return st;
}

bti_status bti_postcov_diag_probe(bti_handle h, const double* V, int64_t S, double* diag) {
  bti_status st = check_handle(h);
  if (st != BTI_OK) return st;
  if (S <= 0) return fail(h, BTI_ERR_ARG, "postcov_diag_probe: S must be > 0");
  if (!V || !diag) return fail(h, BTI_ERR_ARG, "postcov_diag_probe: null pointer");
  if (!h->prior_set) return fail(h, BTI_ERR_STATE, "postcov_diag_probe: no prior set");
  if (!h->K_factored || !h->op[BTI_OP_G].set) return fail(h, BTI_ERR_STATE, "postcov_diag_probe: K not factored");
  const int64_t npar = h->Nt * h->Nm;
  const int64_t Bp = S < 64 ? S : 64;  // probes per batch of Gamma_post(m) actions
  double* U = nullptr;
  st = dev_alloc(h, (void**)&U, sizeof(double) * ((size_t)Bp * npar + 2 * (size_t)npar), "probe temporaries");
  if (st != BTI_OK) return st;
  double* num = U + (size_t)Bp * npar;
  double* den = num + npar;
  cudaMemsetAsync(num, 0, sizeof(double) * 2 * (size_t)npar, h->stream);
  for (int64_t s0 = 0; s0 < S && st == BTI_OK; s0 += Bp) {
    const int64_t nb = S - s0 < Bp ? S - s0 : Bp;
    const double* Vb = V + (size_t)s0 * npar;
    st = bti_apply_postcov(h, Vb, U, nb);
    if (st == BTI_OK) {
      count_dense(h, probe_accumulate(Vb, U, nb, npar, num, den, h->stream));
      st = launched(h, "postcov_diag_probe");
    }
  }
  if (st == BTI_OK) {
    count_dense(h, probe_finish(num, den, diag, npar, h->stream));
    st = launched(h, "postcov_diag_probe");
  }
  cudaStreamSynchronize(h->stream);
  dev_freep(U);
  return st;
}

bti_status bti_infer_map_prior(bti_handle h, const double* d_obs, const double* m_prior, double* m_map, int64_t B,
                               int refine_iters) {
  bti_status st = check_handle(h);
  if (st != BTI_OK) return st;
  if (B < 0) return fail(h, BTI_ERR_ARG, "infer_map_prior: B < 0");
  if (B == 0) return BTI_OK;
  if (!d_obs || !m_prior || !m_map || m_prior == m_map)
    return fail(h, BTI_ERR_ARG, "infer_map_prior: null or aliased pointers");
  if (!h->K_factored || !h->op[BTI_OP_G].set) return fail(h, BTI_ERR_STATE, "infer_map_prior: K not factored");
  const int64_t n = h->Nt * h->Nd, npar = h->Nt * h->Nm;
  // Eq. (4.13) + Eq. (4.8): m_map = m_prior + G^* K^{-1} (d_obs - F m_prior)
  double* r = nullptr;
  st = dev_alloc(h, (void**)&r, sizeof(double) * (size_t)B * n, "prior-mean residual");
  if (st != BTI_OK) return st;
  st = apply_op(h, BTI_OP_F, false, m_prior, r, B, BTI_P_F64, "infer_map_prior F");
  if (st == BTI_OK) {
    count_dense(h, axpby_f64(r, d_obs, 1.0, -1.0, B * n, h->stream));
    st = infer_map_impl(h, r, m_map, B, refine_iters);
  }
  if (st == BTI_OK) {
    count_dense(h, axpby_f64(m_map, m_prior, 1.0, 1.0, B * npar, h->stream));
    st = launched(h, "infer_map_prior");
  }
  cudaStreamSynchronize(h->stream);
  dev_freep(r);
  return st;
}

bti_status bti_apply_elliptic(bti_handle h, int gx, int gy, double alpha1, double alpha2, const double* m,
                              double* out, int64_t B, int squared) {
  bti_status st = check_handle(h);
  if (st != BTI_OK) return st;
  if (gx <= 0 || gy <= 0 || B < 0 || !(alpha1 > 0.0) || !(alpha2 >= 0.0))
    return fail(h, BTI_ERR_ARG, "apply_elliptic: bad argument");
  if ((int64_t)gx * gy != h->Nm) return fail(h, BTI_ERR_SHAPE, "apply_elliptic: gx * gy != N_m");
  if (B == 0) return BTI_OK;
  if (!m || !out || m == out) return fail(h, BTI_ERR_ARG, "apply_elliptic: null or aliased pointers");
  const int64_t nblocks = B * h->Nt;
  if (!squared) {
    count_dense(h, elliptic_apply(m, out, gx, gy, alpha1, alpha2, nblocks, h->stream));
    return launched(h, "apply_elliptic");
  }
  // A_s^2 m = A_s (A_s m) through a temporary (A_s is symmetric, so this is A_s^T A_s m)
  double* tmp = nullptr;
  st = dev_alloc(h, (void**)&tmp, sizeof(double) * (size_t)nblocks * h->Nm, "elliptic temporary");
  if (st != BTI_OK) return st;
  int64_t nl = elliptic_apply(m, tmp, gx, gy, alpha1, alpha2, nblocks, h->stream);
  nl += elliptic_apply(tmp, out, gx, gy, alpha1, alpha2, nblocks, h->stream);
  count_dense(h, nl);
  st = launched(h, "apply_elliptic");
  cudaStreamSynchronize(h->stream);
  dev_freep(tmp);
  return st;
}

bti_status bti_predict_qoi(bti_handle h, const double* m_map, double* q_map, int64_t B) {
  return apply_op(h, BTI_OP_FQ, false, m_map, q_map, B, BTI_P_F64, "predict_qoi");
}

// Workspace the online phase needs for B vectors, allocated before a capture.
static bti_status reserve_online(bti_ctx* h, int64_t B) {
  bti_status st = reserve_solve(h, B);
  if (st != BTI_OK) return st;
  if (h->online_via_Q && Q_planes_ready(h) && B >= 16) {
    st = ensure(h, (void**)&h->wsolve, &h->wsolve_bytes, sizeof(double) * apply_Q_work_elems(h, B), "solve workspace");
    if (st != BTI_OK) return st;
  }
  if (h->online_via_Q && Q_pairs_ready(h) && B <= 2) {
    const int64_t n = h->Nt * h->Nd;
    st = ensure(h, (void**)&h->wsolve, &h->wsolve_bytes,
                sizeof(double) * ((size_t)2 * B * n + gemv_pairs_work_elems(n, B)), "solve workspace");
    if (st != BTI_OK) return st;
  }
  // spectral workspace: the larger of an adjoint (G*) and a forward (F, F_q) product
  const int64_t nf = h->nf, Nm = h->Nm;
  size_t adj = 16 * ((size_t)B * nf * Nm + (size_t)B * nf * h->Nd);
  if (h->op[BTI_OP_G].dig) adj += adj_digits_work_bytes(nf, h->Nd, B);
  size_t fwd = 0;
  for (int op = 0; op < 3; ++op) {
    if (op == BTI_OP_G || !h->op[op].set) continue;
    int64_t R = h->op[op].R;
    size_t f = 16 * ((size_t)B * nf * Nm + prod_fwd_partial_elems(nf, R, Nm, B) + (size_t)B * nf * R);
    if (h->op[op].dig_f) f += fwd_digits_work_bytes(nf, R, Nm);
    if (f > fwd) fwd = f;
  }
  size_t ws = adj > fwd ? adj : fwd;
  return ensure(h, &h->ws, &h->ws_bytes, ws, "workspace");
}

bti_status bti_online(bti_handle h, const double* d_obs, double* m_map, double* q_map, int64_t B,
                      int refine_iters) {
  bti_status st = check_handle(h);
  if (st != BTI_OK) return st;
  if (B <= 0 || refine_iters < 0) return fail(h, BTI_ERR_ARG, "online: B must be > 0 and refine_iters >= 0");
  const bool f32 = h->online_prec == BTI_P_F32;
  if (f32 && refine_iters > 0)
    return fail(h, BTI_ERR_ARG, "online: refinement needs the FP64-level form (bti_set_online_precision)");
  if (!d_obs || !m_map) return fail(h, BTI_ERR_ARG, "online: null pointer");
  if (!h->K_factored) return fail(h, BTI_ERR_STATE, "online: K not factored");
  if (!h->op[BTI_OP_G].set) return fail(h, BTI_ERR_STATE, "online: G blocks not set");
  if (q_map && !h->online_via_Q && !h->op[BTI_OP_FQ].set) return fail(h, BTI_ERR_STATE, "online: F_q blocks not set");
  if (q_map && h->online_via_Q && !h->Q_built) return fail(h, BTI_ERR_STATE, "online: q_map via Q but Q not built");
  if (!h->stream) return fail(h, BTI_ERR_STATE, "online: graph capture needs a non-default stream");
  const bool same = h->online_exec && h->og_d == d_obs && h->og_m == m_map && h->og_q == q_map && h->og_B == B &&
                    h->og_refine == refine_iters && h->og_prec == h->online_prec && h->og_stream == h->stream;
  if (!same) {
    drop_online_graph_any(h);
    st = reserve_online(h, B);
    if (st != BTI_OK) return st;
    const bool prof = h->prof_on;
    h->prof_on = false;  // no event records inside the graph
    st = cuda_check(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    if (st != BTI_OK) {
      h->prof_on = prof;
      return st;
    }
    if (f32) {
      // FP32-level form: the top five digit planes for K^{-1} (its error grows with kappa(K)),
      // four for G^*, F_q and Q
      h->planes_kinv = 5;
      h->planes_op = 4;
    }
    bti_status run = infer_map_impl(h, d_obs, m_map, B, refine_iters);
    if (run == BTI_OK && q_map)
      run = h->online_via_Q ? apply_Q_impl(h, d_obs, q_map, B)
                            : apply_op(h, BTI_OP_FQ, false, m_map, q_map, B, BTI_P_F64, "online F_q");
    h->planes_kinv = h->planes_op = 6;
    cudaGraph_t graph = nullptr;
    cudaError_t ee = cudaStreamEndCapture(h->stream, &graph);
    h->prof_on = prof;
    if (run != BTI_OK) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return run;
    }
    st = cuda_check(h, ee, "end capture");
    if (st != BTI_OK) return st;
    cudaGraphExec_t exec = nullptr;
    cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    st = cuda_check(h, ie, "instantiate online graph");
    if (st != BTI_OK) return st;
    h->online_exec = exec;
    h->og_d = d_obs;
    h->og_m = m_map;
    h->og_q = q_map;
    h->og_B = B;
    h->og_refine = refine_iters;
    h->og_prec = h->online_prec;
    h->og_stream = h->stream;
  }
  return cuda_check(h, cudaGraphLaunch(h->online_exec, h->stream), "launch online graph");
}

bti_status bti_autotune(bti_handle h, bti_op op, int64_t B, char* report, int64_t report_len) {
  bti_status st = check_handle(h);
  if (st != BTI_OK) return st;
  if (op < BTI_OP_F || op > BTI_OP_FQ || B <= 0) return fail(h, BTI_ERR_ARG, "autotune: bad op or B");
  OpStore& o = h->op[op];
  if (!o.set) return fail(h, BTI_ERR_STATE, "autotune: operator blocks not set");
  const int64_t Nt = h->Nt, Nm = h->Nm, R = o.R;
  // zeroed stand-in vectors (values do not affect the timing of these kernels)
  double *vin = nullptr, *vout = nullptr;
  size_t nvec = (size_t)B * Nt * Nm;
  st = dev_alloc(h, (void**)&vin, sizeof(double) * nvec, "autotune vectors");
  if (st != BTI_OK) return st;
  st = dev_alloc(h, (void**)&vout, sizeof(double) * nvec, "autotune vectors");
  if (st != BTI_OK) { dev_freep(vin); return st; }
  cudaMemsetAsync(vin, 0, sizeof(double) * nvec, h->stream);
  cudaMemsetAsync(vout, 0, sizeof(double) * nvec, h->stream);
  const bool prof = h->prof_on;
  h->prof_on = false;
  Tune& t = h->tune[o.prec];
  const Tune saved = t;
  auto fwd = [&]() { apply_op(h, op, false, vin, vout, B, BTI_P_F64, "autotune"); };
  auto adj = [&]() { apply_op(h, op, true, vout, vin, B, BTI_P_F64, "autotune"); };
  std::string rep = "{\"op\": " + std::to_string((int)op) + ", \"tier\": " + std::to_string((int)o.prec) +
                    ", \"B\": " + std::to_string(B);
  // 1. column pairs per FFT CTA, timed on the transforms alone: the forward FFT of the
  //    N_m-column input and the inverse FFT back to N_m columns (within a whole call the
  //    products' time would drown the difference)
  fwd();  // sizes the spectral workspace for B vectors
  const int64_t nf = h->nf;
  auto ffts = [&]() {
    if (double_path(o.prec)) {
      C2<double>* X = (C2<double>*)h->ws;
      rfft_in<double>(h, o, vin, Nm, Nt * Nm, X, nf * Nm, Nm, B, BTI_P_F64);
      irfft_out<double>(h, o, X, Nm, nf * Nm, vout, Nt * Nm, Nm, B, BTI_P_F64);
    } else {
      C2<float>* X = (C2<float>*)h->ws;
      rfft_in<float>(h, o, vin, Nm, Nt * Nm, X, nf * Nm, Nm, B, BTI_P_F64);
      irfft_out<float>(h, o, X, Nm, nf * Nm, vout, Nt * Nm, Nm, B, BTI_P_F64);
    }
  };
  {
    int best = 0;
    float best_ms = 1e30f;
    rep += ", \"fft_p\": {";
    bool first = true;
    for (int p = h->plan.P; p >= 1; p /= 2) {
      t.fft_p = p;
      float ms = time_ms(h, ffts, 5);
      rep += std::string(first ? "" : ", ") + "\"" + std::to_string(p) + "\": " + std::to_string(ms);
      first = false;
      if (ms < best_ms) { best_ms = ms; best = p; }
      if (p <= h->plan.P / 4) break;
    }
    t.fft_p = best;
    rep += "}, \"fft_p_chosen\": " + std::to_string(best);
  }
  // 2. columns per CTA of the forward product
  {
    const int cand[4] = {512, 1024, 2048, 4096};
    const int g = fwd_group(B);
    const size_t col_bytes = (o.prec == BTI_P_F64 || o.prec == BTI_P_DF64) ? 16 : 8;  // staged m-hat
    int& jc = t.jc[g == 4];
    int best = 0;
    float best_ms = 1e30f;
    rep += ", \"jc\": {";
    for (int c = 0; c < 4; ++c) {
      if (c > 0 && cand[c - 1] >= Nm) break;
      if ((size_t)g * cand[c] * col_bytes > kFwdSmemMax) break;
      jc = cand[c];
      float ms = time_ms(h, fwd, 3);
      rep += std::string(c ? ", " : "") + "\"" + std::to_string(cand[c]) + "\": " + std::to_string(ms);
      if (ms < best_ms) { best_ms = ms; best = cand[c]; }
    }
    jc = best;
    rep += "}, \"jc_chosen\": " + std::to_string(best);
  }
  // 3. columns per thread of the adjoint product (single-vector kernel)
  if (B < 4) {
    const int cand[3] = {2, 4, 8};
    int best = 0;
    float best_ms = 1e30f;
    rep += ", \"vpt\": {";
    for (int c = 0; c < 3; ++c) {
      t.vpt = cand[c];
      float ms = time_ms(h, adj, 3);
      rep += std::string(c ? ", " : "") + "\"" + std::to_string(cand[c]) + "\": " + std::to_string(ms);
      if (ms < best_ms) { best_ms = ms; best = cand[c]; }
    }
    t.vpt = best;
    rep += "}, \"vpt_chosen\": " + std::to_string(best);
  }
  rep += "}";
  h->prof_on = prof;
  (void)R;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  dev_freep(vin);
  dev_freep(vout);
  st = launched(h, "autotune");
  if (st == BTI_OK && e != cudaSuccess) st = cuda_check(h, e, "autotune sync");
  if (st != BTI_OK) {
    t = saved;
    return st;
  }
  if (report && report_len > 0) {
    size_t nc = rep.size() < (size_t)(report_len - 1) ? rep.size() : (size_t)(report_len - 1);
    memcpy(report, rep.data(), nc);
    report[nc] = 0;
  }
  return BTI_OK;
}

bti_status bti_sync(bti_handle h) {
  bti_status st = check_handle(h);
  if (st != BTI_OK) return st;
  int stat[2] = {0, 0};
  st = cuda_check(h, cudaMemcpyAsync(stat, h->status, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->stream),
                  "status");
  if (st != BTI_OK) return st;
  st = cuda_check(h, cudaStreamSynchronize(h->stream), "sync");
  if (st != BTI_OK) return st;
  st = launched(h, "sync");
  if (st != BTI_OK) return st;
  if (stat[1] != 0) {
    cudaMemsetAsync(h->status + 1, 0, sizeof(int), h->stream);  // reported once
    return fail(h, BTI_ERR_TIMEOUT, "device status: a bounded wait in a tensor-core product gave up");
  }
  if (stat[0] != 0) return fail(h, BTI_ERR_NOT_SPD, "device status: non-positive pivot " + std::to_string(stat[0]));
  return BTI_OK;
}

const char* bti_last_error(bti_handle h) { return h ? h->err.c_str() : "null handle"; }

}  // extern "C"

