// bti_apply_F_noalloc: d = F m for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc / cudaFree: code whose device memory is
// owned entirely by another allocator (a framework's pool, or a fixed budget
// reserved at start-up), and latency-critical online callers, for which
// cudaFree's implicit device-wide synchronisation and cudaMalloc's unbounded
// cost are not acceptable.  This entry point gives them the p2o matvec without
// any handle or allocation: every intermediate (twiddle table, spectral
// blocks, frequency-domain vectors, reduction partials) lives in one
// file-scope device array of fixed size that is part of the loaded library.
#include "bti_internal.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

namespace {

// Scratch shared by every call on a device.  Holds the last call's contents;
// every element a call reads is written by that call first, so nothing needs
// clearing.  Calls that overlap on the GPU (different streams, or other host
// threads) race on it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[BTI_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
// per device: the context the address was resolved in, and the address
void* g_ctx[kMaxDevices] = {nullptr};
void* g_ptr[kMaxDevices] = {nullptr};

// The driver's current context (null if none is current yet), through the runtime's
// entry-point query, so the library needs no link to the driver library.
cudaError_t current_context(void** ctx) {
  static PFN_cuCtxGetCurrent_v4000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !p) return cudaErrorNotSupported;
    fn = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p);
  }
  CUcontext c = nullptr;
  if (fn(&c) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
  *ctx = c;
  return cudaSuccess;
}

// Device address of the scratch array in the current context.  Set-up, once per device and
// context: with that device current, cudaGetSymbolAddress resolves the address (initialising
// the device's primary context if no context is current yet), and the address is kept with
// the context it belongs to.  A different current context on the same device (after
// cudaDeviceReset, or a caller's own context) holds its own copy of the module, so the address
// is resolved again there rather than reused.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  void* ctx = nullptr;
  e = current_context(&ctx);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!ctx || !g_ptr[dev] || g_ctx[dev] != ctx) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    e = current_context(&ctx);
    if (e != cudaSuccess) return e;
    g_ptr[dev] = p;
    g_ctx[dev] = ctx;
  }
  *out = g_ptr[dev];
  return cudaSuccess;
}

// tw[k] = e^{-2 pi i k / L}
__global__ void twiddle_kernel(double2* tw, int L) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= L) return;
  double s, c;
  sincospi(2.0 * (double)k / (double)L, &s, &c);
  tw[k] = make_double2(c, -s);
}

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

extern "C" bti_status bti_apply_F_noalloc(const double* blocks, const double* m, double* d, int64_t Nm,
                                          int64_t Nd, int64_t Nt, int64_t B, void* cuda_stream) {
  using namespace bti;
  if (!blocks || !m || !d || Nm <= 0 || Nd <= 0 || Nt <= 0 || B <= 0) return BTI_ERR_ARG;
  FftPlan plan;
  if (2 * Nt > kMaxL || !fft_plan_factor(plan, (int)(2 * Nt))) return BTI_ERR_ARG;
  const int64_t nf = Nt + 1, L = 2 * Nt;
  // scratch layout, each piece 256-byte aligned (elements are double2)
  const size_t c = sizeof(double2);
  const size_t b_tw = round256(c * (size_t)L);
  const size_t b_F = round256(c * (size_t)(nf * Nd) * (size_t)Nm);
  const size_t b_m = round256(c * (size_t)(B * nf) * (size_t)Nm);
  const size_t b_p = round256(c * prod_fwd_partial_elems(nf, Nd, Nm, B));
  const size_t b_d = round256(c * (size_t)(B * nf * Nd));
  // overflow-safe size check: each factor is bounded before the products above matter
  if ((double)Nm * (double)nf * (double)(Nd + B) * (double)c > (double)BTI_NOALLOC_SCRATCH_BYTES ||
      b_tw + b_F + b_m + b_p + b_d > (size_t)BTI_NOALLOC_SCRATCH_BYTES)
    return BTI_ERR_SHAPE;
  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) {
    cudaGetLastError();
    return BTI_ERR_CUDA;
  }
  unsigned char* p = static_cast<unsigned char*>(base);
  double2* tw = reinterpret_cast<double2*>(p);
  double2* Fhat = reinterpret_cast<double2*>(p + b_tw);
  double2* mhat = reinterpret_cast<double2*>(p + b_tw + b_F);
  double2* part = reinterpret_cast<double2*>(p + b_tw + b_F + b_m);
  double2* dhat = reinterpret_cast<double2*>(p + b_tw + b_F + b_m + b_p);
  plan.tw64 = tw;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  twiddle_kernel<<<(unsigned)((L + 255) / 256), 256, 0, s>>>(tw, (int)L);
  // spectral blocks of F (Sec. 4: block circulant embedding diagonalised by the DFT)
  launch_rfft_cols<double, double, double>(plan, (int)Nt, blocks, Nd * Nm, 0, Fhat, 0, Nd * Nm, 1, s);
  launch_rfft_cols<double, double, double>(plan, (int)Nt, m, Nm, Nt * Nm, mhat, nf * Nm, Nm, B, s);
  launch_prod_fwd<double, double>(Fhat, mhat, part, nf, Nd, Nm, B, s);
  launch_reduce_chunks<double>(part, dhat, nf, Nd, Nm, B, s);
  launch_irfft_cols<double, double, double>(plan, (int)Nt, dhat, Nd, nf * Nd, d, Nt * Nd, Nd, B, 1.0 / (double)L, s);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? BTI_OK : BTI_ERR_CUDA;
}
