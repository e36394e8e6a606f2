// Vector kernels of the matrix-free data-space solve: batched dot products with a
// fixed reduction order, the conjugate-gradient updates with per-vector scalars kept
// on the device, and the scaled conversions between the FP64 refinement loop and the
// FP32 inner iteration.  Vectors are [B][n] row-major; blockIdx.y selects the vector.

#include "bti_internal.cuh"

namespace bti {

namespace {

constexpr int kDotBlocks = 128;  // partial sums per vector (fixed: the order is deterministic)

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// part[b][blk] = sum over the block's grid-stride slice of x[b][i] y[b][i]
template <typename T>
__global__ void __launch_bounds__(256) dot_partial_kernel(const T* __restrict__ x, const T* __restrict__ y,
                                                          int64_t n, double* __restrict__ part) {
  __shared__ double red[8];
  const int64_t b = blockIdx.y;
  const T* xb = x + b * n;
  const T* yb = y + b * n;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc = fma((double)xb[i], (double)yb[i], acc);
  acc = warp_sum(acc);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = acc;
  __syncthreads();
  if (wid == 0) {
    double v = lane < 8 ? red[lane] : 0.0;
    v = warp_sum(v);
    if (lane == 0) part[b * gridDim.x + blockIdx.x] = v;
  }
}

// out[b] = sum of the kDotBlocks partials of vector b, one warp per vector
__global__ void dot_final_kernel(const double* __restrict__ part, double* __restrict__ out, int64_t B) {
  const int64_t b = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (b >= B) return;
  double v = 0.0;
  for (int k = lane; k < kDotBlocks; k += 32) v += part[b * kDotBlocks + k];
  v = warp_sum(v);
  if (lane == 0) out[b] = v;
}

inline dim3 vec_grid(int64_t n, int64_t B) {
  int64_t gx = (n + 1023) / 1024;
  if (gx > 1024) gx = 1024;
  if (gx < 1) gx = 1;
  return dim3((unsigned)gx, (unsigned)B);
}

// x[b] += alpha_b p[b], r[b] -= alpha_b q[b], alpha_b = rr[b] / pq[b] (0 on breakdown)
template <typename T>
__global__ void cg_xr_kernel(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p, const T* __restrict__ q,
                             const double* __restrict__ rr, const double* __restrict__ pq, int64_t n) {
  const int64_t b = blockIdx.y;
  const double den = pq[b];
  const T alpha = (T)((den > 0.0 && rr[b] > 0.0) ? rr[b] / den : 0.0);
  T* xb = x + b * n;
  T* rb = r + b * n;
  const T* pb = p + b * n;
  const T* qb = q + b * n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    xb[i] += alpha * pb[i];
    rb[i] -= alpha * qb[i];
  }
}

// p[b] = r[b] + beta_b p[b], beta_b = rr_new[b] / rr_old[b] (0 on breakdown)
template <typename T>
__global__ void cg_p_kernel(T* __restrict__ p, const T* __restrict__ r, const double* __restrict__ rr_new,
                            const double* __restrict__ rr_old, int64_t n) {
  const int64_t b = blockIdx.y;
  const double den = rr_old[b];
  const T beta = (T)(den > 0.0 ? rr_new[b] / den : 0.0);
  T* pb = p + b * n;
  const T* rb = r + b * n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    pb[i] = rb[i] + beta * pb[i];
}

// q[b][i] = y[b][i] + nz_i p[b][i] with nz_i = diag[i] (diag != null) or sigma2; q may alias y
template <typename T>
__global__ void add_noise_kernel(T* q, const T* y, const T* __restrict__ p,
                                 const double* __restrict__ diag, double sigma2, int64_t n) {
  const int64_t b = blockIdx.y;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const T nz = (T)(diag ? diag[i] : sigma2);
    q[b * n + i] = y[b * n + i] + nz * p[b * n + i];
  }
}

// out[b][i] = (float)(x[b][i] / norm[b]) (zero vector when norm[b] == 0)
__global__ void normalize_to_f32_kernel(const double* __restrict__ x, const double* __restrict__ nrm2,
                                        float* __restrict__ out, int64_t n) {
  const int64_t b = blockIdx.y;
  const double nb = sqrt(nrm2[b]);
  const double s = nb > 0.0 ? 1.0 / nb : 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[b * n + i] = (float)(x[b * n + i] * s);
}

// x[b][i] += sqrt(nrm2[b]) * (double)d[b][i]
__global__ void add_scaled_f32_kernel(double* __restrict__ x, const float* __restrict__ d,
                                      const double* __restrict__ nrm2, int64_t n) {
  const int64_t b = blockIdx.y;
  const double s = sqrt(nrm2[b]);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[b * n + i] = fma(s, (double)d[b * n + i], x[b * n + i]);
}

template <typename TI, typename TO>
__global__ void convert_kernel(const TI* __restrict__ x, TO* __restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (TO)x[i];
}

// z[b][t][i] = sum_j P[t][i][j] r[b][t][j]: the block-Jacobi preconditioner, one R x R block
// per time step.  grid (N_t, ceil(R / 32)); each warp takes 4 rows, lanes stride the row
// (coalesced), and the vectors' block r_t is staged in shared memory 8 vectors at a time.
constexpr int kPcVec = 8;
template <typename T>
__global__ void __launch_bounds__(256) block_precond_kernel(const double* __restrict__ P, const T* __restrict__ r,
                                                            T* __restrict__ z, int64_t Nt, int64_t R, int64_t B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* rs = reinterpret_cast<double*>(smem_raw);  // [kPcVec][R]
  const int64_t t = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n = Nt * R;
  const double* Pt = P + t * R * R;
  for (int64_t b0 = 0; b0 < B; b0 += kPcVec) {
    const int nb = (int)((B - b0) < kPcVec ? (B - b0) : kPcVec);
    __syncthreads();
    for (int64_t e = threadIdx.x; e < (int64_t)nb * R; e += blockDim.x) {
      const int64_t bb = e / R, j = e - bb * R;
      rs[bb * R + j] = (double)r[(b0 + bb) * n + t * R + j];
    }
    __syncthreads();
    for (int q = 0; q < 4; ++q) {
      const int64_t i = (int64_t)blockIdx.y * 32 + warp * 4 + q;
      if (i >= R) break;
      double acc[kPcVec];
#pragma unroll
      for (int bb = 0; bb < kPcVec; ++bb) acc[bb] = 0.0;
      const double* row = Pt + i * R;
      for (int64_t j = lane; j < R; j += 32) {
        const double pv = __ldg(row + j);
#pragma unroll
        for (int bb = 0; bb < kPcVec; ++bb)
          if (bb < nb) acc[bb] = fma(pv, rs[bb * R + j], acc[bb]);
      }
#pragma unroll
      for (int bb = 0; bb < kPcVec; ++bb) {
        double v = warp_sum(acc[bb]);
        if (lane == 0 && bb < nb) z[(b0 + bb) * n + t * R + i] = (T)v;
      }
    }
  }
}

}  // namespace

size_t dot_workspace_elems(int64_t B) { return (size_t)B * kDotBlocks; }

template <typename T>
int block_precond_apply(const double* P, const T* r, T* z, int64_t Nt, int64_t R, int64_t B, cudaStream_t s) {
  if (Nt <= 0 || R <= 0 || B <= 0) return 0;
  const size_t smem = sizeof(double) * kPcVec * (size_t)R;
  if (smem > 48 * 1024) cudaFuncSetAttribute(block_precond_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dim3 grid((unsigned)Nt, (unsigned)((R + 31) / 32));
  block_precond_kernel<T><<<grid, 256, smem, s>>>(P, r, z, Nt, R, B);
  return 1;
}
template int block_precond_apply<float>(const double*, const float*, float*, int64_t, int64_t, int64_t, cudaStream_t);
template int block_precond_apply<double>(const double*, const double*, double*, int64_t, int64_t, int64_t,
                                         cudaStream_t);

int convert_f32_f64(const float* x, double* y, int64_t n, cudaStream_t s) {
  if (n <= 0) return 0;
  convert_kernel<float, double><<<vec_grid(n, 1), 256, 0, s>>>(x, y, n);
  return 1;
}
int convert_f64_f32(const double* x, float* y, int64_t n, cudaStream_t s) {
  if (n <= 0) return 0;
  convert_kernel<double, float><<<vec_grid(n, 1), 256, 0, s>>>(x, y, n);
  return 1;
}

template <typename T>
int dot_batched(const T* x, const T* y, int64_t n, int64_t B, double* part, double* out, cudaStream_t s) {
  if (B <= 0) return 0;
  dot_partial_kernel<T><<<dim3(kDotBlocks, (unsigned)B), 256, 0, s>>>(x, y, n, part);
  dot_final_kernel<<<(unsigned)((B + 7) / 8), 256, 0, s>>>(part, out, B);
  return 2;
}

template <typename T>
int cg_update_xr(T* x, T* r, const T* p, const T* q, const double* rr, const double* pq, int64_t n, int64_t B,
                 cudaStream_t s) {
  if (B <= 0 || n <= 0) return 0;
  cg_xr_kernel<T><<<vec_grid(n, B), 256, 0, s>>>(x, r, p, q, rr, pq, n);
  return 1;
}

template <typename T>
int cg_update_p(T* p, const T* r, const double* rr_new, const double* rr_old, int64_t n, int64_t B, cudaStream_t s) {
  if (B <= 0 || n <= 0) return 0;
  cg_p_kernel<T><<<vec_grid(n, B), 256, 0, s>>>(p, r, rr_new, rr_old, n);
  return 1;
}

template <typename T>
int add_noise(T* q, const T* y, const T* p, const double* diag, double sigma2, int64_t n, int64_t B, cudaStream_t s) {
  if (B <= 0 || n <= 0) return 0;
  add_noise_kernel<T><<<vec_grid(n, B), 256, 0, s>>>(q, y, p, diag, sigma2, n);
  return 1;
}

int normalize_to_f32(const double* x, const double* nrm2, float* out, int64_t n, int64_t B, cudaStream_t s) {
  if (B <= 0 || n <= 0) return 0;
  normalize_to_f32_kernel<<<vec_grid(n, B), 256, 0, s>>>(x, nrm2, out, n);
  return 1;
}

int add_scaled_f32(double* x, const float* d, const double* nrm2, int64_t n, int64_t B, cudaStream_t s) {
  if (B <= 0 || n <= 0) return 0;
  add_scaled_f32_kernel<<<vec_grid(n, B), 256, 0, s>>>(x, d, nrm2, n);
  return 1;
}

template int dot_batched<float>(const float*, const float*, int64_t, int64_t, double*, double*, cudaStream_t);
template int dot_batched<double>(const double*, const double*, int64_t, int64_t, double*, double*, cudaStream_t);
template int cg_update_xr<float>(float*, float*, const float*, const float*, const double*, const double*, int64_t,
                                 int64_t, cudaStream_t);
template int cg_update_xr<double>(double*, double*, const double*, const double*, const double*, const double*,
                                  int64_t, int64_t, cudaStream_t);
template int cg_update_p<float>(float*, const float*, const double*, const double*, int64_t, int64_t, cudaStream_t);
template int cg_update_p<double>(double*, const double*, const double*, const double*, int64_t, int64_t,
                                 cudaStream_t);
template int add_noise<float>(float*, const float*, const float*, const double*, double, int64_t, int64_t,
                              cudaStream_t);
template int add_noise<double>(double*, const double*, const double*, const double*, double, int64_t, int64_t,
                               cudaStream_t);

// ------------------------------------------------------------------ variance probes
// num[e] += sum_k V[k][e] U[k][e], den[e] += sum_k V[k][e]^2 over nb probes (fixed order k),
// for the probe estimate of the pointwise posterior variances.
__global__ void probe_accumulate_kernel(const double* __restrict__ V, const double* __restrict__ U, int64_t nb,
                                        int64_t n, double* __restrict__ num, double* __restrict__ den) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  double a = num[e], b = den[e];
  for (int64_t k = 0; k < nb; ++k) {
    const double v = V[k * n + e];
    a = fma(v, U[k * n + e], a);
    b = fma(v, v, b);
  }
  num[e] = a;
  den[e] = b;
}
__global__ void probe_finish_kernel(const double* __restrict__ num, const double* __restrict__ den,
                                    double* __restrict__ out, int64_t n) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) out[e] = den[e] > 0.0 ? num[e] / den[e] : 0.0;
}
int probe_accumulate(const double* V, const double* U, int64_t nb, int64_t n, double* num, double* den,
                     cudaStream_t s) {
  if (n <= 0 || nb <= 0) return 0;
  probe_accumulate_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(V, U, nb, n, num, den);
  return 1;
}
int probe_finish(const double* num, const double* den, double* out, int64_t n, cudaStream_t s) {
  if (n <= 0) return 0;
  probe_finish_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(num, den, out, n);
  return 1;
}


}  // namespace bti
