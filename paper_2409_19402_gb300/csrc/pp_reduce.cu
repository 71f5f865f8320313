// pp_reduce.cu -- FP64-accumulated reductions (energies of Thm. 4.2 / 4.4:
// |A|_F^2 and |A-hat|_F^2), input checks (Q^T Q = I for Q in St_{n,p}, finite
// input) and the device-written report.  Every reduction runs on a fixed grid
// with a fixed combination order, so results are bitwise reproducible.
#include <atomic>

#include "pp_internal.h"

namespace pp {
namespace {

constexpr int RED_MAX_BLOCKS = 2048;   // bound of the partial-sum buffers
constexpr int RED_THREADS = 256;

// two CTAs per SM, within the partial-buffer bound
int red_blocks() {
  const int b = 2 * num_sms();
  return b < RED_MAX_BLOCKS ? b : RED_MAX_BLOCKS;
}

// Sum over the CTA (result in thread 0) in a fixed tree: a shuffle tree in
// each warp, then one over the warp totals in warp 0 (FP64 adds are slow on
// this part, so no thread walks the 32 totals one dependent add at a time).
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[32];
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (warp == 0) {
    s = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  }
  __syncthreads();
  return s;
}

__global__ void __launch_bounds__(RED_THREADS) sumsq_kernel(const float *__restrict__ x, int64_t n,
                                                            double *__restrict__ partials) {
  double acc = 0.0;
  const int64_t n4 = ((reinterpret_cast<uintptr_t>(x) & 15) == 0) ? n / 4 : 0;
  const float4 *x4 = reinterpret_cast<const float4 *>(x);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float4 v = x4[i];
    acc += (double)v.x * v.x + (double)v.y * v.y + (double)v.z * v.z + (double)v.w * v.w;
  }
  for (int64_t i = 4 * n4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    acc += (double)x[i] * x[i];
  const double s = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void sum_partials_kernel(const double *__restrict__ partials, int n,
                                    double *__restrict__ out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partials[i];
  const double s = block_sum(acc);
  if (threadIdx.x == 0) *out = s;
}

// max |(Q^T Q)_{ab} - delta_ab| > tol -> PP_ENOTORTHO; one thread per (a, b), b >= a
__global__ void check_q_kernel(const float *__restrict__ Q, int64_t n, int64_t p, float tol,
                               int32_t *status) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= p * p) return;
  const int64_t a = idx / p, b = idx % p;
  if (b < a) return;
  double acc = 0.0;
  for (int64_t s = 0; s < n; ++s) acc += (double)Q[s * p + a] * Q[s * p + b];
  const double dev = fabs(acc - (a == b ? 1.0 : 0.0));
  if (!(dev <= (double)tol)) set_status(status, PP_ENOTORTHO);
}

__global__ void check_finite_kernel(const float *__restrict__ x, int64_t n, int32_t *status) {
  bool bad = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    bad |= !isfinite(x[i]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) set_status(status, PP_ENONFINITE);
}

// the sum of n partials in the order of sum_partials_kernel (blockDim 1024)
__device__ __forceinline__ double sum_partials_block(const double *partials, int n) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partials[i];
  return block_sum(acc);
}

__global__ void __launch_bounds__(1024) report_kernel(ReportArgs a) {
  __shared__ int32_t sw_warp[32];
  double e[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int i = 0; i < 3; ++i)
    if (a.parts[i]) e[i] = sum_partials_block(a.parts[i], a.nparts[i]);
  // the largest sweep count, every thread taking a share of the slices (one
  // thread walking all of them waits for each load in turn)
  int32_t sw = 0;
  for (int64_t t = threadIdx.x; t < a.p; t += blockDim.x) sw = max(sw, a.sweeps[t]);
  sw = __reduce_max_sync(0xffffffffu, sw);
  if ((threadIdx.x & 31) == 0) sw_warp[threadIdx.x >> 5] = sw;
  // fixed-k path: kept and discarded energies, summed like the partials
  double kept = 0.0, disc = 0.0;
  if (!a.sel_scal) {
    kept = sum_partials_block(a.kept_partial, (int)a.p);
    disc = sum_partials_block(a.disc_partial, (int)a.p);
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sw = max(sw, sw_warp[w]);
#pragma unroll
  for (int i = 0; i < 3; ++i)
    if (a.parts[i]) a.sums[i] = e[i];
  pp_report r;
  r.status = *a.status;
  r.sweeps = sw;
  r.normA2 = a.parts[0] ? e[0] : *a.normA2;
  r.normAh2 = a.parts[1] ? e[1] : *a.normAh2;
  r.err2 = a.parts[2] ? e[2] : (a.err2 ? *a.err2 : -1.0);
  if (a.sel_scal) {
    r.K = *a.K;
    r.kappa = a.offs[a.p];
    r.kept2 = a.sel_scal[0];
    r.discarded2 = a.sel_scal[1] - a.sel_scal[0];
  } else {
    r.K = 0;
    r.kappa = a.kappa_fixed;
    r.kept2 = kept;
    r.discarded2 = disc;
  }
  r.proj_err2 = r.normA2 - r.normAh2;
  *a.rep = r;
}

__global__ void hosvd_report_kernel(HosvdReportArgs a) {   // one warp
  int32_t sw = 0;
  for (int64_t t = threadIdx.x; t < a.p; t += 32) sw = max(sw, a.sweeps[t]);
  sw = __reduce_max_sync(0xffffffffu, sw);
  if (threadIdx.x != 0) return;
  pp_hosvd_report r;
  r.status = *a.status;
  r.sweeps = sw;
  r.k1 = a.k1;
  r.k2 = a.k2;
  r.k = a.k;
  r.normA2 = *a.normA2;
  r.err2_hosvd = *a.err2_hosvd;
  r.err2_tsvdq = *a.err2_tsvdq;
  r.proj_err2 = r.normA2 - *a.normAh2;
  *a.rep = r;
}

}  // namespace

int64_t sumsq_max_partials() { return RED_MAX_BLOCKS; }

int num_sms() {
  constexpr int MAXDEV = 64;
  static std::atomic<int> cached[MAXDEV];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAXDEV) return 152;
  const int c = cached[dev].load(std::memory_order_relaxed);
  if (c > 0) return c;
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
    cudaGetLastError();
    return 152;
  }
  cached[dev].store(n, std::memory_order_relaxed);   // concurrent first calls store the same value
  return n;
}

cudaError_t launch_hosvd_report(const HosvdReportArgs &a, cudaStream_t st) {
  count_launch(1);
  hosvd_report_kernel<<<1, 32, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_sumsq(const float *x, int64_t n, double *partials, int *n_partials,
                         cudaStream_t st) {
  const int blocks = red_blocks();
  *n_partials = blocks;
  count_launch(1);
  sumsq_kernel<<<blocks, RED_THREADS, 0, st>>>(x, n, partials);
  return cudaGetLastError();
}

cudaError_t launch_sum_partials(const double *partials, int n_partials, double *out,
                                cudaStream_t st) {
  count_launch(1);
  sum_partials_kernel<<<1, 1024, 0, st>>>(partials, n_partials, out);
  return cudaGetLastError();
}

cudaError_t launch_check_q(const float *Q, int64_t n, int64_t p, float tol, int32_t *status,
                           cudaStream_t st) {
  const int64_t total = p * p;
  count_launch(1);
  check_q_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(Q, n, p, tol, status);
  return cudaGetLastError();
}

cudaError_t launch_check_finite(const float *x, int64_t n, int32_t *status, cudaStream_t st) {
  count_launch(1);
  check_finite_kernel<<<red_blocks(), RED_THREADS, 0, st>>>(x, n, status);
  return cudaGetLastError();
}

cudaError_t launch_report(const ReportArgs &a, cudaStream_t st) {
  count_launch(1);
  report_kernel<<<1, 1024, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace pp
