// pp_select.cu -- the global energy selection of the *Q-SVDII (Alg. 4.2,
// steps 4-7): order all p*b squared singular values, find the first K whose
// cumulative energy reaches gamma times the total, and count each slice's
// members among the first K (rho_t).
//
// The order is the one the algorithm's permutation pi defines, made unique by
// a tie rule: sigma^2 descending, then slice ascending, then position within
// the slice ascending.  Each slice's values arrive sorted (descending), so
// the global position of entry (t, j) is
//   j + sum_{t' < t} #{sigma_{t'}^2 >= key} + sum_{t' > t} #{sigma_{t'}^2 > key},
// computed with one binary search per other slice (a merge-path rank), the
// slices split over the lanes of one warp per entry.  This
// is exact and deterministic, unlike a histogram-based radix select whose
// FP64 bucket sums would depend on atomic ordering.  Keys are sigma^2 formed
// in FP64 from the FP32 sigma (exact: a 24-bit significand squared fits).
//
// The cumulative sums run in FP64 in one CTA: 1024 contiguous chunks summed
// sequentially, a fixed-order scan of the chunk sums (warp shuffles, then the
// warp totals), then a second pass over each chunk to find the first crossing.
// rho_t is read off where the slice's ranks cross K (ranks increase along a
// slice), one writer per slice.  The result is deterministic.
#include "pp_internal.h"

namespace pp {
namespace {

constexpr int SEL_THREADS = 1024;

// Number of entries of the descending row `row` (length b) that come before a
// value v from another slice: sigma' >= v (ge, the other slice has the lower
// index) or sigma' > v.  sigma >= 0, so comparing the FP32 sigma is the same
// as comparing the FP64 keys sigma^2 (exact squares, monotone).
__device__ __forceinline__ int count_desc(const float *row, int b, float v, bool ge) {
  int lo = 0, hi = b;   // first index where the predicate fails
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const float s2 = row[mid];
    const bool in = ge ? (s2 >= v) : (s2 > v);
    if (in) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// One warp per entry (t, j): the lanes split the other slices' binary searches.
__global__ void select_rank_kernel(const float *__restrict__ sig, int64_t p, int b,
                                   double *__restrict__ keys_sorted, int32_t *__restrict__ rank,
                                   int use_smem) {
  extern __shared__ float ssig[];
  const int64_t N = p * b;
  const float *src = sig;
  if (use_smem) {
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) ssig[i] = sig[i];
    __syncthreads();
    src = ssig;
  }
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t e = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); e < N;
       e += warps) {
    const int64_t t = e / b;
    const int j = (int)(e % b);
    const float v = src[e];
    int64_t cnt = 0;
    for (int64_t t2 = lane; t2 < p; t2 += 32) {
      if (t2 == t) continue;
      cnt += count_desc(src + t2 * b, b, v, t2 < t);
    }
    for (int off = 16; off > 0; off >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
    if (lane == 0) {
      const int64_t pos = j + cnt;
      rank[e] = (int32_t)pos;
      keys_sorted[pos] = (double)v * (double)v;
    }
  }
}

// Inclusive scan of v over the CTA in a fixed order: a shuffle scan inside each
// warp, the warp totals scanned by warp 0, their prefix added back.
__device__ double block_inclusive_scan(double v, double *wsum) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (int)(blockDim.x >> 5);
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const double u = __shfl_up_sync(0xffffffffu, v, off);
    if (lane >= off) v += u;
  }
  if (lane == 31) wsum[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double w = lane < nw ? wsum[lane] : 0.0;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const double u = __shfl_up_sync(0xffffffffu, w, off);
      if (lane >= off) w += u;
    }
    wsum[lane] = w;
  }
  __syncthreads();
  if (warp > 0) v += wsum[warp - 1];
  __syncthreads();                            // wsum is reused by the next scan
  return v;
}

// The same scan for integers (exact in any order).
__device__ int64_t block_inclusive_scan_i64(int64_t v, int64_t *wsum) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (int)(blockDim.x >> 5);
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int64_t u = __shfl_up_sync(0xffffffffu, v, off);
    if (lane >= off) v += u;
  }
  if (lane == 31) wsum[warp] = v;
  __syncthreads();
  if (warp == 0) {
    int64_t w = lane < nw ? wsum[lane] : 0;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int64_t u = __shfl_up_sync(0xffffffffu, w, off);
      if (lane >= off) w += u;
    }
    wsum[lane] = w;
  }
  __syncthreads();
  if (warp > 0) v += wsum[warp - 1];
  __syncthreads();
  return v;
}

__global__ void __launch_bounds__(SEL_THREADS) select_finish_kernel(
    const double *__restrict__ keys_sorted, const int32_t *__restrict__ rank, int64_t p, int b,
    double gamma, int32_t *__restrict__ rho, int64_t *__restrict__ offs, double *__restrict__ scal,
    int64_t *__restrict__ Kout) {
  __shared__ double wsum[32];
  __shared__ int64_t isum[32];
  __shared__ double buf[SEL_THREADS];
  __shared__ unsigned long long Ksh;
  __shared__ double keptsh;
  const int tid = threadIdx.x;
  const int64_t N = p * b;
  const int64_t chunk = (N + SEL_THREADS - 1) / SEL_THREADS;
  const int64_t lo = tid * chunk, hi = min(N, lo + chunk);
  double s = 0.0;
  for (int64_t q = lo; q < hi; ++q) s += keys_sorted[q];
  // the exclusive prefix of a chunk is the previous thread's inclusive value,
  // so that the running sums below continue exactly where the scan left them
  buf[tid] = block_inclusive_scan(s, wsum);
  if (tid == 0) { Ksh = 0xffffffffffffffffull; keptsh = 0.0; }
  __syncthreads();
  const double total = buf[SEL_THREADS - 1];
  const double before = tid == 0 ? 0.0 : buf[tid - 1];
  if (total > 0.0 && lo < hi) {
    // running sums c_q = before + k_lo + ... + k_q in this order; a chunk whose
    // prefix already reaches the threshold crosses at its first key (keys are
    // >= 0), so only the chunks before the crossing walk their keys (FP64 is
    // a narrow pipe on this part)
    const double thresh = gamma * total;
    if (before >= thresh) {
      atomicMin(&Ksh, (unsigned long long)(lo + 1));
    } else {
      double c = before;
      for (int64_t q = lo; q < hi; ++q) {
        c += keys_sorted[q];
        if (c >= thresh) {
          atomicMin(&Ksh, (unsigned long long)(q + 1));
          break;
        }
      }
    }
  }
  __syncthreads();
  int64_t K = (total > 0.0) ? (int64_t)Ksh : 0;
  if (total > 0.0 && Ksh == 0xffffffffffffffffull) K = N;   // unreachable for gamma <= 1
  // kept energy c_K: the owning thread recomputes its running sum up to K
  if (K > 0 && lo < K && K <= hi) {
    double c = before;
    for (int64_t q = lo; q < K; ++q) c += keys_sorted[q];
    keptsh = c;
  }
  // per-slice ranks: rank[t*b + j] increases with j, so rho_t is the j where
  // the slice's ranks cross K; exactly one entry of each slice writes it
  for (int64_t e = tid; e < N; e += SEL_THREADS) {
    const int64_t t = e / b;
    const int j = (int)(e % b);
    const bool in = rank[e] < K;
    const bool next_in = j + 1 < b && rank[e + 1] < K;
    if (in && !next_in) rho[t] = j + 1;
    if (j == 0 && !in) rho[t] = 0;
  }
  __syncthreads();
  // offsets: exclusive scan of rho over p slices (chunked like the energies)
  const int64_t pchunk = (p + SEL_THREADS - 1) / SEL_THREADS;
  const int64_t plo = tid * pchunk, phi = min(p, plo + pchunk);
  int64_t cnt = 0;
  for (int64_t t = plo; t < phi; ++t) cnt += rho[t];
  const int64_t inc2 = block_inclusive_scan_i64(cnt, isum);
  int64_t run = inc2 - cnt;
  for (int64_t t = plo; t < phi; ++t) {
    offs[t] = run;
    run += rho[t];
  }
  if (tid == SEL_THREADS - 1) offs[p] = inc2;
  if (tid == 0) {
    scal[0] = keptsh;
    scal[1] = total;
    *Kout = K;
  }
}

}  // namespace

cudaError_t launch_select(const SelectArgs &a, cudaStream_t st) {
  const int64_t N = a.p * a.b;
  const size_t smem_need = (size_t)N * sizeof(float);
  const int use_smem = smem_need <= 160 * 1024;
  // at most one CTA per SM: each CTA stages all of sigma once, its 32 warps
  // then take entries in turn
  int blocks = (int)((N + 31) / 32);
  if (blocks > num_sms()) blocks = num_sms();
  cudaError_t e;
  if (use_smem) {
    e = cudaFuncSetAttribute(select_rank_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_need);
    if (e != cudaSuccess) return e;
  }
  count_launch(1);
  select_rank_kernel<<<blocks, 1024, use_smem ? smem_need : 0, st>>>(
      a.sig, a.p, (int)a.b, a.keys_sorted, a.rank, use_smem);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  count_launch(1);
  select_finish_kernel<<<1, SEL_THREADS, 0, st>>>(a.keys_sorted, a.rank, a.p, (int)a.b,
                                                  a.gamma, a.rho, a.offs, a.scal, a.K);
  return cudaGetLastError();
}

}  // namespace pp
