// pp_jacobi.cu -- batched one-sided (Hestenes) Jacobi SVD of the p frontal
// slices of A-hat (the "truncated matrix SVDs of frontal slices" of Alg. 4.1
// step 3 and the facewise SVD of Alg. 4.2 step 3).
//
// One CTA per slice.  The b = min(l, m) vectors of length a = max(l, m) (rows
// of the slice if l <= m, else its columns) live in shared memory, padded to
// a_pad floats.  A sweep is b-1 rounds of the round-robin ("circle") pairing;
// the b/2 pairs of a round are disjoint and processed concurrently, one pair
// per group of G lanes.  Each lane holds a_pad/(4G) float4 chunks of both
// vectors in registers, forms the three inner products, reduces them across
// the group with xor shuffles (bitwise identical in every lane), and applies
// the symmetric 2x2 Schur rotation in Rutishauser's tau form.  A pair whose
// |cos| is at most `tol` is left alone; a sweep without any rotation ends the
// iteration.
//
// Slices that do not fit in shared memory are processed block-cyclically:
// the vectors live in global memory (the W output array, resident in L2),
// and each outer sweep visits every pair of blocks (I, J), loads the 2*bs
// vectors into shared memory and runs one round-robin pass over their union.
//
// Output per slice: the converged vectors W (unnormalised: w_j = sigma_j y_j),
// sigma descending (FP64-accumulated norms rounded to FP32), the permutation
// sorted position -> vector index (ties: lower vector index first) and the
// number of sweeps.  Non-convergence within max_sweeps writes PP_ENOCONV.
//
// All arithmetic is FP32 except the final norms (FP64 accumulation).  The
// rotation angle is computed in FP32 with IEEE division and square roots;
// FP64 is avoided in the inner loop because this part's FP64 rate is a small
// fraction of its FP32 rate.
#include "pp_internal.h"

namespace pp {
namespace {

constexpr int NV_MAX = 6;                 // float4 chunks per lane per vector
constexpr int SMEM_BUDGET = 200 * 1024;   // bytes of shared memory for vectors

// Circle-method pairing of N (even) players: round r in [0, N-1), slot in [0, N/2).
__device__ __forceinline__ void circle_pair(int N, int r, int slot, int &j, int &k) {
  if (slot == 0) {
    j = r;
    k = N - 1;
  } else {
    j = (r + slot) % (N - 1);
    k = (r - slot + (N - 1)) % (N - 1);
  }
}

template <int G>
__device__ __forceinline__ float group_sum(float v, unsigned mask) {
#pragma unroll
  for (int off = G / 2; off > 0; off >>= 1) v += __shfl_xor_sync(mask, v, off, G);
  return v;
}

// Process one pair held in shared memory; returns true if a rotation was applied.
template <int G>
__device__ __forceinline__ bool jacobi_pair(float *__restrict__ x, float *__restrict__ y, int nv,
                                            float tol, int lg, unsigned mask) {
  float4 xv[NV_MAX], yv[NV_MAX];
  float al = 0.f, be = 0.f, ga = 0.f;
#pragma unroll
  for (int q = 0; q < NV_MAX; ++q) {
    if (q < nv) {
      xv[q] = reinterpret_cast<const float4 *>(x)[lg + q * G];
      yv[q] = reinterpret_cast<const float4 *>(y)[lg + q * G];
      al = fmaf(xv[q].x, xv[q].x, al); al = fmaf(xv[q].y, xv[q].y, al);
      al = fmaf(xv[q].z, xv[q].z, al); al = fmaf(xv[q].w, xv[q].w, al);
      be = fmaf(yv[q].x, yv[q].x, be); be = fmaf(yv[q].y, yv[q].y, be);
      be = fmaf(yv[q].z, yv[q].z, be); be = fmaf(yv[q].w, yv[q].w, be);
      ga = fmaf(xv[q].x, yv[q].x, ga); ga = fmaf(xv[q].y, yv[q].y, ga);
      ga = fmaf(xv[q].z, yv[q].z, ga); ga = fmaf(xv[q].w, yv[q].w, ga);
    }
  }
  al = group_sum<G>(al, mask);
  be = group_sum<G>(be, mask);
  ga = group_sum<G>(ga, mask);
  if (ga == 0.f || fabsf(ga) <= tol * sqrtf(al) * sqrtf(be)) return false;
  const float zeta = (be - al) / (2.f * ga);
  const float az = fabsf(zeta);
  float t;
  if (az > 1e15f) t = 0.5f / zeta;
  else t = copysignf(1.f, zeta) / (az + sqrtf(1.f + zeta * zeta));
  const float c = 1.f / sqrtf(1.f + t * t);
  const float s = c * t;
  // Rutishauser's form x' = x - s (y + tau x), y' = y + s (x - tau y) with
  // tau = s / (1 + c): the implied cosine 1 - s tau stays accurate when c
  // itself rounds to 1 (small angles), so the rotation stays orthogonal to
  // working precision instead of growing the norms by ~t^2/2 per rotation.
  const float tau = s / (1.f + c);
#pragma unroll
  for (int q = 0; q < NV_MAX; ++q) {
    if (q < nv) {
      float4 nx, ny;
      nx.x = fmaf(-s, fmaf(tau, xv[q].x, yv[q].x), xv[q].x);
      ny.x = fmaf(s, fmaf(-tau, yv[q].x, xv[q].x), yv[q].x);
      nx.y = fmaf(-s, fmaf(tau, xv[q].y, yv[q].y), xv[q].y);
      ny.y = fmaf(s, fmaf(-tau, yv[q].y, xv[q].y), yv[q].y);
      nx.z = fmaf(-s, fmaf(tau, xv[q].z, yv[q].z), xv[q].z);
      ny.z = fmaf(s, fmaf(-tau, yv[q].z, xv[q].z), yv[q].z);
      nx.w = fmaf(-s, fmaf(tau, xv[q].w, yv[q].w), xv[q].w);
      ny.w = fmaf(s, fmaf(-tau, yv[q].w, xv[q].w), yv[q].w);
      reinterpret_cast<float4 *>(x)[lg + q * G] = nx;
      reinterpret_cast<float4 *>(y)[lg + q * G] = ny;
    }
  }
  return true;
}

// One round-robin pass over the nvec vectors held in Ws (rows of a_pad floats).
// Returns this thread's rotation count (counted once per group, by lane 0).
template <int G>
__device__ int round_robin_pass(float *Ws, int nvec, int a_pad, int nv, float tol) {
  const int lane = threadIdx.x & 31;
  const int lg = lane % G;                       // lane within the group
  const int grp = threadIdx.x / G;
  const int ngroups = blockDim.x / G;
  const unsigned mask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane - lg));
  const int N = nvec + (nvec & 1);
  int rot = 0;
  for (int r = 0; r < N - 1; ++r) {
    for (int slot = grp; slot < N / 2; slot += ngroups) {
      int j, k;
      circle_pair(N, r, slot, j, k);
      if (j >= nvec || k >= nvec) continue;
      if (jacobi_pair<G>(Ws + (size_t)j * a_pad, Ws + (size_t)k * a_pad, nv, tol, lg, mask) &&
          lg == 0)
        ++rot;
    }
    __syncthreads();
  }
  return rot;
}

__device__ __forceinline__ int block_or_count(int v, int *flag) {
  // returns the CTA-wide sum of v (all threads see it)
  __syncthreads();
  if (threadIdx.x == 0) *flag = 0;
  __syncthreads();
  if (v) atomicAdd(flag, v);
  __syncthreads();
  const int s = *flag;
  __syncthreads();
  return s;
}

constexpr int JAC_MAX_THREADS = 512;

template <int G>
__global__ void __launch_bounds__(JAC_MAX_THREADS) jacobi_kernel(JacobiArgs A, int a_pad, int bs) {
  extern __shared__ __align__(16) float Ws[];
  __shared__ int flag;
  const int64_t f = blockIdx.x;
  const int l = (int)A.l, m = (int)A.m;
  const bool rows = l <= m;                // vectors are rows (length m) or columns (length l)
  const int b = rows ? l : m, a = rows ? m : l;
  const int nv = a_pad / (4 * G);
  const float *Xf = A.X + f * (int64_t)l * m;
  float *Wg = A.W + f * (int64_t)b * a_pad;

  int sweeps = 0;
  bool converged = false;
  if (bs >= b) {
    // ---------------- resident: the whole slice lives in shared memory
    for (int idx = threadIdx.x; idx < b * a_pad; idx += blockDim.x) {
      const int j = idx / a_pad, e = idx % a_pad;
      Ws[idx] = e < a ? (rows ? Xf[(int64_t)j * m + e] : Xf[(int64_t)e * m + j]) : 0.f;
    }
    __syncthreads();
    while (sweeps < A.max_sweeps) {
      ++sweeps;
      const int rot = round_robin_pass<G>(Ws, b, a_pad, nv, A.tol);
      if (block_or_count(rot, &flag) == 0) { converged = true; break; }
    }
    for (int idx = threadIdx.x; idx < b * a_pad / 4; idx += blockDim.x)
      reinterpret_cast<float4 *>(Wg)[idx] = reinterpret_cast<const float4 *>(Ws)[idx];
  } else {
    // ---------------- blocked: vectors in global memory, block pairs in shared memory
    for (int64_t idx = threadIdx.x; idx < (int64_t)b * a_pad; idx += blockDim.x) {
      const int j = (int)(idx / a_pad), e = (int)(idx % a_pad);
      Wg[idx] = e < a ? (rows ? Xf[(int64_t)j * m + e] : Xf[(int64_t)e * m + j]) : 0.f;
    }
    __syncthreads();
    const int nb = (b + bs - 1) / bs;
    while (sweeps < A.max_sweeps) {
      ++sweeps;
      int rot = 0;
      for (int I = 0; I < nb - 1; ++I)
        for (int J = I + 1; J < nb; ++J) {
          const int i0 = I * bs, ni = min(bs, b - i0);
          const int j0 = J * bs, nj = min(bs, b - j0);
          const int n4 = a_pad / 4;
          float4 *W4 = reinterpret_cast<float4 *>(Wg);
          float4 *S4 = reinterpret_cast<float4 *>(Ws);
          for (int idx = threadIdx.x; idx < (ni + nj) * n4; idx += blockDim.x) {
            const int s = idx / n4, e = idx % n4;
            const int g = s < ni ? i0 + s : j0 + (s - ni);
            S4[idx] = W4[(int64_t)g * n4 + e];
          }
          __syncthreads();
          rot += round_robin_pass<G>(Ws, ni + nj, a_pad, nv, A.tol);
          for (int idx = threadIdx.x; idx < (ni + nj) * n4; idx += blockDim.x) {
            const int s = idx / n4, e = idx % n4;
            const int g = s < ni ? i0 + s : j0 + (s - ni);
            W4[(int64_t)g * n4 + e] = S4[idx];
          }
          __syncthreads();
        }
      if (block_or_count(rot, &flag) == 0) { converged = true; break; }
    }
  }
  __syncthreads();

  // ---------------- singular values (FP64 accumulation) and the per-slice sort
  float *sig_tmp = A.sig + f * b;          // unsorted norms first, then sorted in place below
  int32_t *perm = A.perm + f * b;
  // reuse shared memory: [0, b) floats hold the norms
  float *nrm = Ws;
  __syncthreads();
  {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = warp; j < b; j += nw) {
      double acc = 0.0;
      for (int e = lane; e < a_pad; e += 32) {
        const float v = Wg[(int64_t)j * a_pad + e];
        acc = fma((double)v, (double)v, acc);
      }
      for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
      if (lane == 0) nrm[j] = (float)sqrt(acc);
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < b; j += blockDim.x) {
    const float sj = nrm[j];
    int rank = 0;
    for (int k = 0; k < b; ++k) {
      const float sk = nrm[k];
      rank += (sk > sj) || (sk == sj && k < j);
    }
    sig_tmp[rank] = sj;
    perm[rank] = j;
  }
  if (threadIdx.x == 0) {
    A.sweeps[f] = sweeps;
    if (!converged) set_status(A.status, PP_ENOCONV);
  }
}

int pick_group(int64_t a) {
  if (a <= 192) return 8;
  if (a <= 384) return 16;
  return 32;
}

}  // namespace

int64_t jacobi_apad(int64_t l, int64_t m) {
  const int64_t a = l > m ? l : m;
  const int G = pick_group(a);
  return round_up(a, 4 * G);
}

cudaError_t launch_jacobi(const JacobiArgs &A, cudaStream_t st) {
  const int64_t a = A.l > A.m ? A.l : A.m;
  const int64_t b = A.l < A.m ? A.l : A.m;
  if (a > 4 * 32 * NV_MAX) return cudaErrorInvalidValue;   // > 768: not built
  const int G = pick_group(a);
  const int a_pad = (int)round_up(a, 4 * G);
  const int64_t row_bytes = (int64_t)a_pad * 4;
  int bs;                // block size in vectors; bs >= b means resident
  int64_t cap;           // vectors held in shared memory at once
  if (b * row_bytes <= SMEM_BUDGET) {
    bs = (int)b;
    cap = b;
  } else {
    bs = (int)(SMEM_BUDGET / (2 * row_bytes));
    if (bs < 2) return cudaErrorInvalidValue;
    cap = 2 * bs;
  }
  int64_t groups = (cap + 1) / 2;
  if (groups * G > JAC_MAX_THREADS) groups = JAC_MAX_THREADS / G;
  int threads = (int)round_up(groups * G, 32);
  if (threads < 64) threads = 64;
  size_t smem = (size_t)(cap * row_bytes);
  if ((int64_t)smem < b * 4) smem = (size_t)(b * 4);   // norms reuse the buffer
  cudaError_t e;
  switch (G) {
    case 8:
      e = cudaFuncSetAttribute(jacobi_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem);
      if (e != cudaSuccess) return e;
      count_launch(1);
      jacobi_kernel<8><<<(unsigned)A.p, threads, smem, st>>>(A, a_pad, bs);
      break;
    case 16:
      e = cudaFuncSetAttribute(jacobi_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem);
      if (e != cudaSuccess) return e;
      count_launch(1);
      jacobi_kernel<16><<<(unsigned)A.p, threads, smem, st>>>(A, a_pad, bs);
      break;
    default:
      e = cudaFuncSetAttribute(jacobi_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem);
      if (e != cudaSuccess) return e;
      count_launch(1);
      jacobi_kernel<32><<<(unsigned)A.p, threads, smem, st>>>(A, a_pad, bs);
      break;
  }
  return cudaGetLastError();
}

}  // namespace pp
