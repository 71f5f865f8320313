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
// sigma descending (norms accumulated in FP32 pairs without rounding loss,
// rounded to FP32), the permutation sorted position -> vector index (ties:
// lower vector index first) and the number of sweeps.  Non-convergence within
// max_sweeps writes PP_ENOCONV.
//
// All arithmetic is FP32.  FP64 is avoided because this part's FP64 rate is a
// small fraction of its FP32 rate: the rotation angles use FP32 (fast
// reciprocals and square roots refined by Newton steps) and the final norms
// exact FP32-pair sums.
#include <cooperative_groups.h>
#include <stdio.h>
#include <stdlib.h>

#include <map>
#include <mutex>
#include <tuple>

#include "pp_internal.h"

namespace pp {
namespace {

namespace cg = cooperative_groups;

constexpr int NV_MAX = 6;                 // float4 chunks per lane per vector
constexpr int SMEM_BUDGET = 200 * 1024;   // bytes of shared memory for vectors

// Circle-method pairing of N (even) players: round r in [0, N-1), slot in [0, N/2).
// Slot 0 pairs r with the fixed player N-1; slot s pairs r+s and r-s (mod N-1).
__device__ __forceinline__ void circle_pair(int N, int r, int slot, int &j, int &k) {
  if (slot == 0) {
    j = r;
    k = N - 1;
  } else {
    j = r + slot;
    if (j >= N - 1) j -= N - 1;
    k = r - slot;
    if (k < 0) k += N - 1;
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

// hi + lo += b exactly up to the rounding of lo (Knuth's two-sum; the _rn
// intrinsics keep the compiler from contracting the error-free steps)
__device__ __forceinline__ void pair_add(float &hi, float &lo, float b) {
  const float t = __fadd_rn(hi, b);
  const float bp = __fsub_rn(t, hi);
  lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(b, bp)));
  hi = t;
}

// Singular values of one slice from its converged vectors in global memory
// and the per-slice descending sort (ties: lower vector index first).  nrm is
// b floats of shared scratch.  Each squared norm is summed as an FP32 pair
// (every square split exactly into its rounded value and rounding error,
// two-sum accumulation and warp reduction), about as accurate as FP64
// accumulation without the narrow FP64 pipe; its square root is sqrtf of the
// high part corrected by one Newton step on the exact residual.
__device__ void finish_slice(const float *Wg, int b, int a_pad, float *sig, int32_t *perm,
                             float *nrm) {
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = warp; j < b; j += nw) {
    float hi = 0.f, lo = 0.f;
    for (int e = lane; e < a_pad; e += 32) {
      const float v = Wg[(int64_t)j * a_pad + e];
      const float sq = __fmul_rn(v, v);
      lo = __fadd_rn(lo, fmaf(v, v, -sq));   // v*v - sq, exact
      pair_add(hi, lo, sq);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float ohi = __shfl_xor_sync(0xffffffffu, hi, off);
      const float olo = __shfl_xor_sync(0xffffffffu, lo, off);
      // the same sum in both lanes of a pair: two-sum of the high parts
      // (exact, symmetric), low parts added
      const float t = __fadd_rn(hi, ohi);
      const float bp = __fsub_rn(t, hi);
      const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(ohi, bp));
      lo = __fadd_rn(err, __fadd_rn(lo, olo));
      hi = t;
    }
    if (lane == 0) {
      const float r = sqrtf(hi);
      float s = r;
      if (r > 0.f) s = fmaf(__fadd_rn(fmaf(-r, r, hi), lo), __fdiv_rn(0.5f, r), r);
      nrm[j] = s;
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
    sig[rank] = sj;
    perm[rank] = j;
  }
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

  finish_slice(Wg, b, a_pad, A.sig + f * b, A.perm + f * b, Ws);
  if (threadIdx.x == 0) {
    A.sweeps[f] = sweeps;
    if (!converged) set_status(A.status, PP_ENOCONV);
  }
}


// ------------------------------------------------------------------ cluster kernel
// One slice per thread-block cluster of C CTAs (C >= 2).  The b vectors are cut
// into 2C blocks of bs vectors (vectors past b are zero and never rotate).
// CTA c holds two blocks, on "seats" c and 2C-1-c of the round-robin circle
// over blocks.  A sweep is 2C-1 block rounds: in each, a CTA orthogonalises
// every cross pair of its two resident blocks (bs rounds of bs disjoint pairs
// i <-> (i+r) mod bs); the first block round also covers the pairs inside each
// block.  Between block rounds the blocks move one seat along the circle (seat
// 0 fixed), which is a copy of at most two blocks into other CTAs' shared
// memory (DSMEM) followed by one cluster barrier; shared memory is double
// buffered so a CTA never overwrites blocks that are still being rotated.
// After 2C-1 moves every block is back on its first seat.
//
// Few pairs are in flight per round here, so each pair gets a whole warp:
// every lane holds at most CW float4 of each vector, and only the inner
// product x.y is reduced across the warp.  The squared norms are tracked
// (alpha' = alpha - t g, beta' = beta + t g for the rotation that zeroes g)
// travel with their blocks; they are recomputed from the vectors at the start
// of every sweep, so a sweep that rotates nothing tests orthogonality against
// freshly computed norms.

// CW: float4 per lane per vector in the cluster kernel (a <= 128 * CW); 2, 4 or 6
constexpr int CLU_MAX_BS = 64;   // largest block (vectors) the cluster kernel takes

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Sum of v over the GW lanes of this thread's group, bitwise identical in all
// of them: each lane posts its partial to its warp's 32-float scratch (wred)
// and reads the group's GW partials back, added in a fixed tree.  One
// shared-memory round trip is much shorter than log2(GW) dependent shuffles.
template <int GW>
__device__ __forceinline__ float group_sum_smem(float v, float *wred, unsigned mask) {
  const int wl = threadIdx.x & 31;
  wred[wl] = v;
  __syncwarp(mask);
  const float4 *rp = reinterpret_cast<const float4 *>(wred + (wl & ~(GW - 1)));
  float sv[GW / 4];
#pragma unroll
  for (int k = 0; k < GW / 4; ++k) {
    const float4 q = rp[k];
    sv[k] = (q.x + q.y) + (q.z + q.w);
  }
#pragma unroll
  for (int w = GW / 8; w > 0; w >>= 1)
#pragma unroll
    for (int k = 0; k < w; ++k) sv[k] += sv[k + w];
  __syncwarp(mask);
  return sv[0];
}

// Rotation parameters for a pair with squared norms al, be and inner product g:
// the Rutishauser form x' = x - s (y + tau x), y' = y + s (x - tau y) of the
// symmetric Schur rotation that zeroes g; t is its tangent.
__device__ __forceinline__ void pair_angle(float g, float al, float be, float &t, float &s,
                                           float &tau) {
  // With d = be - al and h = sqrt(d^2 + 4 g^2) (1/h from rsqrt refined by one
  // Newton step): the rotation angle theta has cos(2 theta) = |d| / h, so
  // cos^2(theta) = (h + |d|) / (2h) and t = tan(theta) = sign(d) 2g / (h + |d|)
  // (the symmetric Schur tangent).  c and 1/(h + |d|) come from two
  // independent MUFU operations, each refined by one Newton step; then
  // tau = s / (1 + c) (Rutishauser: implied cosine 1 - s tau), also refined.
  const float d = be - al, g2x = 2.f * g;
  const float r = fmaf(d, d, g2x * g2x);
  float ih = rsqrtf(r);
  ih = ih * fmaf(-0.5f * r * ih, ih, 1.5f);
  const float q = fmaf(r, ih, fabsf(d));          // h + |d|, in [h, 2h]
  const float c2 = 0.5f * q * ih;                 // cos^2(theta), in [1/2, 1]
  float rc = rsqrtf(c2);
  float iq = __fdividef(1.f, q);
  rc = rc * fmaf(-0.5f * c2 * rc, rc, 1.5f);
  iq = fmaf(iq, fmaf(-q, iq, 1.f), iq);
  const float c = c2 * rc;
  t = copysignf(1.f, d) * g2x * iq;
  s = c * t;
  const float onec = 1.f + c;                     // in [1.7, 2]: no special cases
  float rp = __fdividef(1.f, onec);
  rp = fmaf(rp, fmaf(-onec, rp, 1.f), rp);
  tau = s * rp;
}

__device__ __forceinline__ void rotate4(float4 &x, float4 &y, float s, float tau) {
  float4 nx, ny;
  nx.x = fmaf(-s, fmaf(tau, x.x, y.x), x.x);
  ny.x = fmaf(s, fmaf(-tau, y.x, x.x), y.x);
  nx.y = fmaf(-s, fmaf(tau, x.y, y.y), x.y);
  ny.y = fmaf(s, fmaf(-tau, y.y, x.y), y.y);
  nx.z = fmaf(-s, fmaf(tau, x.z, y.z), x.z);
  ny.z = fmaf(s, fmaf(-tau, y.z, x.z), y.z);
  nx.w = fmaf(-s, fmaf(tau, x.w, y.w), x.w);
  ny.w = fmaf(s, fmaf(-tau, y.w, x.w), y.w);
  x = nx;
  y = ny;
}

// One pair per group of GW lanes (8, 16 or 32).  na, nb: tracked squared norms
// in shared memory; lane is the lane index within the group; wred is the
// warp's 32-float reduction scratch.
template <int GW, int CW>
__device__ __forceinline__ bool jacobi_pair_warp(float *__restrict__ x, float *__restrict__ y,
                                                 float *na, float *nb, int n4, float tol2,
                                                 int lane, unsigned mask, float *wred) {
  float4 xv[CW], yv[CW];
  float g0 = 0.f, g1 = 0.f, g2 = 0.f, g3 = 0.f;
#pragma unroll
  for (int q = 0; q < CW; ++q) {
    const int e4 = lane + GW * q;
    if (e4 < n4) {
      xv[q] = reinterpret_cast<const float4 *>(x)[e4];
      yv[q] = reinterpret_cast<const float4 *>(y)[e4];
      g0 = fmaf(xv[q].x, yv[q].x, g0);
      g1 = fmaf(xv[q].y, yv[q].y, g1);
      g2 = fmaf(xv[q].z, yv[q].z, g2);
      g3 = fmaf(xv[q].w, yv[q].w, g3);
    }
  }
  const float g = group_sum_smem<GW>((g0 + g1) + (g2 + g3), wred, mask);
  const float al = *na, be = *nb;
  if (g == 0.f || g * g <= tol2 * al * be) return false;
  float t, s, tau;
  pair_angle(g, al, be, t, s, tau);
#pragma unroll
  for (int q = 0; q < CW; ++q) {
    const int e4 = lane + GW * q;
    if (e4 < n4) {
      rotate4(xv[q], yv[q], s, tau);
      reinterpret_cast<float4 *>(x)[e4] = xv[q];
      reinterpret_cast<float4 *>(y)[e4] = yv[q];
    }
  }
  if (lane == 0) {
    *na = fmaxf(fmaf(-t, g, al), 0.f);
    *nb = fmaf(t, g, be);
  }
  return true;
}

// The same rotation with x held in registers (xv) and its tracked squared norm
// al in a register of every lane of the group (every lane gets the same g, so
// every lane updates al identically).
template <int GW, int CW>
__device__ __forceinline__ bool jacobi_pair_reg(float4 (&xv)[CW], float &al,
                                                float *__restrict__ y, float *nb, int n4,
                                                float tol2, int lane, unsigned mask,
                                                float *wred) {
  float4 yv[CW];
  float g0 = 0.f, g1 = 0.f, g2 = 0.f, g3 = 0.f;
#pragma unroll
  for (int q = 0; q < CW; ++q) {
    const int e4 = lane + GW * q;
    if (e4 < n4) {
      yv[q] = reinterpret_cast<const float4 *>(y)[e4];
      g0 = fmaf(xv[q].x, yv[q].x, g0);
      g1 = fmaf(xv[q].y, yv[q].y, g1);
      g2 = fmaf(xv[q].z, yv[q].z, g2);
      g3 = fmaf(xv[q].w, yv[q].w, g3);
    }
  }
  const float g = group_sum_smem<GW>((g0 + g1) + (g2 + g3), wred, mask);
  const float be = *nb;
  if (g == 0.f || g * g <= tol2 * al * be) return false;
  float t, s, tau;
  pair_angle(g, al, be, t, s, tau);
#pragma unroll
  for (int q = 0; q < CW; ++q) {
    const int e4 = lane + GW * q;
    if (e4 < n4) {
      rotate4(xv[q], yv[q], s, tau);
      reinterpret_cast<float4 *>(y)[e4] = yv[q];
    }
  }
  al = fmaxf(fmaf(-t, g, al), 0.f);
  if (lane == 0) *nb = fmaf(t, g, be);
  return true;
}

// The last round of a cross pass with the blocks' next seats known: the same
// rotation (or none) as jacobi_pair_reg, after which the bottom vector and its
// tracked norm are always stored to (yo, nbo), its seat for the next block
// round in this CTA or another CTA of the cluster.
template <int GW, int CW>
__device__ __forceinline__ bool jacobi_pair_reg_out(float4 (&xv)[CW], float &al,
                                                    const float *__restrict__ y, const float *nb,
                                                    float *yo, float *nbo, int n4, float tol2,
                                                    int lane, unsigned mask, float *wred) {
  float4 yv[CW];
  float g0 = 0.f, g1 = 0.f, g2 = 0.f, g3 = 0.f;
#pragma unroll
  for (int q = 0; q < CW; ++q) {
    const int e4 = lane + GW * q;
    if (e4 < n4) {
      yv[q] = reinterpret_cast<const float4 *>(y)[e4];
      g0 = fmaf(xv[q].x, yv[q].x, g0);
      g1 = fmaf(xv[q].y, yv[q].y, g1);
      g2 = fmaf(xv[q].z, yv[q].z, g2);
      g3 = fmaf(xv[q].w, yv[q].w, g3);
    }
  }
  const float g = group_sum_smem<GW>((g0 + g1) + (g2 + g3), wred, mask);
  float be = *nb;
  const bool rot = !(g == 0.f || g * g <= tol2 * al * be);
  if (rot) {
    float t, s, tau;
    pair_angle(g, al, be, t, s, tau);
#pragma unroll
    for (int q = 0; q < CW; ++q)
      if (lane + GW * q < n4) rotate4(xv[q], yv[q], s, tau);
    al = fmaxf(fmaf(-t, g, al), 0.f);
    be = fmaf(t, g, be);
  }
#pragma unroll
  for (int q = 0; q < CW; ++q) {
    const int e4 = lane + GW * q;
    if (e4 < n4) reinterpret_cast<float4 *>(yo)[e4] = yv[q];
  }
  if (lane == 0) *nbo = be;
  return rot;
}

// squared norms of `count` vectors (rows of a_pad floats), one warp per vector
__device__ void block_norms(const float *v, float *nrm, int count, int n4) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = warp; j < count; j += nw) {
    float acc = 0.f;
    for (int e4 = lane; e4 < n4; e4 += 32) {
      const float4 w = reinterpret_cast<const float4 *>(v)[(size_t)j * n4 + e4];
      acc = fmaf(w.x, w.x, fmaf(w.y, w.y, fmaf(w.z, w.z, fmaf(w.w, w.w, acc))));
    }
    acc = warp_sum(acc);
    if (lane == 0) nrm[j] = acc;
  }
}

template <int GW>
__device__ __forceinline__ unsigned group_mask() {
  const int lane = threadIdx.x & 31;
  return GW == 32 ? 0xffffffffu : (((1u << GW) - 1u) << (lane & ~(GW - 1)));
}

template <int GW, int CW>
__device__ int cross_pass_warp(float *top, float *bot, float *ntop, float *nbot, int bs,
                               int a_pad, float tol2, float *wred) {
  const int lane = threadIdx.x % GW, warp = threadIdx.x / GW, nw = blockDim.x / GW;
  const unsigned mask = group_mask<GW>();
  const int n4 = a_pad / 4;
  int rot = 0;
  for (int r = 0; r < bs; ++r) {
    for (int i = warp; i < bs; i += nw) {
      int j = i + r;
      if (j >= bs) j -= bs;
      if (jacobi_pair_warp<GW, CW>(top + (size_t)i * a_pad, bot + (size_t)j * a_pad, ntop + i,
                                   nbot + j, n4, tol2, lane, mask, wred) &&
          lane == 0)
        ++rot;
    }
    __syncthreads();
  }
  return rot;
}

// Cross pass with the top block in registers: group i owns top vector i for
// all bs rounds (round r pairs it with bottom vector (i + r) mod bs), so only
// the bottom vectors travel through shared memory; the top vectors and their
// norms are written back once at the end.  Needs blockDim.x / GW >= bs.  The
// arithmetic is that of cross_pass_warp, so the results are identical.
//
// SEATS: the blocks' seats for the next block round (rtop, rntop, rbot, rnbot,
// possibly in other CTAs of the cluster) are known, and the last round stores
// each bottom vector there and the top vectors go there from the registers,
// in place of the local write-back and a separate block copy; the caller's
// cluster barrier then orders those stores.
template <int GW, int CW, bool SEATS = false>
__device__ int cross_pass_reg(float *top, float *bot, float *ntop, float *nbot, int bs,
                              int a_pad, float tol2, float *wred, float *rtop = nullptr,
                              float *rntop = nullptr, float *rbot = nullptr,
                              float *rnbot = nullptr) {
  const int lane = threadIdx.x % GW, i = threadIdx.x / GW;
  const unsigned mask = group_mask<GW>();
  const int n4 = a_pad / 4;
  const bool act = i < bs;
  float4 xv[CW];
  float al = 0.f;
  float4 *xt = reinterpret_cast<float4 *>(top + (size_t)(act ? i : 0) * a_pad);
  if (act) {
#pragma unroll
    for (int q = 0; q < CW; ++q) {
      const int e4 = lane + GW * q;
      if (e4 < n4) xv[q] = xt[e4];
    }
    al = ntop[i];
  }
  int rot = 0;
  for (int r = 0; r < (SEATS ? bs - 1 : bs); ++r) {
    if (act) {
      int j = i + r;
      if (j >= bs) j -= bs;
      if (jacobi_pair_reg<GW, CW>(xv, al, bot + (size_t)j * a_pad, nbot + j, n4, tol2, lane,
                                  mask, wred) &&
          lane == 0)
        ++rot;
    }
    __syncthreads();
  }
  if (SEATS) {
    if (act) {
      int j = i + bs - 1;
      if (j >= bs) j -= bs;
      if (jacobi_pair_reg_out<GW, CW>(xv, al, bot + (size_t)j * a_pad, nbot + j,
                                      rbot + (size_t)j * a_pad, rnbot + j, n4, tol2, lane, mask,
                                      wred) &&
          lane == 0)
        ++rot;
      float4 *xo = reinterpret_cast<float4 *>(rtop + (size_t)i * a_pad);
#pragma unroll
      for (int q = 0; q < CW; ++q) {
        const int e4 = lane + GW * q;
        if (e4 < n4) xo[e4] = xv[q];
      }
      if (lane == 0) rntop[i] = al;
    }
    return rot;
  }
  if (act) {
#pragma unroll
    for (int q = 0; q < CW; ++q) {
      const int e4 = lane + GW * q;
      if (e4 < n4) xt[e4] = xv[q];
    }
    if (lane == 0) ntop[i] = al;
  }
  __syncthreads();
  return rot;
}

template <int GW, int CW>
__device__ int intra_pass_warp(float *top, float *bot, float *ntop, float *nbot, int bs,
                               int a_pad, float tol2, float *wred) {
  const int lane = threadIdx.x % GW, warp = threadIdx.x / GW, nw = blockDim.x / GW;
  const unsigned mask = group_mask<GW>();
  const int n4 = a_pad / 4;
  const int N = bs + (bs & 1), half = N / 2;
  int rot = 0;
  for (int r = 0; r < N - 1; ++r) {
    for (int slot = warp; slot < 2 * half; slot += nw) {
      const bool upper = slot < half;
      float *base = upper ? top : bot;
      float *nb = upper ? ntop : nbot;
      int j, k;
      circle_pair(N, r, upper ? slot : slot - half, j, k);
      if (j >= bs || k >= bs) continue;
      if (jacobi_pair_warp<GW, CW>(base + (size_t)j * a_pad, base + (size_t)k * a_pad, nb + j,
                                   nb + k, n4, tol2, lane, mask, wred) &&
          lane == 0)
        ++rot;
    }
    __syncthreads();
  }
  return rot;
}

// threads per CTA: GW lanes per pair, capped so that the registers fit
__host__ __device__ constexpr int clu_max_threads(int gw, int cw) {
  return (gw * cw <= 64 && gw >= 32) ? 1024 : 512;
}

// REG variants hold each group's top vector in registers across the cross pass
// (cross_pass_reg).  They exist for the shapes whose registers allow it without
// spills (-Xptxas -v): GW = 16 within the 512-thread bound, GW = 8 with a
// 256-thread bound (up to 255 registers, so fewer CTAs per SM).
__host__ __device__ constexpr bool clu_has_reg(int gw, int cw) {
  return (gw == 16 && cw <= 3) || (gw == 8 && cw <= 8);
}
// REG variants whose registers also hold the last round's seats (no spills)
__host__ __device__ constexpr bool clu_seats(int gw, int cw, bool reg) {
  return reg && ((gw == 16 && cw <= 2) || (gw == 8 && cw <= 5));
}
__host__ __device__ constexpr int clu_bound(int gw, int cw, bool reg) {
  return (reg && gw == 8) ? 256 : clu_max_threads(gw, cw);
}

template <int GW, int CW, bool REG>
__global__ void __launch_bounds__(clu_bound(GW, CW, REG), 1) jacobi_cluster_kernel(JacobiArgs A, int a_pad,
                                                                            int C, int bs) {
  extern __shared__ __align__(16) float sm[];
  __shared__ int blk[2][2];        // block id held in [buffer][top/bottom]
  __shared__ int rot_total;
  __shared__ __align__(16) float red_scratch[clu_bound(GW, CW, REG)];   // 32 floats per warp
  float *wred = red_scratch + (threadIdx.x & ~31);
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int64_t f = blockIdx.x / C;
  const int l = (int)A.l, m = (int)A.m;
  const bool rows = l <= m;
  const int b = rows ? l : m, a = rows ? m : l;
  const int n4 = a_pad / 4;
  const int blk_floats = bs * a_pad;
  const float tol2 = A.tol * A.tol;
  const float *Xf = A.X + f * (int64_t)l * m;
  float *Wg = A.W + f * (int64_t)b * a_pad;
  auto slot = [&](int buf, int tb) { return sm + (size_t)(buf * 2 + tb) * blk_floats; };
  // tracked squared norms, double buffered like the blocks: [buf][top/bottom][bs]
  float *nrm_base = sm + (size_t)4 * blk_floats;
  auto nslot = [&](int buf, int tb) { return nrm_base + (size_t)(buf * 2 + tb) * bs; };

  // initial seats: top = block rank, bottom = block 2C-1-rank
#pragma unroll
  for (int tb = 0; tb < 2; ++tb) {
    float *dst = slot(0, tb);
    const int v0 = (tb == 0 ? rank : 2 * C - 1 - rank) * bs;
    for (int idx = threadIdx.x; idx < blk_floats; idx += blockDim.x) {
      const int j = v0 + idx / a_pad, e = idx % a_pad;
      float v = 0.f;
      if (j < b && e < a) v = rows ? Xf[(int64_t)j * m + e] : Xf[(int64_t)e * m + j];
      dst[idx] = v;
    }
  }
  if (threadIdx.x == 0) {
    blk[0][0] = rank;
    blk[0][1] = 2 * C - 1 - rank;
    rot_total = 0;
  }
  cl.sync();

  int cur = 0, sweeps = 0;
  bool converged = false;
  // destinations of this CTA's blocks when they move one seat
  const int dst_top_rank = (rank == 0) ? 0 : (rank == C - 1 ? C - 1 : rank + 1);
  const int dst_top_tb = (rank == C - 1) ? 1 : 0;
  const int dst_bot_rank = (rank == 0) ? 1 : rank - 1;
  const int dst_bot_tb = (rank == 0) ? 0 : 1;
  while (sweeps < A.max_sweeps) {
    ++sweeps;
    int rot = 0;
    for (int br = 0; br < 2 * C - 1; ++br) {
      float *top = slot(cur, 0), *bot = slot(cur, 1);
      float *ntop = nslot(cur, 0), *nbot = nslot(cur, 1);
      if (br == 0) {   // fresh norms once per sweep; afterwards they travel with the blocks
        block_norms(top, ntop, bs, n4);
        block_norms(bot, nbot, bs, n4);
        __syncthreads();
        rot += intra_pass_warp<GW, CW>(top, bot, ntop, nbot, bs, a_pad, tol2, wred);
      }
      // then move the two blocks one seat along the circle (DSMEM): stored into
      // their next seats by the last round of the register pass where the
      // registers allow it, else copied after the pass
      const int nxt = cur ^ 1;
      const bool regpass = REG && (int)(blockDim.x / GW) >= bs;
      if (clu_seats(GW, CW, REG) && regpass) {
        rot += cross_pass_reg<GW, CW, clu_seats(GW, CW, REG)>(
            top, bot, ntop, nbot, bs, a_pad, tol2, wred,
            cl.map_shared_rank(slot(nxt, dst_top_tb), dst_top_rank),
            cl.map_shared_rank(nslot(nxt, dst_top_tb), dst_top_rank),
            cl.map_shared_rank(slot(nxt, dst_bot_tb), dst_bot_rank),
            cl.map_shared_rank(nslot(nxt, dst_bot_tb), dst_bot_rank));
      } else {
        if (regpass)
          rot += cross_pass_reg<GW, CW>(top, bot, ntop, nbot, bs, a_pad, tol2, wred);
        else
          rot += cross_pass_warp<GW, CW>(top, bot, ntop, nbot, bs, a_pad, tol2, wred);
#pragma unroll
        for (int tb = 0; tb < 2; ++tb) {
          const int dr = tb == 0 ? dst_top_rank : dst_bot_rank;
          const int dtb = tb == 0 ? dst_top_tb : dst_bot_tb;
          float4 *dst = reinterpret_cast<float4 *>(cl.map_shared_rank(slot(nxt, dtb), dr));
          const float4 *src = reinterpret_cast<const float4 *>(slot(cur, tb));
          for (int idx = threadIdx.x; idx < blk_floats / 4; idx += blockDim.x) dst[idx] = src[idx];
          float *dn = cl.map_shared_rank(nslot(nxt, dtb), dr);
          const float *sn = nslot(cur, tb);
          for (int i = threadIdx.x; i < bs; i += blockDim.x) dn[i] = sn[i];
        }
      }
      if (threadIdx.x == 0) {
        cl.map_shared_rank(&blk[0][0], dst_top_rank)[nxt * 2 + dst_top_tb] = blk[cur][0];
        cl.map_shared_rank(&blk[0][0], dst_bot_rank)[nxt * 2 + dst_bot_tb] = blk[cur][1];
      }
      cl.sync();
      cur = nxt;
    }
    if (rot) atomicAdd(cl.map_shared_rank(&rot_total, 0), rot);
    cl.sync();
    const int total = *cl.map_shared_rank(&rot_total, 0);
    cl.sync();
    if (rank == 0 && threadIdx.x == 0) rot_total = 0;   // next add is at least one barrier away
    if (total == 0) {
      converged = true;
      break;
    }
  }
  // write both resident blocks back to their places in W
#pragma unroll
  for (int tb = 0; tb < 2; ++tb) {
    const int v0 = blk[cur][tb] * bs;
    const float4 *src = reinterpret_cast<const float4 *>(slot(cur, tb));
    for (int idx = threadIdx.x; idx < blk_floats / 4; idx += blockDim.x) {
      const int j = v0 + idx / n4;
      if (j < b) reinterpret_cast<float4 *>(Wg)[(int64_t)j * n4 + idx % n4] = src[idx];
    }
  }
  __threadfence();
  cl.sync();
  if (rank == 0) {
    finish_slice(Wg, b, a_pad, A.sig + f * b, A.perm + f * b, sm);
    if (threadIdx.x == 0) {
      A.sweeps[f] = sweeps;
      if (!converged) set_status(A.status, PP_ENOCONV);
    }
  }
}

int pick_group(int64_t a) {
  if (a <= 192) return 8;
  if (a <= 384) return 16;
  return 32;
}

// ------------------------------------------------------------------ grid kernel
// Slices too large for one CTA's shared memory (e.g. 512 x 512), spread over
// the whole device.  The b vectors of a slice are cut into nb (even) blocks of
// bs vectors; a sweep is nb-1 block rounds of the round-robin circle over
// blocks, and the nb/2 block pairs of a round -- of every slice -- are
// independent work items, taken by the CTAs of one persistent cooperative
// launch in turn.  An item loads its two blocks from W (global memory, L2
// resident) into shared memory, computes their squared norms, orthogonalises
// every cross pair of the two blocks (bs rounds of bs disjoint pairs, one pair
// per group of GW lanes; the first block round of a sweep also covers the
// pairs inside each block) and stores the blocks back.  A bounded grid
// barrier separates block rounds.  Each item adds its rotation count to a
// per-slice, per-sweep counter; a slice whose sweep rotated nothing is done
// (every CTA reads the same counters after the barrier, so every CTA takes the
// same decisions).  The pair arithmetic is that of the cluster kernel.
//
// aux (global, zeroed before the launch): [0] barrier arrivals, [1] barrier
// generation, [2] abort flag, [8 ...] counters cnt[sweep * p + slice].
constexpr long long GRID_WAIT_CYCLES = 4000000000LL;   // ~2 s at 2 GHz per barrier
constexpr int GRID_AUX_HEAD = 8;

// Bounded barrier over all CTAs of a cooperative launch.  false: the wait
// expired here or in another CTA (PP_ETIMEOUT recorded); the caller returns.
__device__ bool grid_barrier(int32_t *aux, int32_t *status, int *flag_sh) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned *cnt = reinterpret_cast<unsigned *>(aux);
    volatile unsigned *gen = reinterpret_cast<volatile unsigned *>(aux + 1);
    volatile int32_t *abort_flag = aux + 2;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(cnt, 1u) == gridDim.x - 1) {
      atomicExch(cnt, 0u);
      __threadfence();
      atomicAdd(reinterpret_cast<unsigned *>(aux + 1), 1u);
    } else {
      const long long t0 = clock64();
      while (*gen == g) {
        if (*abort_flag || clock64() - t0 > GRID_WAIT_CYCLES) {
          ok = 0;
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    if (!ok) {
      aux[2] = 1;
      set_status(status, PP_ETIMEOUT);
    }
    *flag_sh = ok;
  }
  __syncthreads();
  return *flag_sh != 0;
}

// the two passes of a block-pair item, kept out of line so that each has the
// kernel's registers to itself (inlined together they spill)
template <int GW, int CW>
__device__ __noinline__ int grid_intra(float *top, float *bot, float *ntop, float *nbot, int bs,
                                       int a_pad, float tol2, float *wred) {
  return intra_pass_warp<GW, CW>(top, bot, ntop, nbot, bs, a_pad, tol2, wred);
}
template <int GW, int CW>
__device__ __noinline__ int grid_cross(float *top, float *bot, float *ntop, float *nbot, int bs,
                                       int a_pad, float tol2, float *wred) {
  return cross_pass_reg<GW, CW>(top, bot, ntop, nbot, bs, a_pad, tol2, wred);
}

constexpr int GRID_MAX_P = 4096;   // slices the device-wide kernel takes (activity flags)

// THREADS >= bs * GW: one group of GW lanes per cross pair of a round
template <int GW, int CW, int THREADS>
__global__ void __launch_bounds__(THREADS, 1) jacobi_grid_kernel(JacobiArgs A,
                                                                             int a_pad, int bs,
                                                                             int nb) {
  extern __shared__ __align__(16) float sm[];   // top block | bottom block | 2 bs norms
  __shared__ __align__(16) float red_scratch[THREADS];
  __shared__ int flag_sh, rot_sh, any_sh;
  __shared__ unsigned char active[GRID_MAX_P];   // slice still iterating in this sweep
  float *wred = red_scratch + (threadIdx.x & ~31);
  const int l = (int)A.l, m = (int)A.m;
  const bool rows = l <= m;
  const int b = rows ? l : m, a = rows ? m : l;
  const int n4 = a_pad / 4;
  const int64_t p = A.p;
  const float tol2 = A.tol * A.tol;
  int32_t *aux = A.aux;
  int32_t *cnt = aux + GRID_AUX_HEAD;
  float *top = sm, *bot = sm + (size_t)bs * a_pad;
  float *ntop = sm + (size_t)2 * bs * a_pad, *nbot = ntop + bs;

  // W <- the slices' vectors (rows, or columns when l > m), zero padded
  const int64_t total = p * b * (int64_t)a_pad;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = idx / ((int64_t)b * a_pad);
    const int64_t r = idx % ((int64_t)b * a_pad);
    const int j = (int)(r / a_pad), e = (int)(r % a_pad);
    const float *Xf = A.X + f * (int64_t)l * m;
    A.W[idx] = e < a ? (rows ? Xf[(int64_t)j * m + e] : Xf[(int64_t)e * m + j]) : 0.f;
  }
  for (int64_t f = threadIdx.x; f < p; f += blockDim.x) active[f] = 1;
  if (!grid_barrier(aux, A.status, &flag_sh)) return;

  const int64_t items = p * (nb / 2);
  int s = 0;
  for (; s < A.max_sweeps; ++s) {
    // a slice whose previous sweep rotated nothing is done (the counters of
    // the earlier sweeps are final here, and the same for every CTA)
    if (threadIdx.x == 0) any_sh = 0;
    __syncthreads();
    for (int64_t f = threadIdx.x; f < p; f += blockDim.x) {
      if (s > 0 && active[f] && ((volatile const int32_t *)cnt)[(int64_t)(s - 1) * p + f] == 0)
        active[f] = 0;
      if (active[f]) any_sh = 1;
    }
    __syncthreads();
    if (!any_sh) break;
    for (int br = 0; br < nb - 1; ++br) {
      for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const int64_t f = it / (nb / 2);
        const int q = (int)(it % (nb / 2));
        if (!active[f]) continue;   // uniform across the CTA
        int I, J;
        circle_pair(nb, br, q, I, J);
        float4 *W4 = reinterpret_cast<float4 *>(A.W + f * (int64_t)b * a_pad);
        for (int idx = threadIdx.x; idx < 2 * bs * n4; idx += blockDim.x) {
          const int row = idx / n4, e4 = idx % n4;
          const int v = row < bs ? I * bs + row : J * bs + (row - bs);
          reinterpret_cast<float4 *>(sm)[idx] =
              v < b ? W4[(int64_t)v * n4 + e4] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
        block_norms(top, ntop, bs, n4);
        block_norms(bot, nbot, bs, n4);
        __syncthreads();
        int rot = 0;
        if (br == 0) rot += grid_intra<GW, CW>(top, bot, ntop, nbot, bs, a_pad, tol2, wred);
        rot += grid_cross<GW, CW>(top, bot, ntop, nbot, bs, a_pad, tol2, wred);
        for (int idx = threadIdx.x; idx < 2 * bs * n4; idx += blockDim.x) {
          const int row = idx / n4, e4 = idx % n4;
          const int v = row < bs ? I * bs + row : J * bs + (row - bs);
          if (v < b) W4[(int64_t)v * n4 + e4] = reinterpret_cast<const float4 *>(sm)[idx];
        }
        if (threadIdx.x == 0) rot_sh = 0;
        __syncthreads();
        if (rot) atomicAdd(&rot_sh, rot);
        __syncthreads();
        if (threadIdx.x == 0 && rot_sh) atomicAdd(&cnt[(int64_t)s * p + f], rot_sh);
      }
      if (!grid_barrier(aux, A.status, &flag_sh)) return;
    }
  }
  // singular values, order and sweep counts, one slice per CTA in turn
  for (int64_t f = blockIdx.x; f < p; f += gridDim.x) {
    int sw = 0;
    while (sw < s && ((volatile const int32_t *)cnt)[(int64_t)sw * p + f] != 0) ++sw;
    const bool conv = sw < s;
    finish_slice(A.W + f * (int64_t)b * a_pad, b, a_pad, A.sig + f * b, A.perm + f * b, sm);
    if (threadIdx.x == 0) {
      A.sweeps[f] = conv ? sw + 1 : s;
      if (!conv) set_status(A.status, PP_ENOCONV);
    }
    __syncthreads();
  }
}

// Grid-kernel launch shape: one warp per pair, bs = 16 vectors per block (at
// most half the vectors) on 512 threads, or bs = 20 on 640 threads (one group
// per block vector in a cross round; the top block held in registers across
// the cross pass), whichever costs less per sweep: the rounds (nb - 1) times
// the waves of items a round takes on the resident CTAs times an item's bs^2
// pair rotations (measured on 512 x 512 slices, an item's time grows like bs^2:
// the SM is throughput-bound).  p = 10 slices of 512 vectors: bs = 16 gives
// 160 items a round, two waves on 152 SMs; bs = 20 gives 130, one wave, and the
// SVD stage goes from 14.2 to 9.8 ms; from p = 25 on, bs = 16 is kept.
struct GridCfg {
  int GW = 0, CW = 0, bs = 0, nb = 0, grid = 0, threads = 0;
  size_t smem = 0;
};

template <int GW, int CW, int THREADS>
cudaError_t grid_launch(const JacobiArgs &A, int a_pad, GridCfg &g, cudaStream_t st) {
  auto kern = jacobi_grid_kernel<GW, CW, THREADS>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)g.smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, g.smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int64_t items = A.p * (g.nb / 2);
  const int64_t cap = (int64_t)per_sm * num_sms();
  g.grid = (int)(items < cap ? items : cap);
  if (g.grid < 1) g.grid = 1;
  e = cudaMemsetAsync(A.aux, 0, jacobi_aux_bytes(A.p), st);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)g.grid, 1, 1);
  cfg.blockDim = dim3(THREADS, 1, 1);
  cfg.dynamicSmemBytes = g.smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  count_launch(1);
  JacobiArgs Ac = A;
  if (Ac.max_sweeps > JACOBI_GRID_MAX_SWEEPS) Ac.max_sweeps = JACOBI_GRID_MAX_SWEEPS;
  return cudaLaunchKernelEx(&cfg, kern, Ac, a_pad, g.bs, g.nb);
}

cudaError_t launch_grid_jacobi(const JacobiArgs &A, int a_pad, cudaStream_t st) {
  const int64_t a = A.l > A.m ? A.l : A.m;
  const int64_t b = A.l < A.m ? A.l : A.m;
  (void)a;
  GridCfg g;
  const int n4 = a_pad / 4;
  if (A.p > GRID_MAX_P) return cudaErrorInvalidValue;
  g.GW = 32;
  g.CW = n4 <= 128 ? 4 : 6;
  if (n4 > g.GW * g.CW) return cudaErrorInvalidValue;
  auto blocks = [&](int bs) {
    int nb = (int)((b + bs - 1) / bs);
    return nb + (nb & 1);
  };
  auto steps = [&](int bs) {   // item steps per sweep, one resident CTA per SM
    const int nb = blocks(bs);
    const int64_t items = A.p * (nb / 2);
    const int64_t waves = (items + num_sms() - 1) / num_sms();
    return (int64_t)(nb - 1) * waves * bs * bs;
  };
  g.bs = 16;
  if (g.bs > (b + 1) / 2) g.bs = (int)((b + 1) / 2);
  // the 640-thread shape only where its registers hold the vectors (CW = 4)
  const bool wide = g.CW == 4 && b >= 40 && 10 * steps(20) < 9 * steps(16);
  if (wide) g.bs = 20;
  g.nb = blocks(g.bs);
  g.smem = (size_t)2 * g.bs * a_pad * sizeof(float) + (size_t)2 * g.bs * sizeof(float);
  if ((int64_t)g.smem < b * 4) g.smem = (size_t)b * 4;   // finish_slice: b norms
  // the cross pass needs one group per block vector: THREADS / GW >= bs
  if (wide) return grid_launch<32, 4, 640>(A, a_pad, g, st);
  return g.CW == 4 ? grid_launch<32, 4, 512>(A, a_pad, g, st)
                   : grid_launch<32, 6, 512>(A, a_pad, g, st);
}


constexpr int MAX_CLUSTER = 8;

// registered launch shapes (pp_set_jacobi_shape): (l, m, p) -> (C, GW)
std::mutex g_shape_mu;
std::map<std::tuple<int64_t, int64_t, int64_t>, std::pair<int, int>> g_shapes;

size_t cluster_smem(int bs, int a_pad, int64_t b) {
  size_t smem = (size_t)4 * bs * a_pad * sizeof(float) + (size_t)4 * bs * sizeof(float);
  if ((int64_t)smem < b * 4) smem = (size_t)b * 4;   // finish_slice: b norms
  return smem;
}

// One cluster configuration: C CTAs per slice, GW lanes per pair, CW float4 per lane.
struct ClusterCfg {
  int C = 0, bs = 0, GW = 0, CW = 0, threads = 0;
  bool reg = false;        // REG variant (top vectors in registers)
  size_t smem = 0;
  int max_clusters = 0;   // co-resident clusters of this shape on the device
};

template <int GW, int CW, bool REG>
cudaError_t cluster_cfg_query(const JacobiArgs &A, int a_pad, int C, ClusterCfg &cc) {
  const int64_t b = A.l < A.m ? A.l : A.m;
  cc.C = C;
  cc.bs = (int)((b + 2 * C - 1) / (2 * C));
  cc.GW = GW;
  cc.CW = CW;
  cc.reg = REG;
  int threads = GW * cc.bs;
  if (threads > clu_bound(GW, CW, REG)) threads = clu_bound(GW, CW, REG);
  cc.threads = (int)round_up(threads < 64 ? 64 : threads, 32);
  cc.smem = cluster_smem(cc.bs, a_pad, b);
  cudaError_t e = cudaFuncSetAttribute(jacobi_cluster_kernel<GW, CW, REG>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cc.smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(A.p * C), 1, 1);
  cfg.blockDim = dim3((unsigned)cc.threads, 1, 1);
  cfg.dynamicSmemBytes = cc.smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaOccupancyMaxActiveClusters(&cc.max_clusters, jacobi_cluster_kernel<GW, CW, REG>, &cfg);
}

template <int GW, int CW, bool REG>
cudaError_t cluster_launch(const JacobiArgs &A, int a_pad, const ClusterCfg &cc,
                           cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(A.p * cc.C), 1, 1);
  cfg.blockDim = dim3((unsigned)cc.threads, 1, 1);
  cfg.dynamicSmemBytes = cc.smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cc.C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  count_launch(1);
  return cudaLaunchKernelEx(&cfg, jacobi_cluster_kernel<GW, CW, REG>, A, a_pad, cc.C, cc.bs);
}

// Estimated cost of a launch shape: waves x (pair rounds + cluster barriers, each
// barrier counted as two rounds) per sweep, where a sweep has 2 C bs - 1 pair
// rounds (bs = ceil(b / 2C): padding vectors cost rounds), the round time grows
// with the group's reduction depth log2(GW), and a REG round (top vectors in
// registers) costs about three quarters of a plain one (measured per round).
double shape_cost(const JacobiArgs &A, const ClusterCfg &cc) {
  const double waves = (double)((A.p + cc.max_clusters - 1) / cc.max_clusters);
  const double depth = cc.GW == 8 ? 3.0 : (cc.GW == 16 ? 4.0 : 5.0);
  return waves * (2.0 * cc.C * cc.bs - 1.0 + 2.0 * (2 * cc.C + 1)) * (1.0 + 0.15 * depth) *
         (cc.reg ? 0.75 : 1.0);
}

// One (GW, CW) shape: the cheaper of the plain and (where it exists) the REG variant.
template <int GW, int CW>
cudaError_t query_shape(const JacobiArgs &A, int a_pad, int C, ClusterCfg &cc) {
  cudaError_t e = cluster_cfg_query<GW, CW, false>(A, a_pad, C, cc);
  if (e != cudaSuccess) return e;
  if constexpr (clu_has_reg(GW, CW)) {
    ClusterCfg r;
    if (cluster_cfg_query<GW, CW, true>(A, a_pad, C, r) == cudaSuccess && r.max_clusters >= 1 &&
        r.threads >= GW * r.bs &&
        (cc.max_clusters < 1 || shape_cost(A, r) < shape_cost(A, cc)))
      cc = r;
    cudaGetLastError();
  }
  return cudaSuccess;
}

template <int GW, int CW>
cudaError_t launch_shape(const JacobiArgs &A, int a_pad, const ClusterCfg &cc, cudaStream_t st) {
  if constexpr (clu_has_reg(GW, CW)) {
    if (cc.reg) return cluster_launch<GW, CW, true>(A, a_pad, cc, st);
  }
  return cluster_launch<GW, CW, false>(A, a_pad, cc, st);
}

cudaError_t query(const JacobiArgs &A, int a_pad, int C, int GW, ClusterCfg &cc) {
  const int n4 = a_pad / 4;
  if (GW == 8) {
    if (n4 <= 32) return query_shape<8, 4>(A, a_pad, C, cc);
    if (n4 <= 40) return query_shape<8, 5>(A, a_pad, C, cc);
    return query_shape<8, 8>(A, a_pad, C, cc);
  }
  if (GW == 16) {
    if (n4 <= 32) return query_shape<16, 2>(A, a_pad, C, cc);
    if (n4 <= 48) return query_shape<16, 3>(A, a_pad, C, cc);
    if (n4 <= 64) return query_shape<16, 4>(A, a_pad, C, cc);
    return query_shape<16, 8>(A, a_pad, C, cc);
  }
  if (n4 <= 64) return query_shape<32, 2>(A, a_pad, C, cc);
  if (n4 <= 128) return query_shape<32, 4>(A, a_pad, C, cc);
  return query_shape<32, 6>(A, a_pad, C, cc);
}

cudaError_t launch(const JacobiArgs &A, int a_pad, const ClusterCfg &cc, cudaStream_t st) {
  if (cc.GW == 8) {
    if (cc.CW == 4) return launch_shape<8, 4>(A, a_pad, cc, st);
    if (cc.CW == 5) return launch_shape<8, 5>(A, a_pad, cc, st);
    return launch_shape<8, 8>(A, a_pad, cc, st);
  }
  if (cc.GW == 16) {
    if (cc.CW == 2) return launch_shape<16, 2>(A, a_pad, cc, st);
    if (cc.CW == 3) return launch_shape<16, 3>(A, a_pad, cc, st);
    if (cc.CW == 4) return launch_shape<16, 4>(A, a_pad, cc, st);
    return launch_shape<16, 8>(A, a_pad, cc, st);
  }
  if (cc.CW == 2) return launch_shape<32, 2>(A, a_pad, cc, st);
  if (cc.CW == 4) return launch_shape<32, 4>(A, a_pad, cc, st);
  return launch_shape<32, 6>(A, a_pad, cc, st);
}

// Pick the cluster shape: among C in [2, 8] and GW in {8, 16, 32} whose shared
// memory fits, minimise shape_cost.  Returns false when no shape applies.
bool pick_cluster(const JacobiArgs &A, int a_pad, ClusterCfg &best) {
  const int64_t b = A.l < A.m ? A.l : A.m;
  double best_cost = 1e300;
  bool found = false;
  // tuning overrides (environment): PP_JACOBI_C in [2, 8], PP_JACOBI_GW in {16, 32}
  const char *envC = getenv("PP_JACOBI_C"), *envG = getenv("PP_JACOBI_GW");
  const int forceC = envC ? atoi(envC) : 0, forceG = envG ? atoi(envG) : 0;
  for (int C = MAX_CLUSTER; C >= 2; --C) {
    if (forceC && C != forceC) continue;
    if (b < 4 * C) continue;
    const int bs = (int)((b + 2 * C - 1) / (2 * C));
    if (bs > CLU_MAX_BS) continue;
    if ((int64_t)cluster_smem(bs, a_pad, b) > SMEM_BUDGET) continue;
    for (int GW : {8, 16, 32}) {
      if (forceG && GW != forceG) continue;
      if (GW == 8 && a_pad / 4 > 64) continue;
      ClusterCfg cc;
      if (query(A, a_pad, C, GW, cc) != cudaSuccess || cc.max_clusters < 1) {
        cudaGetLastError();
        continue;
      }
      const double cost = shape_cost(A, cc);
      if (cost < best_cost * (1.0 - 1e-9)) {
        best_cost = cost;
        best = cc;
        found = true;
      }
    }
  }
  return found;
}

}  // namespace

bool set_jacobi_shape(int64_t l, int64_t m, int64_t p, int C, int GW) {
  if (l < 1 || m < 1 || p < 1 || C < 0 || C > MAX_CLUSTER) return false;
  if (C >= 2 && GW != 8 && GW != 16 && GW != 32) return false;
  std::lock_guard<std::mutex> lock(g_shape_mu);
  const auto key = std::make_tuple(l, m, p);
  if (C == 0) g_shapes.erase(key);
  else g_shapes[key] = std::make_pair(C, GW);
  return true;
}

size_t jacobi_aux_bytes(int64_t p) {
  return (size_t)(GRID_AUX_HEAD + (int64_t)JACOBI_GRID_MAX_SWEEPS * p) * sizeof(int32_t);
}

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
  // cluster split when slices are few relative to the SMs
  const bool log = getenv("PP_LOG_LAUNCH") != nullptr;   // shape of the chosen launch to stderr
  int regC = -1, regG = 0;
  {
    std::lock_guard<std::mutex> lock(g_shape_mu);
    auto it = g_shapes.find(std::make_tuple(A.key_l > 0 ? A.key_l : A.l,
                                            A.key_m > 0 ? A.key_m : A.m, A.p));
    if (it != g_shapes.end()) { regC = it->second.first; regG = it->second.second; }
  }
  if (regC >= 2) {   // a registered cluster shape, if it can be launched
    ClusterCfg cc;
    const int bs = (int)((b + 2 * regC - 1) / (2 * regC));
    if (b >= 4 * regC && bs <= CLU_MAX_BS &&
        (int64_t)cluster_smem(bs, a_pad, b) <= SMEM_BUDGET &&
        query(A, a_pad, regC, regG, cc) == cudaSuccess && cc.max_clusters >= 1) {
      if (log)
        fprintf(stderr, "[pprod] jacobi cluster (registered): p=%lld C=%d bs=%d GW=%d reg=%d\n",
                (long long)A.p, cc.C, cc.bs, cc.GW, (int)cc.reg);
      return launch(A, a_pad, cc, st);
    }
    cudaGetLastError();
  }
  if (regC < 0 && A.p < num_sms() / 2) {
    ClusterCfg cc;
    if (pick_cluster(A, a_pad, cc)) {
      if (log)
        fprintf(stderr, "[pprod] jacobi cluster: p=%lld C=%d bs=%d GW=%d CW=%d reg=%d threads=%d "
                        "smem=%zu max_clusters=%d\n",
                (long long)A.p, cc.C, cc.bs, cc.GW, cc.CW, (int)cc.reg, cc.threads, cc.smem,
                cc.max_clusters);
      return launch(A, a_pad, cc, st);
    }
  }
  // slices too large for one CTA's shared memory: the device-wide kernel
  if (b * row_bytes > SMEM_BUDGET && A.aux && A.allow_grid) {
    const cudaError_t e = launch_grid_jacobi(A, a_pad, st);
    if (log)
      fprintf(stderr, "[pprod] jacobi grid: p=%lld a_pad=%d -> %s\n", (long long)A.p, a_pad,
              cudaGetErrorString(e));
    if (e == cudaSuccess) return e;
    cudaGetLastError();
  }
  if (log) fprintf(stderr, "[pprod] jacobi single-CTA: p=%lld a_pad=%d\n", (long long)A.p, a_pad);
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
