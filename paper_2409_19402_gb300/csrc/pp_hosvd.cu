// pp_hosvd.cu -- the truncated HOSVD comparison of Sec. 4.2: the Gram
// matrices of the mode-1 and mode-2 unfoldings (whose leading eigenvectors are
// the HOSVD factors U1, U2), and the orthogonal projectors P = U U^T that the
// rebuild applies to every transform-domain slice, both on the tensor-core
// kernel of pp_gemm_tc.cu.
//
// Gram of the mode-1 unfolding: G1(i, i') = sum_t sum_j A(i,j,t) A(i',j,t)
// (l x l); mode 2: G2(j, j') = sum_t sum_i A(i,j,t) A(i,j',t) (m x m).  The
// slice products run on the tensor-core kernel (launch_reduce_tc: 3-pass split
// TF32, FP32 sums of 32-term chunks), consecutive slices summed in one grid
// layer, the layers' partial Grams added by a second kernel in layer order
// (deterministic).
#include "pp_internal.h"

namespace pp {
namespace {

__global__ void sum_slices_kernel(const float *__restrict__ part, int64_t count, int64_t nparts,
                                  float *__restrict__ out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int64_t z = 0; z < nparts; ++z) s += part[z * count + e];   // fixed order
    out[e] = s;
  }
}

// U3 builder epilogue (Thm. 4.3, Cor. 4.1).  V (n x p, row-major) holds the
// leading eigenvectors of the mode-3 Gram G (n x n) and s (p) their eigenvalues;
// one CTA of 256 threads, n <= U3_MAX_N.
//  1. Q = V.
//  2. Zero eigenvalues (A_(3) of rank < p) leave zero columns, always the
//     trailing ones (s is sorted).  Each is replaced by the next unit vector e_i
//     (i ascending, never revisited) whose residual after two passes of
//     classical Gram-Schmidt against the columns before it has squared norm
//     above 1/(2n), normalised.  Some e_i always qualifies: the residuals'
//     squared norms of all n unit vectors sum to n - q >= 1.
//  3. Each column's sign makes its largest-magnitude entry (the first such row
//     on ties) positive.
constexpr int U3_MAX_N = 768;

__device__ float block_sum256(float v, float *red) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  float t = 0.f;
#pragma unroll
  for (int w = 0; w < 8; ++w) t += red[w];   // same order in every thread
  return t;
}

__global__ void __launch_bounds__(256) u3_finish_kernel(const float *__restrict__ V,
                                                        const float *__restrict__ s,
                                                        const float *__restrict__ G, int64_t n,
                                                        int64_t p, float *__restrict__ Q,
                                                        float *__restrict__ lambda,
                                                        int32_t *status, const int32_t *sweeps,
                                                        pp_report *rep) {
  __shared__ float vs[U3_MAX_N], ds[U3_MAX_N], red[8];
  __shared__ float wv[8];
  __shared__ int64_t wi[8];
  __shared__ float sgn;
  __shared__ int first_def;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // 1. copy
  for (int64_t e = tid; e < n * p; e += 256) Q[e] = V[e];
  if (tid == 0) first_def = (int)p;
  __syncthreads();
  // 2. completion of a rank-deficient basis
  for (int64_t q = warp; q < p; q += 8) {
    float nn = 0.f;
    for (int64_t e = lane; e < n; e += 32) nn = fmaf(Q[e * p + q], Q[e * p + q], nn);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
    if (lane == 0 && nn < 0.5f) atomicMin(&first_def, (int)q);
  }
  __syncthreads();
  int64_t cand = 0;
  const float accept = 0.5f / (float)n;
  for (int64_t q = first_def; q < p; ++q) {
    bool done = false;
    while (!done && cand < n) {
      for (int64_t e = tid; e < n; e += 256) vs[e] = e == cand ? 1.f : 0.f;
      __syncthreads();
      for (int pass = 0; pass < 2; ++pass) {
        for (int64_t c = warp; c < q; c += 8) {
          float d = 0.f;
          for (int64_t e = lane; e < n; e += 32) d = fmaf(Q[e * p + c], vs[e], d);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
          if (lane == 0) ds[c] = d;
        }
        __syncthreads();
        for (int64_t e = tid; e < n; e += 256) {
          float acc = vs[e];
          for (int64_t c = 0; c < q; ++c) acc = fmaf(-ds[c], Q[e * p + c], acc);
          vs[e] = acc;
        }
        __syncthreads();
      }
      float r2 = 0.f;
      for (int64_t e = tid; e < n; e += 256) r2 = fmaf(vs[e], vs[e], r2);
      r2 = block_sum256(r2, red);
      ++cand;
      if (r2 > accept) {
        const float inv = rsqrtf(r2);
        for (int64_t e = tid; e < n; e += 256) Q[e * p + q] = vs[e] * inv;
        done = true;
      }
      __syncthreads();
    }
    if (!done) {            // not reachable in exact arithmetic; reported, never silent
      if (tid == 0) set_status(status, PP_ENOCONV);
      break;
    }
  }
  __syncthreads();
  // 3. sign convention
  for (int64_t q = 0; q < p; ++q) {
    float best = -1.f;
    int64_t bi = n;
    for (int64_t e = tid; e < n; e += 256) {
      const float v = fabsf(Q[e * p + q]);
      if (v > best) { best = v; bi = e; }         // e ascending per thread: first wins
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ov = __shfl_down_sync(0xffffffffu, best, o);
      const int64_t oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) { wv[warp] = best; wi[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      float bv = wv[0];
      int64_t bj = wi[0];
      for (int w = 1; w < 8; ++w)
        if (wv[w] > bv || (wv[w] == bv && wi[w] < bj)) { bv = wv[w]; bj = wi[w]; }
      sgn = (bj < n && Q[bj * p + q] < 0.f) ? -1.f : 1.f;
    }
    __syncthreads();
    const float sg = sgn;
    if (sg < 0.f)
      for (int64_t e = tid; e < n; e += 256) Q[e * p + q] = -Q[e * p + q];
    __syncthreads();
  }
  if (lambda)
    for (int64_t q = tid; q < p; q += 256) lambda[q] = s[q];
  if (tid == 0 && rep) {
    double tr = 0.0, kept = 0.0;
    for (int64_t e = 0; e < n; ++e) tr += (double)G[e * n + e];
    for (int64_t q = 0; q < p; ++q) kept += (double)s[q];
    rep->status = *status;
    rep->sweeps = *sweeps;
    rep->K = p;
    rep->kappa = p;
    rep->normA2 = tr;
    rep->normAh2 = kept;
    rep->kept2 = kept;
    rep->discarded2 = tr - kept;
    rep->err2 = 0.0;
    rep->proj_err2 = tr - kept;
  }
}

}  // namespace

cudaError_t launch_u3_finish(const float *V, const float *s, const float *G, int64_t n, int64_t p,
                             float *Q, float *lambda, int32_t *status, const int32_t *sweeps,
                             pp_report *rep, cudaStream_t st) {
  if (n > U3_MAX_N) return cudaErrorInvalidValue;
  count_launch(1);
  u3_finish_kernel<<<1, 256, 0, st>>>(V, s, G, n, p, Q, lambda, status, sweeps, rep);
  return cudaGetLastError();
}

int64_t gram_groups(int64_t n) {
  // enough slice groups to give the Gram launch a few waves of CTAs
  const int64_t g = n < 64 ? n : 64;
  return g < 1 ? 1 : g;
}

cudaError_t launch_gram(const float *A, int64_t l, int64_t m, int64_t n, int mode, float *part,
                        float *G, cudaStream_t st) {
  // slice t: A_t A_t^T (mode 1: M(i, j) = A_t[i m + j], X(j, i') = A_t[i' m + j])
  // or A_t^T A_t (mode 2: M(j, i) = A_t[i m + j], X(i, j') = A_t[i m + j']),
  // the slices summed on the tensor cores in groups of consecutive slices
  const int64_t d = mode == 1 ? l : m;
  const int64_t rz = (n + gram_groups(n) - 1) / gram_groups(n);
  const int64_t nz = (n + rz - 1) / rz;
  cudaError_t e = mode == 1
                      ? launch_reduce_tc(A, m, 1, l * m, A, l * m, 1, m, part, d * d, d, m, d, n,
                                         nz, st)
                      : launch_reduce_tc(A, 1, m, l * m, A, l * m, m, 1, part, d * d, d, l, d, n,
                                         nz, st);
  if (e != cudaSuccess) return e;
  const int64_t count = d * d;
  int blocks = (int)((count + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  count_launch(1);
  sum_slices_kernel<<<blocks, 256, 0, st>>>(part, count, nz, G);
  return cudaGetLastError();
}

cudaError_t launch_projector(const float *U, int64_t d, int64_t k, float *P, cudaStream_t st) {
  // P (d x d) = U U^T on the tensor cores: M(i, q) = U[i k + q], X(q, j) = U[j k + q]
  return launch_batched_tc(U, k, 1, 0, U, 0, 1, k, P, 0, d, k, d, 1, 0, nullptr, st);
}

}  // namespace pp
