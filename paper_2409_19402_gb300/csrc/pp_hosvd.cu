// pp_hosvd.cu -- kernels for the truncated HOSVD comparison of Sec. 4.2:
// the Gram matrices of the mode-1 and mode-2 unfoldings (whose leading
// eigenvectors are the HOSVD factors U1, U2), and the orthogonal projectors
// P = U U^T that the rebuild applies to every transform-domain slice.
//
// Gram of the mode-1 unfolding: G1(i, i') = sum_t sum_j A(i,j,t) A(i',j,t)
// (l x l); mode 2: G2(j, j') = sum_t sum_i A(i,j,t) A(i,j',t) (m x m).  The sum
// over slices is split across CTAs (grid.z) into FP32 partial Grams that a
// second kernel adds in slice-group order (deterministic).
#include "pp_internal.h"

namespace pp {
namespace {

constexpr int GT = 64;   // output tile
constexpr int GK = 16;   // contraction chunk

// partial[z] (d x d) = sum over slices t in group z of the mode-`mode` Gram of slice t
__global__ void __launch_bounds__(256) gram_partial_kernel(const float *__restrict__ A, int64_t l,
                                                           int64_t m, int64_t n, int mode,
                                                           int64_t tpg, float *__restrict__ part) {
  const int64_t d = mode == 1 ? l : m;         // Gram size
  const int64_t kc = mode == 1 ? m : l;        // contracted extent inside a slice
  const int64_t i0 = (int64_t)blockIdx.y * GT, j0 = (int64_t)blockIdx.x * GT;
  const int64_t t0 = (int64_t)blockIdx.z * tpg, t1 = min(n, t0 + tpg);
  __shared__ float As[GK][GT + 1], Bs[GK][GT + 1];
  const int tid = threadIdx.x, ti = tid / 16, tj = tid % 16;
  float acc[4][4] = {};
  for (int64_t t = t0; t < t1; ++t) {
    const float *At = A + t * l * m;
    for (int64_t k0 = 0; k0 < kc; k0 += GK) {
      for (int e = tid; e < GT * GK; e += 256) {
        int rr, kk;
        if (mode == 1) { kk = e % GK; rr = e / GK; } else { rr = e % GT; kk = e / GT; }
        const int64_t k = k0 + kk;
        const int64_t ia = i0 + rr, jb = j0 + rr;
        float va = 0.f, vb = 0.f;
        if (k < kc) {
          if (mode == 1) {   // A(i, k, t) = At[i*m + k]
            if (ia < d) va = At[ia * m + k];
            if (jb < d) vb = At[jb * m + k];
          } else {           // A(k, j, t) = At[k*m + j]
            if (ia < d) va = At[k * m + ia];
            if (jb < d) vb = At[k * m + jb];
          }
        }
        As[kk][rr] = va;
        Bs[kk][rr] = vb;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < GK; ++kk) {
        float a[4], bb[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) { a[r] = As[kk][ti + 16 * r]; bb[r] = Bs[kk][tj + 16 * r]; }
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(a[r], bb[c], acc[r][c]);
      }
      __syncthreads();
    }
  }
  float *P = part + (int64_t)blockIdx.z * d * d;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int64_t i = i0 + ti + 16 * r;
    if (i >= d) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int64_t j = j0 + tj + 16 * c;
      if (j < d) P[i * d + j] = acc[r][c];
    }
  }
}

__global__ void sum_slices_kernel(const float *__restrict__ part, int64_t count, int64_t nparts,
                                  float *__restrict__ out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int64_t z = 0; z < nparts; ++z) s += part[z * count + e];   // fixed order
    out[e] = s;
  }
}

// P (d x d) = U U^T, U is d x k row-major
__global__ void projector_kernel(const float *__restrict__ U, int64_t d, int64_t k,
                                 float *__restrict__ P) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < d * d;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / d, j = e % d;
    float s = 0.f;
    for (int64_t q = 0; q < k; ++q) s = fmaf(U[i * k + q], U[j * k + q], s);
    P[e] = s;
  }
}

}  // namespace

int64_t gram_groups(int64_t n) {
  // enough slice groups to give the Gram launch a few waves of CTAs
  const int64_t g = n < 64 ? n : 64;
  return g < 1 ? 1 : g;
}

cudaError_t launch_gram(const float *A, int64_t l, int64_t m, int64_t n, int mode, float *part,
                        float *G, cudaStream_t st) {
  const int64_t d = mode == 1 ? l : m;
  const int64_t groups = gram_groups(n);
  const int64_t tpg = (n + groups - 1) / groups;
  const int64_t nz = (n + tpg - 1) / tpg;
  const dim3 grid((unsigned)((d + GT - 1) / GT), (unsigned)((d + GT - 1) / GT), (unsigned)nz);
  count_launch(1);
  gram_partial_kernel<<<grid, 256, 0, st>>>(A, l, m, n, mode, tpg, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t count = d * d;
  int blocks = (int)((count + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  count_launch(1);
  sum_slices_kernel<<<blocks, 256, 0, st>>>(part, count, nz, G);
  return cudaGetLastError();
}

cudaError_t launch_projector(const float *U, int64_t d, int64_t k, float *P, cudaStream_t st) {
  int blocks = (int)((d * d + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  count_launch(1);
  projector_kernel<<<blocks, 256, 0, st>>>(U, d, k, P);
  return cudaGetLastError();
}

}  // namespace pp
