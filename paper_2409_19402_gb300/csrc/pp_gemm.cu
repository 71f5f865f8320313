// pp_gemm.cu -- FP32 CUDA-core tiled GEMMs for the mode-3 product (Def. 2.2)
// and the facewise product (Def. 2.3).
//
// The mode-3 product Y = X x_3 M is one GEMM over the mode-3 unfolding:
// Y_(3) (P x N) = M (P x S) * X_(3) (S x N) with N = l*m pixels, S the input
// slice count and P the output slice count.  X_(3) is the tensor itself in the
// frontal-slice-major layout, so the kernel streams it row by row (coalesced
// along pixels).  M is addressed through two strides so that the same kernel
// applies Q^T (projection) or Q (back-projection) without a transposed copy.
//
// Optionally the epilogue accumulates sum (Aref - Y)^2 in FP64 per CTA (the
// reconstruction error |A - A_k|_F^2 of Thm. 4.2, fused into the
// back-projection so A_k is never re-read), and the projection accumulates the
// energies |X|_F^2 (from the tiles it streams in) and |Y|_F^2 (from its
// outputs) so that neither tensor is read a second time.
#include "pp_internal.h"

namespace pp {
namespace {

constexpr int BM = 64;   // output slices per CTA
constexpr int BN = 128;  // pixels per CTA
constexpr int BK = 16;   // contraction step
constexpr int NT = 256;  // threads per CTA

__device__ __forceinline__ double block_sum_double(double v, double *red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];  // fixed order
  }
  return s;
}

// Y[z] (P x N) = M[z] (P x S) * X[z] (S x N); M(r, c) = Qm[z*sMz + r*sr + c*sc].
__global__ void __launch_bounds__(NT) gemm_tile_kernel(
    const float *__restrict__ Qm, int64_t sr, int64_t sc, int64_t sMz,
    const float *__restrict__ X, int64_t sXz, int64_t sxc, int64_t sxn, float *__restrict__ Y,
    int64_t sYz, int64_t P, int64_t S, int64_t N, const float *__restrict__ Aref,
    double *__restrict__ errp, double *__restrict__ xpart, double *__restrict__ ypart) {
  // X(c, n) = X[z*sXz + c*sxc + n*sxn] (row-major: sxc = N, sxn = 1)
  // Y may be nullptr (only the error partials are produced); xpart / ypart may be
  // nullptr.  xpart[blockIdx.x] (CTAs of the first row tile only) and
  // ypart[CTA] receive the FP64 sums of squares of the X tiles and Y tile.
  __shared__ float Ms[BK][BM + 4];
  __shared__ __align__(16) float Xs[BK][BN];
  __shared__ double red[NT / 32];

  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t z = blockIdx.z;
  const int64_t r0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;
  Qm += z * sMz;
  X += z * sXz;
  if (Y) Y += z * sYz;

  float acc[4][8];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  double xs = 0.0;
  const bool do_x = xpart != nullptr && blockIdx.y == 0;
  for (int64_t c0 = 0; c0 < S; c0 += BK) {
    for (int e = tid; e < BM * BK; e += NT) {
      const int rr = e % BM, cc = e / BM;
      const int64_t r = r0 + rr, c = c0 + cc;
      Ms[cc][rr] = (r < P && c < S) ? Qm[r * sr + c * sc] : 0.f;
    }
    for (int e = tid; e < BK * BN; e += NT) {
      const int cc = e / BN, nn = e % BN;
      const int64_t c = c0 + cc, n = n0 + nn;
      const float v = (c < S && n < N) ? X[c * sxc + n * sxn] : 0.f;
      Xs[cc][nn] = v;
      if (do_x) xs += (double)v * v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = Ms[kk][ty * 4 + i];
      const float4 b0 = *reinterpret_cast<const float4 *>(&Xs[kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4 *>(&Xs[kk][64 + tx * 4]);
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }

  double err = 0.0, ys = 0.0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t r = r0 + ty * 4 + i;
    if (r >= P) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int64_t n = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
      if (n >= N) continue;
      if (Y) Y[r * N + n] = acc[i][j];
      ys += (double)acc[i][j] * acc[i][j];
      if (Aref) {
        const double d = (double)Aref[z * sYz + r * N + n] - (double)acc[i][j];
        err += d * d;
      }
    }
  }
  const int64_t cta = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  if (Aref) {  // uniform branches: every thread of the CTA takes them
    const double s = block_sum_double(err, red);
    if (tid == 0) errp[cta] = s;
    __syncthreads();
  }
  if (ypart) {
    const double s = block_sum_double(ys, red);
    if (tid == 0) ypart[cta] = s;
    __syncthreads();
  }
  if (do_x) {
    const double s = block_sum_double(xs, red);
    if (tid == 0) xpart[blockIdx.x] = s;
  }
}

}  // namespace

int64_t mode3_gemm_max_partials(int64_t P, int64_t N) {
  return ((N + BN - 1) / BN) * ((P + BM - 1) / BM);
}

cudaError_t launch_mode3_gemm(const float *Qm, int64_t sr, int64_t sc, const float *X,
                              float *Y, int64_t P, int64_t S, int64_t N, const float *Aref,
                              double *err_partials, int *n_partials, cudaStream_t st,
                              double *xpart, int *n_xpart, double *ypart) {
  const dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((P + BM - 1) / BM), 1);
  if (n_partials) *n_partials = (int)(grid.x * grid.y);
  if (n_xpart) *n_xpart = (int)grid.x;
  count_launch(1);
  gemm_tile_kernel<<<grid, NT, 0, st>>>(Qm, sr, sc, 0, X, 0, N, 1, Y, 0, P, S, N, Aref,
                                        err_partials, xpart, ypart);
  return cudaGetLastError();
}

cudaError_t launch_batched_gemm(const float *Mm, int64_t sr, int64_t sc, int64_t sMz,
                                const float *X, int64_t sXz, float *Y, int64_t sYz, int64_t P,
                                int64_t S, int64_t N, int64_t batch, cudaStream_t st,
                                int64_t sxc, int64_t sxn) {
  if (sxc < 0) { sxc = N; sxn = 1; }
  const dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((P + BM - 1) / BM), (unsigned)batch);
  count_launch(1);
  gemm_tile_kernel<<<grid, NT, 0, st>>>(Mm, sr, sc, sMz, X, sXz, sxc, sxn, Y, sYz, P, S, N,
                                        nullptr, nullptr, nullptr, nullptr);
  return cudaGetLastError();
}

namespace {

// ---------------------------------------------------------------- A B^T, split over K
// part[z] (R x S) = A[:, kz] B[:, kz]^T over the z-th chunk of the common dimension K;
// A (R x K) and B (S x K) row-major.  Tiles 64 x 64, 256 threads.
__global__ void __launch_bounds__(256) nt_partial_kernel(const float *__restrict__ A,
                                                         const float *__restrict__ B, int64_t R,
                                                         int64_t S, int64_t K, int64_t kchunk,
                                                         float *__restrict__ part) {
  __shared__ float As[16][64 + 1], Bs[16][64 + 1];
  const int64_t r0 = (int64_t)blockIdx.y * 64, s0 = (int64_t)blockIdx.x * 64;
  const int64_t k0 = (int64_t)blockIdx.z * kchunk, k1 = min(K, k0 + kchunk);
  const int tid = threadIdx.x, ti = tid / 16, tj = tid % 16;
  float acc[4][4] = {};
  for (int64_t kb = k0; kb < k1; kb += 16) {
    for (int e = tid; e < 64 * 16; e += 256) {
      const int kk = e % 16, rr = e / 16;
      const int64_t k = kb + kk;
      As[kk][rr] = (k < k1 && r0 + rr < R) ? A[(r0 + rr) * K + k] : 0.f;
      Bs[kk][rr] = (k < k1 && s0 + rr < S) ? B[(s0 + rr) * K + k] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { a[q] = As[kk][ti + 16 * q]; b[q] = Bs[kk][tj + 16 * q]; }
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[q][c] = fmaf(a[q], b[c], acc[q][c]);
    }
    __syncthreads();
  }
  float *P = part + (int64_t)blockIdx.z * R * S;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int64_t r = r0 + ti + 16 * q;
    if (r >= R) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int64_t s = s0 + tj + 16 * c;
      if (s < S) P[r * S + s] = acc[q][c];
    }
  }
}

// out (R x S) (+)= sum over z of part[z], in z order
__global__ void sum_parts_kernel(const float *__restrict__ part, int64_t count, int64_t nz,
                                 float *__restrict__ out, int accumulate) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    float s = accumulate ? out[e] : 0.f;
    for (int64_t z = 0; z < nz; ++z) s += part[z * count + e];
    out[e] = s;
  }
}

// S (p x p) = Q^T D; then D <- D - Q sym(S) (tangent projection at Q on St_{n,p})
__global__ void qtd_kernel(const float *__restrict__ Q, const float *__restrict__ D, int64_t n,
                           int64_t p, float *__restrict__ Sm) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < p * p;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = e / p, b = e % p;
    float s = 0.f;
    for (int64_t i = 0; i < n; ++i) s = fmaf(Q[i * p + a], D[i * p + b], s);
    Sm[e] = s;
  }
}

__global__ void stiefel_kernel(const float *__restrict__ Q, const float *__restrict__ D,
                               const float *__restrict__ Sm, int64_t n, int64_t p,
                               float *__restrict__ out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * p;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / p, b = e % p;
    float s = 0.f;
    for (int64_t a = 0; a < p; ++a) s = fmaf(Q[i * p + a], 0.5f * (Sm[a * p + b] + Sm[b * p + a]), s);
    out[e] = D[e] - s;
  }
}

}  // namespace

int64_t nt_splits(int64_t R, int64_t S, int64_t K) {
  const int64_t tiles = ((R + 63) / 64) * ((S + 63) / 64);
  int64_t z = ((int64_t)num_sms() * 3 + tiles - 1) / tiles;
  const int64_t zmax = (K + 255) / 256;   // at least 256 of K per split
  if (z > zmax) z = zmax;
  return z < 1 ? 1 : z;
}

cudaError_t launch_nt_accumulate(const float *A, const float *B, int64_t R, int64_t S, int64_t K,
                                 float *part, float *out, int accumulate, cudaStream_t st) {
  const int64_t nz = nt_splits(R, S, K);
  const int64_t kchunk = (K + nz - 1) / nz;
  const dim3 grid((unsigned)((S + 63) / 64), (unsigned)((R + 63) / 64), (unsigned)nz);
  count_launch(1);
  nt_partial_kernel<<<grid, 256, 0, st>>>(A, B, R, S, K, kchunk, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t count = R * S;
  int blocks = (int)((count + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  count_launch(1);
  sum_parts_kernel<<<blocks, 256, 0, st>>>(part, count, nz, out, accumulate);
  return cudaGetLastError();
}

cudaError_t launch_stiefel(const float *Q, const float *D, int64_t n, int64_t p, float *Sm,
                           float *out, cudaStream_t st) {
  int b1 = (int)((p * p + 255) / 256);
  if (b1 > 4096) b1 = 4096;
  count_launch(1);
  qtd_kernel<<<b1, 256, 0, st>>>(Q, D, n, p, Sm);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int b2 = (int)((n * p + 255) / 256);
  if (b2 > 4096) b2 = 4096;
  count_launch(1);
  stiefel_kernel<<<b2, 256, 0, st>>>(Q, D, Sm, n, p, out);
  return cudaGetLastError();
}

cudaError_t launch_facewise_gemm(const float *A, const float *B, float *C, int64_t n1,
                                 int64_t m, int64_t n2, int64_t p, cudaStream_t st) {
  // slice t: C_t (n1 x n2) = A_t (n1 x m) * B_t (m x n2); A_t(r, c) = A[t*n1*m + r*m + c]
  const dim3 grid((unsigned)((n2 + BN - 1) / BN), (unsigned)((n1 + BM - 1) / BM),
                  (unsigned)p);
  count_launch(1);
  gemm_tile_kernel<<<grid, NT, 0, st>>>(A, m, 1, n1 * m, B, m * n2, n2, 1, C, n1 * n2, n1, m,
                                        n2, nullptr, nullptr, nullptr, nullptr);
  return cudaGetLastError();
}

}  // namespace pp
