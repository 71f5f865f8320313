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
    const float *__restrict__ X, int64_t sXz, float *__restrict__ Y, int64_t sYz, int64_t P,
    int64_t S, int64_t N, const float *__restrict__ Aref, double *__restrict__ errp,
    double *__restrict__ xpart, double *__restrict__ ypart) {
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
      const float v = (c < S && n < N) ? X[c * N + n] : 0.f;
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
  gemm_tile_kernel<<<grid, NT, 0, st>>>(Qm, sr, sc, 0, X, 0, Y, 0, P, S, N, Aref,
                                        err_partials, xpart, ypart);
  return cudaGetLastError();
}

cudaError_t launch_batched_gemm(const float *Mm, int64_t sr, int64_t sc, int64_t sMz,
                                const float *X, int64_t sXz, float *Y, int64_t sYz, int64_t P,
                                int64_t S, int64_t N, int64_t batch, cudaStream_t st) {
  const dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((P + BM - 1) / BM), (unsigned)batch);
  count_launch(1);
  gemm_tile_kernel<<<grid, NT, 0, st>>>(Mm, sr, sc, sMz, X, sXz, Y, sYz, P, S, N, nullptr,
                                        nullptr, nullptr, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_facewise_gemm(const float *A, const float *B, float *C, int64_t n1,
                                 int64_t m, int64_t n2, int64_t p, cudaStream_t st) {
  // slice t: C_t (n1 x n2) = A_t (n1 x m) * B_t (m x n2); A_t(r, c) = A[t*n1*m + r*m + c]
  const dim3 grid((unsigned)((n2 + BN - 1) / BN), (unsigned)((n1 + BM - 1) / BM),
                  (unsigned)p);
  count_launch(1);
  gemm_tile_kernel<<<grid, NT, 0, st>>>(A, m, 1, n1 * m, B, m * n2, C, n1 * n2, n1, m, n2,
                                        nullptr, nullptr, nullptr, nullptr);
  return cudaGetLastError();
}

}  // namespace pp
