// pp_gemm.cu -- the batched products of the library on the tensor cores: the
// facewise product (Def. 2.3), the strided facewise products of the backward
// pass, the slice-wise projector products of the HOSVD, and A B^T contracted
// over all pixels (the Q gradient and the mode-3 Gram of the U3 builder), the
// last split over the contraction into partial products summed in a fixed
// order.  All of them run on launch_batched_tc (tcgen05, 3-pass split TF32,
// FP32 sums of 32-term chunks; pp_gemm_tc.cu), as does Q^T D of the Stiefel
// projection; only its last n x p product Q sym(Q^T D) stays on the CUDA cores.
#include "pp_internal.h"

namespace pp {
namespace {

// ---------------------------------------------------------------- A B^T, split over K
// out (R x S) (+)= sum over z of part[z], in z order; the parts hold R x S
// (transposed = 0) or S x R (transposed = 1) products.  One CTA of 1024
// threads per 32 x 32 tile of the parts, one entry per thread summed over z
// with the parts read along their rows; a transposed tile goes out through
// shared memory so that the writes run along out's rows as well.
__global__ void __launch_bounds__(1024) sum_parts_kernel(const float *__restrict__ part,
                                                         int64_t R, int64_t S, int64_t nz,
                                                         float *__restrict__ out, int accumulate,
                                                         int transposed) {
  __shared__ float tile[32][33];
  const int64_t count = R * S;
  // the parts are rows x cols: S x R when transposed, else R x S
  const int64_t rows = transposed ? S : R, cols = transposed ? R : S;
  const int64_t tiles_c = (cols + 31) / 32;
  const int64_t r0 = (int64_t)(blockIdx.x / tiles_c) * 32, c0 = (int64_t)(blockIdx.x % tiles_c) * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t r = r0 + ty, c = c0 + tx;
  float v = 0.f;
  if (r < rows && c < cols) {
    const float *pz = part + r * cols + c;
#pragma unroll 8
    for (int64_t z = 0; z < nz; ++z) v += pz[z * count];   // fixed order
  }
  if (!transposed) {
    if (r < rows && c < cols) {
      const int64_t e = r * cols + c;
      out[e] = accumulate ? out[e] + v : v;
    }
    return;
  }
  tile[ty][tx] = v;
  __syncthreads();
  // out (R x S): out row = part column, out column = part row
  const int64_t oc = c0 + ty, orow = r0 + tx;   // part column c0 + ty, part row r0 + tx
  if (orow < rows && oc < cols) {
    const int64_t e = oc * S + orow;
    const float w = tile[tx][ty];
    out[e] = accumulate ? out[e] + w : w;
  }
}

// out = D - Q sym(S) with S = Q^T D (tangent projection at Q on St_{n,p})
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

// one CTA per 32 x 32 tile of the R x S output
unsigned sum_parts_blocks(int64_t R, int64_t S) {
  return (unsigned)(((R + 31) / 32) * ((S + 31) / 32));
}

}  // namespace

// The product behind A B^T: the tensor-core tile puts 128 rows of its output
// on the MMA's M and 64 on its N, so when S (the columns of A B^T) is the
// smaller side the product is formed transposed, B A^T (S x R), with R on M.
bool nt_transposed(int64_t R, int64_t S) { return S < R; }

// Splits of the contraction: enough (64 x 128)-tile members to cover the SMs
// three times, each with at least 256 of the K terms.
int64_t nt_splits(int64_t R, int64_t S, int64_t K) {
  const int64_t rows = nt_transposed(R, S) ? S : R, cols = nt_transposed(R, S) ? R : S;
  const int64_t tiles = ((rows + 63) / 64) * ((cols + 127) / 128);
  int64_t z = ((int64_t)num_sms() * 3 + tiles - 1) / tiles;
  const int64_t zmax = (K + 255) / 256;   // at least 256 of K per split
  if (z > zmax) z = zmax;
  return z < 1 ? 1 : z;
}

cudaError_t launch_nt_accumulate(const float *A, const float *B, int64_t R, int64_t S, int64_t K,
                                 float *part, float *out, int accumulate, cudaStream_t st,
                                 void *img, size_t img_bytes, int64_t part_floats) {
  if (img) {   // the warp-specialised kernel, the smaller operand's tf32 image in img
    bool used = false, trw = false;
    int64_t nzw = 0;
    cudaError_t e = launch_nt_ws(A, B, R, S, K, part, part_floats, img, img_bytes, &nzw, &trw, st,
                                 &used);
    if (e != cudaSuccess) return e;
    if (used) {
      count_launch(1);
      sum_parts_kernel<<<sum_parts_blocks(R, S), 1024, 0, st>>>(part, R, S, nzw, out, accumulate,
                                                                trw ? 1 : 0);
      return cudaGetLastError();
    }
  }
  const int64_t nz = nt_splits(R, S, K);
  int64_t kchunk = (K + nz - 1) / nz;
  kchunk = (kchunk + 31) / 32 * 32;            // whole 32-term chunks per split
  const int64_t nzu = (K + kchunk - 1) / kchunk;
  const bool tr = nt_transposed(R, S);
  // member z: part[z] = A[:, zk..] B[:, zk..]^T (R x S), or its transpose
  // B[:, zk..] A[:, zk..]^T (S x R); M(r, c) = first[r K + c], X(c, n) = second[n K + c]
  const float *first = tr ? B : A, *second = tr ? A : B;
  const int64_t P = tr ? S : R, N = tr ? R : S;
  cudaError_t e = launch_batched_tc(first, K, 1, kchunk, second, kchunk, 1, K, part, R * S, P,
                                    kchunk, N, nzu, K, nullptr, st);
  if (e != cudaSuccess) return e;
  count_launch(1);
  sum_parts_kernel<<<sum_parts_blocks(R, S), 1024, 0, st>>>(part, R, S, nzu, out, accumulate,
                                                            tr ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_batched_gemm(const float *Mm, int64_t sr, int64_t sc, int64_t sMz,
                                const float *X, int64_t sXz, float *Y, int64_t sYz, int64_t P,
                                int64_t S, int64_t N, int64_t batch, cudaStream_t st,
                                int64_t sxc, int64_t sxn) {
  if (sxc < 0) { sxc = N; sxn = 1; }
  return launch_batched_tc(Mm, sr, sc, sMz, X, sXz, sxc, sxn, Y, sYz, P, S, N, batch, 0,
                           nullptr, st);
}

cudaError_t launch_stiefel(const float *Q, const float *D, int64_t n, int64_t p, float *Sm,
                           float *out, cudaStream_t st, float *part, int64_t part_floats) {
  // Sm (p x p) = Q^T D on the tensor cores: M(a, i) = Q[i p + a], X = D (n x p).
  // One output tile contracted over all n rows is one CTA; with scratch for
  // the parts, the n rows are split into up to 8 members of at least
  // max(p, 32) rows (whole 32-row chunks) summed afterwards in a fixed order.
  int64_t kchunk = (n + 7) / 8;
  if (kchunk < p) kchunk = p;
  kchunk = (kchunk + 31) / 32 * 32;
  const int64_t nz = (n + kchunk - 1) / kchunk;
  cudaError_t e;
  if (nz > 1 && part && nz * p * p <= part_floats) {
    e = launch_batched_tc(Q, 1, p, kchunk * p, D, kchunk * p, p, 1, part, p * p, p, kchunk, p, nz,
                          n, nullptr, st);
    if (e != cudaSuccess) return e;
    count_launch(1);
    sum_parts_kernel<<<sum_parts_blocks(p, p), 1024, 0, st>>>(part, p, p, nz, Sm, 0, 0);
    e = cudaGetLastError();
  } else {
    e = launch_batched_tc(Q, 1, p, 0, D, 0, p, 1, Sm, 0, p, n, p, 1, 0, nullptr, st);
  }
  if (e != cudaSuccess) return e;
  int b2 = (int)((n * p + 255) / 256);
  if (b2 > 4096) b2 = 4096;
  count_launch(1);
  stiefel_kernel<<<b2, 256, 0, st>>>(Q, D, Sm, n, p, out);
  return cudaGetLastError();
}

size_t facewise_img_bytes(int64_t rows, int64_t inner, int64_t cols, int64_t p) {
  const size_t face = batched_img_bytes(rows > cols ? cols : rows, inner, 1);
  const size_t total = face * (size_t)(p < 1 ? 0 : p);
  const size_t cap = face > FACEWISE_IMG_CAP ? face : FACEWISE_IMG_CAP;
  return total < cap ? total : cap;
}

cudaError_t launch_facewise_strided(const float *L, int64_t sLi, int64_t sLk, int64_t sLz,
                                    const float *Rm, int64_t sRk, int64_t sRj, int64_t sRz,
                                    float *C, int64_t rows, int64_t inner, int64_t cols,
                                    int64_t p, cudaStream_t st, void *img, size_t img_bytes) {
  const size_t face = batched_img_bytes(rows > cols ? cols : rows, inner, 1);
  int64_t t0 = 0;   // faces before t0 are done
  if (img && face > 0 && img_bytes >= face) {
    // the faces in groups whose images fit in img; the larger of rows and
    // cols along the 128-row MMA tiles (rows: C_t^T = R_t^T L_t^T, C stored
    // transposed)
    const int64_t per = (int64_t)(img_bytes / face);
    for (; t0 < p; t0 += per) {
      const int64_t nb = p - t0 < per ? p - t0 : per;
      bool used = false;
      cudaError_t e = cudaSuccess;
      if (rows > cols) {
        const bool mn = sLi == 1, km = !mn && sLk == 1;
        if (mn || km)
          e = launch_batched_ws(Rm + t0 * sRz, sRj, sRk, sRz, L + t0 * sLz, sLz, mn ? sLk : sLi,
                                km, C + t0 * rows * cols, rows * cols, cols, true, cols, inner,
                                rows, nb, img, img_bytes, st, &used);
      } else {
        const bool mn = sRj == 1, km = !mn && sRk == 1;
        if (mn || km)
          e = launch_batched_ws(L + t0 * sLz, sLi, sLk, sLz, Rm + t0 * sRz, sRz, mn ? sRk : sRj,
                                km, C + t0 * rows * cols, rows * cols, cols, false, rows, inner,
                                cols, nb, img, img_bytes, st, &used);
      }
      if (e != cudaSuccess) return e;
      if (!used) break;
    }
    if (t0 >= p) return cudaSuccess;
  }
  return launch_batched_tc(L + t0 * sLz, sLi, sLk, sLz, Rm + t0 * sRz, sRz, sRk, sRj,
                           C + t0 * rows * cols, rows * cols, rows, inner, cols, p - t0, 0,
                           nullptr, st);
}

cudaError_t launch_facewise_gemm(const float *A, const float *B, float *C, int64_t n1,
                                 int64_t m, int64_t n2, int64_t p, cudaStream_t st, void *img,
                                 size_t img_bytes) {
  // slice t: C_t (n1 x n2) = A_t (n1 x m) * B_t (m x n2); A_t(r, c) = A[t*n1*m + r*m + c]
  return launch_facewise_strided(A, m, 1, n1 * m, B, n2, 1, m * n2, C, n1, m, n2, p, st, img,
                                 img_bytes);
}

}  // namespace pp
