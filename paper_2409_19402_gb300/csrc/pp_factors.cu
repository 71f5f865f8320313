// pp_factors.cu -- transform-domain factors and the low-rank rebuild
// (Alg. 4.1 step 3 output / Alg. 4.2 step 8 truncation, and the
// U-hat S-hat V-hat^T product that precedes the reverse transform).
//
// After the Jacobi iteration the converged vectors are w_q = sigma_q y_q,
// where y_q is the singular vector along the slice's long side (length a).
// The short-side singular vector follows from the slice itself:
//   short_q = X y_q / sigma_q = X w_q / sigma_q^2   (X oriented a_short x a),
// so no rotation accumulator is needed in the Jacobi kernel.  For a zero
// singular value both vectors are returned as zero.
//
// With the QR preconditioner (pp_qrcp.cu) the roles swap: the Jacobi vectors
// are the short-side singular vectors (scaled, in pivoted order) and the
// long-side vector is long_q = X^T short_q / sigma_q.
//
// Rank per slice: R_t = k (fixed, Alg. 4.1) or rho_t (Alg. 4.2, packed at
// offs[t]).  Output layouts (row-major blocks):
//   fixed:  Uh[t] is l x k at t*l*k, Vh[t] is m x k at t*m*k, s at t*k
//   ragged: Uh block l x rho_t at l*offs[t], Vh block m x rho_t at m*offs[t],
//           s at offs[t]
// The rebuild forms A-hat_k(:,:,t) = sum_{q < R_t} sigma_q u_q v_q^T.
#include "pp_internal.h"

namespace pp {
namespace {

struct Geo {
  int64_t rank;   // R_t
  int64_t soff;   // offset of s block
  int64_t uoff;   // offset of Uh block
  int64_t voff;   // offset of Vh block
};

__device__ __forceinline__ Geo geo(const FactorArgs &a, int64_t t) {
  Geo g;
  if (a.kfix > 0) {
    g.rank = a.kfix;
    g.soff = t * a.kfix;
    g.uoff = t * a.l * a.kfix;
    g.voff = t * a.m * a.kfix;
  } else {
    g.rank = a.rho[t];
    g.soff = a.offs[t];
    g.uoff = a.l * a.offs[t];
    g.voff = a.m * a.offs[t];
  }
  return g;
}

// long-side vectors and sigma; one CTA per slice
__global__ void factor_long_kernel(FactorArgs a) {
  const int64_t t = blockIdx.x;
  const Geo g = geo(a, t);
  const bool rows = a.l <= a.m;       // long side is V (length m) when l <= m
  const int64_t alen = rows ? a.m : a.l;
  float *out = rows ? a.Vh + g.voff : a.Uh + g.uoff;
  const float *sg = a.sig + t * a.b;
  const int32_t *pm = a.perm + t * a.b;
  const float *Wt = a.W + t * a.b * a.a_pad;
  for (int64_t idx = threadIdx.x; idx < alen * g.rank; idx += blockDim.x) {
    const int64_t e = idx / g.rank, q = idx % g.rank;
    const float sq = sg[q];
    out[e * g.rank + q] = sq > 0.f ? Wt[(int64_t)pm[q] * a.a_pad + e] / sq : 0.f;
  }
  for (int64_t q = threadIdx.x; q < g.rank; q += blockDim.x) a.s[g.soff + q] = sg[q];
  if (threadIdx.x == 0 && a.kept_partial) {
    double kept = 0.0, disc = 0.0;
    for (int64_t q = 0; q < a.b; ++q) {
      const double v = (double)sg[q] * (double)sg[q];
      if (q < g.rank) kept += v; else disc += v;
    }
    a.kept_partial[t] = kept;
    a.disc_partial[t] = disc;
  }
}

// short-side vectors: out(e2, q) = sum_e X(e2, e) w_{perm q}(e) / sigma_q^2
// tile 64 (e2) x 32 (q), 256 threads, each 4 x 2 outputs
__global__ void __launch_bounds__(256) factor_short_kernel(FactorArgs a) {
  const int64_t t = blockIdx.z;
  const Geo g = geo(a, t);
  const bool rows = a.l <= a.m;
  const int64_t nshort = rows ? a.l : a.m, nlong = rows ? a.m : a.l;
  const int64_t e20 = (int64_t)blockIdx.y * 64, q0 = (int64_t)blockIdx.x * 32;
  if (e20 >= nshort || q0 >= g.rank) return;
  __shared__ float Xs[16][64 + 1];
  __shared__ float Ws_[16][32 + 1];
  const float *Xf = a.X + t * a.l * a.m;
  const float *sg = a.sig + t * a.b;
  const int32_t *pm = a.perm + t * a.b;
  const float *Wt = a.W + t * a.b * a.a_pad;
  const int tid = threadIdx.x, ti = tid / 16, tj = tid % 16;
  float acc[4][2] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  for (int64_t k0 = 0; k0 < nlong; k0 += 16) {
    for (int e = tid; e < 64 * 16; e += 256) {
      int ii, kk;
      if (rows) { kk = e % 16; ii = e / 16; } else { ii = e % 64; kk = e / 64; }
      const int64_t e2 = e20 + ii, el = k0 + kk;
      float v = 0.f;
      if (e2 < nshort && el < nlong) v = rows ? Xf[e2 * a.m + el] : Xf[el * a.m + e2];
      Xs[kk][ii] = v;
    }
    for (int e = tid; e < 32 * 16; e += 256) {
      const int kk = e % 16, qq = e / 16;
      const int64_t el = k0 + kk, q = q0 + qq;
      Ws_[kk][qq] = (el < nlong && q < g.rank) ? Wt[(int64_t)pm[q] * a.a_pad + el] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float xv = Xs[kk][ti + 16 * r];
        acc[r][0] = fmaf(xv, Ws_[kk][tj], acc[r][0]);
        acc[r][1] = fmaf(xv, Ws_[kk][tj + 16], acc[r][1]);
      }
    }
    __syncthreads();
  }
  float *out = rows ? a.Uh + g.uoff : a.Vh + g.voff;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int64_t e2 = e20 + ti + 16 * r;
    if (e2 >= nshort) continue;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int64_t q = q0 + tj + 16 * c;
      if (q >= g.rank) continue;
      const float sq = sg[q];
      out[e2 * g.rank + q] = sq > 0.f ? acc[r][c] / (sq * sq) : 0.f;
    }
  }
}

// QR-preconditioned Jacobi (pp_qrcp.cu): the converged rows of W have length
// b and hold the short-side vectors in pivoted order,
// W_q[j] = sigma_q u_q[qperm[j]]; one CTA per slice.
__global__ void factor_pc_short_kernel(FactorArgs a) {
  const int64_t t = blockIdx.x;
  const Geo g = geo(a, t);
  const bool rows = a.l <= a.m;
  float *out = rows ? a.Uh + g.uoff : a.Vh + g.voff;
  const float *sg = a.sig + t * a.b;
  const int32_t *pm = a.perm + t * a.b;
  const int32_t *qp = a.qperm + t * a.b;
  const float *Wt = a.W + t * a.b * a.a_pad;
  for (int64_t idx = threadIdx.x; idx < a.b * g.rank; idx += blockDim.x) {
    const int64_t j = idx / g.rank, q = idx % g.rank;
    const float sq = sg[q];
    out[(int64_t)qp[j] * g.rank + q] = sq > 0.f ? Wt[(int64_t)pm[q] * a.a_pad + j] / sq : 0.f;
  }
  for (int64_t q = threadIdx.x; q < g.rank; q += blockDim.x) a.s[g.soff + q] = sg[q];
  if (threadIdx.x == 0 && a.kept_partial) {
    double kept = 0.0, disc = 0.0;
    for (int64_t q = 0; q < a.b; ++q) {
      const double v = (double)sg[q] * (double)sg[q];
      if (q < g.rank) kept += v; else disc += v;
    }
    a.kept_partial[t] = kept;
    a.disc_partial[t] = disc;
  }
}

// ... and the long-side vectors from the slice: long_q(e) = sum_{e2} X(e2, e)
// u_q(e2) / sigma_q over the short index e2 (X oriented short x long);
// tile 64 (e) x 32 (q), 256 threads, each 4 x 2 outputs; used for tall slices (l > m).
__global__ void __launch_bounds__(256) factor_pc_long_kernel(FactorArgs a) {
  const int64_t t = blockIdx.z;
  const Geo g = geo(a, t);
  const bool rows = a.l <= a.m;
  const int64_t nshort = rows ? a.l : a.m, nlong = rows ? a.m : a.l;
  const int64_t e0 = (int64_t)blockIdx.y * 64, q0 = (int64_t)blockIdx.x * 32;
  if (e0 >= nlong || q0 >= g.rank) return;
  __shared__ float Xs[16][64 + 1];
  __shared__ float Us[16][32 + 1];
  const float *Xf = a.X + t * a.l * a.m;
  const float *sg = a.sig + t * a.b;
  const float *U = rows ? a.Uh + g.uoff : a.Vh + g.voff;      // nshort x rank
  const int tid = threadIdx.x, ti = tid / 16, tj = tid % 16;
  float acc[4][2] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  for (int64_t k0 = 0; k0 < nshort; k0 += 16) {
    for (int e = tid; e < 64 * 16; e += 256) {
      int ii, kk;
      if (rows) { ii = e % 64; kk = e / 64; } else { kk = e % 16; ii = e / 16; }
      const int64_t e2 = k0 + kk, el = e0 + ii;
      float v = 0.f;
      if (e2 < nshort && el < nlong) v = rows ? Xf[e2 * a.m + el] : Xf[el * a.m + e2];
      Xs[kk][ii] = v;
    }
    for (int e = tid; e < 32 * 16; e += 256) {
      const int qq = e % 32, kk = e / 32;
      const int64_t e2 = k0 + kk, q = q0 + qq;
      Us[kk][qq] = (e2 < nshort && q < g.rank) ? U[e2 * g.rank + q] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float xv = Xs[kk][ti + 16 * r];
        acc[r][0] = fmaf(xv, Us[kk][tj], acc[r][0]);
        acc[r][1] = fmaf(xv, Us[kk][tj + 16], acc[r][1]);
      }
    }
    __syncthreads();
  }
  float *out = rows ? a.Vh + g.voff : a.Uh + g.uoff;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int64_t el = e0 + ti + 16 * r;
    if (el >= nlong) continue;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int64_t q = q0 + tj + 16 * c;
      if (q >= g.rank) continue;
      const float sq = sg[q];
      out[el * g.rank + q] = sq > 0.f ? acc[r][c] / sq : 0.f;
    }
  }
}

// The same product when the slice is short x long row-major (l <= m): lanes
// run over 32 consecutive long indices e (coalesced rows of X), the 8 warps
// over residues of the short index e2, and the short-side vectors sit in
// shared memory 8 columns at a time.  Small ragged ranks (the usual output of
// Alg. 4.2) then cost one pass over the slice per 8 ranks instead of a tile
// loop over the whole short side per 32.  256 threads; dynamic shared memory
// holds nshort x 8 vector entries and the 8 x 32 x 8 warp partials.
constexpr int PCL_QC = 8;
__global__ void __launch_bounds__(256) factor_pc_long_rows_kernel(FactorArgs a) {
  const int64_t t = blockIdx.y;
  const Geo g = geo(a, t);
  if (g.rank == 0) return;
  const int64_t nshort = a.l, nlong = a.m;
  extern __shared__ float4 pcl_smem4[];
  float4 *Us = pcl_smem4;                                   // nshort x 2 float4
  float *red = reinterpret_cast<float *>(pcl_smem4 + 2 * nshort);   // [8][32][8]
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int64_t e0 = (int64_t)blockIdx.x * 32, e = e0 + lane;
  const float *Xf = a.X + t * a.l * a.m;
  const float *sg = a.sig + t * a.b;
  const float *U = a.Uh + g.uoff;                           // nshort x rank
  float *out = a.Vh + g.voff;                               // nlong x rank
  float *Usf = reinterpret_cast<float *>(Us);
  for (int64_t q0 = 0; q0 < g.rank; q0 += PCL_QC) {
    for (int64_t idx = tid; idx < nshort * PCL_QC; idx += 256) {
      const int64_t e2 = idx / PCL_QC, q = q0 + idx % PCL_QC;
      Usf[idx] = q < g.rank ? U[e2 * g.rank + q] : 0.f;
    }
    __syncthreads();
    float acc[PCL_QC] = {};
    if (e < nlong) {
#pragma unroll 4
      for (int64_t e2 = w; e2 < nshort; e2 += 8) {
        const float x = Xf[e2 * a.m + e];
        const float4 u0 = Us[2 * e2], u1 = Us[2 * e2 + 1];
        acc[0] = fmaf(x, u0.x, acc[0]); acc[1] = fmaf(x, u0.y, acc[1]);
        acc[2] = fmaf(x, u0.z, acc[2]); acc[3] = fmaf(x, u0.w, acc[3]);
        acc[4] = fmaf(x, u1.x, acc[4]); acc[5] = fmaf(x, u1.y, acc[5]);
        acc[6] = fmaf(x, u1.z, acc[6]); acc[7] = fmaf(x, u1.w, acc[7]);
      }
    }
#pragma unroll
    for (int c = 0; c < PCL_QC; ++c) red[(w * 32 + lane) * PCL_QC + c] = acc[c];
    __syncthreads();
    {
      const int el = tid / PCL_QC, c = tid % PCL_QC;          // 32 e x 8 q outputs
      float v = 0.f;
#pragma unroll
      for (int ww = 0; ww < 8; ++ww) v += red[(ww * 32 + el) * PCL_QC + c];
      const int64_t eo = e0 + el, q = q0 + c;
      if (eo < nlong && q < g.rank) {
        const float sq = sg[q];
        out[eo * g.rank + q] = sq > 0.f ? v / sq : 0.f;
      }
    }
    __syncthreads();
  }
}

// rebuild: Ahk(i, j) = sum_{q < R} Uh(i, q) s_q Vh(j, q); tile 64 x 64, 256 threads
__global__ void __launch_bounds__(256) rebuild_kernel(FactorArgs a) {
  const int64_t t = blockIdx.z;
  const Geo g = geo(a, t);
  const int64_t i0 = (int64_t)blockIdx.y * 64, j0 = (int64_t)blockIdx.x * 64;
  if (i0 >= a.l || j0 >= a.m) return;
  __shared__ float Us[16][64 + 1];
  __shared__ float Vs[16][64 + 1];
  const float *U = a.Uh + g.uoff;
  const float *V = a.Vh + g.voff;
  const float *S = a.s + g.soff;
  const int tid = threadIdx.x, ti = tid / 16, tj = tid % 16;
  float acc[4][4] = {};
  for (int64_t k0 = 0; k0 < g.rank; k0 += 16) {
    for (int e = tid; e < 64 * 16; e += 256) {
      const int kk = e % 16, ii = e / 16;
      const int64_t q = k0 + kk;
      const int64_t i = i0 + ii, j = j0 + ii;
      Us[kk][ii] = (q < g.rank && i < a.l) ? U[i * g.rank + q] * S[q] : 0.f;
      Vs[kk][ii] = (q < g.rank && j < a.m) ? V[j * g.rank + q] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float u[4], v[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) { u[r] = Us[kk][ti + 16 * r]; v[r] = Vs[kk][tj + 16 * r]; }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(u[r], v[c], acc[r][c]);
    }
    __syncthreads();
  }
  float *O = a.Ahk + t * a.l * a.m;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int64_t i = i0 + ti + 16 * r;
    if (i >= a.l) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int64_t j = j0 + tj + 16 * c;
      if (j < a.m) O[i * a.m + j] = acc[r][c];
    }
  }
}

}  // namespace

cudaError_t launch_factors(const FactorArgs &a, cudaStream_t st) {
  const int64_t R = a.kfix > 0 ? a.kfix : a.b;   // grid bound; ragged CTAs exit early
  if (a.qperm) {
    count_launch(1);
    factor_pc_short_kernel<<<(unsigned)a.p, 256, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (a.l <= a.m) {
      const size_t smem = sizeof(float) * (size_t)(a.l * PCL_QC + 8 * 32 * PCL_QC);
      if (smem > 48 * 1024) return cudaErrorInvalidValue;   // qrcp_fits keeps l small
      count_launch(1);
      factor_pc_long_rows_kernel<<<dim3((unsigned)((a.m + 31) / 32), (unsigned)a.p), 256, smem,
                                   st>>>(a);
    } else {
      const dim3 g1((unsigned)((R + 31) / 32), (unsigned)((a.l + 63) / 64), (unsigned)a.p);
      count_launch(1);
      factor_pc_long_kernel<<<g1, 256, 0, st>>>(a);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess || !a.Ahk) return e;
    const dim3 g2((unsigned)((a.m + 63) / 64), (unsigned)((a.l + 63) / 64), (unsigned)a.p);
    count_launch(1);
    rebuild_kernel<<<g2, 256, 0, st>>>(a);
    return cudaGetLastError();
  }
  count_launch(1);
  factor_long_kernel<<<(unsigned)a.p, 256, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t nshort = a.l <= a.m ? a.l : a.m;
  const dim3 g1((unsigned)((R + 31) / 32), (unsigned)((nshort + 63) / 64), (unsigned)a.p);
  count_launch(1);
  factor_short_kernel<<<g1, 256, 0, st>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (a.Ahk) {
    const dim3 g2((unsigned)((a.m + 63) / 64), (unsigned)((a.l + 63) / 64), (unsigned)a.p);
    count_launch(1);
    rebuild_kernel<<<g2, 256, 0, st>>>(a);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace pp
