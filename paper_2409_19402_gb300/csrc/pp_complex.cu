// pp_complex.cu -- the hot path with a complex transformation Q in St_{n,p}(C)
// (Sec. 3 defines the projected product over C; the remark after Def. 3.2 notes
// that with Q = F(1:p,:)^H, the DFT rows, the product of real tensors can be
// complex).  Real data A, complex Q:
//   A-hat = A x_3 Q^H is complex (two real mode-3 products: Re Q^T A and -Im Q^T A),
//   facewise complex SVDs by a one-sided Jacobi with unitary 2x2 rotations,
//   the same global energy select (singular values are real),
//   complex factors and rebuild, and A_k = A-hat_k x_3 Q as two real products
//   with the stacked real matrices [Re Q | -Im Q] and [Im Q | Re Q].
//
// Layouts: Q and the returned factors are interleaved complex (re, im float
// pairs, as C99 float complex / torch.complex64); inside the workspace the
// transform domain is planar: the p real slices, then the p imaginary slices.
#include "pp_internal.h"

namespace pp {
namespace {

// ------------------------------------------------------------ real matrices from Q
// Pim (p x n) = -Im(Q)^T;  Bre (n x 2p) = [Re Q | -Im Q];  Bim (n x 2p) = [Im Q | Re Q]
__global__ void qc_build_kernel(const float *__restrict__ Qf, int64_t n, int64_t p,
                                float *__restrict__ Pim, float *__restrict__ Bre,
                                float *__restrict__ Bim) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n * p;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = idx / p, t = idx % p;
    const float re = Qf[2 * idx], im = Qf[2 * idx + 1];
    Pim[t * n + s] = -im;
    Bre[s * 2 * p + t] = re;
    Bre[s * 2 * p + p + t] = -im;
    Bim[s * 2 * p + t] = im;
    Bim[s * 2 * p + p + t] = re;
  }
}

// max |Q^H Q - I| over the p x p entries; entry (i, j) per thread
__global__ void qc_check_kernel(const float *__restrict__ Qf, int64_t n, int64_t p, float tol,
                                int32_t *status) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < p * p;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / p, j = idx % p;
    double re = 0.0, im = 0.0;
    for (int64_t s = 0; s < n; ++s) {
      const double ar = Qf[2 * (s * p + i)], ai = Qf[2 * (s * p + i) + 1];
      const double br = Qf[2 * (s * p + j)], bi = Qf[2 * (s * p + j) + 1];
      re += ar * br + ai * bi;          // conj(a) b
      im += ar * bi - ai * br;
    }
    if (i == j) re -= 1.0;
    if (fabs(re) > tol || fabs(im) > tol) set_status(status, PP_ENOTORTHO);
  }
}

// ------------------------------------------------------------ complex one-sided Jacobi
constexpr int CJ_THREADS = 1024;
constexpr int CJ_G = 16;                       // lanes per pair

__device__ __forceinline__ void cj_circle_pair(int N, int r, int slot, int &j, int &k) {
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

__device__ __forceinline__ float cj_group_sum(float v, unsigned mask) {
#pragma unroll
  for (int off = CJ_G / 2; off > 0; off >>= 1) v += __shfl_xor_sync(mask, v, off, CJ_G);
  return v;
}

// The pair's (real, imaginary) inner-product partials summed over its CJ_G
// lanes through the warp's 32 float2 of scratch, in a fixed order (bitwise the
// same in every lane of the group).
__device__ __forceinline__ float2 cj_group_sum2(float2 v, float2 *wred, unsigned mask) {
  const int wl = threadIdx.x & 31;
  wred[wl] = v;
  __syncwarp(mask);
  const float4 *rp = reinterpret_cast<const float4 *>(wred + (wl & ~(CJ_G - 1)));
  float2 sv[CJ_G / 4];
#pragma unroll
  for (int k = 0; k < CJ_G / 4; ++k) {
    const float4 a = rp[2 * k], b = rp[2 * k + 1];          // four float2
    sv[k] = make_float2((a.x + a.z) + (b.x + b.z), (a.y + a.w) + (b.y + b.w));
  }
#pragma unroll
  for (int w = CJ_G / 8; w > 0; w >>= 1)
#pragma unroll
    for (int k = 0; k < w; ++k) sv[k] = make_float2(sv[k].x + sv[k + w].x, sv[k].y + sv[k + w].y);
  __syncwarp(mask);
  return sv[0];
}

// One pair x, y (complex, length a_pad): with g = x^H y = |g| e^{i phi}, the
// unitary [[c, s e^{i phi}], [-s e^{-i phi}, c]] acting on [x y] gives
// x'^H y' = e^{i phi} (c s (al - be) + (c^2 - s^2) |g|), zero for the real
// symmetric Schur angle of (al, be, |g|); applied in Rutishauser's form
// (1 - s tau = c).  Squared norms are tracked (al - t |g|, be + t |g|).  The
// angle as in the real kernel: cos^2 = (h + |d|) / 2h, each MUFU result
// refined by one Newton step.
__device__ __forceinline__ bool cj_pair(float2 *__restrict__ x, float2 *__restrict__ y,
                                        float *na, float *nb, int a_pad, float tol2, int lane,
                                        unsigned mask, float2 *wred) {
  float gr = 0.f, gi = 0.f;
  for (int e = lane; e < a_pad; e += CJ_G) {
    const float2 u = x[e], v = y[e];
    gr = fmaf(u.x, v.x, fmaf(u.y, v.y, gr));
    gi = fmaf(u.x, v.y, fmaf(-u.y, v.x, gi));
  }
  const float2 g = cj_group_sum2(make_float2(gr, gi), wred, mask);
  const float al = *na, be = *nb;
  const float g2 = fmaf(g.x, g.x, g.y * g.y);
  if (g2 == 0.f || g2 <= tol2 * al * be) return false;
  float iag = rsqrtf(g2);
  iag = iag * fmaf(-0.5f * g2 * iag, iag, 1.5f);
  const float ag = g2 * iag;
  const float cph = g.x * iag, sph = g.y * iag;   // e^{i phi}
  const float d = be - al, g2x = 2.f * ag;
  const float r = fmaf(d, d, g2x * g2x);
  float ih = rsqrtf(r);
  ih = ih * fmaf(-0.5f * r * ih, ih, 1.5f);
  const float q = fmaf(r, ih, fabsf(d));          // h + |d|
  const float c2 = 0.5f * q * ih;                 // cos^2(theta)
  float rc = rsqrtf(c2);
  float iq = __fdividef(1.f, q);
  rc = rc * fmaf(-0.5f * c2 * rc, rc, 1.5f);
  iq = fmaf(iq, fmaf(-q, iq, 1.f), iq);
  const float c = c2 * rc;
  const float t = copysignf(1.f, d) * g2x * iq;
  const float s = c * t;
  const float onec = 1.f + c;
  float rp = __fdividef(1.f, onec);
  rp = fmaf(rp, fmaf(-onec, rp, 1.f), rp);
  const float tau = s * rp;
  // x' = x - s (tau x + e^{-i phi} y),  y' = y + s (e^{i phi} x - tau y): the
  // unitary [[c, s e^{i phi}], [-s e^{-i phi}, c]] (1 - s tau = c) with the phase
  // only in the terms scaled by s, so its rounding moves no norm by more than s u
  for (int e = lane; e < a_pad; e += CJ_G) {
    const float2 u = x[e], v = y[e];
    const float2 pv = make_float2(fmaf(v.x, cph, v.y * sph), fmaf(v.y, cph, -v.x * sph));
    const float2 pu = make_float2(fmaf(u.x, cph, -u.y * sph), fmaf(u.y, cph, u.x * sph));
    x[e] = make_float2(fmaf(-s, fmaf(tau, u.x, pv.x), u.x), fmaf(-s, fmaf(tau, u.y, pv.y), u.y));
    y[e] = make_float2(fmaf(s, fmaf(-tau, v.x, pu.x), v.x), fmaf(s, fmaf(-tau, v.y, pu.y), v.y));
  }
  if (lane == 0) {
    *na = fmaxf(fmaf(-t, ag, al), 0.f);
    *nb = fmaf(t, ag, be);
  }
  return true;
}

// One CTA per slice, the slice's b vectors resident in shared memory (complex,
// rows when l <= m, else columns), cyclic round-robin (circle) ordering.
__global__ void __launch_bounds__(CJ_THREADS) cjacobi_kernel(CJacobiArgs A) {
  extern __shared__ __align__(16) float2 cw[];
  __shared__ int flag;
  __shared__ __align__(16) float2 cj_red[CJ_THREADS];     // 32 float2 per warp
  float2 *wred = cj_red + (threadIdx.x & ~31);
  const int64_t f = blockIdx.x;
  const int l = (int)A.l, m = (int)A.m;
  const bool rows = l <= m;
  const int b = rows ? l : m, a = rows ? m : l;
  const int ap = A.a_pad;
  float *nrm = reinterpret_cast<float *>(cw + (size_t)b * ap);
  const float *Xr = A.Xre + f * (int64_t)l * m;
  const float *Xi = A.Xim + f * (int64_t)l * m;
  const int tid = threadIdx.x, lane = tid % CJ_G, grp = tid / CJ_G, ngrp = CJ_THREADS / CJ_G;
  const unsigned mask = ((1u << CJ_G) - 1u) << ((tid & 31) & ~(CJ_G - 1));
  for (int idx = tid; idx < b * ap; idx += CJ_THREADS) {
    const int j = idx / ap, e = idx % ap;
    float2 v = make_float2(0.f, 0.f);
    if (e < a) {
      const int64_t o = rows ? (int64_t)j * m + e : (int64_t)e * m + j;
      v = make_float2(Xr[o], Xi[o]);
    }
    cw[idx] = v;
  }
  __syncthreads();
  for (int j = grp; j < b; j += ngrp) {
    float s = 0.f;
    for (int e = lane; e < ap; e += CJ_G) {
      const float2 v = cw[(size_t)j * ap + e];
      s = fmaf(v.x, v.x, fmaf(v.y, v.y, s));
    }
    s = cj_group_sum(s, mask);
    if (lane == 0) nrm[j] = s;
  }
  __syncthreads();
  const float tol2 = A.tol * A.tol;
  const int N = b + (b & 1);
  int sweeps = 0;
  bool converged = false;
  while (sweeps < A.max_sweeps) {
    ++sweeps;
    int rot = 0;
    for (int r = 0; r < N - 1; ++r) {
      for (int slot = grp; slot < N / 2; slot += ngrp) {
        int j, k;
        cj_circle_pair(N, r, slot, j, k);
        if (j >= b || k >= b) continue;
        if (cj_pair(cw + (size_t)j * ap, cw + (size_t)k * ap, nrm + j, nrm + k, ap, tol2, lane,
                    mask, wred) &&
            lane == 0)
          ++rot;
      }
      __syncthreads();
    }
    if (tid == 0) flag = 0;
    __syncthreads();
    if (rot) atomicAdd(&flag, rot);
    __syncthreads();
    const int total = flag;
    __syncthreads();
    if (total == 0) {
      converged = true;
      break;
    }
  }
  // singular values from the final vectors, sorted descending (ties: lower index)
  for (int j = grp; j < b; j += ngrp) {
    float s = 0.f;
    for (int e = lane; e < ap; e += CJ_G) {
      const float2 v = cw[(size_t)j * ap + e];
      s = fmaf(v.x, v.x, fmaf(v.y, v.y, s));
    }
    s = cj_group_sum(s, mask);
    if (lane == 0) nrm[j] = sqrtf(s);
  }
  __syncthreads();
  for (int j = tid; j < b; j += CJ_THREADS) {
    const float sj = nrm[j];
    int rank = 0;
    for (int i = 0; i < b; ++i) {
      const float si = nrm[i];
      rank += (si > sj || (si == sj && i < j)) ? 1 : 0;
    }
    A.perm[f * b + rank] = j;
    A.sig[f * b + rank] = sj;
  }
  float2 *Wg = A.W + f * (int64_t)b * ap;
  for (int idx = tid; idx < b * ap; idx += CJ_THREADS) Wg[idx] = cw[idx];
  if (tid == 0) {
    A.sweeps[f] = sweeps;
    if (!converged) set_status(A.status, PP_ENOCONV);
  }
}

// ------------------------------------------------------------ factors and rebuild
struct CGeo {
  int64_t rank, soff, uoff, voff;
};

__device__ __forceinline__ CGeo cgeo(const CFactorArgs &a, int64_t t) {
  CGeo g;
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

// Converged rows (l <= m): W = J X with W W^H = S^2, so v_q = conj(w_q) / sigma_q.
// Columns (l > m): W = X J with W^H W = S^2, so u_q = w_q / sigma_q.  One CTA per slice.
__global__ void cfactor_long_kernel(CFactorArgs a) {
  const int64_t t = blockIdx.x;
  const CGeo g = cgeo(a, t);
  const bool rows = a.l <= a.m;
  const int64_t alen = rows ? a.m : a.l;
  float2 *out = rows ? a.Vh + g.voff : a.Uh + g.uoff;
  const float *sg = a.sig + t * a.b;
  const int32_t *pm = a.perm + t * a.b;
  const float2 *Wt = a.W + t * a.b * a.a_pad;
  for (int64_t idx = threadIdx.x; idx < alen * g.rank; idx += blockDim.x) {
    const int64_t e = idx / g.rank, q = idx % g.rank;
    const float sq = sg[q];
    float2 w = Wt[(int64_t)pm[q] * a.a_pad + e];
    if (rows) w.y = -w.y;
    out[e * g.rank + q] = sq > 0.f ? make_float2(w.x / sq, w.y / sq) : make_float2(0.f, 0.f);
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

// Short side: rows: u_q(i) = sum_e X(i, e) conj(w_q(e)) / sigma_q^2;
//             cols: v_q(e) = sum_i conj(X(i, e)) w_q(i) / sigma_q^2.
// Tile 32 (short index) x 32 (q), 256 threads, 4 outputs each.
__global__ void __launch_bounds__(256) cfactor_short_kernel(CFactorArgs a) {
  const int64_t t = blockIdx.z;
  const CGeo g = cgeo(a, t);
  const bool rows = a.l <= a.m;
  const int64_t nshort = rows ? a.l : a.m, nlong = rows ? a.m : a.l;
  const int64_t e20 = (int64_t)blockIdx.y * 32, q0 = (int64_t)blockIdx.x * 32;
  if (e20 >= nshort || q0 >= g.rank) return;
  __shared__ float2 Xs[16][33];
  __shared__ float2 Ws[16][33];
  const float *Xr = a.Xre + t * a.l * a.m, *Xi = a.Xim + t * a.l * a.m;
  const float *sg = a.sig + t * a.b;
  const int32_t *pm = a.perm + t * a.b;
  const float2 *Wt = a.W + t * a.b * a.a_pad;
  const int tid = threadIdx.x, tq = tid % 32, te = tid / 32;     // te in 0..7
  float2 acc[4] = {};
  for (int64_t k0 = 0; k0 < nlong; k0 += 16) {
    for (int e = tid; e < 32 * 16; e += 256) {
      const int kk = e % 16, ii = e / 16;
      const int64_t e2 = e20 + ii, el = k0 + kk;
      float2 v = make_float2(0.f, 0.f);
      if (e2 < nshort && el < nlong) {
        const int64_t o = rows ? e2 * a.m + el : el * a.m + e2;
        v = make_float2(Xr[o], rows ? Xi[o] : -Xi[o]);       // X(i,e), or conj(X(i,e))
      }
      Xs[kk][ii] = v;
      const int64_t q = q0 + ii;
      float2 w = make_float2(0.f, 0.f);
      if (el < nlong && q < g.rank) {
        w = Wt[(int64_t)pm[q] * a.a_pad + el];
        if (rows) w.y = -w.y;                                   // conj(w) for rows
      }
      Ws[kk][ii] = w;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      const float2 w = Ws[kk][tq];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float2 x = Xs[kk][te + 8 * r];
        acc[r].x = fmaf(x.x, w.x, fmaf(-x.y, w.y, acc[r].x));
        acc[r].y = fmaf(x.x, w.y, fmaf(x.y, w.x, acc[r].y));
      }
    }
    __syncthreads();
  }
  float2 *out = rows ? a.Uh + g.uoff : a.Vh + g.voff;
  const int64_t q = q0 + tq;
  if (q >= g.rank) return;
  const float sq = sg[q];
  const float inv = sq > 0.f ? 1.f / (sq * sq) : 0.f;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int64_t e2 = e20 + te + 8 * r;
    if (e2 < nshort) out[e2 * g.rank + q] = make_float2(acc[r].x * inv, acc[r].y * inv);
  }
}

// A-hat_k(i, j) = sum_q U(i, q) sigma_q conj(V(j, q)), planar outputs; tile 32 x 32
__global__ void __launch_bounds__(256) crebuild_kernel(CFactorArgs a) {
  const int64_t t = blockIdx.z;
  const CGeo g = cgeo(a, t);
  const int64_t i0 = (int64_t)blockIdx.y * 32, j0 = (int64_t)blockIdx.x * 32;
  if (i0 >= a.l || j0 >= a.m) return;
  __shared__ float2 Us[16][33];
  __shared__ float2 Vs[16][33];
  const float2 *U = a.Uh + g.uoff, *V = a.Vh + g.voff;
  const float *S = a.s + g.soff;
  const int tid = threadIdx.x, tj = tid % 32, ti = tid / 32;
  float2 acc[4] = {};
  for (int64_t k0 = 0; k0 < g.rank; k0 += 16) {
    for (int e = tid; e < 32 * 16; e += 256) {
      const int kk = e % 16, ii = e / 16;
      const int64_t q = k0 + kk;
      float2 u = make_float2(0.f, 0.f), v = u;
      if (q < g.rank && i0 + ii < a.l) {
        u = U[(i0 + ii) * g.rank + q];
        u.x *= S[q];
        u.y *= S[q];
      }
      if (q < g.rank && j0 + ii < a.m) {
        v = V[(j0 + ii) * g.rank + q];
        v.y = -v.y;                                   // conj
      }
      Us[kk][ii] = u;
      Vs[kk][ii] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      const float2 v = Vs[kk][tj];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float2 u = Us[kk][ti + 8 * r];
        acc[r].x = fmaf(u.x, v.x, fmaf(-u.y, v.y, acc[r].x));
        acc[r].y = fmaf(u.x, v.y, fmaf(u.y, v.x, acc[r].y));
      }
    }
    __syncthreads();
  }
  const int64_t plm = a.p * a.l * a.m;
  float *Or = a.Ahk + t * a.l * a.m, *Oi = Or + plm;
  const int64_t j = j0 + tj;
  if (j >= a.m) return;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int64_t i = i0 + ti + 8 * r;
    if (i < a.l) {
      Or[i * a.m + j] = acc[r].x;
      Oi[i * a.m + j] = acc[r].y;
    }
  }
}

// complex facewise product C_t = A_t B_t on planar stacked operands; tile 32 x 32
__global__ void __launch_bounds__(256) cfacewise_kernel(const float *__restrict__ Ap,
                                                        const float *__restrict__ Bp,
                                                        float *__restrict__ Cp, int64_t n1,
                                                        int64_t m, int64_t n2, int64_t p) {
  const int64_t t = blockIdx.z;
  const int64_t i0 = (int64_t)blockIdx.y * 32, j0 = (int64_t)blockIdx.x * 32;
  __shared__ float2 As[16][33];
  __shared__ float2 Bs[16][33];
  const float *Ar = Ap + t * n1 * m, *Ai = Ar + p * n1 * m;
  const float *Br = Bp + t * m * n2, *Bi = Br + p * m * n2;
  const int tid = threadIdx.x, tj = tid % 32, ti = tid / 32;
  float2 acc[4] = {};
  for (int64_t k0 = 0; k0 < m; k0 += 16) {
    for (int e = tid; e < 32 * 16; e += 256) {
      const int kk = e % 16, ii = e / 16;
      const int64_t k = k0 + kk;
      float2 u = make_float2(0.f, 0.f), v = u;
      if (k < m && i0 + ii < n1) u = make_float2(Ar[(i0 + ii) * m + k], Ai[(i0 + ii) * m + k]);
      As[kk][ii] = u;
      const int kk2 = e / 32, jj = e % 32;
      const int64_t k2 = k0 + kk2;
      if (k2 < m && j0 + jj < n2) v = make_float2(Br[k2 * n2 + j0 + jj], Bi[k2 * n2 + j0 + jj]);
      Bs[kk2][jj] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      const float2 v = Bs[kk][tj];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float2 u = As[kk][ti + 8 * r];
        acc[r].x = fmaf(u.x, v.x, fmaf(-u.y, v.y, acc[r].x));
        acc[r].y = fmaf(u.x, v.y, fmaf(u.y, v.x, acc[r].y));
      }
    }
    __syncthreads();
  }
  float *Cr = Cp + t * n1 * n2, *Ci = Cr + p * n1 * n2;
  const int64_t j = j0 + tj;
  if (j >= n2) return;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int64_t i = i0 + ti + 8 * r;
    if (i < n1) {
      Cr[i * n2 + j] = acc[r].x;
      Ci[i * n2 + j] = acc[r].y;
    }
  }
}

inline unsigned grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (unsigned)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

}  // namespace

int64_t cjacobi_apad(int64_t l, int64_t m) {
  const int64_t a = l > m ? l : m;
  return round_up(a, CJ_G);
}

size_t cjacobi_smem(int64_t l, int64_t m) {
  const int64_t b = l < m ? l : m;
  return (size_t)b * cjacobi_apad(l, m) * sizeof(float2) + (size_t)b * sizeof(float);
}

cudaError_t launch_qc_build(const float *Qf, int64_t n, int64_t p, float *Pim, float *Bre,
                            float *Bim, cudaStream_t st) {
  count_launch(1);
  qc_build_kernel<<<grid_for(n * p), 256, 0, st>>>(Qf, n, p, Pim, Bre, Bim);
  return cudaGetLastError();
}

cudaError_t launch_qc_check(const float *Qf, int64_t n, int64_t p, float tol, int32_t *status,
                            cudaStream_t st) {
  count_launch(1);
  qc_check_kernel<<<grid_for(p * p), 256, 0, st>>>(Qf, n, p, tol, status);
  return cudaGetLastError();
}

cudaError_t launch_cjacobi(const CJacobiArgs &a, cudaStream_t st) {
  const size_t smem = cjacobi_smem(a.l, a.m);
  cudaError_t e = cudaFuncSetAttribute(cjacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  count_launch(1);
  cjacobi_kernel<<<(unsigned)a.p, CJ_THREADS, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_cfactors(const CFactorArgs &a, cudaStream_t st) {
  const int64_t R = a.kfix > 0 ? a.kfix : a.b;
  count_launch(1);
  cfactor_long_kernel<<<(unsigned)a.p, 256, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t nshort = a.l <= a.m ? a.l : a.m;
  const dim3 g1((unsigned)((R + 31) / 32), (unsigned)((nshort + 31) / 32), (unsigned)a.p);
  count_launch(1);
  cfactor_short_kernel<<<g1, 256, 0, st>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess || !a.Ahk) return e;
  const dim3 g2((unsigned)((a.m + 31) / 32), (unsigned)((a.l + 31) / 32), (unsigned)a.p);
  count_launch(1);
  crebuild_kernel<<<g2, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_cfacewise(const float *A, const float *B, float *C, int64_t n1, int64_t m,
                             int64_t n2, int64_t p, cudaStream_t st) {
  const dim3 g((unsigned)((n2 + 31) / 32), (unsigned)((n1 + 31) / 32), (unsigned)p);
  count_launch(1);
  cfacewise_kernel<<<g, 256, 0, st>>>(A, B, C, n1, m, n2, p);
  return cudaGetLastError();
}

}  // namespace pp
