// pp_qrcp.cu -- QR factorisation with column pivoting of every transform-domain
// slice, the preconditioner of the one-sided Jacobi SVD (Drmac & Veselic,
// "New fast and accurate Jacobi SVD algorithm", SIAM J. Matrix Anal. Appl.
// 29 (2008)).
//
// A slice X (l x m) has b = min(l, m) vectors of length a = max(l, m): its rows
// when l <= m, else its columns.  With Y the a x b matrix whose columns are
// those vectors, Householder QR with column pivoting gives Y P = Q R (R b x b
// upper triangular).  The Jacobi iteration then orthogonalises the rows of R:
// graded, shorter (b instead of a) and much closer to orthogonal than the rows
// of X, they converge in fewer sweeps.  Q is never formed: with J R = W
// (orthogonal rows) the normalised rows of W are the short-side singular
// vectors of X in pivoted order (W_k[j] = sigma_k u_k[perm[j]]), and the
// long-side vectors follow from X itself (X^T u_k / sigma_k, pp_factors.cu).
//
// One CTA per slice holds Y in shared memory; vectors never move.  Step k:
// every warp reduces the per-warp candidates left by the previous update to
// the pivot (the unpivoted vector with the largest trailing norm, the lowest
// index on ties) and forms the scalars of its Householder reflector; all
// threads then apply the reflector to the unpivoted vectors, 4 lanes per
// vector, recompute their trailing norms from the updated entries (no norm
// downdating, hence no cancellation safeguard) and leave the next candidates.
// The unpivoted vectors stay packed in the lowest 4-lane groups (the group
// that held the pivot takes over the last group's vector), so the warps past
// them have nothing to issue.  One barrier per step; R is written at the end.
#include "pp_internal.h"

namespace pp {
namespace {

constexpr int QR_THREADS = 512;
constexpr int QG = 4;                        // lanes per vector in the update
constexpr int QR_SMEM_BUDGET = 200 * 1024;

// row stride of the vector store: a multiple of 4 floats (float4 access) that
// is 16 mod 32, so the 4-lane groups of a warp alternate between the two
// halves of the banks
__host__ __device__ inline int64_t qr_ap(int64_t a) { return (a + 31) / 32 * 32 + 16; }

__host__ __device__ inline int64_t qr_smem_floats(int64_t b, int64_t a) {
  return b * qr_ap(a) + 4 * b;               // vectors, diagonal, order, 2 group maps
}

constexpr int QR_NREG = 11;                  // float4 per lane held in registers in the update

// y -= f h on a float4; the squared entries above k join the trailing norm
// (four partial sums; masked only in the float4 that holds entry k)
__device__ __forceinline__ void qr_update4(float4 &v, const float4 h, float f, int e, int k,
                                           bool edge, float4 &s) {
  v.x = fmaf(-f, h.x, v.x);
  v.y = fmaf(-f, h.y, v.y);
  v.z = fmaf(-f, h.z, v.z);
  v.w = fmaf(-f, h.w, v.w);
  if (edge) {
    s.x = fmaf(e + 0 > k ? v.x : 0.f, v.x, s.x);
    s.y = fmaf(e + 1 > k ? v.y : 0.f, v.y, s.y);
    s.z = fmaf(e + 2 > k ? v.z : 0.f, v.z, s.z);
    s.w = fmaf(e + 3 > k ? v.w : 0.f, v.w, s.w);
  } else {
    s.x = fmaf(v.x, v.x, s.x);
    s.y = fmaf(v.y, v.y, s.y);
    s.z = fmaf(v.z, v.z, s.z);
    s.w = fmaf(v.w, v.w, s.w);
  }
}

// Warp-wide choice among (norm, vector) candidates: the largest norm, the lowest
// vector index on ties; lanes without a candidate pass j = QR_NONE.  Norms are
// >= 0, so their bit patterns order like the values.
constexpr unsigned QR_NONE = 0x7fffffffu;
__device__ __forceinline__ void warp_pivot(float v, unsigned j, unsigned &bv, unsigned &bj) {
  const unsigned bits = j == QR_NONE ? 0u : __float_as_uint(v);
  bv = __reduce_max_sync(0xffffffffu, bits);
  bj = __reduce_min_sync(0xffffffffu, (j != QR_NONE && bits == bv) ? j : QR_NONE);
}

// the reflector's float4 at e4: the pivot vector's entries, with 0 below k and
// vk at k (only the float4 holding entry k differs)
__device__ __forceinline__ float4 qr_h4(const float4 *p4, int e4, int k4, int k, float vk) {
  float4 h = p4[e4];
  if (e4 == k4) {
    const int e = 4 * e4;
    h.x = e + 0 < k ? 0.f : (e + 0 == k ? vk : h.x);
    h.y = e + 1 < k ? 0.f : (e + 1 == k ? vk : h.y);
    h.z = e + 2 < k ? 0.f : (e + 2 == k ? vk : h.z);
    h.w = e + 3 < k ? 0.f : (e + 3 == k ? vk : h.w);
  }
  return h;
}

// The reflector applied to one vector held in registers: NQ float4 per lane
// (the last one guarded), one read and one write of the vector; the squared
// entries above k accumulate in s4.  Instantiated for NQ = 1..QR_NREG so that
// late steps, whose vectors are short, issue only their live chunks.
template <int NQ>
__device__ __forceinline__ void qr_update_regs(float4 *y4, const float4 *p4, int k4, int k,
                                               float vk, float beta, int glane, unsigned gmask,
                                               int ap4, float4 &s4) {
  // only chunk 0 of lane 0 (e4 == k4) holds entries at or below k; every other
  // chunk starts at least 4 float4 past it and takes the plain path
  const bool edge = glane == 0;
  float4 r[NQ];
  float4 c4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int e4 = k4 + glane + QG * q;
    if (q < NQ - 1 || e4 < ap4) {
      r[q] = y4[e4];
      const float4 h = (q == 0 && edge) ? qr_h4(p4, e4, k4, k, vk) : p4[e4];
      c4.x = fmaf(h.x, r[q].x, c4.x);
      c4.y = fmaf(h.y, r[q].y, c4.y);
      c4.z = fmaf(h.z, r[q].z, c4.z);
      c4.w = fmaf(h.w, r[q].w, c4.w);
    }
  }
  float c = (c4.x + c4.y) + (c4.z + c4.w);
#pragma unroll
  for (int o = QG / 2; o > 0; o >>= 1) c += __shfl_xor_sync(gmask, c, o, QG);
  const float fct = beta * c;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int e4 = k4 + glane + QG * q;
    if (q < NQ - 1 || e4 < ap4) {
      if (q == 0 && edge)
        qr_update4(r[q], qr_h4(p4, e4, k4, k, vk), fct, 4 * e4, k, true, s4);
      else
        qr_update4(r[q], p4[e4], fct, 4 * e4, k, false, s4);
      y4[e4] = r[q];
    }
  }
}

__global__ void __launch_bounds__(QR_THREADS) qrcp_kernel(QrArgs A) {
  extern __shared__ __align__(16) float qs[];
  constexpr int NW = QR_THREADS / 32;
  __shared__ unsigned cand_v[2][NW], cand_j[2][NW];   // pivot candidates per warp, by step parity
  const int64_t f = blockIdx.x;
  const int l = (int)A.l, m = (int)A.m;
  const bool rows = l <= m;
  const int b = rows ? l : m, a = rows ? m : l;
  const int ap = (int)qr_ap(a);
  const int ap4 = (a + 3) / 4;   // float4 holding entries (the zero padding past them is skipped)
  float *Y = qs;                             // vector j (original index) at Y + j * ap
  float *diag = Y + (size_t)b * ap;          // R(k, k)
  int *order = reinterpret_cast<int *>(diag + b);  // pivoted position -> vector
  int *gmap = order + b;                     // [2][b]: group -> vector, by step parity
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int glane = tid % QG, grp = tid / QG, ngrp = QR_THREADS / QG;
  const unsigned gmask = ((1u << QG) - 1u) << (lane & ~(QG - 1));
  const float *Xf = A.X + f * (int64_t)l * m;

  if (rows) {
    for (int idx = tid; idx < b * ap; idx += QR_THREADS) {
      const int j = idx / ap, e = idx % ap;
      Y[idx] = e < a ? Xf[(int64_t)j * m + e] : 0.f;
    }
  } else {
    for (int idx = tid; idx < b * a; idx += QR_THREADS) {
      const int e = idx / b, j = idx % b;
      Y[(size_t)j * ap + e] = Xf[(int64_t)e * m + j];
    }
    for (int idx = tid; idx < b * (ap - a); idx += QR_THREADS)
      Y[(size_t)(idx / (ap - a)) * ap + a + idx % (ap - a)] = 0.f;
  }
  for (int j = tid; j < b; j += QR_THREADS) gmap[j] = j;
  __syncthreads();
  {
    float bestv = 0.f;
    unsigned bestj = QR_NONE;
    for (int j = grp; j < b; j += ngrp) {
      const float4 *y4 = reinterpret_cast<const float4 *>(Y + (size_t)j * ap);
      float4 s4 = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int e4 = glane; e4 < ap4; e4 += QG) {
        const float4 v = y4[e4];
        s4.x = fmaf(v.x, v.x, s4.x);
        s4.y = fmaf(v.y, v.y, s4.y);
        s4.z = fmaf(v.z, v.z, s4.z);
        s4.w = fmaf(v.w, v.w, s4.w);
      }
      float s = (s4.x + s4.y) + (s4.z + s4.w);
#pragma unroll
      for (int o = QG / 2; o > 0; o >>= 1) s += __shfl_xor_sync(gmask, s, o, QG);
      if (bestj == QR_NONE || s > bestv) { bestv = s; bestj = (unsigned)j; }
    }
    unsigned bv, bj;
    warp_pivot(bestv, bestj, bv, bj);
    if (lane == 0) { cand_v[0][warp] = bv; cand_j[0][warp] = bj; }
  }
  __syncthreads();

  // One barrier per step: every warp reduces the candidates left by the last
  // update (double-buffered by step parity) to the same pivot sp and computes
  // the reflector's scalars itself; the pivot vector is never written (its
  // entries above k are R's column, entry k becomes vk only inside qr_h4).
  for (int k = 0; k < b; ++k) {
    const int k4 = k / 4;
    const int par = k & 1;
    unsigned bv, bj;
    warp_pivot(lane < NW ? __uint_as_float(cand_v[par][lane]) : 0.f,
               lane < NW ? cand_j[par][lane] : QR_NONE, bv, bj);
    const int sp = bj < (unsigned)b ? (int)bj : 0;
    // Householder reflector H = I - beta v v^T with H y = alpha e_k:
    // alpha = -sign(y_k) |y|, v = y - alpha e_k, v^T v = 2 |y| (|y| + |y_k|),
    // |y|^2 = the pivot's trailing norm (entries k..a-1)
    const float4 *p4 = reinterpret_cast<const float4 *>(Y + (size_t)sp * ap);
    const float x0 = Y[(size_t)sp * ap + k];
    const float nx = sqrtf(__uint_as_float(bv));
    const float alpha = x0 >= 0.f ? -nx : nx;
    const float vk = x0 - alpha;
    const float vtv = 2.f * nx * (nx + fabsf(x0));
    const float beta = vtv > 0.f ? __fdividef(2.f, vtv) : 0.f;
    if (tid == 0) {
      diag[k] = alpha;
      order[k] = sp;
    }
    const bool in_regs = ap4 - k4 <= QG * QR_NREG;
    const int nq = (ap4 - k4 + QG - 1) / QG;
    float bestv = 0.f;
    unsigned bestj = QR_NONE;
    // b - k vectors were live at this step, the pivot among them; its group
    // takes the last group's vector and the remaining b - k - 1 stay packed
    const int nlive = b - k - 1;
    const int *gcur = gmap + par * b;
    int *gnext = gmap + (par ^ 1) * b;
    for (int g = grp; g < nlive; g += ngrp) {
      int j = gcur[g];
      if (j == sp) j = gcur[nlive];
      if (glane == 0) gnext[g] = j;
      float4 *y4 = reinterpret_cast<float4 *>(Y + (size_t)j * ap);
      float4 c4 = make_float4(0.f, 0.f, 0.f, 0.f), s4 = c4;
      if (in_regs) {                           // one read and one write of the vector
        switch (nq) {                          // live float4 per lane, uniform in the CTA
#define QR_CASE(NQ) \
  case NQ:          \
    qr_update_regs<NQ>(y4, p4, k4, k, vk, beta, glane, gmask, ap4, s4); \
    break;
          QR_CASE(1) QR_CASE(2) QR_CASE(3) QR_CASE(4) QR_CASE(5) QR_CASE(6)
          QR_CASE(7) QR_CASE(8) QR_CASE(9) QR_CASE(10) QR_CASE(11)
#undef QR_CASE
          default: break;
        }
      } else {                                 // long vectors: a read pass, then read-write
        for (int e4 = k4 + glane; e4 < ap4; e4 += QG) {
          const float4 h = qr_h4(p4, e4, k4, k, vk), v = y4[e4];
          c4.x = fmaf(h.x, v.x, c4.x);
          c4.y = fmaf(h.y, v.y, c4.y);
          c4.z = fmaf(h.z, v.z, c4.z);
          c4.w = fmaf(h.w, v.w, c4.w);
        }
        float c = (c4.x + c4.y) + (c4.z + c4.w);
#pragma unroll
        for (int o = QG / 2; o > 0; o >>= 1) c += __shfl_xor_sync(gmask, c, o, QG);
        const float fct = beta * c;
        for (int e4 = k4 + glane; e4 < ap4; e4 += QG) {
          float4 v = y4[e4];
          qr_update4(v, qr_h4(p4, e4, k4, k, vk), fct, 4 * e4, k, e4 == k4, s4);
          y4[e4] = v;
        }
      }
      float s = (s4.x + s4.y) + (s4.z + s4.w);
#pragma unroll
      for (int o = QG / 2; o > 0; o >>= 1) s += __shfl_xor_sync(gmask, s, o, QG);
      if (bestj == QR_NONE || s > bestv || (s == bestv && (unsigned)j < bestj)) {
        bestv = s;
        bestj = (unsigned)j;
      }
    }
    warp_pivot(bestv, bestj, bv, bj);
    if (lane == 0) { cand_v[par ^ 1][warp] = bv; cand_j[par ^ 1][warp] = bj; }
    __syncthreads();
  }
  // R(i, j) for j > i: entry i of the vector at pivoted position j (final
  // after step i); the diagonal from diag
  float *Rf = A.R + f * (int64_t)b * b;
  for (int idx = tid; idx < b * b; idx += QR_THREADS) {
    const int i = idx / b, j = idx % b;
    Rf[idx] = j < i ? 0.f : (j == i ? diag[j] : Y[(size_t)order[j] * ap + i]);
  }
  for (int j = tid; j < b; j += QR_THREADS) A.qperm[f * b + j] = order[j];
}

// ---------------------------------------------------------------------------
// Register-resident variant for slices of at most QR_REG_MAXB vectors of at
// most 4 * 4 * QR_REG_NCH entries (the video-shaped 120 x 160 slices): a 4-lane
// group keeps one vector in registers, lane glane holding float4 chunks
// glane, glane + 4, ... of it, so the rank-1 updates touch no shared memory.
// After each step every warp publishes only its pivot candidate (the vector,
// its trailing norm, its index and its group) in a parity-buffered slot; the
// next step reads the reflector from the winning slot and writes R's column k
// from it.  The unpivoted vectors stay packed in the lowest groups: when the
// pivot's group is not the last live one, the last live group hands its
// updated vector to the pivot's group through a parity-buffered slot, taken up
// at the next step.  Same pivot rule, reflector and norms as qrcp_kernel (the
// chunks are split over the lanes differently, so sums round in another order).
constexpr int QR_REG_MAXB = QR_THREADS / QG;    // one vector per group
constexpr int QR_REG_NCH = 11;                  // float4 chunks per lane, at most
constexpr int QR_REG_A4 = QG * QR_REG_NCH;      // float4 per vector (<= 176 entries)

__host__ __device__ inline int64_t qr_reg_smem_bytes(int64_t b, int64_t a) {
  // candidate slots [2][NW] and hand-over slots [2], then staging / R, diag, order
  return (int64_t)sizeof(float4) * (2 * (QR_THREADS / 32) + 2) * QR_REG_A4 +
         (int64_t)sizeof(float) * (b * qr_ap(a) + 2 * b);
}

// one Householder update of the register-resident vector v (NCH chunks per
// lane) from the chunk that holds entry k on (Q0 = k4 / 4)
template <int NCH, int Q0>
__device__ __forceinline__ void qr_reg_update(float4 (&v)[NCH], const float4 *p4, int k4, int k,
                                              float vk, float beta, int glane, unsigned gmask,
                                              int a4, float4 &s4) {
  float4 c4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int q = Q0; q < NCH; ++q) {
    const int e4 = glane + QG * q;
    if ((q > Q0 || e4 >= k4) && (q < NCH - 1 || e4 < a4)) {
      const float4 h = q == Q0 ? qr_h4(p4, e4, k4, k, vk) : p4[e4];
      c4.x = fmaf(h.x, v[q].x, c4.x);
      c4.y = fmaf(h.y, v[q].y, c4.y);
      c4.z = fmaf(h.z, v[q].z, c4.z);
      c4.w = fmaf(h.w, v[q].w, c4.w);
    }
  }
  float c = (c4.x + c4.y) + (c4.z + c4.w);
#pragma unroll
  for (int o = QG / 2; o > 0; o >>= 1) c += __shfl_xor_sync(gmask, c, o, QG);
  const float fct = beta * c;
#pragma unroll
  for (int q = Q0; q < NCH; ++q) {
    const int e4 = glane + QG * q;
    if ((q > Q0 || e4 >= k4) && (q < NCH - 1 || e4 < a4)) {
      if (q == Q0)
        qr_update4(v[q], qr_h4(p4, e4, k4, k, vk), fct, 4 * e4, k, e4 == k4, s4);
      else
        qr_update4(v[q], p4[e4], fct, 4 * e4, k, false, s4);
    }
  }
}

template <int NCH>
__device__ __forceinline__ void qr_reg_store(float4 *dst, const float4 (&v)[NCH], int glane,
                                             int a4) {
#pragma unroll
  for (int q = 0; q < NCH; ++q) {
    const int e4 = glane + QG * q;
    if (q < NCH - 1 || e4 < a4) dst[e4] = v[q];
  }
}

template <int NCH>
__device__ __forceinline__ void qr_reg_load(float4 (&v)[NCH], const float4 *src, int glane,
                                            int a4) {
#pragma unroll
  for (int q = 0; q < NCH; ++q) {
    const int e4 = glane + QG * q;
    v[q] = (q < NCH - 1 || e4 < a4) ? src[e4] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// NCH = float4 chunks per lane: a4 = ceil(a / 4) <= 4 * NCH
template <int NCH>
__global__ void __launch_bounds__(QR_THREADS) qrcp_reg_kernel(QrArgs A) {
  extern __shared__ __align__(16) float qs[];
  constexpr int NW = QR_THREADS / 32;
  // candidates: trailing norm and key = vector << 8 | group that published it
  // (the smallest key among equal norms is the lowest vector index)
  __shared__ unsigned cand_v[2][NW], cand_j[2][NW];
  __shared__ int move_j[2];
  const int64_t f = blockIdx.x;
  const int l = (int)A.l, m = (int)A.m;
  const bool rows = l <= m;
  const int b = rows ? l : m, a = rows ? m : l;
  const int ap = (int)qr_ap(a);
  const int a4 = (a + 3) / 4;
  float4 *cvec = reinterpret_cast<float4 *>(qs);        // [2][NW][QR_REG_A4] candidates
  float4 *mvec = cvec + 2 * NW * QR_REG_A4;             // [2][QR_REG_A4] hand-over
  float *Y = reinterpret_cast<float *>(mvec + 2 * QR_REG_A4);   // staging b x ap, then R b x b
  float *diag = Y + (size_t)b * ap;
  int *order = reinterpret_cast<int *>(diag + b);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int glane = tid % QG, g = tid / QG;
  const unsigned gmask = ((1u << QG) - 1u) << (lane & ~(QG - 1));
  const float *Xf = A.X + f * (int64_t)l * m;

  if (rows) {
    for (int idx = tid; idx < b * ap; idx += QR_THREADS) {
      const int j = idx / ap, e = idx % ap;
      Y[idx] = e < a ? Xf[(int64_t)j * m + e] : 0.f;
    }
  } else {
    for (int idx = tid; idx < b * a; idx += QR_THREADS) {
      const int e = idx / b, j = idx % b;
      Y[(size_t)j * ap + e] = Xf[(int64_t)e * m + j];
    }
    for (int idx = tid; idx < b * (ap - a); idx += QR_THREADS)
      Y[(size_t)(idx / (ap - a)) * ap + a + idx % (ap - a)] = 0.f;
  }
  __syncthreads();
  int myj = g;                        // vector held by this group
  float4 v[NCH];
  {
    const bool live = g < b;
    qr_reg_load<NCH>(v, reinterpret_cast<const float4 *>(Y + (size_t)(live ? g : 0) * ap), glane,
                     a4);
    float4 s4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int q = 0; q < NCH; ++q) {
      s4.x = fmaf(v[q].x, v[q].x, s4.x);
      s4.y = fmaf(v[q].y, v[q].y, s4.y);
      s4.z = fmaf(v[q].z, v[q].z, s4.z);
      s4.w = fmaf(v[q].w, v[q].w, s4.w);
    }
    float s = (s4.x + s4.y) + (s4.z + s4.w);
#pragma unroll
    for (int o = QG / 2; o > 0; o >>= 1) s += __shfl_xor_sync(gmask, s, o, QG);
    unsigned bv, bj;
    const unsigned key = ((unsigned)g << 8) | (unsigned)g;   // group == vector before any hand-over
    warp_pivot(s, live ? key : QR_NONE, bv, bj);
    if (live && key == bj) qr_reg_store<NCH>(cvec + (size_t)warp * QR_REG_A4, v, glane, a4);
    if (lane == 0) {
      cand_v[0][warp] = bv;
      cand_j[0][warp] = bj;
    }
  }
  __syncthreads();

  int gs_prev = -1, gl_prev = -1;     // last step's pivot group and hand-over source
  for (int k = 0; k < b; ++k) {
    const int k4 = k / 4;
    const int par = k & 1;
    // take up the vector handed over at the previous step
    if (gs_prev >= 0 && g == gs_prev) {
      qr_reg_load<NCH>(v, mvec + (size_t)par * QR_REG_A4, glane, a4);
      myj = move_j[par];
    }
    const bool has = lane < NW;
    const unsigned cj = has ? cand_j[par][lane] : QR_NONE;
    unsigned bv, bj;
    warp_pivot(has ? __uint_as_float(cand_v[par][lane]) : 0.f, cj, bv, bj);
    const bool found = bj != QR_NONE;
    const int sp = found ? (int)(bj >> 8) : 0;
    int gs = found ? (int)(bj & 255u) : 0;   // group that published the pivot ...
    const int wi = gs / (32 / QG);           // (its warp's candidate slot)
    if (gs == gl_prev) gs = gs_prev;         // ... unless it has handed it over since
    const float4 *p4 = cvec + ((size_t)par * NW + wi) * QR_REG_A4;
    const float *pf = reinterpret_cast<const float *>(p4);
    const float x0 = pf[k];
    const float nx = sqrtf(__uint_as_float(bv));
    const float alpha = x0 >= 0.f ? -nx : nx;
    const float vk = x0 - alpha;
    const float vtv = 2.f * nx * (nx + fabsf(x0));
    const float beta = vtv > 0.f ? __fdividef(2.f, vtv) : 0.f;
    if (tid == 0) {
      diag[k] = alpha;
      order[k] = sp;
    }
    for (int e = tid; e < k; e += QR_THREADS) Y[(size_t)e * b + k] = pf[e];   // R(e, k)
    // groups 0 .. b-k-1 hold the b-k unpivoted vectors; the pivot's is done
    const bool live = g < b - k && g != gs;
    float4 s4 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (live) {
      switch (k4 / QG) {                      // uniform in the CTA
#define QR_RCASE(Q0)                                                              \
  case Q0:                                                                        \
    if (Q0 < NCH) qr_reg_update<NCH, (Q0 < NCH ? Q0 : 0)>(v, p4, k4, k, vk, beta, \
                                                          glane, gmask, a4, s4);  \
    break;
        QR_RCASE(0) QR_RCASE(1) QR_RCASE(2) QR_RCASE(3) QR_RCASE(4) QR_RCASE(5)
        QR_RCASE(6) QR_RCASE(7)
#undef QR_RCASE
        default: break;
      }
    }
    float s = (s4.x + s4.y) + (s4.z + s4.w);
#pragma unroll
    for (int o = QG / 2; o > 0; o >>= 1) s += __shfl_xor_sync(gmask, s, o, QG);
    const unsigned mykey = ((unsigned)myj << 8) | (unsigned)g;
    warp_pivot(s, live ? mykey : QR_NONE, bv, bj);
    if (live && mykey == bj)
      qr_reg_store<NCH>(cvec + ((size_t)(par ^ 1) * NW + warp) * QR_REG_A4, v, glane, a4);
    if (lane == 0) {
      cand_v[par ^ 1][warp] = bv;
      cand_j[par ^ 1][warp] = bj;
    }
    // hand the last live group's vector to the pivot's group
    const int gl = b - k - 1;
    if (gl != gs && g == gl) {
      qr_reg_store<NCH>(mvec + (size_t)(par ^ 1) * QR_REG_A4, v, glane, a4);
      if (glane == 0) move_j[par ^ 1] = myj;
    }
    gs_prev = gl != gs ? gs : -1;
    gl_prev = gl != gs ? gl : -1;
    __syncthreads();
  }
  float *Rf = A.R + f * (int64_t)b * b;
  for (int idx = tid; idx < b * b; idx += QR_THREADS) {
    const int i = idx / b, j = idx % b;
    Rf[idx] = j < i ? 0.f : (j == i ? diag[j] : Y[idx]);
  }
  for (int j = tid; j < b; j += QR_THREADS) A.qperm[f * b + j] = order[j];
}

}  // namespace

bool qrcp_fits(int64_t l, int64_t m) {
  const int64_t b = l < m ? l : m, a = l < m ? m : l;
  return b >= 2 && (int64_t)sizeof(float) * qr_smem_floats(b, a) <= QR_SMEM_BUDGET;
}

cudaError_t launch_qrcp(const QrArgs &A, cudaStream_t st) {
  const int64_t b = A.l < A.m ? A.l : A.m, a = A.l < A.m ? A.m : A.l;
  const int64_t nch = ((a + 3) / 4 + QG - 1) / QG;   // float4 chunks per lane
  if (b <= QR_REG_MAXB && nch <= QR_REG_NCH) {
    const size_t rsmem = (size_t)qr_reg_smem_bytes(b, a);
    auto kern = nch <= 4 ? qrcp_reg_kernel<4>
              : nch <= 6 ? qrcp_reg_kernel<6>
              : nch <= 8 ? qrcp_reg_kernel<8>
              : nch <= 10 ? qrcp_reg_kernel<10> : qrcp_reg_kernel<11>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)rsmem);
    if (e != cudaSuccess) return e;
    count_launch(1);
    kern<<<(unsigned)A.p, QR_THREADS, rsmem, st>>>(A);
    return cudaGetLastError();
  }
  const size_t smem = sizeof(float) * (size_t)qr_smem_floats(b, a);
  cudaError_t e = cudaFuncSetAttribute(qrcp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  count_launch(1);
  qrcp_kernel<<<(unsigned)A.p, QR_THREADS, smem, st>>>(A);
  return cudaGetLastError();
}

}  // namespace pp
