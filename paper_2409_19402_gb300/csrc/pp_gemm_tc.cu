// pp_gemm_tc.cu -- the mode-3 product (Def. 2.2) on the 5th-generation tensor
// cores: Y (P x N) = M (P x S) * X (S x N) over the mode-3 unfolding, N = l*m
// pixels.  This is the transform A x_3 Q^T of Alg. 4.1 step 2 and the reverse
// transform x_3 Q of step 4.
//
// Tile: one CTA computes 128 pixels x NT = 64 output slices as
// D[128 x NT] = X^T[128 x S] * M^T[S x NT] with tcgen05.mma kind::tf32, the
// accumulator in tensor memory (TMEM).  FP32 accuracy is recovered with the
// 3-pass split: every operand is written as hi = tf32(x) and lo = tf32(x - hi)
// and the MMA accumulates hi*hi + hi*lo + lo*hi (the dropped lo*lo term and
// the rounding of lo are below 2^-22 of each product).  The tensor core's own
// accumulation is not round-to-nearest, and its error grows with the
// magnitude of the accumulator; so each 32-wide chunk of S is accumulated
// from zero in one of two TMEM buffers, and the chunk sums are added in FP32
// registers (round to nearest) while the next chunk's MMAs run.
//
// Operands: the tensor is pixel-contiguous, i.e. MN-major for this product,
// and M is tiny; both are streamed in chunks of 32 along S and written into
// shared memory in the K-major,
// 128-byte-swizzled canonical layout (row = pixel or slice, 32 tf32 = 128 bytes per row, 8-row
// atoms of 1024 bytes, 16-byte chunk index XOR (row mod 8)).  The tensor's
// chunks arrive either through the threads' registers (each thread's values
// for chunk c + 1 are requested while chunk c is written and issued; each load
// of a warp covers 32 consecutive pixels), or, for longer contractions whose
// rows are 16-byte aligned, by TMA: 32 x 128 FP32 boxes of the S x N matrix
// into a ring of TMA_STAGES raw stages, so that several chunks are in flight
// per SM (out-of-range rows and pixels read as zero); the threads then convert
// from shared memory.  Two
// stages: while the MMAs of chunk c run, the threads fill chunk c+1; a stage
// is refilled only after the tcgen05.commit of its previous MMAs has arrived
// on that stage's mbarrier.  Every mbarrier wait is bounded; on expiry the
// kernel records PP_ETIMEOUT, releases its TMEM and returns.
//
// 256 threads: threads r and r + 128 share pixel row r (each converts half of
// the chunk's 32 values) and, in the epilogue, half of the 64 output columns
// of TMEM lane r (tcgen05.ld), which they store as coalesced 128-byte rows of
// Y, fusing the optional sums |Aref - Y|^2, |Y|^2 and |X|^2 (FP32 over a few
// terms, FP64 beyond).
#include <cuda.h>

#include <cstring>

#include "pp_internal.h"
#include "pp_tc.cuh"
#include "pp_tma.h"

namespace pp {
namespace {

using namespace tc;

constexpr int TM = 128;        // pixels per CTA (MMA M)
constexpr int TK = 32;         // S per stage: one 128-byte swizzle row of tf32
constexpr int THREADS = 256;   // two threads per pixel row (halves of K and of the columns)
constexpr int TMA_STAGES = 4;                     // raw FP32 chunks in flight (TMA path)
constexpr int RAW_BYTES = TK * TM * 4;            // one 32 x 128 FP32 box

// one 2-D box of the tensor map at (x = pixel, y = S row) into shared memory,
// completing `bytes` on the mbarrier
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mbar)
      : "memory");
}

constexpr int NT = 64;   // output slices per CTA (MMA N)

// Batch and layout of a product launch: member z reads M at Qm + z sMz and X at
// X + z sXz, X(s, n) = X[s sxc + n sxn], and writes Y + z sYz; s_total > 0
// marks a split of one contraction of s_total terms into members of S terms.
struct BatchStrides {
  int64_t sMz = 0, sXz = 0, sYz = 0;
  int64_t sxc = 0, sxn = 1;
  int64_t s_total = 0;
  // contraction-contiguous operands with 16-byte aligned rows: a thread's 16
  // consecutive terms come in as four 16-byte loads (register path)
  int vec_x = 0, vec_m = 0;
  // rz > 0 (register path): grid member z sums the products of members
  // z rz ... min(nmem, (z + 1) rz) - 1 (operands sMz, sXz apart) into one
  // output at Y + z sYz, chunk by chunk, in member order
  int64_t rz = 0, nmem = 0;
};

// X(c, n) = X[c + n sxn] (sxc = 1) with every member's rows 16-byte aligned
bool vec_rows(const float *base, int64_t stride, int64_t member_stride) {
  return (reinterpret_cast<uintptr_t>(base) & 15) == 0 && stride % 4 == 0 &&
         member_stride % 4 == 0;
}

// warp w adds columns [32 (w / 4), 32 (w / 4) + 32) of TMEM lanes 32 (w % 4) ... + 31 of
// buffer `buf` (chunk partial sums) into acc[] (one TMEM lane per thread)
__device__ __forceinline__ void tmem_accumulate(uint32_t tmem, int buf, int warp, float *acc) {
#pragma unroll
  for (int j0 = 0; j0 < NT / 2; j0 += 16) {
    uint32_t r[16];
    const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) +
                           (uint32_t)(buf * NT + (warp >> 2) * (NT / 2) + j0);
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[j0 + q] += __uint_as_float(r[q]);
  }
}

// TMA: chunks of X arrive by TMA through `tmap` (X's S x N matrix), else
// through the threads' registers
template <bool TMA>
__global__ void __launch_bounds__(THREADS, TMA ? 1 : 2) mode3_tc_kernel(
    const __grid_constant__ CUtensorMap tmap, const float *__restrict__ Qm, int64_t sr,
    int64_t sc, const float *__restrict__ X,
    float *__restrict__ Y, int64_t P, int64_t S, int64_t N, const BatchStrides bz,
    const float *__restrict__ Aref,
    double *__restrict__ errp, double *__restrict__ xpart, double *__restrict__ ypart,
    int32_t *status) {
  // stage layout (bytes): A_hi 16K | A_lo 16K | B_hi 8K | B_lo 8K
  constexpr int A_BYTES = TM * 128, B_BYTES = NT * 128;
  constexpr int STAGE = 2 * A_BYTES + 2 * B_BYTES;
  constexpr int TMEM_COLS = 2 * NT;   // two chunk accumulators
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // the 1024-byte aligned base, offset from smem_raw itself so that the
  // compiler still sees shared-memory accesses (not generic ones) through it
  unsigned char *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ __align__(8) uint64_t full[TMA_STAGES];   // TMA path: raw stage filled
  __shared__ uint32_t tmem_base_sh;
  __shared__ double red[THREADS / 32];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // batch member z (blockIdx.z): its operands and output; split-K members
  // (s_total > 0) each take S of the s_total contraction terms, the last fewer
  int nm = 1;   // members summed by this CTA
  {
    const int64_t z = blockIdx.z;
    const int64_t m0 = bz.rz > 0 ? z * bz.rz : z;
    Qm += m0 * bz.sMz;
    X += m0 * bz.sXz;
    if (Y) Y += z * bz.sYz;
    if (bz.s_total > 0) {
      const int64_t rem = bz.s_total - z * S;
      S = rem < S ? rem : S;
    }
    if (bz.rz > 0) {
      const int64_t left = bz.nmem - m0;
      nm = (int)(left < bz.rz ? left : bz.rz);
    }
  }
  const int64_t sxc = bz.sxc, sxn = bz.sxn;
  const int64_t n0 = (int64_t)blockIdx.x * TM;
  const int64_t y0 = (int64_t)blockIdx.y * NT;
  const bool do_x = xpart != nullptr && blockIdx.y == 0;
  constexpr uint32_t IDESC = tf32_idesc(TM, NT);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_sh)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
    if (TMA)
      for (int i = 0; i < TMA_STAGES; ++i)
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[i])));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base_sh;

  float acc[NT / 2];
#pragma unroll
  for (int j = 0; j < NT / 2; ++j) acc[j] = 0.f;
  const int row = tid & (TM - 1);          // pixel row / slice row owned by this thread
  const int khalf = tid >> 7;              // which 16 of the 32 K values (0 or 1)
  const int nch = (int)((S + TK - 1) / TK);   // chunks per member
  const int nchunks = nm * nch;
  double xs = 0.0;
  bool ok = true;
  // TMA path: raw FP32 stages after the two converted stages; chunk c goes to
  // raw stage c % TMA_STAGES, and is refilled with chunk c + TMA_STAGES once
  // every thread has converted it (the barrier before the MMA issue)
  unsigned char *raw = smem + 2 * STAGE;
  int issued = 0;                          // TMA boxes issued (thread 0)
  auto tma_issue = [&](int c) {
    const int rs = c % TMA_STAGES;
    const uint32_t fb = smem_u32(&full[rs]);
    mbar_expect_tx(fb, (uint32_t)RAW_BYTES);
    tma_load_2d(smem_u32(raw + rs * RAW_BYTES), &tmap, (int)n0, c * TK, fb);
    ++issued;
  };
  if (TMA && tid == 0) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap)) : "memory");
    for (int c = 0; c < nchunks && c < TMA_STAGES; ++c) tma_issue(c);
  }
  // chunk c's operands are loaded into registers one iteration ahead, so the
  // global-memory latency overlaps the previous chunk's barrier and MMA issue
  const int64_t pix = n0 + row;
  const int64_t trow = y0 + row;
  const float *const X_ = X, *const Qm_ = Qm;
  float va[TK / 2], vb[TK / 2];
  auto load_chunk = [&](int cc) {
    // chunk cc: chunk c of member mem (one member unless the CTA sums several)
    const int mem = nm > 1 ? cc / nch : 0;
    const int c = nm > 1 ? cc % nch : cc;
    const float *X = X_ + mem * bz.sXz;
    const float *Qm = Qm_ + mem * bz.sMz;
    const int64_t s0 = (int64_t)c * TK;
    const int64_t sk = s0 + khalf * (TK / 2);   // this thread's first term of the chunk
    if (!TMA) {
      if (bz.vec_x && pix < N && sk + TK / 2 <= S) {
        const float4 *p4 = reinterpret_cast<const float4 *>(X + pix * sxn + sk);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 t = p4[q];
          va[4 * q] = t.x; va[4 * q + 1] = t.y; va[4 * q + 2] = t.z; va[4 * q + 3] = t.w;
        }
      } else {
#pragma unroll
        for (int k = 0; k < TK / 2; ++k) {
          const int64_t s = sk + k;
          va[k] = (pix < N && s < S) ? X[s * sxc + pix * sxn] : 0.f;
        }
      }
    }
    if (bz.vec_m && row < NT && trow < P && sk + TK / 2 <= S) {
      const float4 *p4 = reinterpret_cast<const float4 *>(Qm + trow * sr + sk);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 t = p4[q];
        vb[4 * q] = t.x; vb[4 * q + 1] = t.y; vb[4 * q + 2] = t.z; vb[4 * q + 3] = t.w;
      }
    } else {
#pragma unroll
      for (int k = 0; k < TK / 2; ++k) {
        const int64_t s = sk + k;
        vb[k] = (row < NT && trow < P && s < S) ? Qm[trow * sr + s * sc] : 0.f;
      }
    }
  };
  if (nchunks > 0) load_chunk(0);
  for (int c = 0; c < nchunks; ++c) {
    const int st = c & 1;   // smem stage and TMEM buffer
    unsigned char *base = smem + st * STAGE;
    if (c >= 2) {   // chunk c-2 (same stage and buffer) must be complete: add its sums
      if (!mbar_wait(smem_u32(&mbar[st]), (uint32_t)(((c - 2) >> 1) & 1))) ok = false;
      if (__syncthreads_or(!ok)) { ok = false; break; }
      asm volatile("tcgen05.fence::after_thread_sync;");
      tmem_accumulate(tmem, st, warp, acc);
    }
    if (TMA) {   // this chunk's raw stage: row s of the box is 128 pixels
      const int rs = c % TMA_STAGES;
      if (!mbar_wait(smem_u32(&full[rs]), (uint32_t)((c / TMA_STAGES) & 1))) ok = false;
      if (__syncthreads_or(!ok)) { ok = false; break; }
      const float *rp = reinterpret_cast<const float *>(raw + rs * RAW_BYTES);
#pragma unroll
      for (int k = 0; k < TK / 2; ++k) va[k] = rp[(khalf * (TK / 2) + k) * TM + row];
    }
    // ---- A: pixel row `row`, 16 values along S (this thread's half of the chunk)
    {
      unsigned char *ah = base, *al = base + A_BYTES;
      float xq = 0.f;
#pragma unroll
      for (int c4 = 0; c4 < 4; ++c4) {
        const int ch = khalf * 4 + c4;
        float4 h, l;
        h.x = tf32_rna(va[4 * c4 + 0]); l.x = tf32_rna(va[4 * c4 + 0] - h.x);
        h.y = tf32_rna(va[4 * c4 + 1]); l.y = tf32_rna(va[4 * c4 + 1] - h.y);
        h.z = tf32_rna(va[4 * c4 + 2]); l.z = tf32_rna(va[4 * c4 + 2] - h.z);
        h.w = tf32_rna(va[4 * c4 + 3]); l.w = tf32_rna(va[4 * c4 + 3] - h.w);
        const uint32_t off = sw128_chunk(row, ch);
        *reinterpret_cast<float4 *>(ah + off) = h;
        *reinterpret_cast<float4 *>(al + off) = l;
        xq = fmaf(va[4 * c4], va[4 * c4], fmaf(va[4 * c4 + 1], va[4 * c4 + 1],
             fmaf(va[4 * c4 + 2], va[4 * c4 + 2], fmaf(va[4 * c4 + 3], va[4 * c4 + 3], xq))));
      }
      if (do_x) xs += (double)xq;   // FP32 over 16 values, FP64 across chunks
    }
    // ---- B: output-slice row `row` (< NT), 16 values along S: M(y0 + row, s0 + k)
    if (row < NT) {
      unsigned char *bh = base + 2 * A_BYTES, *bl = bh + B_BYTES;
#pragma unroll
      for (int c4 = 0; c4 < 4; ++c4) {
        const int ch = khalf * 4 + c4;
        float4 h, l;
        h.x = tf32_rna(vb[4 * c4 + 0]); l.x = tf32_rna(vb[4 * c4 + 0] - h.x);
        h.y = tf32_rna(vb[4 * c4 + 1]); l.y = tf32_rna(vb[4 * c4 + 1] - h.y);
        h.z = tf32_rna(vb[4 * c4 + 2]); l.z = tf32_rna(vb[4 * c4 + 2] - h.z);
        h.w = tf32_rna(vb[4 * c4 + 3]); l.w = tf32_rna(vb[4 * c4 + 3] - h.w);
        const uint32_t off = sw128_chunk(row, ch);
        *reinterpret_cast<float4 *>(bh + off) = h;
        *reinterpret_cast<float4 *>(bl + off) = l;
      }
    }
    if (c + 1 < nchunks) load_chunk(c + 1);   // next chunk's loads in flight
    // generic-proxy writes -> visible to the tensor core (async proxy); the
    // TMEM reads above are ordered before the MMAs that overwrite the buffer
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t a_hi = smem_u32(base), a_lo = a_hi + A_BYTES;
      const uint32_t b_hi = a_hi + 2 * A_BYTES, b_lo = b_hi + B_BYTES;
      const uint32_t d = tmem + (uint32_t)(st * NT);
      // the descriptors' address field is (address >> 4) and every address here
      // is below 256 KB, so a K step of 32 bytes adds 2 to each descriptor
      const uint64_t dah = sw128_desc(a_hi), dal = sw128_desc(a_lo);
      const uint64_t dbh = sw128_desc(b_hi), dbl = sw128_desc(b_lo);
#pragma unroll
      for (int kk = 0; kk < TK / 8; ++kk) {   // 8 tf32 = 32 bytes of K per MMA
        const uint64_t o = 2u * (uint32_t)kk;
        mma_tf32(d, dal + o, dbh + o, IDESC, kk > 0 ? 1u : 0u);
        mma_tf32(d, dah + o, dbl + o, IDESC, 1u);
        mma_tf32(d, dah + o, dbh + o, IDESC, 1u);
      }
      mma_commit(smem_u32(&mbar[st]));
      if (TMA && c + TMA_STAGES < nchunks) tma_issue(c + TMA_STAGES);
    }
  }
  // TMA path: on an early exit, let the boxes in flight land before the CTA
  // (and its shared memory) goes away; every wait is bounded
  if (TMA && tid == 0 && !ok) {
    for (int c = 0; c < issued; ++c) {
      // boxes below the failed chunk were consumed; the rest are waited here
      if (!mbar_try(smem_u32(&full[c % TMA_STAGES]), (uint32_t)((c / TMA_STAGES) & 1)))
        (void)mbar_wait(smem_u32(&full[c % TMA_STAGES]), (uint32_t)((c / TMA_STAGES) & 1));
    }
  }
  // the last two chunks
  for (int c = (nchunks >= 2 ? nchunks - 2 : 0); ok && c < nchunks; ++c) {
    const int st = c & 1;
    if (!mbar_wait(smem_u32(&mbar[st]), (uint32_t)((c >> 1) & 1))) ok = false;
    if (__syncthreads_or(!ok)) { ok = false; break; }
    asm volatile("tcgen05.fence::after_thread_sync;");
    tmem_accumulate(tmem, st, warp, acc);
  }
  ok = __syncthreads_and(ok);

  double err = 0.0, ys = 0.0;
  if (ok) {
    const int64_t pix = n0 + (warp & 3) * 32 + lane;       // TMEM lane of this thread
    const int64_t c0 = y0 + (warp >> 2) * (NT / 2);        // first of its 32 columns
    if (pix < N) {
#pragma unroll
      for (int g = 0; g < NT / 2; g += 8) {     // FP32 over 8 values, FP64 across groups
        float e8 = 0.f, y8 = 0.f;
#pragma unroll
        for (int q = g; q < g + 8; ++q) {
          const int64_t t = c0 + q;
          if (t < P) {
            const float v = acc[q];
            if (Y) Y[t * N + pix] = v;
            y8 = fmaf(v, v, y8);
            if (Aref) {
              const float d = Aref[t * N + pix] - v;
              e8 = fmaf(d, d, e8);
            }
          }
        }
        ys += (double)y8;
        err += (double)e8;
      }
    }
  } else if (tid == 0 && status) {
    atomicCAS(status, 0, PP_ETIMEOUT);
  }
  // reductions (fixed order) of the fused sums
  auto block_sum = [&](double v) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (tid == 0)
      for (int w = 0; w < THREADS / 32; ++w) s += red[w];
    __syncthreads();
    return s;
  };
  const int64_t cta = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
  if (Aref) {
    const double s = block_sum(err);
    if (tid == 0) errp[cta] = s;
  }
  if (ypart) {
    const double s = block_sum(ys);
    if (tid == 0) ypart[cta] = s;
  }
  if (do_x) {
    const double s = block_sum(xs);
    if (tid == 0) xpart[blockIdx.x] = s;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS));
  }
}

size_t tc_smem(bool tma) {
  // 2 converted stages (+ the TMA ring) + alignment slack
  return (size_t)2 * (2 * TM * 128 + 2 * NT * 128) + (tma ? (size_t)TMA_STAGES * RAW_BYTES : 0) +
         1024;
}

// The S x N FP32 matrix X as a TMA map with 32 x 128 boxes; false when X's
// rows are not 16-byte aligned or the driver refuses
bool make_x_map(const float *X, int64_t S, int64_t N, CUtensorMap *map) {
  return encode_rows_2d(map, X, N, S, (uint32_t)TM, (uint32_t)TK, true);
}

}  // namespace

int64_t mode3_tc_partials(int64_t P, int64_t N) {
  // this kernel: one per CTA tile; the warp-specialised one: four per unit
  // (errp, ypart) and eight per pixel tile (xpart)
  return ((N + TM - 1) / TM) * ((P + NT - 1) / NT) * 8;
}

cudaError_t launch_mode3_tc(const float *Qm, int64_t sr, int64_t sc, const float *X, float *Y,
                            int64_t P, int64_t S, int64_t N, const float *Aref, double *errp,
                            int *n_partials, double *xpart, int *n_xpart, double *ypart,
                            int32_t *status, cudaStream_t st, void *img, size_t img_bytes,
                            bool *img_ready) {
  if (img) {
    bool used = false;
    cudaError_t e = launch_mode3_ws(Qm, sr, sc, X, Y, P, S, N, Aref, errp, n_partials, xpart,
                                    n_xpart, ypart, status, img, img_bytes, st, &used, img_ready);
    if (used || e != cudaSuccess) return e;
  }
  if (n_partials) *n_partials = (int)(((N + TM - 1) / TM) * ((P + NT - 1) / NT));
  if (n_xpart) *n_xpart = (int)((N + TM - 1) / TM);
  // TMA for contractions of more than two chunks (two CTAs per SM otherwise)
  CUtensorMap map;
  std::memset(&map, 0, sizeof(map));
  const bool tma = S > 2 * TK && make_x_map(X, S, N, &map);
  const size_t smem = tc_smem(tma);
  auto kern = tma ? mode3_tc_kernel<true> : mode3_tc_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)((N + TM - 1) / TM), (unsigned)((P + NT - 1) / NT), 1);
  BatchStrides bz;
  bz.sxc = N;
  bz.vec_m = sc == 1 && vec_rows(Qm, sr, 0) ? 1 : 0;
  count_launch(1);
  kern<<<grid, THREADS, smem, st>>>(map, Qm, sr, sc, X, Y, P, S, N, bz, Aref, errp, xpart,
                                    ypart, status);
  return cudaGetLastError();
}

cudaError_t launch_batched_tc(const float *Mm, int64_t sr, int64_t sc, int64_t sMz,
                              const float *X, int64_t sXz, int64_t sxc, int64_t sxn, float *Y,
                              int64_t sYz, int64_t P, int64_t S, int64_t N, int64_t batch,
                              int64_t s_total, int32_t *status, cudaStream_t st) {
  if (batch < 1 || P < 1 || N < 1) return cudaSuccess;
  if (batch > 65535) return cudaErrorInvalidValue;
  CUtensorMap map;
  std::memset(&map, 0, sizeof(map));
  const size_t smem = tc_smem(false);
  cudaError_t e = cudaFuncSetAttribute(mode3_tc_kernel<false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  BatchStrides bz;
  bz.sMz = sMz;
  bz.sXz = sXz;
  bz.sYz = sYz;
  bz.sxc = sxc;
  bz.sxn = sxn;
  bz.s_total = s_total;
  bz.vec_x = sxc == 1 && vec_rows(X, sxn, batch > 1 ? sXz : 0) ? 1 : 0;
  bz.vec_m = sc == 1 && vec_rows(Mm, sr, batch > 1 ? sMz : 0) ? 1 : 0;
  const dim3 grid((unsigned)((N + TM - 1) / TM), (unsigned)((P + NT - 1) / NT), (unsigned)batch);
  count_launch(1);
  mode3_tc_kernel<false><<<grid, THREADS, smem, st>>>(map, Mm, sr, sc, X, Y, P, S, N, bz,
                                                      nullptr, nullptr, nullptr, nullptr,
                                                      status);
  return cudaGetLastError();
}

cudaError_t launch_reduce_tc(const float *Mm, int64_t sr, int64_t sc, int64_t sMz,
                             const float *X, int64_t sXz, int64_t sxc, int64_t sxn, float *Y,
                             int64_t sYz, int64_t P, int64_t S, int64_t N, int64_t nmem,
                             int64_t groups, cudaStream_t st) {
  if (nmem < 1 || P < 1 || N < 1 || S < 1) return cudaSuccess;
  if (groups < 1) groups = 1;
  if (groups > nmem) groups = nmem;
  const int64_t rz = (nmem + groups - 1) / groups;
  groups = (nmem + rz - 1) / rz;   // every group has at least one member
  if (groups > 65535) return cudaErrorInvalidValue;
  CUtensorMap map;
  std::memset(&map, 0, sizeof(map));
  const size_t smem = tc_smem(false);
  cudaError_t e = cudaFuncSetAttribute(mode3_tc_kernel<false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  BatchStrides bz;
  bz.sMz = sMz;
  bz.sXz = sXz;
  bz.sYz = sYz;
  bz.sxc = sxc;
  bz.sxn = sxn;
  bz.rz = rz;
  bz.nmem = nmem;
  bz.vec_x = sxc == 1 && vec_rows(X, sxn, sXz) ? 1 : 0;
  bz.vec_m = sc == 1 && vec_rows(Mm, sr, sMz) ? 1 : 0;
  const dim3 grid((unsigned)((N + TM - 1) / TM), (unsigned)((P + NT - 1) / NT), (unsigned)groups);
  count_launch(1);
  mode3_tc_kernel<false><<<grid, THREADS, smem, st>>>(map, Mm, sr, sc, X, Y, P, S, N, bz, nullptr,
                                                      nullptr, nullptr, nullptr, nullptr);
  return cudaGetLastError();
}

}  // namespace pp
