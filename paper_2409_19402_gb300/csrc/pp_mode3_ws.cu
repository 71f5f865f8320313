// pp_mode3_ws.cu -- the mode-3 product (Def. 2.2) as a persistent,
// warp-specialised tcgen05 kernel: Y (P x N) = M (P x S) X (S x N) over the
// mode-3 unfolding, N = l m pixels, for the transform A x_3 Q^T of Alg. 4.1
// step 2 and the reverse transform x_3 Q of step 4 when the caller provides a
// small scratch buffer for M's converted image; with X contraction-
// contiguous and the contraction split into members, the A B^T over all
// pixels of the Q gradient (launch_nt_ws); and, with the members independent
// products, the facewise products of Def. 2.3 in the projected product and
// its backward, stored directly or transposed (launch_batched_ws).
//
// Arithmetic (the same as the one-CTA-per-tile kernel of pp_gemm_tc.cu): the
// 3-pass split tf32 product hi.hi + hi.lo + lo.hi with hi = tf32(x) and
// lo = tf32(x - hi) (round to nearest, ties away), FP32 accumulation; the
// tensor core sums each 32-wide chunk of the contraction into its own TMEM
// accumulator from zero and the chunk sums are added in FP32 registers (round
// to nearest), in chunk order.  (Summing the 64 terms of a stage in one
// accumulator raised the projection error by half and took a hyperspectral
// A_k check past its bound.)
//
// Layout of the work: a unit is 128 pixels x 64 output rows (MMA M = 128
// pixels, N = 64 rows of M); the CTA, one per SM, walks the units
// u = blockIdx.x, + gridDim.x, ... (row tile fastest, so that the CTAs that
// run at the same time share a pixel tile of X through L2).  Each unit runs
// over S in stages of KC = 64 terms.  The roles, tied together by mbarrier
// rings whose every wait is bounded:
//   - producer warp: per stage, X's terms [64 c, 64 c + 64) for the unit's 128
//     pixels into a ring of R raw stages: one unswizzled 128 x 64 box when X
//     is pixel-contiguous, two 128-byte-swizzled 32 x 128 boxes when it is
//     contraction-contiguous;
//   - image warp: one bulk copy per stage of the hi/lo image of M (two
//     32-wide chunks, K-major, 128-byte swizzle: the MMA's B operand), built
//     once per call by prep_image_kernel, into a ring of SB stages;
//   - converter warps (four, one per TMEM lane quarter): a thread per pixel
//     row reads its 64 raw values, splits them into tf32 hi/lo and stores them
//     into TMEM (tcgen05.st), where the MMA takes its A operand from (SA
//     stages of 128 columns);
//   - MMA thread: 24 tcgen05.mma kind::tf32 per stage into one of DB pairs of
//     TMEM accumulators (one per 32-wide chunk), then tcgen05.commit to the
//     barriers that free the A stage, the image stage and hand the
//     accumulators to the epilogue;
//   - epilogue warps (four, one per TMEM lane quarter): add each stage's sums
//     into registers; at the end of a unit write the 64 x 32-pixel tile of
//     each warp into shared memory and store it with one TMA store, fusing
//     sum Y^2 and, against a reference A (its tile brought in by TMA while
//     the stages run), sum (A - Y)^2.
// Partial sums are written per (unit, warp) and summed later in index order,
// so the results are deterministic.
//
// Every ring has one consumer that takes its uses in order, so a waiter is
// never more than one phase ahead of the barrier it waits on, which the
// parity waits require.  (Two converter groups taking alternate stages broke
// this: a group could reach a slot whose previous use, the other group's, had
// not landed yet, read the parity as complete one phase early and over-arrive
// on the barrier.)
#include <cuda.h>

#include <cstring>

#include "pp_internal.h"
#include "pp_tc.cuh"
#include "pp_tma.h"

namespace pp {
namespace {

using namespace tc;

constexpr int TM = 128;               // pixels per unit (MMA M)
constexpr int NT = 64;                // output rows per unit (MMA N)
constexpr int TK = 32;                // terms per image chunk (one 128-byte swizzle row)
constexpr int KC = 64;                // terms per stage
constexpr int R = 3;                  // raw X stages
constexpr int SB = 2;                 // image stages
constexpr int SA = 2;                 // A stages in TMEM
constexpr int DB = 2;                 // accumulator pairs in TMEM (one per 32-wide chunk of a stage)
constexpr int NCG = 1;                // converter groups (one: see the ring rule above)
constexpr int OB = 2;                 // staging tiles per epilogue warp
constexpr int WPROD = 4 + 4 * NCG, WIMG = WPROD + 1, WMMA = WPROD + 2;
constexpr int THREADS = 32 * (WMMA + 1);
constexpr int RAW = KC * TM * 4;      // 32 KB: 64 rows x 128 pixels
constexpr int BCH = 2 * NT * 128;     // one 32-wide image chunk, hi and lo: 16 KB
constexpr int BST = (KC / TK) * BCH;  // one image stage: 32 KB
constexpr int OSTG = NT * 32 * 4;     // a warp's 64 x 32 output tile: 8 KB
constexpr int ACOLS = 2 * KC;         // TMEM columns of an A stage (hi, lo)
constexpr int DCOL = SA * ACOLS;      // first accumulator column
constexpr int DCOLS = (KC / TK) * NT; // TMEM columns of an accumulator pair
constexpr int TMEM_COLS = 512;
static_assert(DCOL + DB * DCOLS <= TMEM_COLS, "TMEM budget");
constexpr size_t SMEM_BYTES =
    (size_t)SB * BST + (size_t)R * RAW + (size_t)4 * OB * OSTG + 1024;   // + alignment slack

// position in a ring of n slots and the phase parity of its current use
struct Ring {
  uint32_t i = 0, ph = 0;
  __device__ __forceinline__ void next(uint32_t n) {
    if (++i == n) {
      i = 0;
      ph ^= 1u;
    }
  }
};

__device__ __forceinline__ bool test_phase(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}

// try_wait with a suspend-time hint (20 us): the thread sleeps until the phase
// completes instead of spinning on its SMSP's issue slots
__device__ __forceinline__ bool try_sleep(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity), "r"(20000u)
      : "memory");
  return ok != 0;
}

// Wait for the phase of parity `parity` to complete.  False once any role of
// the CTA has given up (abort flag) or after ~2 s, which raises the flag.
__device__ __forceinline__ bool wait_or_abort(uint32_t mbar, uint32_t parity,
                                              volatile int *abort_flag) {
  if (test_phase(mbar, parity)) return true;
  const long long t0 = clock64();
  while (!try_sleep(mbar, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > WAIT_CYCLES) {
      *abort_flag = 1;
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void init_bar(uint64_t *b, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}

// D (TMEM) (+)= A (TMEM) * B (shared-memory descriptor), kind::tf32
__device__ __forceinline__ void mma_tf32_ta(uint32_t d, uint32_t a_tmem, uint64_t b,
                                            uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d),
      "r"(a_tmem), "l"(b), "r"(idesc), "r"(accumulate));
}

// 32 consecutive 32-bit TMEM columns of this thread's lane (32x32b shape)
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const float *v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
      "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
      "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]),
      "f"(v[8]), "f"(v[9]), "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]),
      "f"(v[15]), "f"(v[16]), "f"(v[17]), "f"(v[18]), "f"(v[19]), "f"(v[20]), "f"(v[21]),
      "f"(v[22]), "f"(v[23]), "f"(v[24]), "f"(v[25]), "f"(v[26]), "f"(v[27]), "f"(v[28]),
      "f"(v[29]), "f"(v[30]), "f"(v[31]));
}

// An FP32 pair (hi, lo) whose sum carries a running total of FP32 terms
// without rounding loss (Knuth's branch-free two-sum: hi + e is exactly the
// sum of hi and the term; the errors e collect in lo).  The energy partials
// are accumulated this way, FP32 within a group of terms and exactly beyond,
// instead of in FP64, whose pipe is narrow on this part and sat on the
// converters' and the epilogue's critical paths.
struct F2 {
  float hi = 0.f, lo = 0.f;
};

__device__ __forceinline__ void f2_add(F2 &s, float b) {
  const float t = s.hi + b;
  const float bp = t - s.hi;
  const float e = (s.hi - (t - bp)) + (b - bp);
  s.hi = t;
  s.lo += e;
}

// a + b (two-sum of the high parts, low parts added): the same result for
// (a, b) and (b, a), so an xor-shuffle reduction leaves it in every lane
__device__ __forceinline__ F2 f2_sum(const F2 &a, const F2 &b) {
  F2 r;
  const float t = a.hi + b.hi;
  const float bp = t - a.hi;
  const float e = (a.hi - (t - bp)) + (b.hi - bp);
  r.hi = t;
  r.lo = e + (a.lo + b.lo);
  return r;
}

__device__ __forceinline__ F2 f2_warp_sum(F2 v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    F2 o;
    o.hi = __shfl_xor_sync(0xffffffffu, v.hi, off);
    o.lo = __shfl_xor_sync(0xffffffffu, v.lo, off);
    v = f2_sum(v, o);
  }
  return v;
}

__device__ __forceinline__ double f2_value(const F2 &v) { return (double)v.hi + (double)v.lo; }

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mbar)
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            int z, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(mbar)
      : "memory");
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes,
                                          uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(dst),
      "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(mbar)
      : "memory");
}

// The image of M: for row tile ty and 32-wide chunk c (2 nst chunks per tile,
// nst = stages), the K-major 128-byte-swizzled tf32 hi tile of
// M(64 ty + t, 32 c + k), t < 64, k < 32, followed by its lo tile; zero outside
// P x S; batch members one after the other.  One thread per 16-byte group of
// four terms.
__global__ void prep_image_kernel(const float *__restrict__ Qm, int64_t sr, int64_t sc, int64_t sMz,
                                  int64_t P, int64_t S, int64_t nchunk, int64_t tiles_y,
                                  int64_t batch, unsigned char *__restrict__ img) {
  // members z < batch, M[z](r, c) = Qm[z sMz + r sr + c sc], one after the other
  const int64_t total = batch * tiles_y * nchunk * NT * 8;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(e & 7);
    const int t = (int)((e >> 3) % NT);
    const int64_t tc = e / (8 * NT);   // (member * tiles_y + tile) * nchunk + chunk
    const int64_t c = tc % nchunk;
    const int64_t zt = tc / nchunk;
    const int64_t row = (zt % tiles_y) * NT + t;
    const float *Mz = Qm + (zt / tiles_y) * sMz;
    float hv[4], lv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t k = c * TK + 4 * q + j;
      const float x = (row < P && k < S) ? Mz[row * sr + k * sc] : 0.f;
      hv[j] = tf32_rna(x);
      lv[j] = tf32_rna(x - hv[j]);
    }
    unsigned char *base = img + tc * BCH;
    const uint32_t off = sw128_chunk(t, q);
    *reinterpret_cast<float4 *>(base + off) = make_float4(hv[0], hv[1], hv[2], hv[3]);
    *reinterpret_cast<float4 *>(base + NT * 128 + off) = make_float4(lv[0], lv[1], lv[2], lv[3]);
  }
}

// KMAJ: X is contraction-contiguous (X(s, n) = X[n ldx + s]) and comes in as
// two 128-byte-swizzled 32 x 128 boxes per stage; else X(s, n) = X[s ldx + n],
// one unswizzled 128 x 64 box.  There are nz members (the third coordinate of
// the X and Y maps): with batch = 0 they split one contraction of S terms into
// kchunk terms each (a multiple of KC; all read layer 0 of X at a term
// offset and one image), with batch = 1 they are independent products (X
// layer z, image z).  TRANS: Y is stored transposed, Y(t, n) at n P + t (the
// 64 x 32 tile of a warp as two 128-byte-swizzled 32 x 32 boxes), else at t N + n.
template <bool KMAJ, bool TRANS>
__global__ void __launch_bounds__(THREADS, 1) mode3_ws_kernel(
    const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap ymap,
    const __grid_constant__ CUtensorMap amap, const unsigned char *__restrict__ img, int has_y,
    int has_ref, int P, int S, int N, int nz, int kchunk, int batch, double *__restrict__ errp,
    double *__restrict__ xpart, double *__restrict__ ypart, int32_t *status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // the 1024-byte aligned base, offset from smem_raw itself so that the
  // compiler still sees shared-memory accesses (not generic ones) through it
  unsigned char *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  unsigned char *bimg = smem;              // SB image stages (1024-aligned for the swizzle)
  unsigned char *xraw = smem + SB * BST;   // R raw X stages
  unsigned char *ostg = xraw + R * RAW;    // 4 warps x OB output staging tiles
  __shared__ __align__(8) uint64_t x_full[R], x_empty[R], a_full[SA], a_empty[SA];
  __shared__ __align__(8) uint64_t b_full[SB], b_empty[SB], t_full[DB], t_empty[DB];
  __shared__ __align__(8) uint64_t ref_full[4];   // epilogue warp w: its A tile arrived
  __shared__ uint32_t tmem_sh;
  __shared__ volatile int abort_flag;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tiles_x = (N + TM - 1) / TM, tiles_y = (P + NT - 1) / NT;
  const int per = tiles_x * tiles_y;     // units per member
  const int U = nz * per;
  const int nst_total = (S + KC - 1) / KC;   // image stages per row tile
  // unit u: member z, row tile ty (fastest), pixel tile tx; its stages
  auto unit = [&](int u, int &z, int &ty, int &tx) {
    z = u / per;
    const int r = u - z * per;
    ty = r % tiles_y;
    tx = r / tiles_y;
    if (batch) return nst_total;
    const int sz = S - z * kchunk;
    return ((sz < kchunk ? sz : kchunk) + KC - 1) / KC;
  };
  if (tid == 0) {
    for (int i = 0; i < R; ++i) {
      init_bar(&x_full[i], 1);
      init_bar(&x_empty[i], 4);   // one arrival per converter warp of the group
    }
    for (int i = 0; i < SA; ++i) {
      init_bar(&a_full[i], 4);
      init_bar(&a_empty[i], 1);   // tcgen05.commit
    }
    for (int i = 0; i < SB; ++i) {
      init_bar(&b_full[i], 1);
      init_bar(&b_empty[i], 1);
    }
    for (int i = 0; i < DB; ++i) {
      init_bar(&t_full[i], 1);
      init_bar(&t_empty[i], 4);   // one arrival per epilogue warp
    }
    for (int i = 0; i < 4; ++i) init_bar(&ref_full[i], 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == WMMA) tmem_alloc(&tmem_sh, TMEM_COLS);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_sh;

  if (warp == WPROD) {
    // ---------------- X stages by TMA
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&xmap)) : "memory");
      Ring xr;
      int g = 0;
      bool ok = true;
      for (int u = blockIdx.x; ok && u < U; u += gridDim.x) {
        int z, ty, tx;
        const int nst = unit(u, z, ty, tx);
        for (int c = 0; c < nst; ++c, ++g) {
          if (g >= R && !wait_or_abort(smem_u32(&x_empty[xr.i]), xr.ph ^ 1u, &abort_flag)) {
            ok = false;
            break;
          }
          const uint32_t dst = smem_u32(xraw + xr.i * RAW), fb = smem_u32(&x_full[xr.i]);
          const int s0 = (batch ? 0 : z * kchunk) + c * KC;   // first term of the stage
          const int layer = batch ? z : 0;
          mbar_expect_tx(fb, (uint32_t)RAW);
          if (KMAJ) {
            tma_load_3d(dst, &xmap, s0, tx * TM, layer, fb);
            tma_load_3d(dst + RAW / 2, &xmap, s0 + TK, tx * TM, layer, fb);
          } else {
            tma_load_3d(dst, &xmap, tx * TM, s0, layer, fb);
          }
          xr.next(R);
        }
      }
      // the boxes still in flight (the last use of each slot) land before exit
      for (int h = (g > R ? g - R : 0); h < g; ++h)
        (void)mbar_wait(smem_u32(&x_full[h % R]), (uint32_t)((h / R) & 1));
    }
  } else if (warp == WIMG) {
    // ---------------- image stages of M by bulk copy
    if (lane == 0) {
      Ring br;
      int g = 0;
      bool ok = true;
      for (int u = blockIdx.x; ok && u < U; u += gridDim.x) {
        int z, ty, tx;
        const int nst = unit(u, z, ty, tx);
        for (int c = 0; c < nst; ++c, ++g) {
          if (g >= SB && !wait_or_abort(smem_u32(&b_empty[br.i]), br.ph ^ 1u, &abort_flag)) {
            ok = false;
            break;
          }
          mbar_expect_tx(smem_u32(&b_full[br.i]), (uint32_t)BST);
          const int64_t stage = batch ? ((int64_t)z * tiles_y + ty) * nst_total + c
                                      : (int64_t)ty * nst_total + (int64_t)z * (kchunk / KC) + c;
          bulk_load(smem_u32(bimg + br.i * BST), img + stage * BST, (uint32_t)BST,
                    smem_u32(&b_full[br.i]));
          br.next(SB);
        }
      }
      for (int h = (g > SB ? g - SB : 0); h < g; ++h)
        (void)mbar_wait(smem_u32(&b_full[h % SB]), (uint32_t)((h / SB) & 1));
    }
  } else if (warp == WMMA) {
    // ---------------- MMA issue
    if (lane == 0) {
      constexpr uint32_t IDESC = tf32_idesc(TM, NT);
      // the descriptors' address field is (address >> 4), every address here is
      // below 256 KB, so offsets add to it directly
      const uint64_t desc0 = sw128_desc(smem_u32(bimg));
      Ring ar, br, dr;
      int g = 0;
      bool ok = true;
      for (int u = blockIdx.x; ok && u < U; u += gridDim.x) {
        int z, ty, tx;
        const int nst = unit(u, z, ty, tx);
        for (int c = 0; c < nst; ++c, ++g) {
          if (!wait_or_abort(smem_u32(&a_full[ar.i]), ar.ph, &abort_flag) ||
              !wait_or_abort(smem_u32(&b_full[br.i]), br.ph, &abort_flag) ||
              (g >= DB && !wait_or_abort(smem_u32(&t_empty[dr.i]), dr.ph ^ 1u, &abort_flag))) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t ta0 = tmem + ar.i * (uint32_t)ACOLS;
          // Chunk h of the stage goes into its own accumulator, from zero, as
          // lo.hi + hi.lo + hi.hi per 8-term K step (the small products
          // first).  The two chunks' MMAs alternate, so consecutive MMAs never
          // accumulate into the same TMEM columns; each accumulator takes its
          // products in the same order as with the chunks one after the other.
#pragma unroll
          for (int kk = 0; kk < TK / 8; ++kk) {   // 8 tf32 of K per MMA
#pragma unroll
            for (int h = 0; h < KC / TK; ++h) {
              const uint32_t td =
                  tmem + (uint32_t)DCOL + dr.i * (uint32_t)DCOLS + (uint32_t)(h * NT);
              const uint64_t dbh = desc0 + (uint64_t)((br.i * BST + h * BCH) >> 4);
              const uint64_t dbl = dbh + (uint64_t)((NT * 128) >> 4);
              const uint32_t ta = ta0 + (uint32_t)(h * 2 * TK);   // chunk h: hi, then lo
              mma_tf32_ta(td, ta + TK + 8 * kk, dbh + 2 * kk, IDESC, kk > 0 ? 1u : 0u);
              mma_tf32_ta(td, ta + 8 * kk, dbl + 2 * kk, IDESC, 1u);
              mma_tf32_ta(td, ta + 8 * kk, dbh + 2 * kk, IDESC, 1u);
            }
          }
          mma_commit(smem_u32(&a_empty[ar.i]));
          mma_commit(smem_u32(&b_empty[br.i]));
          mma_commit(smem_u32(&t_full[dr.i]));
          ar.next(SA);
          br.next(SB);
          dr.next(DB);
        }
      }
      // Every commit's arrival lands before the CTA exits (and with it the MMAs
      // that read shared memory and TMEM): the three commits of a stage arrive
      // independently, and nobody else waits for the last uses of a ring, so
      // the last phase of every barrier a commit arrives on is waited here.
      auto drain = [&](uint64_t *bars, int n) {
        for (int i = 0; i < n && i < g; ++i) {
          const int uses = (g - i + n - 1) / n;   // stages g' < g with g' = i (mod n)
          (void)mbar_wait(smem_u32(&bars[i]), (uint32_t)((uses - 1) & 1));
        }
      };
      drain(a_empty, SA);
      drain(b_empty, SB);
      drain(t_full, DB);
    }
  } else if (warp >= 4) {
    // ---------------- converters: X stage -> A hi/lo in TMEM
    const int cg = (warp - 4) >> 2;
    const int row = (warp & 3) * 32 + lane;   // pixel row = TMEM lane
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    Ring xr, ar;
    int g = 0;
    bool ok = true;
    for (int u = blockIdx.x; ok && u < U; u += gridDim.x) {
      int z, ty, tx;
      const int nst = unit(u, z, ty, tx);
      const bool do_x = xpart != nullptr && ty == 0 && z == 0;
      F2 xs;
      for (int c = 0; c < nst; ++c, ++g, xr.next(R), ar.next(SA)) {
        if (g % NCG != cg) continue;
        if (!__all_sync(0xffffffffu,
                        wait_or_abort(smem_u32(&x_full[xr.i]), xr.ph, &abort_flag))) {
          ok = false;
          break;
        }
        float v[32], w[32];
        if (KMAJ) {
          // two swizzled 32 x 128 boxes: row `row` holds terms 0-31 (and 32-63 in
          // the second box) as eight 16-byte chunks, chunk j at j ^ (row mod 8)
          const unsigned char *rb = xraw + xr.i * RAW + row * 128;
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const uint32_t off = (uint32_t)(((j ^ row) & 7) << 4);
            const float4 a = *reinterpret_cast<const float4 *>(rb + off);
            const float4 b = *reinterpret_cast<const float4 *>(rb + RAW / 2 + off);
            v[4 * j] = a.x; v[4 * j + 1] = a.y; v[4 * j + 2] = a.z; v[4 * j + 3] = a.w;
            w[4 * j] = b.x; w[4 * j + 1] = b.y; w[4 * j + 2] = b.z; w[4 * j + 3] = b.w;
          }
        } else {
          const float *rp = reinterpret_cast<const float *>(xraw + xr.i * RAW);
#pragma unroll
          for (int k = 0; k < 32; ++k) {
            v[k] = rp[k * TM + row];
            w[k] = rp[(32 + k) * TM + row];
          }
        }
        __syncwarp();
        if (lane == 0) arrive(smem_u32(&x_empty[xr.i]));
        if (do_x) {   // FP32 over 16 values, exact beyond
          float q0 = 0.f, q1 = 0.f, q2 = 0.f, q3 = 0.f;
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            q0 = fmaf(v[k], v[k], q0);
            q1 = fmaf(v[16 + k], v[16 + k], q1);
            q2 = fmaf(w[k], w[k], q2);
            q3 = fmaf(w[16 + k], w[16 + k], q3);
          }
          f2_add(xs, q0);
          f2_add(xs, q1);
          f2_add(xs, q2);
          f2_add(xs, q3);
        }
        if (g >= SA && !__all_sync(0xffffffffu, wait_or_abort(smem_u32(&a_empty[ar.i]),
                                                               ar.ph ^ 1u, &abort_flag))) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        {
          const uint32_t ta = tmem + lane_base + ar.i * (uint32_t)ACOLS;
          float lo[32];
#pragma unroll
          for (int k = 0; k < 32; ++k) {
            const float h = tf32_rna(v[k]);
            lo[k] = tf32_rna(v[k] - h);
            v[k] = h;
          }
          tmem_st32(ta, v);
          tmem_st32(ta + TK, lo);
#pragma unroll
          for (int k = 0; k < 32; ++k) {
            const float h = tf32_rna(w[k]);
            lo[k] = tf32_rna(w[k] - h);
            w[k] = h;
          }
          tmem_st32(ta + 2 * TK, w);
          tmem_st32(ta + 3 * TK, lo);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncwarp();
        if (lane == 0) arrive(smem_u32(&a_full[ar.i]));
      }
      if (!ok) break;
      if (do_x) {
        xs = f2_warp_sum(xs);
        if (lane == 0) xpart[((int64_t)tx * NCG + cg) * 4 + (warp & 3)] = f2_value(xs);
      }
    }
  } else {
    // ---------------- epilogue (warps 0-3)
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    Ring dr;
    int g = 0, ul = 0;
    bool ok = true;
    for (int u = blockIdx.x; ok && u < U; u += gridDim.x, ++ul) {
      int z, ty, tx;
      const int nst = unit(u, z, ty, tx);
      float *stg = reinterpret_cast<float *>(ostg + (warp * OB + (ul % OB)) * OSTG);
      // this staging tile's store from OB units ago has been read; then the
      // reference tile (A) of this unit comes into it by TMA
      if (lane == 0) {
        asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
        if (has_ref) {
          mbar_expect_tx(smem_u32(&ref_full[warp]), (uint32_t)OSTG);
          tma_load_2d(smem_u32(stg), &amap, tx * TM + warp * 32, ty * NT, smem_u32(&ref_full[warp]));
        }
      }
      float acc[NT];
#pragma unroll
      for (int j = 0; j < NT; ++j) acc[j] = 0.f;
      for (int c = 0; c < nst; ++c, ++g) {
        if (!__all_sync(0xffffffffu,
                        wait_or_abort(smem_u32(&t_full[dr.i]), dr.ph, &abort_flag))) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
        for (int h = 0; h < KC / TK; ++h) {   // the stage's chunk sums, in chunk order
#pragma unroll
          for (int j0 = 0; j0 < NT; j0 += 16) {
            float t16[16];
            tmem_ld16(tmem + lane_base + (uint32_t)DCOL + dr.i * (uint32_t)DCOLS +
                          (uint32_t)(h * NT + j0),
                      t16);
#pragma unroll
            for (int q = 0; q < 16; ++q) acc[j0 + q] += t16[q];
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncwarp();
        if (lane == 0) arrive(smem_u32(&t_empty[dr.i]));
        dr.next(DB);
      }
      const bool ref_ok =
          !has_ref || __all_sync(0xffffffffu, wait_or_abort(smem_u32(&ref_full[warp]),
                                                            (uint32_t)(ul & 1), &abort_flag));
      if (!ok || !ref_ok) {
        ok = false;
        break;
      }
      const int pix = tx * TM + warp * 32 + lane;
      F2 err, ys;
#pragma unroll
      for (int g8 = 0; g8 < NT; g8 += 8) {   // FP32 over 8 values, exact beyond
        float e8 = 0.f, y8 = 0.f;
#pragma unroll
        for (int q = g8; q < g8 + 8; ++q) {
          const float v = acc[q];
          if (ty * NT + q < P && pix < N) {
            y8 = fmaf(v, v, y8);
            if (!TRANS && has_ref) {
              const float d = stg[q * 32 + lane] - v;
              e8 = fmaf(d, d, e8);
            }
          }
          if (!TRANS) stg[q * 32 + lane] = v;
        }
        f2_add(ys, y8);
        f2_add(err, e8);
      }
      if (TRANS) {
        // row `lane` (this pixel) of two 32 x 32 boxes (outputs 0-31, 32-63),
        // 16-byte chunk j of a row at j ^ (row mod 8)
        unsigned char *sb = reinterpret_cast<unsigned char *>(stg) + lane * 128;
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int j = 0; j < 8; ++j)
            *reinterpret_cast<float4 *>(sb + h * 4096 + (((j ^ lane) & 7) << 4)) =
                make_float4(acc[32 * h + 4 * j], acc[32 * h + 4 * j + 1], acc[32 * h + 4 * j + 2],
                            acc[32 * h + 4 * j + 3]);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0 && has_y) {   // out-of-range rows and pixels are clipped by the store
        if (TRANS) {
#pragma unroll
          for (int h = 0; h < 2; ++h)
            asm volatile(
                "cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::
                    "l"(reinterpret_cast<uint64_t>(&ymap)),
                "r"(ty * NT + 32 * h), "r"(tx * TM + warp * 32), "r"(z),
                "r"(smem_u32(stg) + (uint32_t)(h * 4096))
                : "memory");
        } else {
          asm volatile(
              "cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::
                  "l"(reinterpret_cast<uint64_t>(&ymap)),
              "r"(tx * TM + warp * 32), "r"(ty * NT), "r"(z), "r"(smem_u32(stg))
              : "memory");
        }
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      }
      const int64_t part = (((int64_t)z * tiles_y + ty) * tiles_x + tx) * 4 + warp;
      if (errp) {
        err = f2_warp_sum(err);
        if (lane == 0) errp[part] = f2_value(err);
      }
      if (ypart) {
        ys = f2_warp_sum(ys);
        if (lane == 0) ypart[part] = f2_value(ys);
      }
    }
    if (lane == 0) {
      // a reference tile requested for a unit that was given up lands before exit
      if (!ok && has_ref) (void)mbar_wait(smem_u32(&ref_full[warp]), (uint32_t)(ul & 1));
      asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (abort_flag && tid == 0 && status) atomicCAS(status, 0, PP_ETIMEOUT);
  if (warp == WMMA) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

}  // namespace

size_t mode3_img_bytes(int64_t P, int64_t S) {
  if (P < 1 || S < 1) return 0;
  return (size_t)((P + NT - 1) / NT) * (size_t)((S + KC - 1) / KC) * (size_t)BST;
}

int64_t mode3_ws_partials(int64_t P, int64_t N) {
  return ((N + TM - 1) / TM) * ((P + NT - 1) / NT) * 4;
}

namespace {

// The image of M (batch members of P x S, M_z(r, c) = Qm[z sMz + r sr + c sc])
// and one launch of the kernel over nz members (split-K members of kchunk
// terms, or with batch the independent products); Y, when given, a 3-D map of
// nz products.
template <bool KMAJ, bool TRANS>
cudaError_t run_ws(const CUtensorMap &xmap, const CUtensorMap &ymap, const CUtensorMap &amap,
                   const float *Qm, int64_t sr, int64_t sc, int64_t sMz, bool has_y, bool has_ref,
                   int64_t P, int64_t S, int64_t N, int64_t nz, int64_t kchunk, bool batch,
                   double *errp, double *xpart, double *ypart, int32_t *status, void *img,
                   cudaStream_t st, bool prep = true) {
  const int64_t tiles_y = (P + NT - 1) / NT, nst = (S + KC - 1) / KC, tiles_x = (N + TM - 1) / TM;
  if (prep) {
    const int64_t members = batch ? nz : 1;
    const int64_t total = members * tiles_y * 2 * nst * NT * 8;
    int pb = (int)((total + 255) / 256);
    if (pb > 4 * num_sms()) pb = 4 * num_sms();
    count_launch(1);
    prep_image_kernel<<<pb, 256, 0, st>>>(Qm, sr, sc, batch ? sMz : 0, P, S, 2 * nst, tiles_y,
                                          members, static_cast<unsigned char *>(img));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const int64_t U = nz * tiles_x * tiles_y;
  const int grid = (int)(U < num_sms() ? U : num_sms());
  count_launch(1);
  mode3_ws_kernel<KMAJ, TRANS><<<grid, THREADS, SMEM_BYTES, st>>>(
      xmap, ymap, amap, static_cast<const unsigned char *>(img), has_y ? 1 : 0, has_ref ? 1 : 0,
      (int)P, (int)S, (int)N, (int)nz, (int)kchunk, batch ? 1 : 0, errp, xpart, ypart, status);
  return cudaGetLastError();
}

template <bool KMAJ, bool TRANS>
bool ws_attr() {
  if (cudaFuncSetAttribute(mode3_ws_kernel<KMAJ, TRANS>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)SMEM_BYTES) != cudaSuccess) {
    (void)cudaGetLastError();   // this device cannot host it: the caller takes the other kernel
    return false;
  }
  return true;
}

constexpr int64_t DIM_MAX = (int64_t)1 << 30;

}  // namespace

cudaError_t launch_mode3_ws(const float *Qm, int64_t sr, int64_t sc, const float *X, float *Y,
                            int64_t P, int64_t S, int64_t N, const float *Aref, double *errp,
                            int *n_partials, double *xpart, int *n_xpart, double *ypart,
                            int32_t *status, void *img, size_t img_bytes, cudaStream_t st,
                            bool *used, bool *img_ready) {
  *used = false;
  if (!img || img_bytes < mode3_img_bytes(P, S) || P < 1 || S < 1 || N < 1 || N > DIM_MAX ||
      P > DIM_MAX || S > DIM_MAX || (reinterpret_cast<uintptr_t>(img) & 15) != 0)
    return cudaSuccess;
  CUtensorMap xmap, ymap, amap;
  std::memset(&xmap, 0, sizeof(xmap));
  std::memset(&ymap, 0, sizeof(ymap));
  std::memset(&amap, 0, sizeof(amap));
  // X(s, n) = X[s N + n]: one layer of S rows, 64 x 128 boxes
  if (!encode_3d(&xmap, X, N, S, 1, N, N * S, (uint32_t)TM, (uint32_t)KC, true, false))
    return cudaSuccess;
  if (Y && !encode_layers_3d(&ymap, Y, N, P, 1, 32u, (uint32_t)NT)) return cudaSuccess;
  if (Aref && !encode_rows_2d(&amap, Aref, N, P, 32u, (uint32_t)NT, false)) return cudaSuccess;
  if (!ws_attr<false, false>()) return cudaSuccess;
  *used = true;
  const int64_t tiles_y = (P + NT - 1) / NT, tiles_x = (N + TM - 1) / TM;
  if (n_partials) *n_partials = (int)(tiles_x * tiles_y * 4);
  if (n_xpart) *n_xpart = (int)(tiles_x * NCG * 4);
  const int64_t kchunk = (S + KC - 1) / KC * KC;   // one member: the whole contraction
  const cudaError_t e =
      run_ws<false, false>(xmap, ymap, amap, Qm, sr, sc, 0, Y != nullptr, Aref != nullptr, P, S,
                           N, 1, kchunk, false, Aref ? errp : nullptr, xpart, ypart, status, img,
                           st, !(img_ready && *img_ready));
  if (img_ready && e == cudaSuccess) *img_ready = true;
  return e;
}

size_t nt_img_bytes(int64_t R, int64_t S, int64_t K) {
  return mode3_img_bytes(S < R ? S : R, K);
}

cudaError_t launch_nt_ws(const float *A, const float *B, int64_t R, int64_t S, int64_t K,
                         float *part, int64_t part_floats, void *img, size_t img_bytes,
                         int64_t *nz_out, bool *transposed, cudaStream_t st, bool *used) {
  *used = false;
  // part[z] = A[:, z kc ..] B[:, z kc ..]^T (R x S), or its transpose B A^T (S x R) when
  // S < R, so that the larger side runs along the 128-row MMA tiles; M = first, X = second
  const bool tr = S < R;
  const float *first = tr ? B : A, *second = tr ? A : B;
  const int64_t P = tr ? S : R, N = tr ? R : S;
  if (!img || !part || img_bytes < mode3_img_bytes(P, K) || K < 1 || P < 1 || N < 1 ||
      K > DIM_MAX || N > DIM_MAX || K % 4 != 0 || (reinterpret_cast<uintptr_t>(img) & 15) != 0)
    return cudaSuccess;
  // members: about one unit per SM, each at least four stages
  const int64_t per = ((N + TM - 1) / TM) * ((P + NT - 1) / NT);
  int64_t nz = (num_sms() + per - 1) / per;
  const int64_t zmax = (K + 4 * KC - 1) / (4 * KC);
  if (nz > zmax) nz = zmax;
  if (nz < 1) nz = 1;
  int64_t kchunk = (K + nz - 1) / nz;
  kchunk = (kchunk + KC - 1) / KC * KC;
  nz = (K + kchunk - 1) / kchunk;
  if (nz * R * S > part_floats || nz > 65535) return cudaSuccess;
  CUtensorMap xmap, ymap, amap;
  std::memset(&xmap, 0, sizeof(xmap));
  std::memset(&ymap, 0, sizeof(ymap));
  std::memset(&amap, 0, sizeof(amap));
  // X(s, n) = second[n K + s]: one layer of N rows of K terms, 32 x 128 boxes
  // with the 128-byte swizzle
  if (!encode_3d(&xmap, second, K, N, 1, K, K * N, (uint32_t)TK, (uint32_t)TM, true, true))
    return cudaSuccess;
  if (!encode_layers_3d(&ymap, part, N, P, nz, 32u, (uint32_t)NT)) return cudaSuccess;
  if (!ws_attr<true, false>()) return cudaSuccess;
  *used = true;
  *nz_out = nz;
  *transposed = tr;
  return run_ws<true, false>(xmap, ymap, amap, first, K, 1, 0, true, false, P, K, N, nz, kchunk,
                             false, nullptr, nullptr, nullptr, nullptr, img, st);
}

size_t batched_img_bytes(int64_t P, int64_t S, int64_t batch) {
  return batch < 1 ? 0 : (size_t)batch * mode3_img_bytes(P, S);
}

cudaError_t launch_batched_ws(const float *Mm, int64_t sr, int64_t sc, int64_t sMz,
                              const float *X, int64_t sXz, int64_t ldx, bool x_kmaj, float *Y,
                              int64_t sYz, int64_t ldy, bool y_trans, int64_t P, int64_t S,
                              int64_t N, int64_t batch, void *img, size_t img_bytes,
                              cudaStream_t st, bool *used) {
  *used = false;
  if (!img || img_bytes < batched_img_bytes(P, S, batch) || P < 1 || S < 1 || N < 1 ||
      batch < 1 || batch > 65535 || P > DIM_MAX || S > DIM_MAX || N > DIM_MAX ||
      (reinterpret_cast<uintptr_t>(img) & 15) != 0 || (x_kmaj ? S : N) > ldx ||
      (y_trans ? P : N) > ldy ||
      batch * ((N + TM - 1) / TM) * ((P + NT - 1) / NT) > (int64_t)INT32_MAX)
    return cudaSuccess;
  CUtensorMap xmap, ymap, amap;
  std::memset(&xmap, 0, sizeof(xmap));
  std::memset(&ymap, 0, sizeof(ymap));
  std::memset(&amap, 0, sizeof(amap));
  // X_z: rows ldx floats apart, layers sXz apart; contraction-contiguous X in
  // swizzled 32 x 128 boxes, pixel-contiguous X in 64 x 128 boxes
  const bool xok = x_kmaj ? encode_3d(&xmap, X, S, N, batch, ldx, sXz, (uint32_t)TK,
                                      (uint32_t)TM, true, true)
                          : encode_3d(&xmap, X, N, S, batch, ldx, sXz, (uint32_t)TM,
                                      (uint32_t)KC, true, false);
  // Y_z: a warp's tile as one 64 x 32 box, or transposed as two swizzled 32 x 32 boxes
  const bool yok = y_trans ? encode_3d(&ymap, Y, P, N, batch, ldy, sYz, 32u, 32u, false, true)
                           : encode_3d(&ymap, Y, N, P, batch, ldy, sYz, 32u, (uint32_t)NT, false,
                                       false);
  if (!xok || !yok) return cudaSuccess;
  if (x_kmaj ? (y_trans ? !ws_attr<true, true>() : !ws_attr<true, false>())
             : (y_trans ? !ws_attr<false, true>() : !ws_attr<false, false>()))
    return cudaSuccess;
  *used = true;
  const int64_t kchunk = (S + KC - 1) / KC * KC;
  if (x_kmaj && y_trans)
    return run_ws<true, true>(xmap, ymap, amap, Mm, sr, sc, sMz, true, false, P, S, N, batch,
                              kchunk, true, nullptr, nullptr, nullptr, nullptr, img, st);
  if (x_kmaj)
    return run_ws<true, false>(xmap, ymap, amap, Mm, sr, sc, sMz, true, false, P, S, N, batch,
                               kchunk, true, nullptr, nullptr, nullptr, nullptr, img, st);
  if (y_trans)
    return run_ws<false, true>(xmap, ymap, amap, Mm, sr, sc, sMz, true, false, P, S, N, batch,
                               kchunk, true, nullptr, nullptr, nullptr, nullptr, img, st);
  return run_ws<false, false>(xmap, ymap, amap, Mm, sr, sc, sMz, true, false, P, S, N, batch,
                              kchunk, true, nullptr, nullptr, nullptr, nullptr, img, st);
}

}  // namespace pp
