// pp_internal.h -- private declarations shared by the CUDA translation units
// of the projected t-SVD library.  Not part of the public C ABI (pprod.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pprod.h"

namespace pp {

// Count `n` kernel launches in the process-wide counter (pp_kernel_launches).
void count_launch(int n);

// Number of SMs of the current device (cudaDevAttrMultiProcessorCount, cached
// per device; 152 if the query fails).  Grids that fill the device and the
// launch-shape cost model use it; buffers sized from it are sized for the
// device that is current when the size is asked for.
int num_sms();

// Round x up to a multiple of a.
static inline int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// Device-side error word: the first nonzero pp_status written wins.
__device__ inline void set_status(int32_t *status, int32_t code) {
  if (status) atomicCAS(status, 0, code);
}

// ---------------------------------------------------------------- GEMMs
// Y (P x N, row-major, ldY = N) = M (P x S) * X (S x N, row-major) on the
// tensor cores (tcgen05, 3-pass split TF32), M(r, c) = Qm[r * sr + c * sc].
// When Aref != nullptr the launch also writes sum (Aref - Y)^2 over each CTA
// tile to errp[CTA] (FP64); Y may then be nullptr (error only).  Optional
// energy partials: xpart gets *n_xpart sums of X^2 (each X entry counted
// once), ypart one sum of Y^2 per CTA; partial counts from mode3_tc_partials.
// A bounded wait that expires writes PP_ETIMEOUT to *status (if non-null).
// With a scratch buffer img of at least mode3_img_bytes(P, S) bytes (16-byte
// aligned) and TMA-compatible X, Y, Aref (16-byte aligned, N a multiple of 4)
// the product runs on the persistent warp-specialised kernel of
// pp_mode3_ws.cu (one extra launch builds M's tf32 image in img); otherwise on
// the one-CTA-per-tile kernel.  Both compute the same arithmetic.  img_ready
// (optional): true on entry when img already holds the image of this M (an
// earlier call with the same M, P, S and img); set true once it does.
cudaError_t launch_mode3_tc(const float *Qm, int64_t sr, int64_t sc, const float *X, float *Y,
                            int64_t P, int64_t S, int64_t N, const float *Aref, double *errp,
                            int *n_partials, double *xpart, int *n_xpart, double *ypart,
                            int32_t *status, cudaStream_t st, void *img = nullptr,
                            size_t img_bytes = 0, bool *img_ready = nullptr);
// partial-sum slots for errp, xpart and ypart, enough for either kernel
int64_t mode3_tc_partials(int64_t P, int64_t N);
size_t mode3_img_bytes(int64_t P, int64_t S);
// the warp-specialised kernel; *used = false (nothing launched) when the
// arguments do not suit it
cudaError_t launch_mode3_ws(const float *Qm, int64_t sr, int64_t sc, const float *X, float *Y,
                            int64_t P, int64_t S, int64_t N, const float *Aref, double *errp,
                            int *n_partials, double *xpart, int *n_xpart, double *ypart,
                            int32_t *status, void *img, size_t img_bytes, cudaStream_t st,
                            bool *used, bool *img_ready = nullptr);

// The same tensor-core product over a batch (grid z): member z computes
// Y[z] (P x N, row-major) = M[z] (P x S) X[z] (S x N) with M(r, c) =
// Mm[z sMz + r sr + c sc] and X(c, n) = X[z sXz + c sxc + n sxn], Y at
// Y + z sYz.  s_total > 0: the members are the K-chunks of one contraction of
// s_total terms (member z holds terms z S .. min(s_total, (z + 1) S) - 1, its
// operand offsets given by sMz and sXz).
cudaError_t launch_batched_tc(const float *Mm, int64_t sr, int64_t sc, int64_t sMz,
                              const float *X, int64_t sXz, int64_t sxc, int64_t sxn, float *Y,
                              int64_t sYz, int64_t P, int64_t S, int64_t N, int64_t batch,
                              int64_t s_total, int32_t *status, cudaStream_t st);
// Sums of products: Y[g] (P x N) = sum over members z of group g of M[z] X[z]
// (the same operand layout as launch_batched_tc), nmem members split into at
// most `groups` groups of consecutive members; each group is one grid layer
// that accumulates its members' 32-term chunk sums in FP32 in member order.
cudaError_t launch_reduce_tc(const float *Mm, int64_t sr, int64_t sc, int64_t sMz,
                             const float *X, int64_t sXz, int64_t sxc, int64_t sxn, float *Y,
                             int64_t sYz, int64_t P, int64_t S, int64_t N, int64_t nmem,
                             int64_t groups, cudaStream_t st);

// Batched product Y[z] (P x N) = M[z] (P x S) * X[z] (S x N) (launch_batched_tc), M(r, c) =
// Mm[z*sMz + r*sr + c*sc], X and Y row-major with leading dimension N; a batch
// stride of 0 broadcasts an operand over the batch.
// X may be strided: X(c, n) = X[z*sXz + c*sxc + n*sxn] (sxc < 0: row-major, sxc = N).
cudaError_t launch_batched_gemm(const float *Mm, int64_t sr, int64_t sc, int64_t sMz,
                                const float *X, int64_t sXz, float *Y, int64_t sYz, int64_t P,
                                int64_t S, int64_t N, int64_t batch, cudaStream_t st,
                                int64_t sxc = -1, int64_t sxn = 1);

// out (R x S) = [out +] A B^T for A (R x K), B (S x K) row-major, split over K into
// nt_splits(R, S, K) FP32 partials (part) summed in a fixed order.
int64_t nt_splits(int64_t R, int64_t S, int64_t K);
// With img (at least nt_img_bytes(R, S, K) bytes) and part_floats of part,
// the product runs on the warp-specialised kernel (launch_nt_ws).
cudaError_t launch_nt_accumulate(const float *A, const float *B, int64_t R, int64_t S, int64_t K,
                                 float *part, float *out, int accumulate, cudaStream_t st,
                                 void *img = nullptr, size_t img_bytes = 0,
                                 int64_t part_floats = 0);
size_t nt_img_bytes(int64_t R, int64_t S, int64_t K);
// A B^T split over K on the warp-specialised kernel: part[z] for z < *nz_out
// holds member z's R x S product, or its S x R transpose (*transposed);
// *used = false (nothing launched) when the arguments do not suit it
cudaError_t launch_nt_ws(const float *A, const float *B, int64_t R, int64_t S, int64_t K,
                         float *part, int64_t part_floats, void *img, size_t img_bytes,
                         int64_t *nz_out, bool *transposed, cudaStream_t st, bool *used);
// out = D - Q sym(Q^T D) for Q, D n x p (Sm: p x p scratch; part, of
// part_floats floats, lets Q^T D split over the n rows)
cudaError_t launch_stiefel(const float *Q, const float *D, int64_t n, int64_t p, float *Sm,
                           float *out, cudaStream_t st, float *part = nullptr,
                           int64_t part_floats = 0);

// Independent products on the warp-specialised kernel: for z < batch,
// Y_z (P x N) = M_z (P x S) X_z (S x N) with M_z(r, c) = Mm[z sMz + r sr + c sc];
// X_z(s, n) = X[z sXz + n ldx + s] (x_kmaj) or X[z sXz + s ldx + n];
// Y_z(t, n) at Y[z sYz + n ldy + t] (y_trans) or Y[z sYz + t ldy + n].
// img: at least batched_img_bytes(P, S, batch) bytes for the members' tf32
// images.  *used = false (nothing launched) when the arguments do not suit it
// (TMA needs 16-byte aligned bases and strides that are multiples of 4 floats).
size_t batched_img_bytes(int64_t P, int64_t S, int64_t batch);
cudaError_t launch_batched_ws(const float *Mm, int64_t sr, int64_t sc, int64_t sMz,
                              const float *X, int64_t sXz, int64_t ldx, bool x_kmaj, float *Y,
                              int64_t sYz, int64_t ldy, bool y_trans, int64_t P, int64_t S,
                              int64_t N, int64_t batch, void *img, size_t img_bytes,
                              cudaStream_t st, bool *used);

// Facewise products C_t (rows x cols, row-major, faces rows*cols apart) =
// L_t (rows x inner) R_t (inner x cols) for t < p, with L_t(i, k) =
// L[t sLz + i sLi + k sLk] and R_t(k, j) = R[t sRz + k sRk + j sRj].  With img
// (facewise_img_bytes of it, an image budget capped at FACEWISE_IMG_CAP or one
// face) the faces run on the warp-specialised kernel in groups that fit it;
// otherwise, or when the layouts do not suit it, on the one-CTA-per-tile kernel.
constexpr size_t FACEWISE_IMG_CAP = (size_t)32 << 20;
size_t facewise_img_bytes(int64_t rows, int64_t inner, int64_t cols, int64_t p);
cudaError_t launch_facewise_strided(const float *L, int64_t sLi, int64_t sLk, int64_t sLz,
                                    const float *Rm, int64_t sRk, int64_t sRj, int64_t sRz,
                                    float *C, int64_t rows, int64_t inner, int64_t cols,
                                    int64_t p, cudaStream_t st, void *img = nullptr,
                                    size_t img_bytes = 0);
// Batched facewise product C_t = A_t B_t (Def. 2.3).
cudaError_t launch_facewise_gemm(const float *A, const float *B, float *C, int64_t n1,
                                 int64_t m, int64_t n2, int64_t p, cudaStream_t st,
                                 void *img = nullptr, size_t img_bytes = 0);

// ---------------------------------------------------------------- Jacobi
struct JacobiArgs {
  const float *X = nullptr;   // p faces, l x m row-major each (transform domain A-hat)
  float *W = nullptr;         // p * b * a_pad: rotated vectors (output / blocked store)
  float *sig = nullptr;       // p * b: singular values, descending per face
  int32_t *perm = nullptr;    // p * b: sorted position -> vector index
  int32_t *sweeps = nullptr;  // p: sweeps used per face
  int32_t *status = nullptr;  // device status word
  int64_t l = 0, m = 0, p = 0;
  int32_t max_sweeps = 30;
  float tol = 0.f;            // rotation threshold on |cos|
  int64_t key_l = 0, key_m = 0;   // slice shape for registered launch shapes (0: l, m)
  // jacobi_aux_bytes(p) of workspace for the device-wide kernel that takes
  // slices too large for one CTA's shared memory; nullptr (or allow_grid =
  // false, e.g. for launches that run concurrently with other Jacobi launches)
  // keeps such slices on the single-CTA block-cyclic kernel
  int32_t *aux = nullptr;
  bool allow_grid = true;
};
int64_t jacobi_apad(int64_t l, int64_t m);
size_t jacobi_aux_bytes(int64_t p);
constexpr int JACOBI_GRID_MAX_SWEEPS = 64;   // sweep cap of the device-wide kernel
// register (C >= 1) or remove (C = 0) the Jacobi launch shape for l x m slices, p of them
bool set_jacobi_shape(int64_t l, int64_t m, int64_t p, int C, int GW);
cudaError_t launch_jacobi(const JacobiArgs &a, cudaStream_t st);

// ---------------------------------------------------------------- select (Alg. 4.2)
struct SelectArgs {
  const float *sig;        // p x b, descending per face
  int64_t p, b;
  double gamma;
  double *keys_sorted;     // p*b, scratch
  int32_t *rank;           // p*b, scratch: global position of (t, j)
  int32_t *rho;            // p out
  int64_t *offs;           // p+1 out
  double *scal;            // scal[0] = kept2, scal[1] = total2, scal[2] = K (as double)
  int64_t *K;              // out
};
cudaError_t launch_select(const SelectArgs &a, cudaStream_t st);

// ---------------------------------------------------------------- factors / rebuild
// ---------------------------------------------------------------- QR with column pivoting
// Preconditioner of the Jacobi SVD: for each slice, the b = min(l, m) vectors
// (rows if l <= m, else columns) as columns of Y: Y P = Q R.  R (p * b * b,
// row-major upper triangular) becomes the Jacobi input; qperm[t * b + j] is the
// original index of the vector in pivoted position j.  Q is not formed.
struct QrArgs {
  const float *X;
  float *R;
  int32_t *qperm;
  int64_t l, m, p;
};
bool qrcp_fits(int64_t l, int64_t m);   // the slice fits the kernel's shared memory
cudaError_t launch_qrcp(const QrArgs &a, cudaStream_t st);
struct FactorArgs {
  const float *X;          // A-hat, p faces l x m
  const float *W;          // converged vectors, p * b * a_pad
  const float *sig;        // p * b sorted
  const int32_t *perm;     // p * b
  int64_t l, m, p, b, a_pad;
  int64_t kfix;            // fixed rank (tsvdq) or 0 -> ragged from rho/offs
  const int32_t *rho;      // ragged ranks (tsvdqII) or nullptr
  const int64_t *offs;     // ragged offsets or nullptr
  float *Uh, *s, *Vh;      // outputs (fixed: p x l x k etc.; ragged: packed)
  float *Ahk;              // rebuilt transform-domain tensor p x l x m
  double *kept_partial;    // per face kept sigma^2 (FP64) -> used for trunc report
  double *disc_partial;    // per face discarded sigma^2
  // QR-preconditioned Jacobi (launch_qrcp): W holds the rotated rows of R (length
  // b, a_pad = jacobi_apad(b, b)); the orthonormal side is then the short one,
  // u_q[qperm[j]] = W_q[j] / sigma_q, and the long side is X^T u_q / sigma_q.
  const int32_t *qperm = nullptr;
};
cudaError_t launch_factors(const FactorArgs &a, cudaStream_t st);

// ---------------------------------------------------------------- complex Q (pp_complex.cu)
// Real matrices from a complex Q (n x p, interleaved): Pim (p x n) = -Im(Q)^T,
// Bre (n x 2p) = [Re Q | -Im Q], Bim (n x 2p) = [Im Q | Re Q].
cudaError_t launch_qc_build(const float *Qf, int64_t n, int64_t p, float *Pim, float *Bre,
                            float *Bim, cudaStream_t st);
// PP_ENOTORTHO into *status when some |(Q^H Q - I)(i, j)| > tol
cudaError_t launch_qc_check(const float *Qf, int64_t n, int64_t p, float tol, int32_t *status,
                            cudaStream_t st);
struct CJacobiArgs {
  const float *Xre, *Xim;     // p complex slices l x m, planar
  float2 *W;                  // p * b * a_pad converged vectors
  float *sig;                 // p * b, descending per slice
  int32_t *perm;              // p * b: sorted position -> vector index
  int32_t *sweeps;            // p
  int32_t *status;
  int64_t l, m, p;
  int a_pad;                  // cjacobi_apad(l, m)
  int32_t max_sweeps;
  float tol;
};
int64_t cjacobi_apad(int64_t l, int64_t m);
size_t cjacobi_smem(int64_t l, int64_t m);   // the slice must fit one CTA's shared memory
cudaError_t launch_cjacobi(const CJacobiArgs &a, cudaStream_t st);
struct CFactorArgs {
  const float *Xre, *Xim;     // A-hat, planar
  const float2 *W;
  const float *sig;
  const int32_t *perm;
  int64_t l, m, p, b, a_pad;
  int64_t kfix;               // fixed rank, or 0 -> ragged from rho / offs
  const int32_t *rho;
  const int64_t *offs;
  float2 *Uh, *Vh;            // complex factors (interleaved), layouts as the real ones
  float *s;
  float *Ahk;                 // rebuilt transform domain, planar stacked (2 p l m), or nullptr
  double *kept_partial, *disc_partial;
};
cudaError_t launch_cfactors(const CFactorArgs &a, cudaStream_t st);
// C_t = A_t B_t (complex, planar stacked operands: p real slices then p imaginary)
cudaError_t launch_cfacewise(const float *A, const float *B, float *C, int64_t n1, int64_t m,
                             int64_t n2, int64_t p, cudaStream_t st);
// ---------------------------------------------------------------- reductions
// partials[blk] = sum of x^2 over a fixed grid; returns the number of partials.
cudaError_t launch_sumsq(const float *x, int64_t n, double *partials, int *n_partials,
                         cudaStream_t st);
int64_t sumsq_max_partials();
// out[0] = sum of partials[0..n) in a fixed order.
cudaError_t launch_sum_partials(const double *partials, int n_partials, double *out,
                                cudaStream_t st);
cudaError_t launch_check_q(const float *Q, int64_t n, int64_t p, float tol, int32_t *status,
                           cudaStream_t st);
cudaError_t launch_check_finite(const float *x, int64_t n, int32_t *status, cudaStream_t st);

// ---------------------------------------------------------------- HOSVD (Sec. 4.2)
int64_t gram_groups(int64_t n);
// G (d x d) = Gram of the mode-`mode` unfolding (1: d = l, 2: d = m) of A (n slices
// l x m); part holds gram_groups(n) partial d x d matrices.
cudaError_t launch_gram(const float *A, int64_t l, int64_t m, int64_t n, int mode, float *part,
                        float *G, cudaStream_t st);
// P (d x d) = U U^T for U d x k row-major.
cudaError_t launch_projector(const float *U, int64_t d, int64_t k, float *P, cudaStream_t st);

// U3 builder epilogue (n <= 768): Q (n x p) = V, trailing zero columns (zero
// eigenvalues) completed to an orthonormal basis, each column's largest-magnitude
// entry made positive, lambda (p, may be null) = s, rep (may be null) from the Gram's
// trace and the kept eigenvalues (Cor. 4.1).
cudaError_t launch_u3_finish(const float *V, const float *s, const float *G, int64_t n, int64_t p,
                             float *Q, float *lambda, int32_t *status, const int32_t *sweeps,
                             pp_report *rep, cudaStream_t st);
struct HosvdReportArgs {
  pp_hosvd_report *rep;
  const int32_t *status;
  const int32_t *sweeps;
  int64_t p, k1, k2, k;
  const double *normA2, *normAh2, *err2_tsvdq, *err2_hosvd;
};
cudaError_t launch_hosvd_report(const HosvdReportArgs &a, cudaStream_t st);

struct ReportArgs {
  pp_report *rep;
  const int32_t *status;
  const int32_t *sweeps;
  int64_t p;
  const double *normA2, *normAh2, *err2;   // scalars (device)
  const double *kept_partial, *disc_partial;  // per face (trunc) or nullptr
  const double *sel_scal;                     // select scalars (tsvdqII) or nullptr
  const int64_t *K;
  int64_t kappa_fixed;                        // k*p for trunc, -1 for ragged (from offs)
  const int64_t *offs;
  // energies still as partial sums: when parts[i] is set the report kernel sums
  // them (the same fixed order as launch_sum_partials), uses the sum in place of
  // normA2 / normAh2 / err2 (i = 0, 1, 2) and stores it to sums[i]
  const double *parts[3] = {nullptr, nullptr, nullptr};
  int nparts[3] = {0, 0, 0};
  double *sums = nullptr;
};
cudaError_t launch_report(const ReportArgs &a, cudaStream_t st);

}  // namespace pp
