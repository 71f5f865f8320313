/*
 * pprod.h -- C ABI of the GB300 (sm_103a) projected tensor-tensor product
 * library: the projected t-SVD hot path of Keegan & Newman, "Projected
 * Tensor-Tensor Products for Efficient Computation of Optimal Multiway Data
 * Representations" (arXiv 2409.19402).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Tensors.  An n1 x n2 x n3 tensor T is stored frontal-slice-major in FP32:
 *   entry (i, j, t) (0-based) at T[(t*n1 + i)*n2 + j].
 * Frontal slice t is a contiguous row-major n1 x n2 matrix and the mode-3
 * unfolding T_(3) (Def. 2.1) is the row-major n3 x (n1*n2) matrix at the same
 * address (pixel order (i, j) row-major instead of the paper's column-major
 * J(i,j); the mode-3 product acts tube by tube, so this changes nothing).
 * This is a C-contiguous PyTorch tensor of shape (n3, n1, n2).
 *
 * Q.  The transformation is a real n x p matrix with orthonormal columns
 * (Q in St_{n,p}, Sec. 3), row-major FP32 (Q[s*p + t]).  With p = n and Q
 * square orthogonal every call computes the invertible *M form (Def. 2.4,
 * M = Q^T).  Complex Q (Q^H Q = I, e.g. rows of the DFT) with real data is
 * taken by the separate *_c entry points below.
 *
 * Pointers.  Every array argument is a DEVICE pointer, unless stated
 * otherwise, owned by the caller: the library never allocates or frees
 * device memory (its one fixed device array, PP_NOALLOC_SCRATCH_BYTES, is
 * part of its loaded module).  Inputs are read only.  Outputs must not alias inputs.
 * Calls needing scratch take a caller-allocated device workspace of at least
 * pp_workspace_bytes(op, shape) bytes, 256-byte aligned.
 *
 * Execution.  Every call is asynchronous on `stream` (a cudaStream_t passed
 * as void*; NULL = legacy default stream) and returns after enqueueing.
 * Results, including the device-side pp_report, are valid after the stream
 * is synchronised.  The call makes no host<->device copies and no stream or
 * device synchronisation.
 *
 * Errors.  Argument errors the host can see (bad sizes, NULL pointers, a
 * workspace that is too small, gamma outside (0, 1]) return a nonzero
 * pp_status before anything is enqueued.  A failed kernel launch returns
 * PP_ECUDA.  Conditions only the device can see (Q not orthonormal, a
 * non-finite input, Jacobi not converged within the sweep cap) are written to
 * pp_report.status; the outputs are then unspecified.  Nothing in the library
 * aborts, exits or traps.
 */
#ifndef PPROD_H
#define PPROD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Symbols of this ABI are the only ones the shared library exports. */
#if defined(__GNUC__)
#define PP_API __attribute__((visibility("default")))
#else
#define PP_API
#endif

typedef enum pp_status {
    PP_OK = 0,
    PP_EINVAL = 1,      /* bad scalar argument or NULL pointer                 */
    PP_ESHAPE = 2,      /* inconsistent or out-of-range sizes                 */
    PP_ENOTORTHO = 3,   /* device: max |Q^T Q - I| above opts->q_tol           */
    PP_ENONFINITE = 4,  /* device: NaN/Inf in the input tensor                 */
    PP_ENOCONV = 5,     /* device: Jacobi did not converge within max_sweeps   */
    PP_ETIMEOUT = 6,    /* device: a bounded wait gave up                      */
    PP_EWORKSPACE = 7,  /* workspace NULL, misaligned or smaller than needed   */
    PP_ECUDA = 8,       /* a CUDA launch or runtime call failed                */
    PP_ENOSYS = 9       /* requested variant not built                         */
} pp_status;

/* Operation selector for pp_workspace_bytes. */
typedef enum pp_op {
    PP_OP_MODE3 = 0,
    PP_OP_FACEWISE = 1,
    PP_OP_PPROD = 2,
    PP_OP_TSVDQ = 3,
    PP_OP_TSVDQII = 4,
    PP_OP_HOSVD = 5,
    PP_OP_PPROD_BWD = 6,
    PP_OP_U3 = 7,
    PP_OP_PPROD_C = 8,
    PP_OP_TSVDQ_C = 9,
    PP_OP_TSVDQII_C = 10
} pp_op;

/* Problem sizes for pp_workspace_bytes.  Fields an op does not use are
 * ignored.  l x m x n is the tensor A (n frontal slices), p the projection
 * dimension, k the fixed truncation, n2 the second dimension of B in pprod. */
typedef struct pp_shape {
    int64_t l, m, n, p, k, n2;
} pp_shape;

/* Options; pass NULL for the defaults shown. */
typedef struct pp_opts {
    int32_t max_sweeps;   /* Jacobi sweep cap (default 30)                         */
    int32_t check_q;      /* nonzero: device check max|Q^T Q - I| <= q_tol (def 0)  */
    float q_tol;          /* orthonormality tolerance (default 1e-5)                */
    int32_t check_finite; /* nonzero: device scan of A for NaN/Inf (default 0)      */
    float jacobi_tol;     /* rotation threshold on |cos| (0 = sqrt(len) * 2^-24)    */
    int32_t precond;      /* QR preconditioning of the facewise Jacobi SVD: >= 0 on  */
                          /* where the slice fits its kernel (default), < 0 off     */
    int32_t reserved[3];
} pp_opts;

/* Device-written report of a decomposition call.  Energies are sums of FP32
 * partial sums over at most 16 terms (relative error <= 16 * 2^-24), carried
 * beyond that without rounding loss (FP32 pairs, then FP64); the rank-deciding
 * energies kept2 / discarded2 are FP64 sums of FP64 sigma^2. */
typedef struct pp_report {
    int32_t status;       /* PP_OK or a device-detected pp_status                  */
    int32_t sweeps;       /* largest Jacobi sweep count over the p slices          */
    int64_t K;            /* Alg. 4.2 energy index (0 for tsvdq_trunc)             */
    int64_t kappa;        /* implicit rank sum_i rho_i (Def. 4.4); k*p for trunc    */
    double normA2;        /* |A|_F^2                                               */
    double normAh2;       /* |A x_3 Q^T|_F^2, the transform-domain energy           */
    double kept2;         /* sum of retained sigma^2                               */
    double discarded2;    /* sum of discarded sigma^2 (Eckart-Young term, Thm 4.2) */
    double err2;          /* |A - A_k|_F^2 computed from A_k (only if computed)     */
    double proj_err2;     /* |A|^2 - |A x_3 Q^T|^2: projection error of Thm 4.2,    */
                          /* exact only for orthonormal Q; suffers cancellation    */
} pp_report;

/* Device-written report of hosvd_compare. */
typedef struct pp_hosvd_report {
    int32_t status;       /* PP_OK or a device-detected pp_status                  */
    int32_t sweeps;       /* largest Jacobi sweep count over the p slices          */
    int64_t k1, k2, k;    /* HOSVD ranks (k1, k2, p) and the *Q-SVD rank min(k1,k2) */
    double normA2;        /* |A|_F^2                                               */
    double err2_hosvd;    /* |A - A_(k1,k2,p)|_F^2, truncated HOSVD with U3 = Q     */
    double err2_tsvdq;    /* |A - A_k|_F^2, truncated *Q-SVD with k = min(k1, k2)  */
    double proj_err2;     /* |A|^2 - |A x_3 Q^T|^2 (common projection error)       */
} pp_hosvd_report;

/* Human-readable name of a status code (static string). */
PP_API const char *pp_status_str(int32_t status);

/* Library version string, e.g. "pprod-gb300 0.1 sm_103a". */
PP_API const char *pp_version(void);

/* Workspace bytes needed by `op` at `shape` (0 if none).  Returns 0 and sets
 * nothing for invalid shapes; the entry point itself reports the error. */
PP_API size_t pp_workspace_bytes(int32_t op, const pp_shape *shape);

/*
 * Mode-3 product with Q or Q^T (Def. 2.2; the transform and reverse
 * transform of Def. 3.1 / Alg. 4.1 steps 2 and 4).
 *   transpose == 0:  Y = X x_3 Q^T   X is l x m x n, Y is l x m x p
 *   transpose == 1:  Y = X x_3 Q     X is l x m x p, Y is l x m x n
 * i.e. Y(i,j,t) = sum_s M(t,s) X(i,j,s) with M = Q^T or Q.  FP32 in/out,
 * FP32 accumulation in the 3-pass split-TF32 tensor-core path.  No workspace.
 */
PP_API pp_status pprod_mode3(const float *X, int64_t l, int64_t m, int64_t n,
                      const float *Q, int64_t p, int32_t transpose, float *Y,
                      void *stream);

/*
 * Facewise product (Def. 2.3): Ch(:,:,t) = Ah(:,:,t) Bh(:,:,t), t < p.
 * Ah is n1 x m x p, Bh is m x n2 x p, Ch is n1 x n2 x p.  No workspace.
 */
PP_API pp_status pprod_facewise(const float *Ah, const float *Bh, int64_t n1, int64_t m,
                         int64_t n2, int64_t p, float *Ch, void *stream);

/*
 * Projected product (Def. 3.1): C = [(A x_3 Q^T) ^ (B x_3 Q^T)] x_3 Q.
 * A is n1 x m x n, B is m x n2 x n, Q is n x p, C is n1 x n2 x n.
 * Workspace: pp_workspace_bytes(PP_OP_PPROD, {l=n1, m=m, n=n, p=p, n2=n2}):
 * the transform-domain A-hat, B-hat, C-hat, the tf32 images of Q^T and Q
 * (each built once per call) and a region for the facewise operands' images
 * (at most 32 MB or one face's image; the faces then run in groups).
 */
PP_API pp_status pprod(const float *A, const float *B, const float *Q, int64_t n1,
                int64_t m, int64_t n2, int64_t n, int64_t p, float *C,
                void *ws, size_t ws_bytes, void *stream);

/*
 * Backward of the projected product C = A *Q B (Def. 3.1) for a loss L with
 * G = dL/dC, by the chain rule through its three steps (the transform-domain
 * tensors A-hat, B-hat, C-hat are recomputed, not stored):
 *   G-hat = G x_3 Q^T;  dA-hat_t = G-hat_t B-hat_t^T;  dB-hat_t = A-hat_t^T G-hat_t
 *   dA = dA-hat x_3 Q;  dB = dB-hat x_3 Q
 *   dQ_E = G_(3) C-hat_(3)^T + A_(3) dA-hat_(3)^T + B_(3) dB-hat_(3)^T   (n x p)
 *   dQ   = dQ_E - Q sym(Q^T dQ_E)  (projection on the tangent space of St_{n,p})
 * Sizes as in pprod; G, dA, dB have the shapes of C, A, B.  dQ_euclid and dQ
 * (n x p) may each be NULL.  Workspace: pp_workspace_bytes(PP_OP_PPROD_BWD,
 * {l = n1, m, n, p, n2}): as for pprod, plus G-hat, dA-hat, dB-hat, the
 * split-K parts of dQ_E and the image of the smaller operand of each A B^T.
 */
PP_API pp_status pprod_backward(const float *A, const float *B, const float *Q, const float *G,
                                int64_t n1, int64_t m, int64_t n2, int64_t n, int64_t p,
                                float *dA, float *dB, float *dQ_euclid, float *dQ,
                                void *ws, size_t ws_bytes, void *stream);

/*
 * Truncated *Q-SVD (Alg. 4.1; Def. 4.1; error terms of Thm. 4.2).
 *   A is l x m x n, Q is n x p (1 <= p <= n), 1 <= k <= min(l, m).
 * Outputs (transform-domain factors: the storage counted in Sec. 5.1.2):
 *   Uh  p x l x k  -- slice t is U-hat_k(:,:,t), row-major l x k
 *   s   p x k      -- singular values of slice t, descending
 *   Vh  p x m x k  -- slice t is V-hat_k(:,:,t), row-major m x k
 *   Ak  n x l x m  -- A_k = (U-hat_k S-hat_k V-hat_k^T) x_3 Q; may be NULL,
 *                     then A_k is formed in the workspace for rep->err2
 *   rep            -- device pointer, may be NULL
 * For a singular value that is exactly zero the matching short-side vector
 * is returned as zero.  Workspace: pp_workspace_bytes(PP_OP_TSVDQ, ...).
 */
PP_API pp_status tsvdq_trunc(const float *A, const float *Q, int64_t l, int64_t m,
                      int64_t n, int64_t p, int64_t k, float *Uh, float *s,
                      float *Vh, float *Ak, pp_report *rep, const pp_opts *opts,
                      void *ws, size_t ws_bytes, void *stream);

/*
 * *Q-SVDII (Alg. 4.2; Defs. 4.3-4.4; error terms of Thm. 4.4).
 *   A is l x m x n, Q is n x p, gamma in (0, 1].
 * All p*min(l,m) squared singular values are ordered globally (descending
 * sigma^2; ties by slice, then by index within the slice), K is the first
 * index whose cumulative energy reaches gamma * |A x_3 Q^T|^2 (the energy is
 * summed in FP64 from the FP32 singular values), and rho_t counts slice t's
 * values among the first K (K = 0 and rho = 0 when the energy is zero).
 * Outputs:
 *   rho     int32  p       per-slice ranks (the *Q-multirank kept)
 *   offs    int64  p+1     offs[t] = sum_{t'<t} rho_t', offs[p] = kappa
 *   Uh_pk   float  capacity p*min(l,m)*l: slice t's l x rho_t block
 *                  (row-major) starts at l*offs[t]
 *   s_pk    float  capacity p*min(l,m): slice t's rho_t values at offs[t]
 *   Vh_pk   float  capacity p*min(l,m)*m: slice t's m x rho_t block at m*offs[t]
 *   Ak      float  n x l x m (may be NULL), rep (device, may be NULL)
 * Workspace: pp_workspace_bytes(PP_OP_TSVDQII, ...).
 */
PP_API pp_status tsvdqII(const float *A, const float *Q, int64_t l, int64_t m,
                  int64_t n, int64_t p, double gamma, int32_t *rho,
                  int64_t *offs, float *Uh_pk, float *s_pk, float *Vh_pk,
                  float *Ak, pp_report *rep, const pp_opts *opts, void *ws,
                  size_t ws_bytes, void *stream);

/*
 * Truncated HOSVD against the *Q-SVD (Sec. 4.2, Thm. 4.6).
 *   A is l x m x n, Q is n x p (the mode-3 factor U3), 1 <= k1 <= l, 1 <= k2 <= m.
 * U1, U2 are the leading k1 / k2 eigenvectors of the Gram matrices of the
 * mode-1 / mode-2 unfoldings (eq. modek_svd); the HOSVD approximation is
 * A_(k1,k2,p) = A x_1 U1U1^T x_2 U2U2^T x_3 QQ^T.  The *Q-SVD (Alg. 4.1) is run
 * with k = min(k1, k2) on the same Q; Thm. 4.6 states err2_tsvdq <= err2_hosvd
 * when Q = U3(:, 1:p).  Ak_hosvd (n x l x m) may be NULL; rep (device) receives
 * both squared errors.  Workspace: pp_workspace_bytes(PP_OP_HOSVD, {l, m, n, p,
 * k = k1, n2 = k2}).
 */
PP_API pp_status hosvd_compare(const float *A, const float *Q, int64_t l, int64_t m,
                               int64_t n, int64_t p, int64_t k1, int64_t k2,
                               float *Ak_hosvd, pp_hosvd_report *rep,
                               const pp_opts *opts, void *ws, size_t ws_bytes,
                               void *stream);

/*
 * Matched-storage HOSVD truncation (Sec. 5.3, the storage equations that fix
 * the HOSVD rank k2 from the *Q-SVD truncation k).  Returns in *k2 the largest
 * integer k2 >= 1 whose truncated HOSVD costs no more storage than the
 * truncated *Q-SVD with truncation k (both with the n x p factor Q / U3):
 *   variant 0, multirank (l, k2, p):   l k2 p + l^2 + m k2 + n p <= k (l + m) p + n p
 *   variant 1, multirank (k2, k2, p):  k2^2 p + l k2 + m k2 + n p <= k (l + m) p + n p
 * i.e. the equations solved for k2 and rounded down, capped at m (variant 0)
 * or min(l, m) (variant 1).  *k2 = 0 when no k2 >= 1 fits.  Host-only: no
 * device work.  PP_EINVAL for NULL k2 or another variant; PP_ESHAPE unless
 * 1 <= p <= n and 1 <= k <= min(l, m).  The *Q-SVDII energy with the same
 * error bound (Thm. 4.5) is rep.kept2 / rep.normAh2 of the tsvdq_trunc report.
 */
PP_API pp_status pp_hosvd_matched_k2(int64_t l, int64_t m, int64_t n, int64_t p, int64_t k,
                                     int32_t variant, int64_t *k2);

/*
 * U3 transformation (Thm. 4.3, Cor. 4.1; the data-dependent Q of Sec. 5.1.1).
 *   A is l x m x n, 1 <= p <= n <= 768.
 * Q (n x p, row-major) receives the leading p left singular vectors of the
 * mode-3 unfolding A_(3), computed as eigenvectors of the n x n Gram matrix
 * A_(3) A_(3)^T (FP32 products over the l*m pixels, split into partial sums
 * that are added in a fixed order) by the one-sided Jacobi SVD of that
 * symmetric matrix; columns in descending eigenvalue order, each with the sign
 * that makes its largest-magnitude entry (the first on ties) positive.
 * lambda (p, FP32, may be NULL) receives the eigenvalues sigma_j(A_(3))^2.
 * rep (device, may be NULL): status, sweeps, K = kappa = p, normA2 = trace of
 * the Gram (|A|_F^2), normAh2 = kept2 = the sum of the p eigenvalues
 * (|A x_3 Q^T|_F^2 by Cor. 4.1), discarded2 = proj_err2 = normA2 - normAh2
 * (the projection error of Cor. 4.1; cancellation when it is small), err2 = 0.
 * opts: max_sweeps, jacobi_tol and check_finite apply.
 * Workspace: pp_workspace_bytes(PP_OP_U3, {l, m, n, p}).  PP_ENOSYS for n > 768.
 */
PP_API pp_status pprod_u3(const float *A, int64_t l, int64_t m, int64_t n, int64_t p, float *Q,
                          float *lambda, pp_report *rep, const pp_opts *opts, void *ws,
                          size_t ws_bytes, void *stream);

/*
 * Complex transformations (Sec. 3: Q in St_{n,p}(C), Q^H Q = I_p; the remark
 * after Def. 3.2: with Q = F(1:p,:)^H, rows of the unitary DFT, the product
 * of real tensors can be complex).  The data A, B are REAL (as in the paper's
 * experiments); Q is complex, interleaved (Q[2 (s p + t)] = Re Q(s, t),
 * Q[2 (s p + t) + 1] = Im Q(s, t), i.e. C99 float complex / torch.complex64,
 * row-major n x p).  The transform domain A x_3 Q^H is complex; its facewise
 * SVDs use a one-sided Jacobi with unitary 2 x 2 rotations (the pair's phase,
 * then the real rotation), singular values real and sorted descending.
 * Complex factors are interleaved with the layouts of the real entry points;
 * complex tensor outputs are given as separate real and imaginary arrays.
 * pp_report fields as for the real calls: err2 = |A - Re A_k|^2 + |Im A_k|^2.
 * opts: max_sweeps, jacobi_tol, check_finite (A) and check_q (max |Q^H Q - I|)
 * apply; precond does not (no QR preconditioner on this path).  Slices must
 * fit one CTA's shared memory: min(l,m) * roundup(max(l,m), 16) * 8 bytes
 * <= 200 KB, else PP_ENOSYS (the video-shaped 120 x 160 slices fit).
 *
 * pprod_c: C = A *Q B (Def. 3.1 over C), A n1 x m x n, B m x n2 x n real,
 *   C_re, C_im (n1 x n2 x n each).  Workspace PP_OP_PPROD_C {l = n1, m, n, p, n2}.
 * tsvdq_trunc_c: Alg. 4.1 over C; Uh (p, l, k) and Vh (p, m, k) complex,
 *   s (p, k); Ak_re / Ak_im both NULL or both given.  Workspace PP_OP_TSVDQ_C.
 * tsvdqII_c: Alg. 4.2 over C; rho, offs as tsvdqII; Uh_pk / Vh_pk complex
 *   packed blocks (capacity p min(l,m) l and p min(l,m) m complex), s_pk real.
 *   Workspace PP_OP_TSVDQII_C.
 */
PP_API pp_status pprod_c(const float *A, const float *B, const float *Q, int64_t n1, int64_t m,
                         int64_t n2, int64_t n, int64_t p, float *C_re, float *C_im, void *ws,
                         size_t ws_bytes, void *stream);
PP_API pp_status tsvdq_trunc_c(const float *A, const float *Q, int64_t l, int64_t m, int64_t n,
                               int64_t p, int64_t k, float *Uh, float *s, float *Vh,
                               float *Ak_re, float *Ak_im, pp_report *rep, const pp_opts *opts,
                               void *ws, size_t ws_bytes, void *stream);
PP_API pp_status tsvdqII_c(const float *A, const float *Q, int64_t l, int64_t m, int64_t n,
                           int64_t p, double gamma, int32_t *rho, int64_t *offs, float *Uh_pk,
                           float *s_pk, float *Vh_pk, float *Ak_re, float *Ak_im,
                           pp_report *rep, const pp_opts *opts, void *ws, size_t ws_bytes,
                           void *stream);

/*
 * Batched *Q-SVDII over independent tensors of uneven sizes (one item per
 * tensor: its own A, Q, sizes, outputs, report and workspace slice, exactly as
 * the arguments of tsvdqII).  Items are spread over a small set of auxiliary
 * streams that fork from `stream` and join back into it (events), so the
 * tensors' kernels overlap on the GPU; the call enqueues everything and
 * returns, with no allocation and no synchronisation, so the whole batch can
 * be captured into one CUDA graph from `stream` and replayed.  All items are
 * validated on the host before anything is enqueued (the first error is
 * returned).  The auxiliary streams and events are created once per device on
 * first use (make that first call outside any capture); concurrent batched
 * calls on one device must be serialised by the caller.
 */
typedef struct pp_batch_item {
    const float *A;
    const float *Q;
    int64_t l, m, n, p;
    int32_t *rho;
    int64_t *offs;
    float *Uh_pk, *s_pk, *Vh_pk;
    float *Ak;            /* may be NULL */
    pp_report *rep;       /* may be NULL */
    void *ws;
    size_t ws_bytes;
} pp_batch_item;

PP_API pp_status tsvdqII_batched(const pp_batch_item *items, int64_t count, double gamma,
                                 const pp_opts *opts, void *stream);

/*
 * tsvdqII_noalloc: the same computation as tsvdqII for callers that cannot
 * allocate device memory (no counterpart in the paper; it exists for callers
 * whose device memory belongs to another allocator, latency-critical loops
 * that forbid allocation after start-up because allocation can synchronise
 * the device, and foreign-language bindings that only pass pointers they own).
 * The caller passes inputs and outputs exactly as for tsvdqII but no
 * workspace: the library uses one fixed device array of
 * PP_NOALLOC_SCRATCH_BYTES bytes, held on every GPU that loads the library
 * until the process exits.  Shapes whose tsvdqII workspace exceeds it return
 * PP_EWORKSPACE before anything is enqueued (the video-shaped 120 x 160 x 300,
 * p = 50 problem needs about 14.8 MB and fits); argument errors are checked
 * first, in tsvdqII's order, and get tsvdqII's status.
 * Every call looks up the array's device address on the current device; the
 * first call on a device may load the library's device module, so make it
 * before any stream capture.  Calls never allocate or free memory.  All calls
 * on a device share the array and it keeps the last call's contents (each
 * call resets what must start at zero): calls that may overlap on the GPU
 * (unordered streams) race and must be serialised by the caller.
 */
#define PP_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)
PP_API pp_status tsvdqII_noalloc(const float *A, const float *Q, int64_t l, int64_t m,
                                 int64_t n, int64_t p, double gamma, int32_t *rho,
                                 int64_t *offs, float *Uh_pk, float *s_pk, float *Vh_pk,
                                 float *Ak, pp_report *rep, const pp_opts *opts,
                                 void *stream);

/*
 * Instrumentation for benchmarks (no counterpart in the paper).
 *
 * pp_set_stage_events: register up to 8 caller-created CUDA events
 * (cudaEvent_t passed as void*; NULL/0 disables).  While registered,
 * tsvdq_trunc and tsvdqII record events[i] on their stream at stage
 * boundaries: 0 entry, 1 after the projection and energies, 2 after the
 * facewise Jacobi SVD, 3 after the global select (tsvdqII; repeated for
 * tsvdq_trunc), 4 after factors and rebuild, 5 after the back-projection and
 * report.  Process-wide state: not for concurrent use from several threads.
 *
 * pp_kernel_launches: number of kernels this library has launched so far in
 * the process (monotone counter).
 */
PP_API void pp_set_stage_events(void *const *events, int32_t n);
PP_API uint64_t pp_kernel_launches(void);

/*
 * pp_peak_probe: measure an arithmetic peak (instrumentation, no counterpart
 * in the paper).  kind 0: FP32 FMA throughput (a full-device grid of
 * independent register FMA chains, `reps` rounds); kind 1: tcgen05 kind::tf32
 * tensor throughput (one CTA per SM issuing `reps` M128 N256 K8 MMAs from
 * shared memory into TMEM).  Asynchronous on `stream`; the caller times it
 * with CUDA events.  *flops (host) receives the floating-point operations the
 * launch performs; a bounded wait that expires writes PP_ETIMEOUT to *status
 * (device pointer, may be NULL).  PP_EINVAL for another kind, reps < 1 or a
 * NULL flops.
 */
PP_API pp_status pp_peak_probe(int32_t kind, int64_t reps, double *flops, int32_t *status,
                               void *stream);

/*
 * Launch-shape tuning of the facewise Jacobi SVD (no counterpart in the paper).
 * For slices of l x m, p of them per call, use C CTAs per slice (C = 1: one
 * CTA per slice; 2..8: a thread-block cluster of C CTAs exchanging vector
 * blocks through distributed shared memory) and GW lanes per rotated pair (8,
 * 16 or 32).  A registered shape overrides the built-in choice when it can be
 * launched; C = 0 removes the entry.  Process-wide; returns PP_EINVAL for
 * unsupported values.  The Python autotuner (autotune.py) times the candidates
 * and registers the fastest.
 */
PP_API pp_status pp_set_jacobi_shape(int64_t l, int64_t m, int64_t p, int32_t C, int32_t GW);

#ifdef __cplusplus
}
#endif

#endif /* PPROD_H */
