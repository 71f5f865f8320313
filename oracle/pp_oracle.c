/*
 * pp_oracle.c -- plain FP64 CPU oracle for projected tensor-tensor products
 * (Keegan & Newman, "Projected Tensor-Tensor Products for Efficient
 * Computation of Optimal Multiway Data Representations", arXiv 2409.19402).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA path, and the CUDA path never calls
 * it.  Everything here is written for obviousness, not speed: loop nests in
 * the order of the paper's definitions, FP64 throughout, no blocking.
 *
 * Storage convention (shared by every function below).  An order-3 tensor
 * T in R^{n1 x n2 x n3} is stored frontal-slice-major: entry (i, j, t)
 * (0-based) sits at T[(t*n1 + i)*n2 + j].  Each frontal slice T(:,:,t) is a
 * contiguous row-major n1 x n2 matrix.  Matrices are row-major.
 *
 * Function -> passage it follows:
 *   or_mode3            Def. 2.2 (mode-3 product, via the mode-3 unfolding of Def. 2.1)
 *   or_facewise         Def. 2.3 (facewise product)
 *   or_qprod            Def. 3.1 (projected product A *Q B)
 *   or_mprod            Def. 2.4 (*M product with an explicit inverse)
 *   or_svd_jacobi       the matrix SVD used by Alg. 4.1 / Alg. 4.2 (the paper
 *                       leaves the method open; one-sided Hestenes Jacobi)
 *   or_tsvdq            Alg. 4.1 (truncated *Q-SVD) + Thm. 4.2 error terms
 *   or_select_energy    Alg. 4.2 global reordering, energy index K, ranks rho_i
 *   or_tsvdqII          Alg. 4.2 (*Q-SVDII) + Thm. 4.4 error terms
 *   or_sym_eig_jacobi   symmetric eigensolver for the mode-i factor matrices
 *   or_hosvd            truncated HOSVD of Sec. 4.2
 *   or_dct_q, or_householder_q   transformation matrices of Sec. 5.1.1
 *   or_qprod_grad       gradient of L = 1/2 |A *Q B - T|_F^2 with respect to A, B
 *                       and Q (Euclidean and projected on the tangent space of
 *                       the Stiefel manifold St_{n,p} of Sec. 3), by the chain
 *                       rule through the three steps of Def. 3.1
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <float.h>

typedef int64_t i64;

#define OR_OK 0
#define OR_EINVAL 1
#define OR_ENOCONV 5
#define OR_ENOMEM 9

/* entry (i,j,t) of an n1 x n2 x n3 tensor */
#define TIDX(i, j, t, n1, n2) ((((i64)(t)) * (n1) + (i)) * (n2) + (j))

/* ------------------------------------------------------------------ */
/* Def. 2.2: Y = X x_3 M = fold(M X_(3)), M is q x n3.                 */
/*   Y(i,j,t) = sum_{s=1..n3} M(t,s) X(i,j,s),  s ascending.            */
/* ------------------------------------------------------------------ */
void or_mode3(const double *X, i64 n1, i64 n2, i64 n3,
              const double *M, i64 q, double *Y)
{
    /* output slices are independent: with OpenMP (the multi-core baseline
       build only) they are shared out over threads; the arithmetic of each
       entry is the same loop in the same order either way */
#pragma omp parallel for schedule(static)
    for (i64 t = 0; t < q; ++t)
        for (i64 i = 0; i < n1; ++i)
            for (i64 j = 0; j < n2; ++j) {
                double acc = 0.0;
                for (i64 s = 0; s < n3; ++s)
                    acc += M[t * n3 + s] * X[TIDX(i, j, s, n1, n2)];
                Y[TIDX(i, j, t, n1, n2)] = acc;
            }
}

/* ------------------------------------------------------------------ */
/* Def. 2.3: (A ^ B)(:,:,i) = A(:,:,i) B(:,:,i);  A n1 x m x p,         */
/* B m x n2 x p, C n1 x n2 x p.                                         */
/* ------------------------------------------------------------------ */
void or_facewise(const double *A, const double *B, i64 n1, i64 m, i64 n2,
                 i64 p, double *C)
{
    for (i64 t = 0; t < p; ++t)
        for (i64 i = 0; i < n1; ++i)
            for (i64 j = 0; j < n2; ++j) {
                double acc = 0.0;
                for (i64 l = 0; l < m; ++l)
                    acc += A[TIDX(i, l, t, n1, m)] * B[TIDX(l, j, t, m, n2)];
                C[TIDX(i, j, t, n1, n2)] = acc;
            }
}

/* transpose of a rows x cols row-major matrix into cols x rows */
static void transpose(const double *M, i64 rows, i64 cols, double *Mt)
{
    for (i64 r = 0; r < rows; ++r)
        for (i64 c = 0; c < cols; ++c)
            Mt[c * rows + r] = M[r * cols + c];
}

/* ------------------------------------------------------------------ */
/* Def. 3.1: A *Q B = [(A x_3 Q^T) ^ (B x_3 Q^T)] x_3 Q, Q is n3 x p   */
/* with orthonormal columns (real case: Q^H = Q^T).                    */
/* ------------------------------------------------------------------ */
int or_qprod(const double *A, const double *B, const double *Q, i64 n1, i64 m,
             i64 n2, i64 n3, i64 p, double *C)
{
    double *Qt = malloc(sizeof(double) * p * n3);
    double *Ah = malloc(sizeof(double) * n1 * m * p);
    double *Bh = malloc(sizeof(double) * m * n2 * p);
    double *Ch = malloc(sizeof(double) * n1 * n2 * p);
    if (!Qt || !Ah || !Bh || !Ch) {
        free(Qt); free(Ah); free(Bh); free(Ch);
        return OR_ENOMEM;
    }
    transpose(Q, n3, p, Qt);                 /* Q^T is p x n3 */
    or_mode3(A, n1, m, n3, Qt, p, Ah);       /* A-hat = A x_3 Q^T */
    or_mode3(B, m, n2, n3, Qt, p, Bh);       /* B-hat = B x_3 Q^T */
    or_facewise(Ah, Bh, n1, m, n2, p, Ch);   /* facewise product   */
    or_mode3(Ch, n1, n2, p, Q, n3, C);       /* back: x_3 Q (n3 x p) */
    free(Qt); free(Ah); free(Bh); free(Ch);
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Def. 2.4: A *M B = ((A x_3 M) ^ (B x_3 M)) x_3 M^{-1}; the caller    */
/* supplies M (n3 x n3) and its inverse.                               */
/* ------------------------------------------------------------------ */
int or_mprod(const double *A, const double *B, const double *M,
             const double *Minv, i64 n1, i64 m, i64 n2, i64 n3, double *C)
{
    double *Ah = malloc(sizeof(double) * n1 * m * n3);
    double *Bh = malloc(sizeof(double) * m * n2 * n3);
    double *Ch = malloc(sizeof(double) * n1 * n2 * n3);
    if (!Ah || !Bh || !Ch) { free(Ah); free(Bh); free(Ch); return OR_ENOMEM; }
    or_mode3(A, n1, m, n3, M, n3, Ah);
    or_mode3(B, m, n2, n3, M, n3, Bh);
    or_facewise(Ah, Bh, n1, m, n2, n3, Ch);
    or_mode3(Ch, n1, n2, n3, Minv, n3, C);
    free(Ah); free(Bh); free(Ch);
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Matrix SVD by one-sided (Hestenes) Jacobi, FP64.                     */
/*                                                                      */
/* X is rows x cols (row-major), r = min(rows, cols).  The r vectors of */
/* length L = max(rows, cols) (columns of X if rows >= cols, else rows  */
/* of X) are made mutually orthogonal by plane rotations applied in     */
/* cyclic-by-rows order (pairs (j,k), j < k, j ascending then k        */
/* ascending).  For a pair with alpha = |w_j|^2, beta = |w_k|^2,         */
/* g = w_j . w_k the rotation is the symmetric 2x2 Schur rotation of    */
/* Golub & Van Loan (zeta = (beta-alpha)/(2g), t = sign(zeta)/(|zeta| + */
/* sqrt(1+zeta^2)), c = 1/sqrt(1+t^2), s = t c), applied as             */
/* w_j <- c w_j - s w_k, w_k <- s w_j + c w_k and to the accumulator Z. */
/* A pair counts as orthogonal when |g| <= L*eps*sqrt(alpha*beta); the  */
/* sweep loop stops after a sweep with no rotation, or fails with       */
/* OR_ENOCONV after max_sweeps sweeps.                                  */
/*                                                                      */
/* Result: sigma_j = |w_j|; long-side singular vector w_j / sigma_j     */
/* (zero when sigma_j = 0); short-side singular vector = row j of Z.    */
/* Then an explicit stable sort by sigma descending (ties keep the lower */
/* original index first).  Outputs: U rows x r, s r, V cols x r, each   */
/* row-major, so that X = U diag(s) V^T.                                 */
/* ------------------------------------------------------------------ */
int or_svd_jacobi(const double *X, i64 rows, i64 cols, double *U, double *s,
                  double *V, int max_sweeps, int *sweeps_out)
{
    const i64 r = rows < cols ? rows : cols;
    const i64 L = rows < cols ? cols : rows;
    const int tall = rows >= cols;           /* vectors are the columns */
    double *W = malloc(sizeof(double) * r * L);   /* W[j*L + e]         */
    double *Z = malloc(sizeof(double) * r * r);   /* Z[j*r + e]         */
    double *sig = malloc(sizeof(double) * r);
    i64 *order = malloc(sizeof(i64) * r);
    if (!W || !Z || !sig || !order) {
        free(W); free(Z); free(sig); free(order);
        return OR_ENOMEM;
    }
    for (i64 j = 0; j < r; ++j)
        for (i64 e = 0; e < L; ++e)
            W[j * L + e] = tall ? X[e * cols + j] : X[j * cols + e];
    for (i64 j = 0; j < r; ++j)
        for (i64 e = 0; e < r; ++e)
            Z[j * r + e] = (j == e) ? 1.0 : 0.0;

    const double tol = (double)L * DBL_EPSILON;
    int sweep = 0, converged = (r < 2);
    while (!converged && sweep < max_sweeps) {
        ++sweep;
        i64 rotations = 0;
        for (i64 j = 0; j < r - 1; ++j)
            for (i64 k = j + 1; k < r; ++k) {
                double *wj = W + j * L, *wk = W + k * L;
                double alpha = 0.0, beta = 0.0, g = 0.0;
                for (i64 e = 0; e < L; ++e) {
                    alpha += wj[e] * wj[e];
                    beta += wk[e] * wk[e];
                    g += wj[e] * wk[e];
                }
                if (g == 0.0 || fabs(g) <= tol * sqrt(alpha * beta))
                    continue;
                double zeta = (beta - alpha) / (2.0 * g);
                double t = (zeta >= 0.0 ? 1.0 : -1.0) /
                           (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double c = 1.0 / sqrt(1.0 + t * t);
                double sn = c * t;
                for (i64 e = 0; e < L; ++e) {
                    double a = wj[e], b = wk[e];
                    wj[e] = c * a - sn * b;
                    wk[e] = sn * a + c * b;
                }
                double *zj = Z + j * r, *zk = Z + k * r;
                for (i64 e = 0; e < r; ++e) {
                    double a = zj[e], b = zk[e];
                    zj[e] = c * a - sn * b;
                    zk[e] = sn * a + c * b;
                }
                ++rotations;
            }
        if (rotations == 0)
            converged = 1;
    }
    if (sweeps_out)
        *sweeps_out = sweep;
    if (!converged) {
        free(W); free(Z); free(sig); free(order);
        return OR_ENOCONV;
    }
    for (i64 j = 0; j < r; ++j) {
        double acc = 0.0;
        for (i64 e = 0; e < L; ++e)
            acc += W[j * L + e] * W[j * L + e];
        sig[j] = sqrt(acc);
        order[j] = j;
    }
    /* explicit stable insertion sort, descending sigma */
    for (i64 a = 1; a < r; ++a) {
        i64 cur = order[a];
        i64 b = a - 1;
        while (b >= 0 && sig[order[b]] < sig[cur]) {
            order[b + 1] = order[b];
            --b;
        }
        order[b + 1] = cur;
    }
    for (i64 q = 0; q < r; ++q) {
        const i64 j = order[q];
        const double sj = sig[j];
        s[q] = sj;
        for (i64 e = 0; e < L; ++e) {
            double y = sj > 0.0 ? W[j * L + e] / sj : 0.0;
            if (tall) U[e * r + q] = y; else V[e * r + q] = y;
        }
        for (i64 e = 0; e < r; ++e) {
            if (tall) V[e * r + q] = Z[j * r + e]; else U[e * r + q] = Z[j * r + e];
        }
    }
    free(W); free(Z); free(sig); free(order);
    return OR_OK;
}

/* Error / energy terms shared by Alg. 4.1 and Alg. 4.2 (Thm. 4.2, 4.4,
 * metric RE of Sec. 5.1.2).  All computed directly, not via identities. */
typedef struct {
    double normA2;      /* |A|_F^2                                   */
    double normAh2;     /* |A x_3 Q^T|_F^2 (transform-domain energy)  */
    double err2;        /* |A - A_k|_F^2, computed entrywise         */
    double discarded2;  /* sum of discarded sigma^2 (Eckart-Young)    */
    double proj_err2;   /* |A - A x_3 Q Q^T|_F^2, computed entrywise  */
    i64 K;              /* Alg. 4.2 energy index (0 for Alg. 4.1)     */
    i64 kappa;          /* implicit rank sum_i rho_i (Def. 4.4)       */
    int max_sweeps;     /* largest Jacobi sweep count over the faces  */
    int status;
} or_report;

static double sumsq(const double *x, i64 n)
{
    double acc = 0.0;
    for (i64 e = 0; e < n; ++e) acc += x[e] * x[e];
    return acc;
}

/* projection error |A - A x_3 QQ^T|_F^2 given A and A-hat */
static double projection_error2(const double *A, const double *Ah, const double *Q,
                                i64 l, i64 m, i64 n, i64 p)
{
    double *P = malloc(sizeof(double) * l * m * n);
    if (!P) return NAN;
    or_mode3(Ah, l, m, p, Q, n, P);          /* (A x_3 Q^T) x_3 Q */
    double acc = 0.0;
    for (i64 e = 0; e < l * m * n; ++e) {
        double d = A[e] - P[e];
        acc += d * d;
    }
    free(P);
    return acc;
}

/* ------------------------------------------------------------------ */
/* Alg. 4.1 (truncated *Q-SVD).  A is l x m x n, Q is n x p, 1<=k<=min(l,m).
 *   step 2: A-hat = A x_3 Q^T
 *   step 3: rank-k truncated SVD of each frontal slice of A-hat
 *   step 4: A_k = (U-hat_k S-hat_k V-hat_k^T) x_3 Q
 * Outputs (transform-domain factors, the storage the paper counts):
 *   Uh p x l x k, s p x k, Vh p x m x k (slice t holds U-hat_k(:,:,t) etc.),
 *   Ak n x l x m (may be NULL), rep.                                    */
/* ------------------------------------------------------------------ */
int or_tsvdq(const double *A, const double *Q, i64 l, i64 m, i64 n, i64 p,
             i64 k, int max_sweeps, double *Uh, double *s, double *Vh,
             double *Ak, or_report *rep)
{
    const i64 r = l < m ? l : m;
    memset(rep, 0, sizeof(*rep));
    if (k < 1 || k > r || p < 1 || p > n) { rep->status = OR_EINVAL; return OR_EINVAL; }
    double *Qt = malloc(sizeof(double) * p * n);
    double *Ah = malloc(sizeof(double) * l * m * p);
    double *Ahk = malloc(sizeof(double) * l * m * p);
    double *Uf = malloc(sizeof(double) * l * r);
    double *sf = malloc(sizeof(double) * r);
    double *Vf = malloc(sizeof(double) * m * r);
    double *Akl = malloc(sizeof(double) * l * m * n);
    if (!Qt || !Ah || !Ahk || !Uf || !sf || !Vf || !Akl) {
        free(Qt); free(Ah); free(Ahk); free(Uf); free(sf); free(Vf); free(Akl);
        rep->status = OR_ENOMEM;
        return OR_ENOMEM;
    }
    transpose(Q, n, p, Qt);
    or_mode3(A, l, m, n, Qt, p, Ah);                      /* step 2 */
    int st = OR_OK;
    for (i64 t = 0; t < p && st == OR_OK; ++t) {          /* step 3 */
        int sw = 0;
        st = or_svd_jacobi(Ah + t * l * m, l, m, Uf, sf, Vf, max_sweeps, &sw);
        if (sw > rep->max_sweeps) rep->max_sweeps = sw;
        if (st != OR_OK) break;
        for (i64 i = 0; i < l; ++i)
            for (i64 q = 0; q < k; ++q) Uh[(t * l + i) * k + q] = Uf[i * r + q];
        for (i64 j = 0; j < m; ++j)
            for (i64 q = 0; q < k; ++q) Vh[(t * m + j) * k + q] = Vf[j * r + q];
        for (i64 q = 0; q < k; ++q) s[t * k + q] = sf[q];
        for (i64 q = k; q < r; ++q) rep->discarded2 += sf[q] * sf[q];
        /* rebuild A-hat_k(:,:,t) = sum_{q<k} s_q u_q v_q^T */
        for (i64 i = 0; i < l; ++i)
            for (i64 j = 0; j < m; ++j) {
                double acc = 0.0;
                for (i64 q = 0; q < k; ++q) acc += Uf[i * r + q] * sf[q] * Vf[j * r + q];
                Ahk[(t * l + i) * m + j] = acc;
            }
    }
    if (st == OR_OK) {
        or_mode3(Ahk, l, m, p, Q, n, Akl);                /* step 4 */
        rep->normA2 = sumsq(A, l * m * n);
        rep->normAh2 = sumsq(Ah, l * m * p);
        double acc = 0.0;
        for (i64 e = 0; e < l * m * n; ++e) {
            double d = A[e] - Akl[e];
            acc += d * d;
        }
        rep->err2 = acc;
        rep->proj_err2 = projection_error2(A, Ah, Q, l, m, n, p);
        rep->kappa = k * p;
        if (Ak) memcpy(Ak, Akl, sizeof(double) * l * m * n);
    }
    rep->status = st;
    free(Qt); free(Ah); free(Ahk); free(Uf); free(sf); free(Vf); free(Akl);
    return st;
}

/* ------------------------------------------------------------------ */
/* Alg. 4.2 steps 4-7 on given singular values.  sig is p x r (row t =  */
/* the r singular values of frontal slice t, descending).               */
/*  - list every (sigma^2, t, j); sort by sigma^2 descending, ties by    */
/*    slice t ascending, then by j ascending (the permutation pi of      */
/*    eq. (4.x) "singvalreorder", made unique by this tie rule);         */
/*  - prefix sums c_1..c_N in that order, sequentially in FP64;          */
/*  - K = first index with c_K >= gamma * c_N (the ratio of step 5,      */
/*    written without a division); K = 0 when c_N = 0;                   */
/*  - rho_t = number of entries of slice t among the first K.            */
/* sigma^2 is formed in FP64 from the FP64 value given.                   */
/* ------------------------------------------------------------------ */
typedef struct { double key; i64 t; i64 j; } or_entry;

static int entry_before(const or_entry *a, const or_entry *b)
{
    if (a->key != b->key) return a->key > b->key;
    if (a->t != b->t) return a->t < b->t;
    return a->j < b->j;
}

static void merge_sort_entries(or_entry *x, or_entry *tmp, i64 n)
{
    if (n < 2) return;
    i64 h = n / 2;
    merge_sort_entries(x, tmp, h);
    merge_sort_entries(x + h, tmp, n - h);
    i64 a = 0, b = h, o = 0;
    while (a < h && b < n) tmp[o++] = entry_before(&x[b], &x[a]) ? x[b++] : x[a++];
    while (a < h) tmp[o++] = x[a++];
    while (b < n) tmp[o++] = x[b++];
    memcpy(x, tmp, sizeof(or_entry) * n);
}

int or_select_energy(const double *sig, i64 p, i64 r, double gamma,
                     i64 *K_out, int32_t *rho, double *kept2, double *total2)
{
    if (!(gamma > 0.0 && gamma <= 1.0)) return OR_EINVAL;
    const i64 N = p * r;
    or_entry *e = malloc(sizeof(or_entry) * (N > 0 ? N : 1));
    or_entry *tmp = malloc(sizeof(or_entry) * (N > 0 ? N : 1));
    if (!e || !tmp) { free(e); free(tmp); return OR_ENOMEM; }
    for (i64 t = 0; t < p; ++t)
        for (i64 j = 0; j < r; ++j) {
            double sv = sig[t * r + j];
            e[t * r + j].key = sv * sv;
            e[t * r + j].t = t;
            e[t * r + j].j = j;
        }
    merge_sort_entries(e, tmp, N);
    double cN = 0.0;
    for (i64 q = 0; q < N; ++q) cN += e[q].key;
    i64 K = 0;
    double c = 0.0;
    if (cN > 0.0) {
        const double thresh = gamma * cN;
        for (i64 q = 0; q < N; ++q) {
            c += e[q].key;
            if (c >= thresh) { K = q + 1; break; }
        }
        if (K == 0) { K = N; }   /* unreachable for gamma <= 1; kept for safety */
    }
    for (i64 t = 0; t < p; ++t) rho[t] = 0;
    double kept = 0.0;
    for (i64 q = 0; q < K; ++q) { rho[e[q].t] += 1; kept += e[q].key; }
    *K_out = K;
    if (kept2) *kept2 = kept;
    if (total2) *total2 = cN;
    free(e); free(tmp);
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Alg. 4.2 (*Q-SVDII).  Packed outputs: offs[t] = sum_{t'<t} rho_t';   */
/* slice t's factors are Uh_p[l*offs[t] ...] (l x rho_t row-major),     */
/* s_p[offs[t] ...] (rho_t), Vh_p[m*offs[t] ...] (m x rho_t row-major). */
/* Capacities: p*min(l,m)*l, p*min(l,m), p*min(l,m)*m.  sig_all (p x r, */
/* may be NULL) receives every singular value for the select tests.     */
/* ------------------------------------------------------------------ */
int or_tsvdqII(const double *A, const double *Q, i64 l, i64 m, i64 n, i64 p,
               double gamma, int max_sweeps, int32_t *rho, i64 *offs,
               double *Uh_p, double *s_p, double *Vh_p, double *Ak,
               double *sig_all, or_report *rep)
{
    const i64 r = l < m ? l : m;
    memset(rep, 0, sizeof(*rep));
    if (!(gamma > 0.0 && gamma <= 1.0) || p < 1 || p > n) {
        rep->status = OR_EINVAL;
        return OR_EINVAL;
    }
    double *Qt = malloc(sizeof(double) * p * n);
    double *Ah = malloc(sizeof(double) * l * m * p);
    double *Ahk = malloc(sizeof(double) * l * m * p);
    double *Uf = malloc(sizeof(double) * p * l * r);
    double *sf = malloc(sizeof(double) * p * r);
    double *Vf = malloc(sizeof(double) * p * m * r);
    double *Akl = malloc(sizeof(double) * l * m * n);
    if (!Qt || !Ah || !Ahk || !Uf || !sf || !Vf || !Akl) {
        free(Qt); free(Ah); free(Ahk); free(Uf); free(sf); free(Vf); free(Akl);
        rep->status = OR_ENOMEM;
        return OR_ENOMEM;
    }
    transpose(Q, n, p, Qt);
    or_mode3(A, l, m, n, Qt, p, Ah);                      /* step 2 */
    int st = OR_OK, msw = 0;
    /* step 3: the slices' SVDs are independent (shared out over threads in
       the OpenMP build; each slice's arithmetic is unchanged) */
#pragma omp parallel for schedule(dynamic) reduction(max : msw)
    for (i64 t = 0; t < p; ++t) {
        int sw = 0;
        const int e = or_svd_jacobi(Ah + t * l * m, l, m, Uf + t * l * r, sf + t * r,
                                    Vf + t * m * r, max_sweeps, &sw);
        if (sw > msw) msw = sw;
        if (e != OR_OK) {
#pragma omp critical
            st = e;
        }
    }
    rep->max_sweeps = msw;
    if (st == OR_OK) {
        i64 K = 0;
        double kept = 0.0, total = 0.0;
        st = or_select_energy(sf, p, r, gamma, &K, rho, &kept, &total);  /* steps 4-7 */
        rep->K = K;
        if (st == OR_OK) {
            offs[0] = 0;
            for (i64 t = 0; t < p; ++t) offs[t + 1] = offs[t] + rho[t];
            rep->kappa = offs[p];
            for (i64 t = 0; t < p; ++t) {                  /* step 8 */
                const i64 rt = rho[t], o = offs[t];
                for (i64 i = 0; i < l; ++i)
                    for (i64 q = 0; q < rt; ++q)
                        Uh_p[l * o + i * rt + q] = Uf[(t * l + i) * r + q];
                for (i64 j = 0; j < m; ++j)
                    for (i64 q = 0; q < rt; ++q)
                        Vh_p[m * o + j * rt + q] = Vf[(t * m + j) * r + q];
                for (i64 q = 0; q < rt; ++q) s_p[o + q] = sf[t * r + q];
                for (i64 q = rt; q < r; ++q) rep->discarded2 += sf[t * r + q] * sf[t * r + q];
                for (i64 i = 0; i < l; ++i)
                    for (i64 j = 0; j < m; ++j) {
                        double acc = 0.0;
                        for (i64 q = 0; q < rt; ++q)
                            acc += Uf[(t * l + i) * r + q] * sf[t * r + q] *
                                   Vf[(t * m + j) * r + q];
                        Ahk[(t * l + i) * m + j] = acc;
                    }
            }
            or_mode3(Ahk, l, m, p, Q, n, Akl);
            rep->normA2 = sumsq(A, l * m * n);
            rep->normAh2 = sumsq(Ah, l * m * p);
            double acc = 0.0;
            for (i64 e = 0; e < l * m * n; ++e) {
                double d = A[e] - Akl[e];
                acc += d * d;
            }
            rep->err2 = acc;
            rep->proj_err2 = projection_error2(A, Ah, Q, l, m, n, p);
            if (Ak) memcpy(Ak, Akl, sizeof(double) * l * m * n);
            if (sig_all) memcpy(sig_all, sf, sizeof(double) * p * r);
        }
    }
    rep->status = st;
    free(Qt); free(Ah); free(Ahk); free(Uf); free(sf); free(Vf); free(Akl);
    return st;
}

/* ------------------------------------------------------------------ */
/* Symmetric eigendecomposition G = E diag(w) E^T by the cyclic two-    */
/* sided Jacobi method (Golub & Van Loan, cyclic Jacobi with the same   */
/* symmetric 2x2 Schur rotation as above).  G is n x n symmetric.       */
/* Output: w descending, E n x n row-major with eigenvector q in column */
/* q, sign fixed so that the entry of largest magnitude is positive.    */
/* ------------------------------------------------------------------ */
int or_sym_eig_jacobi(const double *G, i64 n, double *w, double *E, int max_sweeps)
{
    double *S = malloc(sizeof(double) * n * n);
    double *Z = malloc(sizeof(double) * n * n);
    i64 *order = malloc(sizeof(i64) * n);
    double *d = malloc(sizeof(double) * n);
    if (!S || !Z || !order || !d) { free(S); free(Z); free(order); free(d); return OR_ENOMEM; }
    memcpy(S, G, sizeof(double) * n * n);
    for (i64 i = 0; i < n; ++i)
        for (i64 j = 0; j < n; ++j) Z[i * n + j] = (i == j) ? 1.0 : 0.0;
    /* converged when |offdiag(S)|_F <= n*eps*|diag(S)|_F */
    const double tol2 = ((double)n * DBL_EPSILON) * ((double)n * DBL_EPSILON);
    int converged = (n < 2), sweep = 0;
    while (!converged && sweep < max_sweeps) {
        ++sweep;
        double off = 0.0, diag = 0.0;
        for (i64 i = 0; i < n; ++i)
            for (i64 j = 0; j < n; ++j) {
                if (i == j) diag += S[i * n + j] * S[i * n + j];
                else off += S[i * n + j] * S[i * n + j];
            }
        if (off <= tol2 * diag || off == 0.0) { converged = 1; break; }
        for (i64 pp = 0; pp < n - 1; ++pp)
            for (i64 qq = pp + 1; qq < n; ++qq) {
                double apq = S[pp * n + qq];
                if (apq == 0.0) continue;
                double app = S[pp * n + pp], aqq = S[qq * n + qq];
                double tau = (aqq - app) / (2.0 * apq);
                double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t), sn = t * c;
                /* S <- J^T S J with J = [[c, s], [-s, c]] in the (pp, qq) plane */
                for (i64 k = 0; k < n; ++k) {        /* columns pp, qq */
                    double a = S[k * n + pp], b = S[k * n + qq];
                    S[k * n + pp] = c * a - sn * b;
                    S[k * n + qq] = sn * a + c * b;
                }
                for (i64 k = 0; k < n; ++k) {        /* rows pp, qq */
                    double a = S[pp * n + k], b = S[qq * n + k];
                    S[pp * n + k] = c * a - sn * b;
                    S[qq * n + k] = sn * a + c * b;
                }
                for (i64 k = 0; k < n; ++k) {        /* Z <- Z J */
                    double a = Z[k * n + pp], b = Z[k * n + qq];
                    Z[k * n + pp] = c * a - sn * b;
                    Z[k * n + qq] = sn * a + c * b;
                }
            }
    }
    if (!converged) {
        /* one last check after the final sweep */
        double off = 0.0, diag = 0.0;
        for (i64 i = 0; i < n; ++i)
            for (i64 j = 0; j < n; ++j) {
                if (i == j) diag += S[i * n + j] * S[i * n + j];
                else off += S[i * n + j] * S[i * n + j];
            }
        converged = off <= tol2 * diag || off == 0.0;
    }
    for (i64 i = 0; i < n; ++i) { d[i] = S[i * n + i]; order[i] = i; }
    for (i64 a = 1; a < n; ++a) {               /* stable sort, descending */
        i64 cur = order[a], b = a - 1;
        while (b >= 0 && d[order[b]] < d[cur]) { order[b + 1] = order[b]; --b; }
        order[b + 1] = cur;
    }
    for (i64 q = 0; q < n; ++q) {
        const i64 j = order[q];
        w[q] = d[j];
        i64 arg = 0;
        for (i64 k = 1; k < n; ++k)
            if (fabs(Z[k * n + j]) > fabs(Z[arg * n + j])) arg = k;
        const double sg = Z[arg * n + j] < 0.0 ? -1.0 : 1.0;
        for (i64 k = 0; k < n; ++k) E[k * n + q] = sg * Z[k * n + j];
    }
    free(S); free(Z); free(order); free(d);
    return converged ? OR_OK : OR_ENOCONV;
}

/* Gram matrix of the mode-d unfolding (d = 1, 2, 3) of an n1 x n2 x n3 tensor:
 * G = A_(d) A_(d)^T, of size n_d x n_d, computed entry by entry. */
void or_mode_gram(const double *A, i64 n1, i64 n2, i64 n3, int d, double *G)
{
    const i64 nd = d == 1 ? n1 : (d == 2 ? n2 : n3);
    for (i64 a = 0; a < nd; ++a)
        for (i64 b = 0; b < nd; ++b) G[a * nd + b] = 0.0;
    for (i64 t = 0; t < n3; ++t)
        for (i64 i = 0; i < n1; ++i)
            for (i64 j = 0; j < n2; ++j) {
                /* fibres along mode d are indexed by the other two indices */
                for (i64 b = 0; b < nd; ++b) {
                    i64 ii = i, jj = j, tt = t;
                    i64 a;
                    if (d == 1) { a = i; ii = b; }
                    else if (d == 2) { a = j; jj = b; }
                    else { a = t; tt = b; }
                    G[a * nd + b] += A[TIDX(i, j, t, n1, n2)] * A[TIDX(ii, jj, tt, n1, n2)];
                }
            }
}

/* ------------------------------------------------------------------ */
/* Truncated HOSVD (Sec. 4.2): U_d = leading k_d left singular vectors  */
/* of the mode-d unfolding (here: leading eigenvectors of A_(d)A_(d)^T)  */
/* for d = 1, 2; the mode-3 factor is the given U3 (n3 x k3).            */
/* Core G = A x_1 U1^T x_2 U2^T x_3 U3^T; A_k = G x_1 U1 x_2 U2 x_3 U3.  */
/* Returns |A - A_k|_F^2 in *err2 and A_k in Ak (may be NULL).            */
/* ------------------------------------------------------------------ */
int or_hosvd(const double *A, i64 n1, i64 n2, i64 n3, i64 k1, i64 k2,
             const double *U3, i64 k3, double *Ak, double *err2)
{
    if (k1 < 1 || k1 > n1 || k2 < 1 || k2 > n2 || k3 < 1 || k3 > n3) return OR_EINVAL;
    double *G1 = malloc(sizeof(double) * n1 * n1), *E1 = malloc(sizeof(double) * n1 * n1);
    double *G2 = malloc(sizeof(double) * n2 * n2), *E2 = malloc(sizeof(double) * n2 * n2);
    double *w1 = malloc(sizeof(double) * n1), *w2 = malloc(sizeof(double) * n2);
    double *T1 = malloc(sizeof(double) * k1 * n2 * n3);
    double *T2 = malloc(sizeof(double) * k1 * k2 * n3);
    double *C = malloc(sizeof(double) * k1 * k2 * k3);
    double *R3 = malloc(sizeof(double) * k1 * k2 * n3);
    double *R2 = malloc(sizeof(double) * k1 * n2 * n3);
    double *R1 = malloc(sizeof(double) * n1 * n2 * n3);
    int st = OR_OK;
    if (!G1 || !E1 || !G2 || !E2 || !w1 || !w2 || !T1 || !T2 || !C || !R3 || !R2 || !R1) {
        st = OR_ENOMEM;
        goto done;
    }
    or_mode_gram(A, n1, n2, n3, 1, G1);
    or_mode_gram(A, n1, n2, n3, 2, G2);
    st = or_sym_eig_jacobi(G1, n1, w1, E1, 100);
    if (st == OR_OK) st = or_sym_eig_jacobi(G2, n2, w2, E2, 100);
    if (st != OR_OK) goto done;
    /* T1 = A x_1 U1^T : (a, j, t) = sum_i U1(i,a) A(i,j,t) */
    for (i64 t = 0; t < n3; ++t)
        for (i64 a = 0; a < k1; ++a)
            for (i64 j = 0; j < n2; ++j) {
                double acc = 0.0;
                for (i64 i = 0; i < n1; ++i) acc += E1[i * n1 + a] * A[TIDX(i, j, t, n1, n2)];
                T1[TIDX(a, j, t, k1, n2)] = acc;
            }
    /* T2 = T1 x_2 U2^T : (a, b, t) = sum_j U2(j,b) T1(a,j,t) */
    for (i64 t = 0; t < n3; ++t)
        for (i64 a = 0; a < k1; ++a)
            for (i64 b = 0; b < k2; ++b) {
                double acc = 0.0;
                for (i64 j = 0; j < n2; ++j) acc += E2[j * n2 + b] * T1[TIDX(a, j, t, k1, n2)];
                T2[TIDX(a, b, t, k1, k2)] = acc;
            }
    /* core C = T2 x_3 U3^T : (a, b, c) = sum_t U3(t,c) T2(a,b,t) */
    for (i64 c = 0; c < k3; ++c)
        for (i64 a = 0; a < k1; ++a)
            for (i64 b = 0; b < k2; ++b) {
                double acc = 0.0;
                for (i64 t = 0; t < n3; ++t) acc += U3[t * k3 + c] * T2[TIDX(a, b, t, k1, k2)];
                C[TIDX(a, b, c, k1, k2)] = acc;
            }
    /* reconstruction: R3 = C x_3 U3, R2 = R3 x_2 U2, R1 = R2 x_1 U1 */
    for (i64 t = 0; t < n3; ++t)
        for (i64 a = 0; a < k1; ++a)
            for (i64 b = 0; b < k2; ++b) {
                double acc = 0.0;
                for (i64 c = 0; c < k3; ++c) acc += U3[t * k3 + c] * C[TIDX(a, b, c, k1, k2)];
                R3[TIDX(a, b, t, k1, k2)] = acc;
            }
    for (i64 t = 0; t < n3; ++t)
        for (i64 a = 0; a < k1; ++a)
            for (i64 j = 0; j < n2; ++j) {
                double acc = 0.0;
                for (i64 b = 0; b < k2; ++b) acc += E2[j * n2 + b] * R3[TIDX(a, b, t, k1, k2)];
                R2[TIDX(a, j, t, k1, n2)] = acc;
            }
    for (i64 t = 0; t < n3; ++t)
        for (i64 i = 0; i < n1; ++i)
            for (i64 j = 0; j < n2; ++j) {
                double acc = 0.0;
                for (i64 a = 0; a < k1; ++a) acc += E1[i * n1 + a] * R2[TIDX(a, j, t, k1, n2)];
                R1[TIDX(i, j, t, n1, n2)] = acc;
            }
    {
        double acc = 0.0;
        for (i64 e = 0; e < n1 * n2 * n3; ++e) {
            double dd = A[e] - R1[e];
            acc += dd * dd;
        }
        *err2 = acc;
    }
    if (Ak) memcpy(Ak, R1, sizeof(double) * n1 * n2 * n3);
done:
    free(G1); free(E1); free(G2); free(E2); free(w1); free(w2);
    free(T1); free(T2); free(C); free(R3); free(R2); free(R1);
    return st;
}

/* ------------------------------------------------------------------ */
/* Transformation matrices of Sec. 5.1.1.                               */
/* ------------------------------------------------------------------ */

/* Orthonormal DCT-II basis: C(t, s) = c_t cos(pi (2s+1) t / (2n)),
 * c_0 = sqrt(1/n), c_t = sqrt(2/n).  Q = C(1:p, :)^T, i.e. Q(s, t) = C(t, s),
 * Q is n x p row-major. */
void or_dct_q(i64 n, i64 p, double *Q)
{
    const double pi = 3.14159265358979323846;
    for (i64 s = 0; s < n; ++s)
        for (i64 t = 0; t < p; ++t) {
            double ct = t == 0 ? sqrt(1.0 / (double)n) : sqrt(2.0 / (double)n);
            Q[s * p + t] = ct * cos(pi * (double)(2 * s + 1) * (double)t / (2.0 * (double)n));
        }
}

/* Householder QR of the n x n matrix X (row-major); writes the first p
 * columns of the orthogonal factor into Q (n x p).  Columns are signed so
 * that R has a non-negative diagonal. */
int or_householder_q(const double *X, i64 n, i64 p, double *Q)
{
    double *R = malloc(sizeof(double) * n * n);
    double *H = malloc(sizeof(double) * n * n);   /* accumulated Q = H1 H2 ... */
    double *v = malloc(sizeof(double) * n);
    if (!R || !H || !v) { free(R); free(H); free(v); return OR_ENOMEM; }
    memcpy(R, X, sizeof(double) * n * n);
    for (i64 i = 0; i < n; ++i)
        for (i64 j = 0; j < n; ++j) H[i * n + j] = (i == j) ? 1.0 : 0.0;
    for (i64 c = 0; c < n; ++c) {
        double nrm = 0.0;
        for (i64 i = c; i < n; ++i) nrm += R[i * n + c] * R[i * n + c];
        nrm = sqrt(nrm);
        if (nrm == 0.0) continue;
        double alpha = R[c * n + c] >= 0.0 ? -nrm : nrm;
        for (i64 i = 0; i < n; ++i) v[i] = 0.0;
        for (i64 i = c; i < n; ++i) v[i] = R[i * n + c];
        v[c] -= alpha;
        double vv = 0.0;
        for (i64 i = c; i < n; ++i) vv += v[i] * v[i];
        if (vv == 0.0) continue;
        /* R <- (I - 2 v v^T / vv) R */
        for (i64 j = 0; j < n; ++j) {
            double dot = 0.0;
            for (i64 i = c; i < n; ++i) dot += v[i] * R[i * n + j];
            double f = 2.0 * dot / vv;
            for (i64 i = c; i < n; ++i) R[i * n + j] -= f * v[i];
        }
        /* H <- H (I - 2 v v^T / vv) */
        for (i64 i = 0; i < n; ++i) {
            double dot = 0.0;
            for (i64 k = c; k < n; ++k) dot += H[i * n + k] * v[k];
            double f = 2.0 * dot / vv;
            for (i64 k = c; k < n; ++k) H[i * n + k] -= f * v[k];
        }
    }
    for (i64 t = 0; t < p; ++t) {
        double sg = R[t * n + t] < 0.0 ? -1.0 : 1.0;
        for (i64 s = 0; s < n; ++s) Q[s * p + t] = sg * H[s * n + t];
    }
    free(R); free(H); free(v);
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Gradient of L = 1/2 |C - T|_F^2 with C = A *Q B (Def. 3.1), A n1 x m x n,
 * B m x n2 x n, Q n x p, by the chain rule through the three steps:
 *   A-hat = A x_3 Q^T, B-hat = B x_3 Q^T, C-hat = A-hat ^ B-hat, C = C-hat x_3 Q.
 * With G = C - T:
 *   G-hat = G x_3 Q^T                         (dL/dC-hat, since C_(3) = Q C-hat_(3))
 *   dA-hat_t = G-hat_t B-hat_t^T, dB-hat_t = A-hat_t^T G-hat_t
 *   dA = dA-hat x_3 Q, dB = dB-hat x_3 Q      (A-hat_(3) = Q^T A_(3))
 *   dQ_E = G_(3) C-hat_(3)^T + A_(3) dA-hat_(3)^T + B_(3) dB-hat_(3)^T
 *   dQ = dQ_E - Q sym(Q^T dQ_E), sym(M) = (M + M^T)/2 (tangent projection at Q)
 * Outputs dA (n x n1 x m storage), dB, dQE and dQ (n x p); returns L in *loss. */
int or_qprod_grad(const double *A, const double *B, const double *Q, const double *T,
                  i64 n1, i64 m, i64 n2, i64 n, i64 p, double *dA, double *dB,
                  double *dQE, double *dQ, double *loss)
{
    double *Qt = malloc(sizeof(double) * p * n);
    double *Ah = malloc(sizeof(double) * p * n1 * m), *Bh = malloc(sizeof(double) * p * m * n2);
    double *Ch = malloc(sizeof(double) * p * n1 * n2), *C = malloc(sizeof(double) * n * n1 * n2);
    double *G = malloc(sizeof(double) * n * n1 * n2), *Gh = malloc(sizeof(double) * p * n1 * n2);
    double *dAh = malloc(sizeof(double) * p * n1 * m), *dBh = malloc(sizeof(double) * p * m * n2);
    double *S = malloc(sizeof(double) * p * p);
    int st = OR_OK;
    if (!Qt || !Ah || !Bh || !Ch || !C || !G || !Gh || !dAh || !dBh || !S) { st = OR_ENOMEM; goto out; }
    transpose(Q, n, p, Qt);
    or_mode3(A, n1, m, n, Qt, p, Ah);
    or_mode3(B, m, n2, n, Qt, p, Bh);
    or_facewise(Ah, Bh, n1, m, n2, p, Ch);
    or_mode3(Ch, n1, n2, p, Q, n, C);
    {
        double l2 = 0.0;
        for (i64 e = 0; e < n * n1 * n2; ++e) { G[e] = C[e] - T[e]; l2 += G[e] * G[e]; }
        *loss = 0.5 * l2;
    }
    or_mode3(G, n1, n2, n, Qt, p, Gh);
    for (i64 t = 0; t < p; ++t) {
        for (i64 i = 0; i < n1; ++i)          /* dA-hat_t = G-hat_t B-hat_t^T */
            for (i64 l = 0; l < m; ++l) {
                double acc = 0.0;
                for (i64 j = 0; j < n2; ++j) acc += Gh[TIDX(i, j, t, n1, n2)] * Bh[TIDX(l, j, t, m, n2)];
                dAh[TIDX(i, l, t, n1, m)] = acc;
            }
        for (i64 l = 0; l < m; ++l)           /* dB-hat_t = A-hat_t^T G-hat_t */
            for (i64 j = 0; j < n2; ++j) {
                double acc = 0.0;
                for (i64 i = 0; i < n1; ++i) acc += Ah[TIDX(i, l, t, n1, m)] * Gh[TIDX(i, j, t, n1, n2)];
                dBh[TIDX(l, j, t, m, n2)] = acc;
            }
    }
    or_mode3(dAh, n1, m, p, Q, n, dA);
    or_mode3(dBh, m, n2, p, Q, n, dB);
    for (i64 s = 0; s < n; ++s)               /* dQ_E(s, t) */
        for (i64 t = 0; t < p; ++t) {
            double acc = 0.0;
            for (i64 e = 0; e < n1 * n2; ++e) acc += G[s * n1 * n2 + e] * Ch[t * n1 * n2 + e];
            for (i64 e = 0; e < n1 * m; ++e) acc += A[s * n1 * m + e] * dAh[t * n1 * m + e];
            for (i64 e = 0; e < m * n2; ++e) acc += B[s * m * n2 + e] * dBh[t * m * n2 + e];
            dQE[s * p + t] = acc;
        }
    for (i64 a = 0; a < p; ++a)               /* S = Q^T dQ_E */
        for (i64 b = 0; b < p; ++b) {
            double acc = 0.0;
            for (i64 s = 0; s < n; ++s) acc += Q[s * p + a] * dQE[s * p + b];
            S[a * p + b] = acc;
        }
    for (i64 s = 0; s < n; ++s)
        for (i64 t = 0; t < p; ++t) {
            double acc = 0.0;
            for (i64 a = 0; a < p; ++a) acc += Q[s * p + a] * 0.5 * (S[a * p + t] + S[t * p + a]);
            dQ[s * p + t] = dQE[s * p + t] - acc;
        }
out:
    free(Qt); free(Ah); free(Bh); free(Ch); free(C); free(G); free(Gh); free(dAh); free(dBh); free(S);
    return st;
}
