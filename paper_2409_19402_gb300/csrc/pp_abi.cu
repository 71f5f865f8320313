// pp_abi.cu -- the extern "C" entry points declared in include/pprod.h:
// argument validation, workspace carving and the stream-ordered launch
// sequence of each operation.  No entry point allocates, frees, copies to or
// from the host, or synchronises.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

#include "pp_internal.h"

namespace pp {
namespace {
std::atomic<uint64_t> g_launches{0};
}
void count_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }
}  // namespace pp

namespace {

// benchmark stage events (see pp_set_stage_events)
cudaEvent_t g_events[8];
int g_nevents = 0;

void stage(int i, cudaStream_t st) {
  if (i < g_nevents && g_events[i]) cudaEventRecord(g_events[i], st);
}

using pp::round_up;

// Bump allocator over the caller's workspace; with base == nullptr it only
// measures (used by pp_workspace_bytes).
struct Carve {
  char *base;
  size_t off = 0;
  explicit Carve(void *b) : base(static_cast<char *>(b)) {}
  template <class T>
  T *take(int64_t count) {
    off = (size_t)round_up((int64_t)off, 256);
    T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
    off += (size_t)count * sizeof(T);
    return p;
  }
};

constexpr int64_t MAX_LONG_SIDE = 768;   // longest slice side the Jacobi kernel is built for

// scratch for the tf32 image of the mode-3 operand, enough for both
// directions (Q^T: p x n, Q: n x p)
size_t mode3_img_max(int64_t n, int64_t p) {
  const size_t a = pp::mode3_img_bytes(p, n), b = pp::mode3_img_bytes(n, p);
  return a > b ? a : b;
}

// The projected product's images: Q^T (p x n) and Q (n x p), each built once
// per call and kept for all of its transforms, and one region for the other
// products (facewise and, in the backward, the A B^T of the Q gradient).
struct PprodImg {
  unsigned char *qt, *q, *other;
  size_t qt_bytes, q_bytes, other_bytes;
  bool qt_ready = false, q_ready = false;
};

PprodImg carve_pprod_img(Carve &c, int64_t n, int64_t p, size_t other_bytes) {
  PprodImg g;
  g.qt_bytes = pp::mode3_img_bytes(p, n);
  g.q_bytes = pp::mode3_img_bytes(n, p);
  g.other_bytes = other_bytes;
  g.qt = c.take<unsigned char>((int64_t)g.qt_bytes);
  g.q = c.take<unsigned char>((int64_t)g.q_bytes);
  g.other = c.take<unsigned char>((int64_t)other_bytes);
  return g;
}

struct DecompWs {
  float *Ah, *W, *sig, *Ahk;
  int32_t *perm, *sweeps, *status, *rank;
  int32_t *jaux;       // device-wide Jacobi kernel's counters (jacobi_aux_bytes)
  unsigned char *img;  // tf32 image of Q or Q^T for the mode-3 products (mode3_img_bytes)
  size_t img_bytes;
  double *kept_p, *disc_p, *part_a, *part_h, *part_e, *scal, *keys;
  int64_t *K;
  // QR preconditioner of the Jacobi SVD (slices that fit its shared memory)
  bool pc;
  float *R;            // p * b * b
  int32_t *qperm;      // p * b
  int64_t wpad;        // row stride of W: jacobi_apad(b, b) with pc, else jacobi_apad(l, m)
};

// The workspace always has room for the QR preconditioner where the slice fits
// its kernel; want_pc (pp_opts.precond >= 0) decides whether it runs.
DecompWs carve_decomp(Carve &c, int64_t l, int64_t m, int64_t n, int64_t p, bool ragged,
                      bool want_pc = true) {
  const int64_t b = l < m ? l : m;
  const int64_t a_pad = pp::jacobi_apad(l, m), b_pad = pp::jacobi_apad(b, b);
  DecompWs w{};
  const bool fits = pp::qrcp_fits(l, m);
  w.pc = fits && want_pc;
  w.wpad = w.pc ? b_pad : a_pad;
  w.Ah = c.take<float>(p * l * m);
  w.W = c.take<float>(p * b * (a_pad > b_pad ? a_pad : b_pad));
  w.sig = c.take<float>(p * b);
  w.perm = c.take<int32_t>(p * b);
  w.sweeps = c.take<int32_t>(p);
  w.Ahk = c.take<float>(p * l * m);
  w.kept_p = c.take<double>(p);
  w.disc_p = c.take<double>(p);
  w.part_a = c.take<double>(pp::mode3_tc_partials(p, l * m));
  w.part_h = c.take<double>(pp::mode3_tc_partials(p, l * m));
  w.part_e = c.take<double>(pp::mode3_tc_partials(n, l * m));
  w.scal = c.take<double>(8);
  w.status = c.take<int32_t>(1);
  w.jaux = c.take<int32_t>((int64_t)pp::jacobi_aux_bytes(p) / 4);
  w.img_bytes = mode3_img_max(n, p);
  w.img = c.take<unsigned char>((int64_t)w.img_bytes);
  w.K = c.take<int64_t>(1);
  if (ragged) {
    w.keys = c.take<double>(p * b);
    w.rank = c.take<int32_t>(p * b);
  }
  if (fits) {
    w.R = c.take<float>(p * b * b);
    w.qperm = c.take<int32_t>(p * b);
  }
  return w;
}

// Factor arguments for the Jacobi output of project_and_svd
pp::FactorArgs decomp_factor_args(const DecompWs &w, int64_t l, int64_t m, int64_t p) {
  pp::FactorArgs fa{};
  fa.X = w.Ah;
  fa.W = w.W;
  fa.sig = w.sig;
  fa.perm = w.perm;
  fa.l = l;
  fa.m = m;
  fa.p = p;
  fa.b = l < m ? l : m;
  fa.a_pad = w.wpad;
  fa.qperm = w.pc ? w.qperm : nullptr;
  return fa;
}

struct HosvdWs {
  DecompWs d;
  float *Uk, *sk, *Vk;                       // *Q-SVD factors at k = min(k1, k2)
  float *gpart, *G1, *G2;                    // Gram partials and the two Grams
  float *Wg, *sigg;                          // Jacobi of a Gram matrix (one slice)
  int32_t *permg, *sweepsg, *jauxg;
  float *U1, *s1, *V1, *U2, *s2, *V2;        // leading eigenvectors (V1, V2 are used)
  float *P1, *P2, *T;                        // projectors and the slice-wise temporary
};

HosvdWs carve_hosvd(Carve &c, int64_t l, int64_t m, int64_t n, int64_t p, int64_t k1,
                    int64_t k2, bool want_pc = true) {
  HosvdWs h;
  h.d = carve_decomp(c, l, m, n, p, false, want_pc);
  const int64_t k = k1 < k2 ? k1 : k2;
  const int64_t d = l > m ? l : m;
  h.Uk = c.take<float>(p * l * k);
  h.sk = c.take<float>(p * k);
  h.Vk = c.take<float>(p * m * k);
  h.gpart = c.take<float>(pp::gram_groups(n) * d * d);
  h.G1 = c.take<float>(l * l);
  h.G2 = c.take<float>(m * m);
  h.Wg = c.take<float>(d * pp::jacobi_apad(d, d));
  h.sigg = c.take<float>(d);
  h.permg = c.take<int32_t>(d);
  h.sweepsg = c.take<int32_t>(1);
  h.jauxg = c.take<int32_t>((int64_t)pp::jacobi_aux_bytes(1) / 4);
  h.U1 = c.take<float>(l * k1);
  h.s1 = c.take<float>(k1);
  h.V1 = c.take<float>(l * k1);
  h.U2 = c.take<float>(m * k2);
  h.s2 = c.take<float>(k2);
  h.V2 = c.take<float>(m * k2);
  h.P1 = c.take<float>(l * l);
  h.P2 = c.take<float>(m * m);
  h.T = c.take<float>(p * l * m);
  return h;
}

pp_status cuda_status(cudaError_t e) { return e == cudaSuccess ? PP_OK : PP_ECUDA; }

struct BwdWs {
  float *Ah, *Bh, *Ch, *Gh, *dAh, *dBh, *part, *dQE, *Sm;
  int64_t part_floats;
  PprodImg img;
};

BwdWs carve_bwd(Carve &c, int64_t n1, int64_t m, int64_t n2, int64_t n, int64_t p) {
  BwdWs w;
  w.Ah = c.take<float>(p * n1 * m);
  w.Bh = c.take<float>(p * m * n2);
  w.Ch = c.take<float>(p * n1 * n2);
  w.Gh = c.take<float>(p * n1 * n2);
  w.dAh = c.take<float>(p * n1 * m);
  w.dBh = c.take<float>(p * m * n2);
  int64_t z = pp::nt_splits(n, p, n1 * n2);
  const int64_t z2 = pp::nt_splits(n, p, n1 * m), z3 = pp::nt_splits(n, p, m * n2);
  if (z2 > z) z = z2;
  if (z3 > z) z = z3;
  w.part_floats = z * n * p;
  w.part = c.take<float>(w.part_floats);
  w.dQE = c.take<float>(n * p);
  w.Sm = c.take<float>(p * p);
  size_t other = pp::facewise_img_bytes(n1, m, n2, p);
  for (int64_t K : {n1 * n2, n1 * m, m * n2}) {   // the three A B^T of the Q gradient
    const size_t b = pp::nt_img_bytes(n, p, K);
    if (b > other) other = b;
  }
  // the facewise dA-hat_t = G-hat_t B-hat_t^T and dB-hat_t = A-hat_t^T G-hat_t
  for (size_t b : {pp::facewise_img_bytes(n1, n2, m, p), pp::facewise_img_bytes(m, n1, n2, p)})
    if (b > other) other = b;
  w.img = carve_pprod_img(c, n, p, other);
  return w;
}

struct U3Ws {
  float *part, *G, *W, *sig, *Uh, *s, *Vh;
  int32_t *perm, *sweeps, *status, *jaux;
};

U3Ws carve_u3(Carve &c, int64_t l, int64_t m, int64_t n, int64_t p) {
  U3Ws w;
  w.part = c.take<float>(pp::nt_splits(n, n, l * m) * n * n);
  w.G = c.take<float>(n * n);
  w.W = c.take<float>(n * pp::jacobi_apad(n, n));
  w.sig = c.take<float>(n);
  w.Uh = c.take<float>(n * p);
  w.s = c.take<float>(p);
  w.Vh = c.take<float>(n * p);
  w.perm = c.take<int32_t>(n);
  w.sweeps = c.take<int32_t>(1);
  w.status = c.take<int32_t>(1);
  w.jaux = c.take<int32_t>((int64_t)pp::jacobi_aux_bytes(1) / 4);
  return w;
}

// auxiliary streams and fork/join events for tsvdqII_batched, created once per device
constexpr int AUX_STREAMS = 8;
constexpr int MAX_DEV = 64;
struct AuxSet {
  cudaStream_t s[AUX_STREAMS];
  cudaEvent_t join[AUX_STREAMS];
  cudaEvent_t fork;
  bool ready = false;
};
AuxSet g_aux[MAX_DEV];
std::mutex g_aux_mu;

AuxSet *aux_streams() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEV) return nullptr;
  std::lock_guard<std::mutex> lock(g_aux_mu);
  AuxSet &a = g_aux[dev];
  if (!a.ready) {
    if (cudaEventCreateWithFlags(&a.fork, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    for (int i = 0; i < AUX_STREAMS; ++i) {
      if (cudaStreamCreateWithFlags(&a.s[i], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&a.join[i], cudaEventDisableTiming) != cudaSuccess)
        return nullptr;
    }
    a.ready = true;
  }
  return &a;
}

#define PP_TRY(expr)                            \
  do {                                          \
    cudaError_t _e = (expr);                    \
    if (_e != cudaSuccess) return PP_ECUDA;     \
  } while (0)

pp_status check_ws(const void *ws, size_t ws_bytes, size_t need) {
  if (need == 0) return PP_OK;
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255) != 0 || ws_bytes < need) return PP_EWORKSPACE;
  return PP_OK;
}

struct Opts {
  int32_t max_sweeps = 30;
  bool allow_grid = true;   // false inside tsvdqII_batched (concurrent launches)
  int32_t check_q = 0;
  float q_tol = 1e-5f;
  int32_t check_finite = 0;
  float jacobi_tol = 0.f;
  int32_t precond = 0;
};

// Set while tsvdqII_batched enqueues its items on several streams: their
// Jacobi launches may run at the same time, which the device-wide cooperative
// Jacobi kernel (all its CTAs resident at once, waiting on each other) must not.
thread_local bool t_concurrent = false;
struct ConcurrentScope {
  ConcurrentScope() { t_concurrent = true; }
  ~ConcurrentScope() { t_concurrent = false; }
};

Opts read_opts(const pp_opts *o) {
  Opts r;
  r.allow_grid = !t_concurrent;
  if (o) {
    if (o->max_sweeps > 0) r.max_sweeps = o->max_sweeps;
    r.check_q = o->check_q;
    if (o->q_tol > 0.f) r.q_tol = o->q_tol;
    r.check_finite = o->check_finite;
    r.jacobi_tol = o->jacobi_tol;
    r.precond = o->precond;
  }
  return r;
}

float default_tol(int64_t l, int64_t m) {
  const double a = (double)(l > m ? l : m);
  return (float)(sqrt(a) * 5.9604644775390625e-08);   // sqrt(a) * 2^-24
}

// Steps shared by Alg. 4.1 and Alg. 4.2 up to the facewise SVD.
// Partial-sum counts of the energies |A|^2, |A-hat|^2 and |A - A_k|^2 when
// their final sums are left to the report kernel (one launch instead of three).
struct EnergyParts {
  int np_a = 0, np_h = 0, np_e = 0;
};

pp_status project_and_svd(const float *A, const float *Q, int64_t l, int64_t m, int64_t n,
                          int64_t p, const Opts &o, const DecompWs &w, cudaStream_t st,
                          EnergyParts *defer = nullptr) {
  PP_TRY(cudaMemsetAsync(w.status, 0, sizeof(int32_t), st));
  if (o.check_q) PP_TRY(pp::launch_check_q(Q, n, p, o.q_tol, w.status, st));
  if (o.check_finite) PP_TRY(pp::launch_check_finite(A, n * l * m, w.status, st));
  // Alg. 4.1 step 2: A-hat = A x_3 Q^T;  M(r, c) = Q^T(r, c) = Q[c*p + r], with the
  // energies |A|^2 and |A-hat|^2 accumulated on the way
  int np_h = 0, np_a = 0;
  PP_TRY(pp::launch_mode3_tc(Q, 1, p, A, w.Ah, p, n, l * m, nullptr, nullptr, &np_h, w.part_a,
                             &np_a, w.part_h, w.status, st, w.img, w.img_bytes));
  if (defer) {
    defer->np_a = np_a;
    defer->np_h = np_h;
  } else {
    PP_TRY(pp::launch_sum_partials(w.part_a, np_a, w.scal + 0, st));
    PP_TRY(pp::launch_sum_partials(w.part_h, np_h, w.scal + 1, st));
  }
  stage(1, st);
  // step 3: facewise SVD -- one-sided Jacobi, on the rows of R from a QR with
  // column pivoting of each slice where the slice fits that kernel
  pp::JacobiArgs ja;
  ja.W = w.W;
  ja.sig = w.sig;
  ja.perm = w.perm;
  ja.sweeps = w.sweeps;
  ja.status = w.status;
  ja.p = p;
  ja.key_l = l;
  ja.key_m = m;
  ja.max_sweeps = o.max_sweeps;
  ja.aux = w.jaux;
  ja.allow_grid = o.allow_grid;
  if (w.pc) {
    const int64_t b = l < m ? l : m;
    pp::QrArgs qa{w.Ah, w.R, w.qperm, l, m, p};
    PP_TRY(pp::launch_qrcp(qa, st));
    ja.X = w.R;
    ja.l = b;
    ja.m = b;
    ja.tol = o.jacobi_tol > 0.f ? o.jacobi_tol : default_tol(b, b);
  } else {
    ja.X = w.Ah;
    ja.l = l;
    ja.m = m;
    ja.tol = o.jacobi_tol > 0.f ? o.jacobi_tol : default_tol(l, m);
  }
  PP_TRY(pp::launch_jacobi(ja, st));
  stage(2, st);
  return PP_OK;
}

// Back-projection A_k = A-hat_k x_3 Q with the fused error |A - A_k|^2.
pp_status backproject(const float *A, const float *Q, int64_t l, int64_t m, int64_t n,
                      int64_t p, float *Ak, const DecompWs &w, cudaStream_t st,
                      EnergyParts *defer = nullptr) {
  int np = 0;
  // M(r, c) = Q(r, c) = Q[r*p + c]
  PP_TRY(pp::launch_mode3_tc(Q, p, 1, w.Ahk, Ak, n, p, l * m, A, w.part_e, &np, nullptr, nullptr,
                             nullptr, w.status, st, w.img, w.img_bytes));
  if (defer)
    defer->np_e = np;
  else
    PP_TRY(pp::launch_sum_partials(w.part_e, np, w.scal + 2, st));
  return PP_OK;
}

// The report's energies from the deferred partial sums (written to scal[0..2]
// as well), or nothing to do when no report is wanted.
void report_energies(pp::ReportArgs &ra, const DecompWs &w, const EnergyParts &ep) {
  ra.parts[0] = w.part_a;
  ra.parts[1] = w.part_h;
  ra.parts[2] = w.part_e;
  ra.nparts[0] = ep.np_a;
  ra.nparts[1] = ep.np_h;
  ra.nparts[2] = ep.np_e;
  ra.sums = w.scal;
}

// ---- complex Q (pp_complex.cu)
constexpr size_t CJ_SMEM_BUDGET = 200 * 1024;

struct CDecompWs {
  float *Pim, *Bre, *Bim;      // real matrices from Q
  float *Ah, *Ahk;             // planar stacked transform domain (2 p l m each)
  float2 *W;
  float *sig;
  int32_t *perm, *sweeps, *status, *rank;
  double *kept_p, *disc_p, *part_a, *part_h, *part_e, *scal, *keys;
  int64_t *K;
};

CDecompWs carve_cdecomp(Carve &c, int64_t l, int64_t m, int64_t n, int64_t p, bool ragged) {
  const int64_t b = l < m ? l : m;
  CDecompWs w{};
  w.Pim = c.take<float>(p * n);
  w.Bre = c.take<float>(2 * n * p);
  w.Bim = c.take<float>(2 * n * p);
  w.Ah = c.take<float>(2 * p * l * m);
  w.Ahk = c.take<float>(2 * p * l * m);
  w.W = c.take<float2>(p * b * pp::cjacobi_apad(l, m));
  w.sig = c.take<float>(p * b);
  w.perm = c.take<int32_t>(p * b);
  w.sweeps = c.take<int32_t>(p);
  w.kept_p = c.take<double>(p);
  w.disc_p = c.take<double>(p);
  w.part_a = c.take<double>(pp::mode3_tc_partials(p, l * m));
  w.part_h = c.take<double>(2 * pp::mode3_tc_partials(p, l * m));
  w.part_e = c.take<double>(2 * pp::mode3_tc_partials(n, l * m));
  w.scal = c.take<double>(8);
  w.status = c.take<int32_t>(1);
  w.K = c.take<int64_t>(1);
  if (ragged) {
    w.keys = c.take<double>(p * b);
    w.rank = c.take<int32_t>(p * b);
  }
  return w;
}

// A-hat = A x_3 Q^H (planar: Re = Re(Q)^T A, Im = -Im(Q)^T A) with |A|^2, |A-hat|^2,
// then the complex facewise Jacobi SVD
pp_status cproject_and_svd(const float *A, const float *Q, int64_t l, int64_t m, int64_t n,
                           int64_t p, const Opts &o, const CDecompWs &w, cudaStream_t st) {
  PP_TRY(cudaMemsetAsync(w.status, 0, sizeof(int32_t), st));
  if (o.check_q) PP_TRY(pp::launch_qc_check(Q, n, p, o.q_tol, w.status, st));
  if (o.check_finite) PP_TRY(pp::launch_check_finite(A, n * l * m, w.status, st));
  PP_TRY(pp::launch_qc_build(Q, n, p, w.Pim, w.Bre, w.Bim, st));
  const int64_t plm = p * l * m;
  int np_r = 0, np_i = 0, np_a = 0;
  // Re: M(t, s) = Re Q(s, t) = Q[2 (s p + t)]
  PP_TRY(pp::launch_mode3_tc(Q, 2, 2 * p, A, w.Ah, p, n, l * m, nullptr, nullptr, &np_r, w.part_a,
                             &np_a, w.part_h, w.status, st));
  PP_TRY(pp::launch_mode3_tc(w.Pim, n, 1, A, w.Ah + plm, p, n, l * m, nullptr, nullptr, &np_i,
                             nullptr, nullptr, w.part_h + np_r, w.status, st));
  PP_TRY(pp::launch_sum_partials(w.part_a, np_a, w.scal + 0, st));
  PP_TRY(pp::launch_sum_partials(w.part_h, np_r + np_i, w.scal + 1, st));
  pp::CJacobiArgs ja;
  ja.Xre = w.Ah;
  ja.Xim = w.Ah + plm;
  ja.W = w.W;
  ja.sig = w.sig;
  ja.perm = w.perm;
  ja.sweeps = w.sweeps;
  ja.status = w.status;
  ja.l = l;
  ja.m = m;
  ja.p = p;
  ja.a_pad = (int)pp::cjacobi_apad(l, m);
  ja.max_sweeps = o.max_sweeps;
  ja.tol = o.jacobi_tol > 0.f ? o.jacobi_tol : default_tol(l, m);
  PP_TRY(pp::launch_cjacobi(ja, st));
  return PP_OK;
}

// A_k = A-hat_k x_3 Q: Re = [Re Q | -Im Q] [Re; Im], Im = [Im Q | Re Q] [Re; Im];
// err2 (scal[2]) = |A - Re A_k|^2 + |Im A_k|^2
pp_status cbackproject(const float *A, int64_t l, int64_t m, int64_t n, int64_t p,
                       const float *Xhat, float *Yre, float *Yim, const CDecompWs &w,
                       double *err_out, cudaStream_t st) {
  int np1 = 0, np2 = 0;
  PP_TRY(pp::launch_mode3_tc(w.Bre, 2 * p, 1, Xhat, Yre, n, 2 * p, l * m, A, w.part_e, &np1,
                             nullptr, nullptr, nullptr, w.status, st));
  PP_TRY(pp::launch_mode3_tc(w.Bim, 2 * p, 1, Xhat, Yim, n, 2 * p, l * m, nullptr, nullptr, &np2,
                             nullptr, nullptr, w.part_e + np1, w.status, st));
  if (err_out) PP_TRY(pp::launch_sum_partials(w.part_e, np1 + np2, err_out, st));
  return PP_OK;
}

pp::CFactorArgs cfactor_args(const CDecompWs &w, int64_t l, int64_t m, int64_t p) {
  pp::CFactorArgs fa{};
  fa.Xre = w.Ah;
  fa.Xim = w.Ah + p * l * m;
  fa.W = w.W;
  fa.sig = w.sig;
  fa.perm = w.perm;
  fa.l = l;
  fa.m = m;
  fa.p = p;
  fa.b = l < m ? l : m;
  fa.a_pad = pp::cjacobi_apad(l, m);
  fa.Ahk = w.Ahk;
  return fa;
}

bool bad_dims(int64_t l, int64_t m, int64_t n, int64_t p) {
  return l < 1 || m < 1 || n < 1 || p < 1 || p > n || l > (1 << 20) || m > (1 << 20) ||
         n > (1 << 20) || l * m > (int64_t)1 << 31;
}

}  // namespace

extern "C" {

const char *pp_status_str(int32_t s) {
  switch (s) {
    case PP_OK: return "PP_OK";
    case PP_EINVAL: return "PP_EINVAL: invalid argument";
    case PP_ESHAPE: return "PP_ESHAPE: invalid or unsupported sizes";
    case PP_ENOTORTHO: return "PP_ENOTORTHO: Q does not have orthonormal columns";
    case PP_ENONFINITE: return "PP_ENONFINITE: non-finite input";
    case PP_ENOCONV: return "PP_ENOCONV: Jacobi SVD did not converge within max_sweeps";
    case PP_ETIMEOUT: return "PP_ETIMEOUT: bounded device wait expired";
    case PP_EWORKSPACE: return "PP_EWORKSPACE: workspace missing, misaligned or too small";
    case PP_ECUDA: return "PP_ECUDA: CUDA launch or runtime error";
    case PP_ENOSYS: return "PP_ENOSYS: variant not built";
    default: return "unknown pp_status";
  }
}

const char *pp_version(void) { return "pprod-gb300 0.1 sm_103a"; }

void pp_set_stage_events(void *const *events, int32_t n) {
  if (!events || n <= 0) {
    g_nevents = 0;
    return;
  }
  if (n > 8) n = 8;
  for (int i = 0; i < n; ++i) g_events[i] = static_cast<cudaEvent_t>(events[i]);
  g_nevents = n;
}

uint64_t pp_kernel_launches(void) { return pp::g_launches.load(); }

pp_status pp_set_jacobi_shape(int64_t l, int64_t m, int64_t p, int32_t C, int32_t GW) {
  return pp::set_jacobi_shape(l, m, p, C, GW) ? PP_OK : PP_EINVAL;
}

size_t pp_workspace_bytes(int32_t op, const pp_shape *sh) {
  if (!sh) return 0;
  Carve c(nullptr);
  switch (op) {
    case PP_OP_MODE3:
    case PP_OP_FACEWISE:
      return 0;
    case PP_OP_PPROD:
      if (sh->l < 1 || sh->m < 1 || sh->n2 < 1 || sh->p < 1) return 0;
      c.take<float>(sh->p * sh->l * sh->m);
      c.take<float>(sh->p * sh->m * sh->n2);
      c.take<float>(sh->p * sh->l * sh->n2);
      carve_pprod_img(c, sh->n, sh->p, pp::facewise_img_bytes(sh->l, sh->m, sh->n2, sh->p));
      return c.off;
    case PP_OP_TSVDQ:
    case PP_OP_TSVDQII:
      if (bad_dims(sh->l, sh->m, sh->n, sh->p)) return 0;
      carve_decomp(c, sh->l, sh->m, sh->n, sh->p, op == PP_OP_TSVDQII);
      return c.off;
    case PP_OP_PPROD_BWD:
      if (bad_dims(sh->l, sh->m, sh->n, sh->p) || bad_dims(sh->m, sh->n2, sh->n, sh->p) ||
          bad_dims(sh->l, sh->n2, sh->n, sh->p))
        return 0;
      carve_bwd(c, sh->l, sh->m, sh->n2, sh->n, sh->p);
      return c.off;
    case PP_OP_PPROD_C:
      if (sh->l < 1 || sh->m < 1 || sh->n2 < 1 || bad_dims(sh->l, sh->m, sh->n, sh->p)) return 0;
      c.take<float>(sh->p * sh->n);
      c.take<float>(2 * sh->n * sh->p);
      c.take<float>(2 * sh->n * sh->p);
      c.take<float>(2 * sh->p * sh->l * sh->m);
      c.take<float>(2 * sh->p * sh->m * sh->n2);
      c.take<float>(2 * sh->p * sh->l * sh->n2);
      c.take<int32_t>(1);
      return c.off;
    case PP_OP_TSVDQ_C:
    case PP_OP_TSVDQII_C:
      if (bad_dims(sh->l, sh->m, sh->n, sh->p)) return 0;
      carve_cdecomp(c, sh->l, sh->m, sh->n, sh->p, op == PP_OP_TSVDQII_C);
      return c.off;
    case PP_OP_U3:
      if (bad_dims(sh->l, sh->m, sh->n, sh->p)) return 0;
      carve_u3(c, sh->l, sh->m, sh->n, sh->p);
      return c.off;
    case PP_OP_HOSVD:
      if (bad_dims(sh->l, sh->m, sh->n, sh->p) || sh->k < 1 || sh->k > sh->l || sh->n2 < 1 ||
          sh->n2 > sh->m)
        return 0;
      carve_hosvd(c, sh->l, sh->m, sh->n, sh->p, sh->k, sh->n2);
      return c.off;
    default:
      return 0;
  }
}

pp_status pprod_mode3(const float *X, int64_t l, int64_t m, int64_t n, const float *Q, int64_t p,
                      int32_t transpose, float *Y, void *stream) {
  if (!X || !Q || !Y) return PP_EINVAL;
  if (transpose != 0 && transpose != 1) return PP_EINVAL;
  if (bad_dims(l, m, n, p)) return PP_ESHAPE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (transpose == 0)   // Y (p slices) = X (n slices) x_3 Q^T
    return cuda_status(pp::launch_mode3_tc(Q, 1, p, X, Y, p, n, l * m, nullptr, nullptr, nullptr,
                                           nullptr, nullptr, nullptr, nullptr, st));
  // Y (n slices) = X (p slices) x_3 Q
  return cuda_status(pp::launch_mode3_tc(Q, p, 1, X, Y, n, p, l * m, nullptr, nullptr, nullptr,
                                         nullptr, nullptr, nullptr, nullptr, st));
}

pp_status pprod_facewise(const float *Ah, const float *Bh, int64_t n1, int64_t m, int64_t n2,
                         int64_t p, float *Ch, void *stream) {
  if (!Ah || !Bh || !Ch) return PP_EINVAL;
  if (n1 < 1 || m < 1 || n2 < 1 || p < 1 || p > 65535 || n1 > (1 << 20) || n2 > (1 << 20))
    return PP_ESHAPE;
  return cuda_status(pp::launch_facewise_gemm(Ah, Bh, Ch, n1, m, n2, p,
                                              static_cast<cudaStream_t>(stream)));
}

pp_status pprod(const float *A, const float *B, const float *Q, int64_t n1, int64_t m,
                int64_t n2, int64_t n, int64_t p, float *C, void *ws, size_t ws_bytes,
                void *stream) {
  if (!A || !B || !Q || !C) return PP_EINVAL;
  if (bad_dims(n1, m, n, p) || bad_dims(m, n2, n, p) || bad_dims(n1, n2, n, p) || p > 65535)
    return PP_ESHAPE;
  pp_shape sh{n1, m, n, p, 0, n2};
  const size_t need = pp_workspace_bytes(PP_OP_PPROD, &sh);
  if (pp_status s = check_ws(ws, ws_bytes, need)) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Carve c(ws);
  float *Ah = c.take<float>(p * n1 * m);
  float *Bh = c.take<float>(p * m * n2);
  float *Ch = c.take<float>(p * n1 * n2);
  PprodImg g = carve_pprod_img(c, n, p, pp::facewise_img_bytes(n1, m, n2, p));
  PP_TRY(pp::launch_mode3_tc(Q, 1, p, A, Ah, p, n, n1 * m, nullptr, nullptr, nullptr, nullptr,
                             nullptr, nullptr, nullptr, st, g.qt, g.qt_bytes, &g.qt_ready));
  PP_TRY(pp::launch_mode3_tc(Q, 1, p, B, Bh, p, n, m * n2, nullptr, nullptr, nullptr, nullptr,
                             nullptr, nullptr, nullptr, st, g.qt, g.qt_bytes, &g.qt_ready));
  PP_TRY(pp::launch_facewise_gemm(Ah, Bh, Ch, n1, m, n2, p, st, g.other, g.other_bytes));
  PP_TRY(pp::launch_mode3_tc(Q, p, 1, Ch, C, n, p, n1 * n2, nullptr, nullptr, nullptr, nullptr,
                             nullptr, nullptr, nullptr, st, g.q, g.q_bytes, &g.q_ready));
  return PP_OK;
}

pp_status pprod_backward(const float *A, const float *B, const float *Q, const float *G,
                         int64_t n1, int64_t m, int64_t n2, int64_t n, int64_t p, float *dA,
                         float *dB, float *dQ_euclid, float *dQ, void *ws, size_t ws_bytes,
                         void *stream) {
  if (!A || !B || !Q || !G || !dA || !dB) return PP_EINVAL;
  if (bad_dims(n1, m, n, p) || bad_dims(m, n2, n, p) || bad_dims(n1, n2, n, p) || p > 65535)
    return PP_ESHAPE;
  pp_shape sh{n1, m, n, p, 0, n2};
  if (pp_status e = check_ws(ws, ws_bytes, pp_workspace_bytes(PP_OP_PPROD_BWD, &sh))) return e;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Carve c(ws);
  BwdWs w = carve_bwd(c, n1, m, n2, n, p);
  PprodImg &g = w.img;
  auto fwd = [&](const float *X, int64_t pix, float *Y) {   // Y = X x_3 Q^T
    return pp::launch_mode3_tc(Q, 1, p, X, Y, p, n, pix, nullptr, nullptr, nullptr, nullptr,
                               nullptr, nullptr, nullptr, st, g.qt, g.qt_bytes, &g.qt_ready);
  };
  auto back = [&](const float *X, int64_t pix, float *Y) {  // Y = X x_3 Q
    return pp::launch_mode3_tc(Q, p, 1, X, Y, n, p, pix, nullptr, nullptr, nullptr, nullptr,
                               nullptr, nullptr, nullptr, st, g.q, g.q_bytes, &g.q_ready);
  };
  // recompute the transform-domain operands
  PP_TRY(fwd(A, n1 * m, w.Ah));
  PP_TRY(fwd(B, m * n2, w.Bh));
  PP_TRY(pp::launch_facewise_gemm(w.Ah, w.Bh, w.Ch, n1, m, n2, p, st, g.other, g.other_bytes));
  PP_TRY(fwd(G, n1 * n2, w.Gh));
  // dA-hat_t (n1 x m) = G-hat_t (n1 x n2) B-hat_t^T: R_t(k = j, l) = B-hat_t[l*n2 + j]
  PP_TRY(pp::launch_facewise_strided(w.Gh, n2, 1, n1 * n2, w.Bh, 1, n2, m * n2, w.dAh, n1, n2, m,
                                     p, st, g.other, g.other_bytes));
  // dB-hat_t (m x n2) = A-hat_t^T (m x n1) G-hat_t: L_t(l, k = i) = A-hat_t[i*m + l]
  PP_TRY(pp::launch_facewise_strided(w.Ah, 1, m, n1 * m, w.Gh, n2, 1, n1 * n2, w.dBh, m, n1, n2,
                                     p, st, g.other, g.other_bytes));
  PP_TRY(back(w.dAh, n1 * m, dA));
  PP_TRY(back(w.dBh, m * n2, dB));
  if (dQ_euclid || dQ) {
    float *dQE = dQ_euclid ? dQ_euclid : w.dQE;
    PP_TRY(pp::launch_nt_accumulate(G, w.Ch, n, p, n1 * n2, w.part, dQE, 0, st, g.other,
                                    g.other_bytes, w.part_floats));
    PP_TRY(pp::launch_nt_accumulate(A, w.dAh, n, p, n1 * m, w.part, dQE, 1, st, g.other,
                                    g.other_bytes, w.part_floats));
    PP_TRY(pp::launch_nt_accumulate(B, w.dBh, n, p, m * n2, w.part, dQE, 1, st, g.other,
                                    g.other_bytes, w.part_floats));
    if (dQ) PP_TRY(pp::launch_stiefel(Q, dQE, n, p, w.Sm, dQ, st, w.part, w.part_floats));
  }
  return PP_OK;
}

pp_status tsvdq_trunc(const float *A, const float *Q, int64_t l, int64_t m, int64_t n, int64_t p,
                      int64_t k, float *Uh, float *s, float *Vh, float *Ak, pp_report *rep,
                      const pp_opts *opts, void *ws, size_t ws_bytes, void *stream) {
  if (!A || !Q || !Uh || !s || !Vh) return PP_EINVAL;
  if (bad_dims(l, m, n, p)) return PP_ESHAPE;
  const int64_t b = l < m ? l : m;
  if (k < 1 || k > b) return PP_ESHAPE;
  if ((l > m ? l : m) > MAX_LONG_SIDE) return PP_ENOSYS;
  pp_shape sh{l, m, n, p, k, 0};
  if (pp_status e = check_ws(ws, ws_bytes, pp_workspace_bytes(PP_OP_TSVDQ, &sh))) return e;
  const Opts o = read_opts(opts);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Carve c(ws);
  const DecompWs w = carve_decomp(c, l, m, n, p, false, o.precond >= 0);
  EnergyParts ep;
  stage(0, st);
  if (pp_status e = project_and_svd(A, Q, l, m, n, p, o, w, st, rep ? &ep : nullptr)) return e;
  stage(3, st);
  pp::FactorArgs fa = decomp_factor_args(w, l, m, p);
  fa.kfix = k;
  fa.rho = nullptr;
  fa.offs = nullptr;
  fa.Uh = Uh;
  fa.s = s;
  fa.Vh = Vh;
  fa.Ahk = w.Ahk;
  fa.kept_partial = w.kept_p;
  fa.disc_partial = w.disc_p;
  PP_TRY(pp::launch_factors(fa, st));
  stage(4, st);
  if (pp_status e = backproject(A, Q, l, m, n, p, Ak, w, st, rep ? &ep : nullptr)) return e;
  if (rep) {
    pp::ReportArgs ra;
    ra.rep = rep;
    ra.status = w.status;
    ra.sweeps = w.sweeps;
    ra.p = p;
    ra.normA2 = w.scal + 0;
    ra.normAh2 = w.scal + 1;
    ra.err2 = w.scal + 2;
    ra.kept_partial = w.kept_p;
    ra.disc_partial = w.disc_p;
    ra.sel_scal = nullptr;
    ra.K = nullptr;
    ra.kappa_fixed = k * p;
    ra.offs = nullptr;
    report_energies(ra, w, ep);
    PP_TRY(pp::launch_report(ra, st));
  }
  stage(5, st);
  return PP_OK;
}

pp_status tsvdqII(const float *A, const float *Q, int64_t l, int64_t m, int64_t n, int64_t p,
                  double gamma, int32_t *rho, int64_t *offs, float *Uh_pk, float *s_pk,
                  float *Vh_pk, float *Ak, pp_report *rep, const pp_opts *opts, void *ws,
                  size_t ws_bytes, void *stream) {
  if (!A || !Q || !rho || !offs || !Uh_pk || !s_pk || !Vh_pk) return PP_EINVAL;
  if (!(gamma > 0.0 && gamma <= 1.0)) return PP_EINVAL;
  if (bad_dims(l, m, n, p)) return PP_ESHAPE;
  const int64_t b = l < m ? l : m;
  if ((l > m ? l : m) > MAX_LONG_SIDE) return PP_ENOSYS;
  if (p * b > ((int64_t)1 << 31) - 1) return PP_ESHAPE;
  pp_shape sh{l, m, n, p, 0, 0};
  if (pp_status e = check_ws(ws, ws_bytes, pp_workspace_bytes(PP_OP_TSVDQII, &sh))) return e;
  const Opts o = read_opts(opts);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Carve c(ws);
  const DecompWs w = carve_decomp(c, l, m, n, p, true, o.precond >= 0);
  EnergyParts ep;
  stage(0, st);
  if (pp_status e = project_and_svd(A, Q, l, m, n, p, o, w, st, rep ? &ep : nullptr)) return e;
  // Alg. 4.2 steps 4-7
  pp::SelectArgs sa;
  sa.sig = w.sig;
  sa.p = p;
  sa.b = b;
  sa.gamma = gamma;
  sa.keys_sorted = w.keys;
  sa.rank = w.rank;
  sa.rho = rho;
  sa.offs = offs;
  sa.scal = w.scal + 4;
  sa.K = w.K;
  PP_TRY(pp::launch_select(sa, st));
  stage(3, st);
  // step 8: truncated factors (packed) and the rebuild
  pp::FactorArgs fa = decomp_factor_args(w, l, m, p);
  fa.kfix = 0;
  fa.rho = rho;
  fa.offs = offs;
  fa.Uh = Uh_pk;
  fa.s = s_pk;
  fa.Vh = Vh_pk;
  fa.Ahk = w.Ahk;
  fa.kept_partial = nullptr;
  fa.disc_partial = nullptr;
  PP_TRY(pp::launch_factors(fa, st));
  stage(4, st);
  if (pp_status e = backproject(A, Q, l, m, n, p, Ak, w, st, rep ? &ep : nullptr)) return e;
  if (rep) {
    pp::ReportArgs ra;
    ra.rep = rep;
    ra.status = w.status;
    ra.sweeps = w.sweeps;
    ra.p = p;
    ra.normA2 = w.scal + 0;
    ra.normAh2 = w.scal + 1;
    ra.err2 = w.scal + 2;
    ra.kept_partial = nullptr;
    ra.disc_partial = nullptr;
    ra.sel_scal = w.scal + 4;
    ra.K = w.K;
    ra.kappa_fixed = -1;
    ra.offs = offs;
    report_energies(ra, w, ep);
    PP_TRY(pp::launch_report(ra, st));
  }
  stage(5, st);
  return PP_OK;
}

pp_status tsvdqII_batched(const pp_batch_item *items, int64_t count, double gamma,
                          const pp_opts *opts, void *stream) {
  if (count < 0 || (count > 0 && !items)) return PP_EINVAL;
  if (!(gamma > 0.0 && gamma <= 1.0)) return PP_EINVAL;
  for (int64_t i = 0; i < count; ++i) {   // validate everything before enqueuing anything
    const pp_batch_item &it = items[i];
    if (!it.A || !it.Q || !it.rho || !it.offs || !it.Uh_pk || !it.s_pk || !it.Vh_pk)
      return PP_EINVAL;
    if (bad_dims(it.l, it.m, it.n, it.p)) return PP_ESHAPE;
    if ((it.l > it.m ? it.l : it.m) > MAX_LONG_SIDE) return PP_ENOSYS;
    pp_shape sh{it.l, it.m, it.n, it.p, 0, 0};
    if (pp_status e = check_ws(it.ws, it.ws_bytes, pp_workspace_bytes(PP_OP_TSVDQII, &sh)))
      return e;
  }
  if (count == 0) return PP_OK;
  AuxSet *aux = aux_streams();
  if (!aux) return PP_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int ns = count < AUX_STREAMS ? (int)count : AUX_STREAMS;
  PP_TRY(cudaEventRecord(aux->fork, st));
  for (int k = 0; k < ns; ++k) PP_TRY(cudaStreamWaitEvent(aux->s[k], aux->fork, 0));
  // largest tensors first (host-side order only), round-robin over the streams
  std::vector<int64_t> order((size_t)count);
  for (int64_t i = 0; i < count; ++i) order[(size_t)i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int64_t x, int64_t y) {
    return items[x].l * items[x].m * items[x].n > items[y].l * items[y].m * items[y].n;
  });
  ConcurrentScope concurrent;
  for (int64_t i = 0; i < count; ++i) {
    const pp_batch_item &it = items[order[(size_t)i]];
    if (pp_status e = tsvdqII(it.A, it.Q, it.l, it.m, it.n, it.p, gamma, it.rho, it.offs,
                              it.Uh_pk, it.s_pk, it.Vh_pk, it.Ak, it.rep, opts, it.ws,
                              it.ws_bytes, aux->s[i % ns]))
      return e;
  }
  for (int k = 0; k < ns; ++k) {
    PP_TRY(cudaEventRecord(aux->join[k], aux->s[k]));
    PP_TRY(cudaStreamWaitEvent(st, aux->join[k], 0));
  }
  return PP_OK;
}

pp_status hosvd_compare(const float *A, const float *Q, int64_t l, int64_t m, int64_t n,
                        int64_t p, int64_t k1, int64_t k2, float *Ak_hosvd, pp_hosvd_report *rep,
                        const pp_opts *opts, void *ws, size_t ws_bytes, void *stream) {
  if (!A || !Q) return PP_EINVAL;
  if (bad_dims(l, m, n, p)) return PP_ESHAPE;
  if (k1 < 1 || k1 > l || k2 < 1 || k2 > m) return PP_ESHAPE;
  if ((l > m ? l : m) > MAX_LONG_SIDE) return PP_ENOSYS;
  pp_shape sh{l, m, n, p, k1, k2};
  if (pp_status e = check_ws(ws, ws_bytes, pp_workspace_bytes(PP_OP_HOSVD, &sh))) return e;
  const Opts o = read_opts(opts);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Carve c(ws);
  const HosvdWs h = carve_hosvd(c, l, m, n, p, k1, k2, o.precond >= 0);
  const DecompWs &w = h.d;
  const int64_t k = k1 < k2 ? k1 : k2;
  // (1) *Q-SVD with k = min(k1, k2) (Alg. 4.1), its error in scal[2]
  if (pp_status e = project_and_svd(A, Q, l, m, n, p, o, w, st)) return e;
  pp::FactorArgs fa = decomp_factor_args(w, l, m, p);
  fa.kfix = k;
  fa.rho = nullptr;
  fa.offs = nullptr;
  fa.Uh = h.Uk;
  fa.s = h.sk;
  fa.Vh = h.Vk;
  fa.Ahk = w.Ahk;
  fa.kept_partial = w.kept_p;
  fa.disc_partial = w.disc_p;
  PP_TRY(pp::launch_factors(fa, st));
  if (pp_status e = backproject(A, Q, l, m, n, p, nullptr, w, st)) return e;
  // (2) HOSVD factors: leading eigenvectors of the mode-1 and mode-2 Grams (eq. modek_svd)
  for (int mode = 1; mode <= 2; ++mode) {
    const int64_t d = mode == 1 ? l : m, kd = mode == 1 ? k1 : k2;
    float *G = mode == 1 ? h.G1 : h.G2;
    PP_TRY(pp::launch_gram(A, l, m, n, mode, h.gpart, G, st));
    pp::JacobiArgs ja;
    ja.X = G;
    ja.W = h.Wg;
    ja.sig = h.sigg;
    ja.perm = h.permg;
    ja.sweeps = h.sweepsg;
    ja.status = w.status;
    ja.l = d;
    ja.m = d;
    ja.p = 1;
    ja.max_sweeps = o.max_sweeps;
    ja.aux = h.jauxg;
    ja.allow_grid = o.allow_grid;
    ja.tol = o.jacobi_tol > 0.f ? o.jacobi_tol : default_tol(d, d);
    PP_TRY(pp::launch_jacobi(ja, st));
    pp::FactorArgs fg;
    fg.X = G;
    fg.W = h.Wg;
    fg.sig = h.sigg;
    fg.perm = h.permg;
    fg.l = d;
    fg.m = d;
    fg.p = 1;
    fg.b = d;
    fg.a_pad = pp::jacobi_apad(d, d);
    fg.kfix = kd;
    fg.rho = nullptr;
    fg.offs = nullptr;
    fg.Uh = mode == 1 ? h.U1 : h.U2;
    fg.s = mode == 1 ? h.s1 : h.s2;
    fg.Vh = mode == 1 ? h.V1 : h.V2;
    fg.Ahk = nullptr;
    fg.kept_partial = nullptr;
    fg.disc_partial = nullptr;
    PP_TRY(pp::launch_factors(fg, st));
    PP_TRY(pp::launch_projector(mode == 1 ? h.V1 : h.V2, d, kd, mode == 1 ? h.P1 : h.P2, st));
  }
  // (3) slice-wise P1 A-hat_t P2, then x_3 Q with the fused error in scal[3]
  PP_TRY(pp::launch_batched_gemm(w.Ah, m, 1, l * m, h.P2, 0, h.T, l * m, l, m, m, p, st));
  PP_TRY(pp::launch_batched_gemm(h.P1, l, 1, 0, h.T, l * m, w.Ahk, l * m, l, l, m, p, st));
  {
    int np = 0;
    PP_TRY(pp::launch_mode3_tc(Q, p, 1, w.Ahk, Ak_hosvd, n, p, l * m, A, w.part_e, &np, nullptr,
                               nullptr, nullptr, w.status, st, w.img, w.img_bytes));
    PP_TRY(pp::launch_sum_partials(w.part_e, np, w.scal + 3, st));
  }
  if (rep) {
    pp::HosvdReportArgs ra;
    ra.rep = rep;
    ra.status = w.status;
    ra.sweeps = w.sweeps;
    ra.p = p;
    ra.k1 = k1;
    ra.k2 = k2;
    ra.k = k;
    ra.normA2 = w.scal + 0;
    ra.normAh2 = w.scal + 1;
    ra.err2_tsvdq = w.scal + 2;
    ra.err2_hosvd = w.scal + 3;
    PP_TRY(pp::launch_hosvd_report(ra, st));
  }
  return PP_OK;
}

pp_status pprod_u3(const float *A, int64_t l, int64_t m, int64_t n, int64_t p, float *Q,
                   float *lambda, pp_report *rep, const pp_opts *opts, void *ws, size_t ws_bytes,
                   void *stream) {
  if (!A || !Q) return PP_EINVAL;
  if (bad_dims(l, m, n, p)) return PP_ESHAPE;
  if (n > MAX_LONG_SIDE) return PP_ENOSYS;
  pp_shape sh{l, m, n, p, 0, 0};
  if (pp_status e = check_ws(ws, ws_bytes, pp_workspace_bytes(PP_OP_U3, &sh))) return e;
  const Opts o = read_opts(opts);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Carve c(ws);
  const U3Ws w = carve_u3(c, l, m, n, p);
  PP_TRY(cudaMemsetAsync(w.status, 0, sizeof(int32_t), st));
  if (o.check_finite) PP_TRY(pp::launch_check_finite(A, n * l * m, w.status, st));
  // Gram of the mode-3 unfolding: G = A_(3) A_(3)^T, A_(3) is n x (l m) row-major
  PP_TRY(pp::launch_nt_accumulate(A, A, n, n, l * m, w.part, w.G, 0, st));
  // its eigenvectors: one-sided Jacobi SVD of the symmetric PSD G (one n x n slice)
  pp::JacobiArgs ja;
  ja.X = w.G;
  ja.W = w.W;
  ja.sig = w.sig;
  ja.perm = w.perm;
  ja.sweeps = w.sweeps;
  ja.status = w.status;
  ja.l = n;
  ja.m = n;
  ja.p = 1;
  ja.max_sweeps = o.max_sweeps;
  ja.aux = w.jaux;
  ja.allow_grid = o.allow_grid;
  ja.tol = o.jacobi_tol > 0.f ? o.jacobi_tol : default_tol(n, n);
  PP_TRY(pp::launch_jacobi(ja, st));
  // leading p: the long-side (normalised rotated) vectors, orthonormal to working accuracy
  pp::FactorArgs fa;
  fa.X = w.G;
  fa.W = w.W;
  fa.sig = w.sig;
  fa.perm = w.perm;
  fa.l = n;
  fa.m = n;
  fa.p = 1;
  fa.b = n;
  fa.a_pad = pp::jacobi_apad(n, n);
  fa.kfix = p;
  fa.rho = nullptr;
  fa.offs = nullptr;
  fa.Uh = w.Uh;
  fa.s = w.s;
  fa.Vh = w.Vh;
  fa.Ahk = nullptr;
  fa.kept_partial = nullptr;
  fa.disc_partial = nullptr;
  PP_TRY(pp::launch_factors(fa, st));
  PP_TRY(pp::launch_u3_finish(w.Vh, w.s, w.G, n, p, Q, lambda, w.status, w.sweeps, rep, st));
  return PP_OK;
}

pp_status pp_hosvd_matched_k2(int64_t l, int64_t m, int64_t n, int64_t p, int64_t k,
                              int32_t variant, int64_t *k2) {
  if (!k2 || (variant != 0 && variant != 1)) return PP_EINVAL;
  *k2 = 0;
  if (l < 1 || m < 1 || n < 1 || p < 1 || p > n || k < 1 || k > (l < m ? l : m) ||
      l > (1 << 20) || m > (1 << 20) || n > (1 << 20))
    return PP_ESHAPE;
  // budget: *Q-SVD storage k (l + m) p (Sec. 5.1.2); the n p of Q is on both sides
  const int64_t budget = k * (l + m) * p;
  int64_t r;
  if (variant == 0) {
    // HOSVD(l, k2, p): l k2 p + l^2 + m k2 <= budget, linear in k2
    const int64_t num = budget - l * l, den = l * p + m;
    r = num < 0 ? 0 : num / den;
    if (r > m) r = m;
  } else {
    // HOSVD(k2, k2, p): p k2^2 + (l + m) k2 <= budget; the positive root, then
    // corrected in integers so that r is the largest k2 that fits
    const double b = (double)(l + m), pd = (double)p;
    r = (int64_t)((-b + sqrt(b * b + 4.0 * pd * (double)budget)) / (2.0 * pd));
    auto cost = [&](int64_t x) { return p * x * x + (l + m) * x; };
    while (r > 0 && cost(r) > budget) --r;
    while (cost(r + 1) <= budget) ++r;
    const int64_t cap = l < m ? l : m;
    if (r > cap) r = cap;
  }
  *k2 = r < 1 ? 0 : r;
  return PP_OK;
}

pp_status pprod_c(const float *A, const float *B, const float *Q, int64_t n1, int64_t m,
                  int64_t n2, int64_t n, int64_t p, float *C_re, float *C_im, void *ws,
                  size_t ws_bytes, void *stream) {
  if (!A || !B || !Q || !C_re || !C_im) return PP_EINVAL;
  if (bad_dims(n1, m, n, p) || bad_dims(m, n2, n, p) || bad_dims(n1, n2, n, p)) return PP_ESHAPE;
  pp_shape sh{n1, m, n, p, 0, n2};
  if (pp_status e = check_ws(ws, ws_bytes, pp_workspace_bytes(PP_OP_PPROD_C, &sh))) return e;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Carve c(ws);
  CDecompWs w{};
  w.Pim = c.take<float>(p * n);
  w.Bre = c.take<float>(2 * n * p);
  w.Bim = c.take<float>(2 * n * p);
  float *Ah = c.take<float>(2 * p * n1 * m);
  float *Bh = c.take<float>(2 * p * m * n2);
  float *Ch = c.take<float>(2 * p * n1 * n2);
  w.status = c.take<int32_t>(1);
  PP_TRY(pp::launch_qc_build(Q, n, p, w.Pim, w.Bre, w.Bim, st));
  auto fwd = [&](const float *X, int64_t pix, float *Y) -> cudaError_t {   // X x_3 Q^H
    cudaError_t e = pp::launch_mode3_tc(Q, 2, 2 * p, X, Y, p, n, pix, nullptr, nullptr, nullptr,
                                        nullptr, nullptr, nullptr, nullptr, st);
    if (e != cudaSuccess) return e;
    return pp::launch_mode3_tc(w.Pim, n, 1, X, Y + p * pix, p, n, pix, nullptr, nullptr, nullptr,
                               nullptr, nullptr, nullptr, nullptr, st);
  };
  PP_TRY(fwd(A, n1 * m, Ah));
  PP_TRY(fwd(B, m * n2, Bh));
  PP_TRY(pp::launch_cfacewise(Ah, Bh, Ch, n1, m, n2, p, st));
  PP_TRY(pp::launch_mode3_tc(w.Bre, 2 * p, 1, Ch, C_re, n, 2 * p, n1 * n2, nullptr, nullptr,
                             nullptr, nullptr, nullptr, nullptr, nullptr, st));
  PP_TRY(pp::launch_mode3_tc(w.Bim, 2 * p, 1, Ch, C_im, n, 2 * p, n1 * n2, nullptr, nullptr,
                             nullptr, nullptr, nullptr, nullptr, nullptr, st));
  return PP_OK;
}

pp_status tsvdq_trunc_c(const float *A, const float *Q, int64_t l, int64_t m, int64_t n,
                        int64_t p, int64_t k, float *Uh, float *s, float *Vh, float *Ak_re,
                        float *Ak_im, pp_report *rep, const pp_opts *opts, void *ws,
                        size_t ws_bytes, void *stream) {
  if (!A || !Q || !Uh || !s || !Vh || ((Ak_re == nullptr) != (Ak_im == nullptr)))
    return PP_EINVAL;
  if (bad_dims(l, m, n, p)) return PP_ESHAPE;
  const int64_t b = l < m ? l : m;
  if (k < 1 || k > b) return PP_ESHAPE;
  if (pp::cjacobi_smem(l, m) > CJ_SMEM_BUDGET) return PP_ENOSYS;
  pp_shape sh{l, m, n, p, k, 0};
  if (pp_status e = check_ws(ws, ws_bytes, pp_workspace_bytes(PP_OP_TSVDQ_C, &sh))) return e;
  const Opts o = read_opts(opts);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Carve c(ws);
  const CDecompWs w = carve_cdecomp(c, l, m, n, p, false);
  if (pp_status e = cproject_and_svd(A, Q, l, m, n, p, o, w, st)) return e;
  pp::CFactorArgs fa = cfactor_args(w, l, m, p);
  fa.kfix = k;
  fa.Uh = reinterpret_cast<float2 *>(Uh);
  fa.Vh = reinterpret_cast<float2 *>(Vh);
  fa.s = s;
  fa.kept_partial = w.kept_p;
  fa.disc_partial = w.disc_p;
  PP_TRY(pp::launch_cfactors(fa, st));
  if (pp_status e = cbackproject(A, l, m, n, p, w.Ahk, Ak_re, Ak_im, w, w.scal + 2, st)) return e;
  if (rep) {
    pp::ReportArgs ra;
    ra.rep = rep;
    ra.status = w.status;
    ra.sweeps = w.sweeps;
    ra.p = p;
    ra.normA2 = w.scal + 0;
    ra.normAh2 = w.scal + 1;
    ra.err2 = w.scal + 2;
    ra.kept_partial = w.kept_p;
    ra.disc_partial = w.disc_p;
    ra.sel_scal = nullptr;
    ra.K = nullptr;
    ra.kappa_fixed = k * p;
    ra.offs = nullptr;
    PP_TRY(pp::launch_report(ra, st));
  }
  return PP_OK;
}

pp_status tsvdqII_c(const float *A, const float *Q, int64_t l, int64_t m, int64_t n, int64_t p,
                    double gamma, int32_t *rho, int64_t *offs, float *Uh_pk, float *s_pk,
                    float *Vh_pk, float *Ak_re, float *Ak_im, pp_report *rep,
                    const pp_opts *opts, void *ws, size_t ws_bytes, void *stream) {
  if (!A || !Q || !rho || !offs || !Uh_pk || !s_pk || !Vh_pk ||
      ((Ak_re == nullptr) != (Ak_im == nullptr)))
    return PP_EINVAL;
  if (!(gamma > 0.0 && gamma <= 1.0)) return PP_EINVAL;
  if (bad_dims(l, m, n, p)) return PP_ESHAPE;
  if (pp::cjacobi_smem(l, m) > CJ_SMEM_BUDGET) return PP_ENOSYS;
  pp_shape sh{l, m, n, p, 0, 0};
  if (pp_status e = check_ws(ws, ws_bytes, pp_workspace_bytes(PP_OP_TSVDQII_C, &sh))) return e;
  const Opts o = read_opts(opts);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Carve c(ws);
  const CDecompWs w = carve_cdecomp(c, l, m, n, p, true);
  const int64_t b = l < m ? l : m;
  if (pp_status e = cproject_and_svd(A, Q, l, m, n, p, o, w, st)) return e;
  pp::SelectArgs sa;
  sa.sig = w.sig;
  sa.p = p;
  sa.b = b;
  sa.gamma = gamma;
  sa.keys_sorted = w.keys;
  sa.rank = w.rank;
  sa.rho = rho;
  sa.offs = offs;
  sa.scal = w.scal + 4;
  sa.K = w.K;
  PP_TRY(pp::launch_select(sa, st));
  pp::CFactorArgs fa = cfactor_args(w, l, m, p);
  fa.kfix = 0;
  fa.rho = rho;
  fa.offs = offs;
  fa.Uh = reinterpret_cast<float2 *>(Uh_pk);
  fa.Vh = reinterpret_cast<float2 *>(Vh_pk);
  fa.s = s_pk;
  PP_TRY(pp::launch_cfactors(fa, st));
  if (pp_status e = cbackproject(A, l, m, n, p, w.Ahk, Ak_re, Ak_im, w, w.scal + 2, st)) return e;
  if (rep) {
    pp::ReportArgs ra;
    ra.rep = rep;
    ra.status = w.status;
    ra.sweeps = w.sweeps;
    ra.p = p;
    ra.normA2 = w.scal + 0;
    ra.normAh2 = w.scal + 1;
    ra.err2 = w.scal + 2;
    ra.kept_partial = nullptr;
    ra.disc_partial = nullptr;
    ra.sel_scal = w.scal + 4;
    ra.K = w.K;
    ra.kappa_fixed = -1;
    ra.offs = offs;
    PP_TRY(pp::launch_report(ra, st));
  }
  return PP_OK;
}

}  // extern "C"
