// MPS state, two-site pipeline and the C ABI (include/mps.h).
//
// Device memory of a handle is reserved once at create: every site for the
// largest bond dims the chain allows, plus one workspace sized for the
// largest two-site split.  The per-gate pipeline (Sec. III-C.2 with the split
// of Sec. III-B.2) is fully stream-ordered: bond dims after a split are known
// on the host (k = min(2 chi_l, 2 chi_r, chi_max)), so no step waits for the
// device.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "internal.h"

using namespace mpsg;

namespace {

constexpr int kDefaultNb = 32;
constexpr int kMaxNb = 32;
constexpr int kMaxCoop = 1024;
constexpr int kNormParts = 256;
constexpr size_t kAlign = 256;
constexpr int kDiscLog = 1 << 16;
constexpr int kSvdMaxChi = 4096;  // MPS_TRUNC_SVD: theta at most 8192 x 8192

inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

int max_bond(int n, int b, int chi) {
  // min(2^b, 2^(n-b), chi) without overflow
  int e = std::min(b, n - b);
  if (e >= 30) return chi;
  return std::min(1 << e, chi);
}

// ---------------------------------------------------------------------------
// workspace of one two-site split (either precision); carved from one buffer
struct WsLayout {
  size_t W, Q, F, vn1, vn2, jpvt, inv, tau, Tfac, Wg, Tblk, G12, Y, Z, SK, red_norm, red_w, red_argv, red_argi, alpha,
      bar, err, disc, total;
  int64_t sk_elems;
};

// sk_wide > 0 sizes the split-K partials for that many columns instead of
// max(nmax, kmax): workspaces that must choose the same splits as a larger one
// (the layer lanes) get the larger one's partial capacity.
WsLayout ws_layout(size_t esz, int mmax, int nmax, int kmax, int nb, int G, int64_t& ldw, int64_t& ldq,
                   int sk_wide = 0) {
  WsLayout L;
  ldw = (int64_t)std::max(4, (mmax + 3) / 4 * 4);
  ldq = ldw;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align_up(off + std::max<size_t>(bytes, 1));
    return o;
  };
  int npan = (kmax + nb - 1) / nb;
  int wide = std::max(nmax, kmax);
  L.W = take(esz * (size_t)ldw * std::max(nmax, 1));
  L.Q = take(esz * (size_t)ldq * std::max(kmax, 1));
  L.F = take(esz * (size_t)std::max(nmax, 1) * nb);
  L.vn1 = take(8 * (size_t)std::max(nmax, 1));
  L.vn2 = take(8 * (size_t)std::max(nmax, 1));
  L.jpvt = take(4 * (size_t)std::max(nmax, 1));
  L.inv = take(4 * (size_t)std::max(nmax, 1));
  L.tau = take(esz * (size_t)std::max(kmax, 1));
  L.Tfac = take(esz * (size_t)std::max(npan, 1) * nb * nb);
  L.Wg = take(16 * (size_t)std::max(npan, 1) * nb * nb);
  L.Tblk = take(esz * (size_t)(npan / 2 + 1) * 4 * nb * nb);
  L.G12 = take(esz * (size_t)nb * nb);
  L.Y = take(esz * (size_t)2 * nb * std::max(wide, 1));
  L.Z = take(esz * (size_t)2 * nb * std::max(wide, 1));
  L.sk_elems = (int64_t)kMaxSplit * 2 * nb * std::max(sk_wide > 0 ? sk_wide : wide, 1);
  L.SK = take(esz * (size_t)L.sk_elems);
  L.red_norm = take(8 * (size_t)G);
  L.red_w = take(16 * (size_t)G * nb);
  L.red_argv = take(8 * (size_t)G);
  L.red_argi = take(4 * (size_t)G);
  L.alpha = take(16);
  L.bar = take(16);
  L.err = take(16);
  L.disc = take(8);
  L.total = off;
  return L;
}

template <typename T>
struct Ws {
  T* W;
  int64_t ldw;
  T* Q;
  int64_t ldq;
  T* F;
  double* vn1;
  double* vn2;
  int* jpvt;
  int* inv;
  T* tau;
  T* Tfac;
  c128* Wg;
  T* Tblk;
  T* G12;
  T* Y;
  T* Z;
  T* SK;
  int64_t sk_cap;
  double* red_norm;
  c128* red_w;
  double* red_argv;
  int* red_argi;
  c128* alpha;
  unsigned* bar;
  int* err;
  double* disc;
};

template <typename T>
Ws<T> ws_views(char* base, const WsLayout& L, int64_t ldw, int64_t ldq) {
  Ws<T> w;
  w.W = (T*)(base + L.W);
  w.ldw = ldw;
  w.Q = (T*)(base + L.Q);
  w.ldq = ldq;
  w.F = (T*)(base + L.F);
  w.vn1 = (double*)(base + L.vn1);
  w.vn2 = (double*)(base + L.vn2);
  w.jpvt = (int*)(base + L.jpvt);
  w.inv = (int*)(base + L.inv);
  w.tau = (T*)(base + L.tau);
  w.Tfac = (T*)(base + L.Tfac);
  w.Wg = (c128*)(base + L.Wg);
  w.Tblk = (T*)(base + L.Tblk);
  w.G12 = (T*)(base + L.G12);
  w.Y = (T*)(base + L.Y);
  w.Z = (T*)(base + L.Z);
  w.SK = (T*)(base + L.SK);
  w.sk_cap = L.sk_elems;
  w.red_norm = (double*)(base + L.red_norm);
  w.red_w = (c128*)(base + L.red_w);
  w.red_argv = (double*)(base + L.red_argv);
  w.red_argi = (int*)(base + L.red_argi);
  w.alpha = (c128*)(base + L.alpha);
  w.bar = (unsigned*)(base + L.bar);
  w.err = (int*)(base + L.err);
  w.disc = (double*)(base + L.disc);
  return w;
}

struct Knobs {
  int nb;
  int G;
  double flag_tol;
  unsigned long long timeout_ns;
  unsigned barrier_extra;
  bool use_tc;  // complex64 products on the tensor cores
  bool small;   // splits whose theta fits one CTA run in small_gate_kernel
};

template <typename T>
SmallGate<T> small_item(int cl, int cm, int cr, int k, const T* A, const T* B, const T* g, T* Aout, T* Bout,
                        double* disc, double* disc_total, int* jpvt_out, const T* gdev = nullptr) {
  SmallGate<T> it;
  it.gdev = gdev;
  it.A = A;
  it.B = B;
  it.Aout = Aout;
  it.Bout = Bout;
  it.disc = disc;
  it.disc_total = disc_total;
  it.jpvt_out = jpvt_out;
  it.cl = cl;
  it.cm = cm;
  it.cr = cr;
  it.k = k;
  for (int q = 0; q < 16; ++q) it.g[q] = g[q];
  return it;
}

template <typename T>
QrPlan<T> make_plan(const Ws<T>& w, const Knobs& kn, int m, int n, int k, int pivot, double* disc_slot,
                    double* disc_total) {
  QrPlan<T> p;
  p.m = m;
  p.n = n;
  p.k = k;
  p.nb = kn.nb;
  p.pivot = pivot;
  p.W = w.W;
  p.ldw = w.ldw;
  p.tau = w.tau;
  p.jpvt = w.jpvt;
  p.Tfac = w.Tfac;
  p.Wg = w.Wg;
  p.Tblk = w.Tblk;
  p.G12 = w.G12;
  p.F = w.F;
  p.vn1 = w.vn1;
  p.vn2 = w.vn2;
  p.red_norm = w.red_norm;
  p.red_w = w.red_w;
  p.red_argv = w.red_argv;
  p.red_argi = w.red_argi;
  p.alpha_slot = w.alpha;
  p.bar = w.bar;
  p.err = w.err;
  p.discarded = disc_slot;
  p.disc_total = disc_total;
  p.Y = w.Y;
  p.Z = w.Z;
  p.SK = w.SK;
  p.sk_cap = w.sk_cap;
  p.G = kn.G;
  p.flag_tol = kn.flag_tol;
  p.timeout_ns = kn.timeout_ns;
  p.barrier_extra = kn.barrier_extra;
  p.use_tc = kn.use_tc;
  return p;
}

template <typename T>
void gate_to_T(const mps_c128* g, int count, T* out) {
  using R = typename real_of<T>::type;
  for (int i = 0; i < count; ++i) out[i] = mk<R>((R)g[i].re, (R)g[i].im);
}

#define CKE(x)                               \
  do {                                       \
    cudaError_t e_ = (x);                    \
    if (e_ != cudaSuccess) {                 \
      note_cuda_failure(__FILE__, __LINE__); \
      return e_;                             \
    }                                        \
  } while (0)

// The two-site gate pipeline on raw device pointers (Sec. III-C.2):
// theta contraction + gate -> truncated pivoted QR -> Q formation -> split.
template <typename T>
cudaError_t theta_step(const Ws<T>& w, const Knobs& kn, int cl, int cm, int cr, const T* A, const T* B, const T* g,
                       cudaStream_t s, LaunchHooks* hk, const T* gdev = nullptr) {
  const int m = 2 * cl, n = 2 * cr;
  hook_before(hk, MPS_KCLASS_THETA, ((double)m * cm + (double)cm * n + (double)m * n) * sizeof(T),
              8.0 * m * n * cm + 32.0 * m * n);
  if constexpr (std::is_same<T, c64>::value) {
    if (kn.use_tc)
      CKE(tc_theta(cl, cm, cr, A, B, g, w.W, w.ldw, w.err, kn.timeout_ns, s, gdev));
    else
      CKE(theta_gemm_simt<T>(cl, cm, cr, A, B, g, w.W, w.ldw, s, gdev));
  } else {
    CKE(theta_gemm_simt<T>(cl, cm, cr, A, B, g, w.W, w.ldw, s, gdev));
  }
  hook_after(hk, MPS_KCLASS_THETA, 1);
  return cudaSuccess;
}

struct SketchRef;
template <typename T>
void plan_sketch(QrPlan<T>& p, const SketchRef& sk);

// sk != nullptr: the pivots are chosen on a random sketch (MPS_TRUNC_RQRCP)
template <typename T>
cudaError_t two_site_core(const Ws<T>& w, const Knobs& kn, int cl, int cm, int cr, int chi, const T* A, const T* B,
                          const T* g, T* Aout, T* Bout, double* disc_slot, double* disc_total, cudaStream_t s,
                          LaunchHooks* hk, const SketchRef* sk = nullptr, const T* gdev = nullptr) {
  const int m = 2 * cl, n = 2 * cr;
  const int k = std::min(std::min(m, n), chi);
  if (!sk && kn.small && small_gate_fits(cl, cm, cr)) {
    // the whole split in one CTA
    SmallBatch<T> b;
    b.count = 1;
    b.item[0] = small_item<T>(cl, cm, cr, k, A, B, g, Aout, Bout, disc_slot, disc_total, w.jpvt, gdev);
    hook_before(hk, MPS_KCLASS_PANEL, ((double)m * cm + (double)cm * n + 2.0 * (m + n) * k) * sizeof(T),
                8.0 * m * n * cm + 16.0 * m * n * k + 8.0 * m * k * k);
    CKE(small_gate_launch<T>(b, s));
    hook_after(hk, MPS_KCLASS_PANEL, 1);
    return cudaSuccess;
  }
  CKE(theta_step<T>(w, kn, cl, cm, cr, A, B, g, s, hk, gdev));
  QrPlan<T> p = make_plan<T>(w, kn, m, n, k, 1, disc_slot, disc_total);
  if (sk) plan_sketch<T>(p, *sk);
  CKE(qr_factor<T>(p, s, hk));
  CKE(qr_form_q<T>(p, w.Q, w.ldq, s, hk));
  hook_before(hk, MPS_KCLASS_SPLIT, 2.0 * ((double)m * k + (double)k * n) * sizeof(T), 0);
  // left site (row-major m x k) <- Q (column-major m x k)
  CKE(transpose_copy<T>(w.Q, w.ldq, Aout, k, k, m, 0, s));
  // right site (row-major k x n) <- R P^T
  CKE(split_right<T>(w.W, w.ldw, w.jpvt, w.inv, k, n, Bout, s, w.err));
  hook_after(hk, MPS_KCLASS_SPLIT, 3);
  return cudaSuccess;
}

// scratch of the SVD split (MPS_TRUNC_SVD), carved from one buffer
struct SvdLayout {
  size_t X, V, sig2, tail, perm, rot, sweeps, part, fro2, total;
};

SvdLayout svd_layout(size_t esz, int mmax) {
  SvdLayout L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align_up(off + std::max<size_t>(bytes, 1));
    return o;
  };
  const size_t mm = (size_t)std::max(mmax, 1);
  L.X = take(esz * mm * mm);
  L.V = take(esz * mm * mm);
  L.sig2 = take(8 * mm);
  L.tail = take(8 * mm);
  L.perm = take(4 * mm);
  L.rot = take(4 * (size_t)kSvdMaxSweeps);
  L.sweeps = take(4);
  L.part = take(8 * (size_t)kSvdParts);
  L.fro2 = take(8);
  L.total = off;
  return L;
}

// scratch of the randomized-pivoting split (MPS_TRUNC_RQRCP), carved from one buffer
struct SkLayout {
  size_t Om, Ys, Yw, Ssk, tau, Wg, jpvt, seq, total;
  int lsk = 0;
  int64_t ldy = 0;
};

SkLayout sk_layout(size_t esz, int mmax, int nmax, int nb) {
  SkLayout L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align_up(off + std::max<size_t>(bytes, 1));
    return o;
  };
  L.lsk = 2 * nb + kSketchOversample;  // a block of two panels, plus oversampling
  L.ldy = (L.lsk + 3) / 4 * 4;
  const size_t mm = (size_t)std::max(mmax, 1), nn = (size_t)std::max(nmax, 1);
  L.Om = take(esz * L.ldy * mm);
  L.Ys = take(esz * L.ldy * nn);
  L.Yw = take(1);
  L.Ssk = take(esz * L.ldy * 2 * nb);
  L.tau = take(1);
  L.Wg = take(1);
  L.jpvt = take(1);
  L.seq = take(4 * 2 * (size_t)nb);
  L.total = off;
  return L;
}

// device pointers of that scratch for one split, with the sketch's generator state
struct SketchRef {
  char* base = nullptr;
  const SkLayout* L = nullptr;
  unsigned long long seed = 0;
};

template <typename T>
void plan_sketch(QrPlan<T>& p, const SketchRef& sk) {
  p.pivot = 2;
  p.lsk = sk.L->lsk;
  p.ldy = sk.L->ldy;
  p.Om = (T*)(sk.base + sk.L->Om);
  p.Ys = (T*)(sk.base + sk.L->Ys);
  p.Yw = (T*)(sk.base + sk.L->Yw);
  p.Ssk = (T*)(sk.base + sk.L->Ssk);
  p.sk_tau = (T*)(sk.base + sk.L->tau);
  p.sk_Wg = (c128*)(sk.base + sk.L->Wg);
  p.sk_jpvt = (int*)(sk.base + sk.L->jpvt);
  p.piv_seq = (int*)(sk.base + sk.L->seq);
  p.seed = sk.seed;
}

// The two-site gate with the truncated SVD split (MPS_TRUNC_SVD): theta as in
// two_site_core, then svd_split instead of the pivoted QR.
template <typename T>
cudaError_t two_site_svd(const Ws<T>& w, char* sbase, const SvdLayout& SL, const Knobs& kn, int cl, int cm, int cr,
                         int chi, const T* A, const T* B, const T* g, T* Aout, T* Bout, double* disc_slot,
                         double* disc_total, cudaStream_t s, LaunchHooks* hk) {
  const int m = 2 * cl, n = 2 * cr;
  CKE(theta_step<T>(w, kn, cl, cm, cr, A, B, g, s, hk));
  SvdPlan<T> p;
  p.m = m;
  p.n = n;
  p.k = std::min(std::min(m, n), chi);
  p.W = w.W;
  p.ldw = w.ldw;
  p.X = (T*)(sbase + SL.X);
  p.V = (T*)(sbase + SL.V);
  p.sig2 = (double*)(sbase + SL.sig2);
  p.tail = (double*)(sbase + SL.tail);
  p.perm = (int*)(sbase + SL.perm);
  p.rot = (int*)(sbase + SL.rot);
  p.sweeps = (int*)(sbase + SL.sweeps);
  p.part = (double*)(sbase + SL.part);
  p.fro2 = (double*)(sbase + SL.fro2);
  p.bar = w.bar;
  p.err = w.err;
  p.timeout_ns = kn.timeout_ns;
  p.barrier_extra = kn.barrier_extra;
  p.discarded = disc_slot;
  p.disc_total = disc_total;
  return svd_split<T>(p, Aout, Bout, s, hk);
}

// ---------------------------------------------------------------------------
// profiling / launch accounting
struct PendingEv {
  int kclass;
  cudaEvent_t a, b;
};

struct Profiler {
  LaunchHooks hooks;
  bool enabled = false;
  cudaStream_t stream = nullptr;
  mps_kstat stat[MPS_KCLASS_COUNT];
  std::vector<PendingEv> pending;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t cur_a = nullptr;
  Profiler() {
    memset(stat, 0, sizeof(stat));
    hooks.before = &Profiler::before_cb;
    hooks.after = &Profiler::after_cb;
    hooks.ctx = this;
  }
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  static void before_cb(LaunchHooks* h, int kclass, double bytes, double flops) {
    Profiler* p = (Profiler*)h->ctx;
    p->stat[kclass].alg_bytes += bytes;
    p->stat[kclass].alg_flops += flops;
    if (p->enabled) {
      p->cur_a = p->get();
      cudaEventRecord(p->cur_a, p->stream);
    }
  }
  static void after_cb(LaunchHooks* h, int kclass, int nlaunch) {
    Profiler* p = (Profiler*)h->ctx;
    p->stat[kclass].launches += nlaunch;
    if (p->enabled && p->cur_a) {
      cudaEvent_t b = p->get();
      cudaEventRecord(b, p->stream);
      p->pending.push_back({kclass, p->cur_a, b});
      p->cur_a = nullptr;
    }
  }
  void drain() {
    for (auto& e : pending) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, e.a, e.b) == cudaSuccess) stat[e.kclass].ms += ms;
      pool.push_back(e.a);
      pool.push_back(e.b);
    }
    pending.clear();
  }
  void destroy() {
    drain();
    for (auto e : pool) cudaEventDestroy(e);
    pool.clear();
  }
};

}  // namespace

// ---------------------------------------------------------------------------
// A lane of the layer path: its own stream and a workspace for gates up to
// kLaneDim rows and columns, so that small gates of one layer run concurrently.
struct Lane {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  char* ws = nullptr;
  WsLayout L;
  int64_t ldw = 0, ldq = 0;
};

struct GraphSlot {
  std::string key;  // layer shape: precision, bond cap, (site, bond dims) per gate
  cudaGraphExec_t exec = nullptr;
  char* staging = nullptr;   // pinned host copy of the layer's parameters, read by the graph's first node
  size_t staging_bytes = 0;
  cudaEvent_t done = nullptr;  // the graph's last launch has finished (staging reusable)
  long long launches = 0;
};

struct mps_s {
  int n = 0, chi_max = 0, prec = MPS_PREC_FP64, policy = MPS_POLICY_CANON, device = 0;
  cudaStream_t stream = nullptr, own_stream = nullptr;
  mps_alloc_fn ualloc = nullptr;
  mps_free_fn ufree = nullptr;
  void* actx = nullptr;
  std::vector<void*> allocs;
  std::vector<int> bond, capb;  // bond dims, reserved bond dims
  std::vector<int> physb;       // min(2^b, 2^(n-b), chi_max): the chain's Schmidt-rank bound
  // MPO zip-up scratch (lazy): carried block C and the product Y = C A
  char* mpo_ws = nullptr;
  size_t mpo_half = 0;
  std::vector<char*> site;
  int centre = 0;
  size_t esz = 16;
  // workspace
  char* ws = nullptr;
  WsLayout L;
  int64_t ldw = 0, ldq = 0;
  Knobs kn;
  // SVD split scratch (MPS_TRUNC_SVD only)
  int trunc = MPS_TRUNC_QRCP;
  char* svd_ws = nullptr;
  SvdLayout SL;
  // randomized-pivoting scratch (MPS_TRUNC_RQRCP only)
  char* sk_ws = nullptr;
  SkLayout SKL;
  unsigned long long sketch_seed = 0;
  // FP64 observables scratch
  double* d_partial = nullptr;
  double* d_scalar = nullptr;  // [0] norm, [1] total discarded
  double* d_disclog = nullptr;
  c128* d_vec = nullptr;  // 2 * chicap + 1
  int chicap = 1;
  // transfer-matrix scratch (lazy)
  c128* d_E = nullptr;
  size_t E_elems = 0;
  long long nsplit = 0;
  // shape of the last pivoted split whose pivots are still in the workspace
  // (0 = the workspace was used for something else since)
  int piv_n = 0, piv_k = 0;
  // layer path (lazy)
  std::vector<Lane> lanes;
  cudaEvent_t ev_fork = nullptr;
  // look-ahead of the centre moves' QR: a high-priority stream for its critical path
  // (panels on one cluster) and three events; null when it could not be created
  cudaStream_t la_stream = nullptr;
  cudaEvent_t la_ev[3] = {};
  bool graphs = true;           // layers are captured into CUDA graphs after the first call
  long long layer_calls = 0;
  long long graph_launches = 0;  // layers run as a graph launch
  std::vector<GraphSlot> graph_cache;
  // device parameters of a replayed layer: [0] the split counter of its first gate,
  // from byte 16 the gates in the data type (16 entries each); per-gate discarded
  // weights land in ldisc and are filed into the log by the graph's last kernel
  char* layer_dev = nullptr;
  double* ldisc = nullptr;
  // autotuning (MPS_FLAG_AUTOTUNE): scratch outputs of the timed candidate splits
  bool tune = false;
  char* tune_ws = nullptr;
  size_t tune_half = 0;
  // status
  int status = MPS_OK;
  std::string msg;
  Profiler prof;
};

namespace {

int fail(mps_t h, int code, const std::string& m) {
  if (h) {
    h->msg = m;
    if (code == MPS_E_TIMEOUT || code == MPS_E_CUDA) h->status = code;
  }
  return code;
}

thread_local const char* t_fail_file = nullptr;  // innermost failing call of this thread
thread_local int t_fail_line = 0;

}  // namespace

void mpsg::note_cuda_failure(const char* file, int line) {
  if (t_fail_file) return;  // the innermost site was recorded first
  const char* slash = std::strrchr(file, '/');
  t_fail_file = slash ? slash + 1 : file;
  t_fail_line = line;
}

namespace {

int cuda_fail(mps_t h, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  if (t_fail_file) m += std::string(" (at ") + t_fail_file + ":" + std::to_string(t_fail_line) + ")";
  t_fail_file = nullptr;
  return fail(h, e == cudaErrorMemoryAllocation ? MPS_E_NOMEM : MPS_E_CUDA, m);
}

#define CUTRY(h, x, where)                         \
  do {                                             \
    cudaError_t e_ = (x);                          \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, where); \
  } while (0)

void* dev_alloc(mps_t h, size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = kAlign;
  if (h->ualloc) {
    p = h->ualloc(bytes, h->actx);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) h->allocs.push_back(p);
  return p;
}

void release(mps_t h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (Lane& ln : h->lanes) {
    if (ln.stream) {
      cudaStreamSynchronize(ln.stream);
      cudaStreamDestroy(ln.stream);
    }
    if (ln.done) cudaEventDestroy(ln.done);
  }
  h->lanes.clear();
  for (GraphSlot& g : h->graph_cache) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.done) cudaEventDestroy(g.done);
    if (g.staging) cudaFreeHost(g.staging);
  }
  h->graph_cache.clear();
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  h->ev_fork = nullptr;
  if (h->la_stream) {
    cudaStreamSynchronize(h->la_stream);
    cudaStreamDestroy(h->la_stream);
    h->la_stream = nullptr;
  }
  for (cudaEvent_t& e : h->la_ev) {
    if (e) cudaEventDestroy(e);
    e = nullptr;
  }
  h->prof.destroy();
  for (void* p : h->allocs) {
    if (h->ufree)
      h->ufree(p, h->actx);
    else
      cudaFree(p);
  }
  h->allocs.clear();
  if (h->own_stream) cudaStreamDestroy(h->own_stream);
  h->own_stream = nullptr;
}

template <typename T>
Ws<T> views(mps_t h) {
  return ws_views<T>(h->ws, h->L, h->ldw, h->ldq);
}

int check_device_error(mps_t h) {
  int dev_err = 0;
  cudaError_t e = cudaMemcpyAsync(&dev_err, views<c64>(h).err, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "device sync");
  if (dev_err == DEV_ERR_TIMEOUT) return fail(h, MPS_E_TIMEOUT, "a bounded device-side wait expired");
  if (dev_err != DEV_OK) {
    h->status = MPS_E_CUDA;
    return fail(h, MPS_E_CUDA, "device-side check failed (code " + std::to_string(dev_err) + ")");
  }
  return MPS_OK;
}

int usable(mps_t h) {
  if (!h) return MPS_E_ARG;
  if (h->status != MPS_OK) {
    h->msg = "handle is in an error state: " + h->msg;
    return MPS_E_STATE;
  }
  if (cudaSetDevice(h->device) != cudaSuccess) return fail(h, MPS_E_CUDA, "cudaSetDevice failed");
  return MPS_OK;
}

// ---------------------------------------------------------------------------
// Autotuning of the two-site split.  Per (precision, m, n, k, SM count) the
// candidates panel width nb in {32, 16, 8} x CTAs of the pivoted panel kernel in
// {all, 3/4, 1/2 of the SMs} are timed on the problem itself (CUDA events, the
// best of `reps` runs after one warm-up) and the fastest is kept.  The GEMM tiles
// are not searched: the rank-nb and block-reflector products (K <= 64) always take
// the 64-row tile and the theta contraction the 128-row one.  One process-wide
// cache; when the environment variable MPS_TUNE_CACHE names a file, entries are
// read from it at first use and appended to it, one JSON object per line.
struct TuneEntry {
  int prec = 0, m = 0, n = 0, k = 0, sms = 0;
  int nb = 0, ctas = 0, candidates = 0;
  double ms = 0, default_ms = 0;
};
std::mutex g_tune_mu;
std::vector<TuneEntry> g_tune;
bool g_tune_loaded = false;

bool json_num(const char* line, const char* key, double* v) {
  char pat[64];
  snprintf(pat, sizeof pat, "\"%s\":", key);
  const char* q = strstr(line, pat);
  if (!q) return false;
  q += strlen(pat);
  while (*q == ' ') ++q;
  char* end = nullptr;
  const double x = strtod(q, &end);
  if (end == q) return false;
  *v = x;
  return true;
}

bool tune_parse(const char* line, TuneEntry* e) {
  double v[10];
  const char* keys[10] = {"m", "n", "k", "sms", "panel_width", "panel_ctas", "ms", "default_ms", "candidates",
                          "complex_bytes"};
  for (int i = 0; i < 10; ++i)
    if (!json_num(line, keys[i], &v[i])) return false;
  e->m = (int)v[0];
  e->n = (int)v[1];
  e->k = (int)v[2];
  e->sms = (int)v[3];
  e->nb = (int)v[4];
  e->ctas = (int)v[5];
  e->ms = v[6];
  e->default_ms = v[7];
  e->candidates = (int)v[8];
  e->prec = v[9] == 16 ? MPS_PREC_FP64 : MPS_PREC_MIXED;
  return e->nb >= 1 && e->nb <= kMaxNb && e->ctas >= 1;
}

TuneEntry* tune_find_locked(int prec, int m, int n, int k, int sms) {
  if (!g_tune_loaded) {
    g_tune_loaded = true;
    const char* path = getenv("MPS_TUNE_CACHE");
    if (path && *path) {
      if (FILE* f = fopen(path, "r")) {
        char line[512];
        while (fgets(line, sizeof line, f)) {
          TuneEntry e;
          if (tune_parse(line, &e)) g_tune.push_back(e);  // a later line for the same key wins
        }
        fclose(f);
      }
    }
  }
  TuneEntry* hit = nullptr;
  for (TuneEntry& e : g_tune)
    if (e.prec == prec && e.m == m && e.n == n && e.k == k && e.sms == sms) hit = &e;
  return hit;
}

void tune_store_locked(const TuneEntry& e) {
  g_tune.push_back(e);
  const char* path = getenv("MPS_TUNE_CACHE");
  if (!path || !*path) return;
  if (FILE* f = fopen(path, "a")) {
    fprintf(f,
            "{\"precision\": \"%s\", \"complex_bytes\": %d, \"m\": %d, \"n\": %d, \"k\": %d, \"sms\": %d, "
            "\"panel_width\": %d, \"panel_ctas\": %d, \"ms\": %.6g, \"default_ms\": %.6g, \"candidates\": %d}\n",
            e.prec == MPS_PREC_FP64 ? "c128" : "c64", e.prec == MPS_PREC_FP64 ? 16 : 8, e.m, e.n, e.k, e.sms, e.nb,
            e.ctas, e.ms, e.default_ms, e.candidates);
    fclose(f);
  }
}

// Time the candidates on one split: A, B inputs (read only), Aout, Bout and
// *disc scratch outputs; w a workspace laid out for nb = kMaxNb and base.G CTAs.
template <typename T>
cudaError_t tune_split(const Ws<T>& w, const Knobs& base, int cl, int cm, int cr, int chi, const T* A, const T* B,
                       const T* g, T* Aout, T* Bout, double* disc, cudaStream_t s, const SketchRef* sk,
                       TuneEntry* out) {
  const int sms = num_sms();
  const int nbs[3] = {32, 16, 8};
  const int ctas[3] = {sms, std::max(1, sms * 3 / 4), std::max(1, sms / 2)};
  cudaEvent_t e0, e1;
  CKE(cudaEventCreate(&e0));
  cudaError_t err = cudaEventCreate(&e1);
  if (err != cudaSuccess) {
    cudaEventDestroy(e0);
    return err;
  }
  auto run = [&](const Knobs& kn, int reps, float* best) -> cudaError_t {
    *best = 1e30f;
    for (int r = 0; r < reps; ++r) {
      CKE(cudaEventRecord(e0, s));
      CKE(two_site_core<T>(w, kn, cl, cm, cr, chi, A, B, g, Aout, Bout, disc, nullptr, s, nullptr, sk));
      CKE(cudaEventRecord(e1, s));
      CKE(cudaEventSynchronize(e1));
      float ms = 0.f;
      CKE(cudaEventElapsedTime(&ms, e0, e1));
      *best = std::min(*best, ms);
    }
    return cudaSuccess;
  };
  float t_def = 0.f;
  err = run(base, 1, &t_def);  // warm-up (first-use set-up of the kernels)
  int reps = 3;
  if (err == cudaSuccess) {
    err = run(base, 1, &t_def);
    reps = t_def > 50.f ? 1 : 3;
  }
  float t_best = 1e30f;
  int best_nb = base.nb, best_g = base.G, cand = 0;
  for (int a = 0; a < 3 && err == cudaSuccess; ++a)
    for (int b = 0; b < 3 && err == cudaSuccess; ++b) {
      if (nbs[a] > base.nb || ctas[b] > base.G) continue;
      Knobs kn = base;
      kn.nb = nbs[a];
      kn.G = ctas[b];
      float t = 0.f;
      err = run(kn, reps, &t);
      ++cand;
      if (err == cudaSuccess && t < t_best) {
        t_best = t;
        best_nb = kn.nb;
        best_g = kn.G;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return err;
  out->m = 2 * cl;
  out->n = 2 * cr;
  out->k = std::min(std::min(2 * cl, 2 * cr), chi);
  out->sms = sms;
  out->nb = best_nb;
  out->ctas = best_g;
  out->ms = t_best;
  out->default_ms = t_def;
  out->candidates = cand;
  return cudaSuccess;
}

// Knobs of the split of gate g on (i, i+1) of a handle: the defaults, or with
// MPS_FLAG_AUTOTUNE the cached choice for the shape, tuned now (on the handle's
// stream and workspace, outputs to scratch, the state untouched) if there is none.
template <typename T>
int tuned_knobs(mps_t h, int i, const T* gt, int chi, const SketchRef* sk, Knobs* kn) {
  *kn = h->kn;
  if (!h->tune || h->trunc != MPS_TRUNC_QRCP) return MPS_OK;  // the QP3 split only
  const int cl = h->bond[i], cm = h->bond[i + 1], cr = h->bond[i + 2];
  if (h->kn.small && small_gate_fits(cl, cm, cr)) return MPS_OK;  // one CTA: no knobs
  const int m = 2 * cl, n = 2 * cr, k = std::min(std::min(m, n), chi);
  TuneEntry e;
  bool have = false;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    if (TuneEntry* hit = tune_find_locked(h->prec, m, n, k, num_sms())) {
      e = *hit;
      have = true;
    }
  }
  if (!have) {
    if (!h->tune_ws) {
      h->tune_half = align_up(h->esz * 2 * (size_t)h->chicap * h->chicap);
      h->tune_ws = (char*)dev_alloc(h, 2 * h->tune_half + kAlign);
      if (!h->tune_ws) return fail(h, MPS_E_NOMEM, "autotune: scratch");
    }
    cudaError_t err = tune_split<T>(views<T>(h), h->kn, cl, cm, cr, chi, (const T*)h->site[i],
                                    (const T*)h->site[i + 1], gt, (T*)h->tune_ws, (T*)(h->tune_ws + h->tune_half),
                                    (double*)(h->tune_ws + 2 * h->tune_half), h->stream, sk, &e);
    if (err != cudaSuccess) return cuda_fail(h, err, "autotune");
    e.prec = h->prec;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_store_locked(e);
  }
  kn->nb = std::min(e.nb, h->kn.nb);
  kn->G = std::min(e.ctas, h->kn.G);
  return MPS_OK;
}

// ---- centre moves (Sec. III-C.1): plain QR rightward, LQ leftward, no truncation
// Look-ahead scratch of a centre move's QR: the main stream's GEMM scratch lives in
// the Q buffer, which the factorisation does not use (Q is formed after it).
template <typename T>
void plan_lookahead(mps_t h, QrPlan<T>& p, const Ws<T>& w) {
  if (!h->la_stream) return;
  const int64_t wide = 2 * (int64_t)std::max(h->chicap, 1);
  const int64_t yz = 2 * (int64_t)p.nb * wide;
  if (p.n > wide || p.k > wide || 2 * yz + p.sk_cap > h->ldq * (int64_t)std::max(h->chicap, 1)) return;
  p.s2 = h->la_stream;
  p.la_ev = h->la_ev;
  p.Y2 = w.Q;
  p.Z2 = w.Q + yz;
  p.SK2 = w.Q + 2 * yz;
}

template <typename T>
int move_right(mps_t h, int j) {
  using R = typename real_of<T>::type;
  Ws<T> w = views<T>(h);
  h->piv_n = 0;
  const int cl = h->bond[j], cr = h->bond[j + 1], cn = h->bond[j + 2];
  const int m = 2 * cl, n = cr, k = std::min(m, n);
  T* sj = (T*)h->site[j];
  T* sn = (T*)h->site[j + 1];
  cudaStream_t s = h->stream;
  LaunchHooks* hk = &h->prof.hooks;
  hook_before(hk, MPS_KCLASS_CANON, 2.0 * m * n * sizeof(T), 0);
  CUTRY(h, transpose_copy<T>(sj, n, w.W, w.ldw, m, n, 0, s), "move_right copy");
  hook_after(hk, MPS_KCLASS_CANON, 1);
  QrPlan<T> p = make_plan<T>(w, h->kn, m, n, k, 0, nullptr, nullptr);
  p.kclass = MPS_KCLASS_CANON;
  plan_lookahead<T>(h, p, w);
  CUTRY(h, qr_factor<T>(p, s, hk), "move_right qr");
  CUTRY(h, qr_form_q<T>(p, w.Q, w.ldq, s, hk), "move_right form_q");
  hook_before(hk, MPS_KCLASS_CANON, 2.0 * m * k * sizeof(T), 0);
  CUTRY(h, transpose_copy<T>(w.Q, w.ldq, sj, k, k, m, 0, s), "move_right split");
  hook_after(hk, MPS_KCLASS_CANON, 1);
  // next site (k x 2cn) = R (k x cr, upper) * site_{j+1} (cr x 2cn); computed transposed into Q
  GemmDesc<T> d;
  d.M = 2 * cn;
  d.N = k;
  d.K = cr;
  d.alpha = mk<R>(1, 0);
  d.beta = mk<R>(0, 0);
  d.A = sn;
  d.lda = 2 * cn;
  d.a_row = 0;
  d.a_conj = 0;
  d.a_mask = MASK_NONE;
  d.B = w.W;
  d.ldb = w.ldw;
  d.b_row = 1;
  d.b_conj = 0;
  d.b_mask = MASK_UPPER;
  d.C = w.Q;
  d.ldc = 2 * cn;
  hook_before(hk, MPS_KCLASS_CANON, ((double)2 * cn * cr + (double)k * cr + 2.0 * cn * k) * sizeof(T),
              8.0 * 2 * cn * k * cr);
  CUTRY(h, gemm_auto<T>(d, h->kn.use_tc, w.err, h->kn.timeout_ns, s), "move_right absorb");
  hook_after(hk, MPS_KCLASS_CANON, 1);
  CUTRY(h, cudaMemcpyAsync(sn, w.Q, sizeof(T) * (size_t)k * 2 * cn, cudaMemcpyDeviceToDevice, s), "move_right copy");
  h->bond[j + 1] = k;
  return MPS_OK;
}

template <typename T>
int move_left(mps_t h, int j) {
  using R = typename real_of<T>::type;
  Ws<T> w = views<T>(h);
  h->piv_n = 0;
  const int cp = h->bond[j - 1], cl = h->bond[j], cr = h->bond[j + 1];
  const int m = 2 * cr, n = cl, k = std::min(m, n);
  T* sj = (T*)h->site[j];
  T* sp = (T*)h->site[j - 1];
  cudaStream_t s = h->stream;
  LaunchHooks* hk = &h->prof.hooks;
  // W (column-major 2cr x cl) = M^H, M = site j as cl x 2cr row-major
  hook_before(hk, MPS_KCLASS_CANON, 2.0 * m * n * sizeof(T), 0);
  CUTRY(h, copy2d<T>(sj, m, w.W, w.ldw, cl, m, 1, s), "move_left copy");
  hook_after(hk, MPS_KCLASS_CANON, 1);
  QrPlan<T> p = make_plan<T>(w, h->kn, m, n, k, 0, nullptr, nullptr);
  p.kclass = MPS_KCLASS_CANON;
  plan_lookahead<T>(h, p, w);
  CUTRY(h, qr_factor<T>(p, s, hk), "move_left qr");
  CUTRY(h, qr_form_q<T>(p, w.Q, w.ldq, s, hk), "move_left form_q");
  // site j (k x 2cr row-major) = Q^H
  hook_before(hk, MPS_KCLASS_CANON, 2.0 * m * k * sizeof(T), 0);
  CUTRY(h, copy2d<T>(w.Q, w.ldq, sj, m, k, m, 1, s), "move_left split");
  hook_after(hk, MPS_KCLASS_CANON, 1);
  // previous site (2cp x k) = site_{j-1} (2cp x cl) * R^H; transposed: conj(R) (k x cl) * site^T
  GemmDesc<T> d;
  d.M = k;
  d.N = 2 * cp;
  d.K = cl;
  d.alpha = mk<R>(1, 0);
  d.beta = mk<R>(0, 0);
  d.A = w.W;
  d.lda = w.ldw;
  d.a_row = 0;
  d.a_conj = 1;
  d.a_mask = MASK_UPPER;
  d.B = sp;
  d.ldb = cl;
  d.b_row = 0;
  d.b_conj = 0;
  d.b_mask = MASK_NONE;
  d.C = w.Q;
  d.ldc = k;
  hook_before(hk, MPS_KCLASS_CANON, ((double)2 * cp * cl + (double)k * cl + 2.0 * cp * k) * sizeof(T),
              8.0 * 2 * cp * k * cl);
  CUTRY(h, gemm_auto<T>(d, h->kn.use_tc, w.err, h->kn.timeout_ns, s), "move_left absorb");
  hook_after(hk, MPS_KCLASS_CANON, 1);
  CUTRY(h, cudaMemcpyAsync(sp, w.Q, sizeof(T) * (size_t)k * 2 * cp, cudaMemcpyDeviceToDevice, s), "move_left copy");
  h->bond[j] = k;
  return MPS_OK;
}

template <typename T>
int move_centre_t(mps_t h, int target) {
  while (h->centre < target) {
    int rc = move_right<T>(h, h->centre);
    if (rc) return rc;
    h->centre++;
  }
  while (h->centre > target) {
    int rc = move_left<T>(h, h->centre);
    if (rc) return rc;
    h->centre--;
  }
  return MPS_OK;
}

template <typename T>
int apply_2q_t(mps_t h, int i, const mps_c128* g, int chi) {
  if (h->policy == MPS_POLICY_CANON) {
    int rc = move_centre_t<T>(h, i);
    if (rc) return rc;
  }
  Ws<T> w = views<T>(h);
  T gt[16];
  gate_to_T<T>(g, 16, gt);
  const int cl = h->bond[i], cm = h->bond[i + 1], cr = h->bond[i + 2];
  const int k = std::min(std::min(2 * cl, 2 * cr), chi);
  double* slot = h->d_disclog + (h->nsplit % kDiscLog);
  cudaError_t e;
  h->piv_n = 0;
  SketchRef sk;
  sk.base = h->sk_ws;
  sk.L = &h->SKL;
  sk.seed = h->sketch_seed + (unsigned long long)h->nsplit;  // split number s: seed + s
  const SketchRef* skp = h->trunc == MPS_TRUNC_RQRCP ? &sk : nullptr;
  Knobs kn;
  int rc = tuned_knobs<T>(h, i, gt, chi, skp, &kn);
  if (rc) return rc;
  if (h->trunc == MPS_TRUNC_SVD)
    e = two_site_svd<T>(w, h->svd_ws, h->SL, kn, cl, cm, cr, chi, (const T*)h->site[i], (const T*)h->site[i + 1],
                        gt, (T*)h->site[i], (T*)h->site[i + 1], slot, h->d_scalar + 1, h->stream, &h->prof.hooks);
  else
    e = two_site_core<T>(w, kn, cl, cm, cr, chi, (const T*)h->site[i], (const T*)h->site[i + 1], gt,
                         (T*)h->site[i], (T*)h->site[i + 1], slot, h->d_scalar + 1, h->stream, &h->prof.hooks, skp);
  if (e != cudaSuccess) return cuda_fail(h, e, "apply_2q");
  if (h->trunc != MPS_TRUNC_SVD) {
    h->piv_n = 2 * cr;
    h->piv_k = k;
  }
  h->bond[i + 1] = k;
  h->nsplit++;
  if (h->policy == MPS_POLICY_CANON) h->centre = i + 1;
  return MPS_OK;
}

// ---------------------------------------------------------------------------
// MPO application by zip-up (Sec. III-C.3).  Left to right over the MPO's
// sites: Y = C A_i (C carried from the previous split, identity at the first
// site), Z = W_i contracted into Y, Z split by the truncated pivoted QR (Q to the
// site, R P^T carried on); the last Z is the last site.  The new bond is capped
// by the reserved room (twice the chain's bound), and bonds left above the
// chain's bound are brought back to it by identity-gate splits, right to left.
constexpr mps_c128 kIdentity4[16] = {{1, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {1, 0}, {0, 0}, {0, 0},
                                     {0, 0}, {0, 0}, {1, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {1, 0}};

template <typename T>
int apply_1q_t(mps_t h, int q, const mps_c128* u);

int mpo_ready(mps_t h) {
  if (h->mpo_ws) return MPS_OK;
  h->mpo_half = align_up(h->esz * (size_t)(2 * h->chicap) * (2 * h->chicap));
  h->mpo_ws = (char*)dev_alloc(h, 2 * h->mpo_half);
  if (!h->mpo_ws) return fail(h, MPS_E_NOMEM, "apply_mpo: scratch");
  return MPS_OK;
}

template <typename T>
int apply_mpo_t(mps_t h, int first, int count, const int* bonds, const mps_c128* W, int chi) {
  if (count == 1) return apply_1q_t<T>(h, first, W);  // W[0][0] is the 2 x 2 operator (out, in)
  int rc = mpo_ready(h);
  if (rc) return rc;
  if (h->policy == MPS_POLICY_CANON) {
    rc = move_centre_t<T>(h, first);
    if (rc) return rc;
  }
  Ws<T> w = views<T>(h);
  h->piv_n = 0;
  LaunchHooks* hk = &h->prof.hooks;
  T* Y = (T*)h->mpo_ws;
  T* C = (T*)(h->mpo_ws + h->mpo_half);
  const int last = first + count - 1;
  int kk = h->bond[first], adim = 1;
  int cl = h->bond[first];  // left bond of site i as stored (bond[i] already holds the new k)
  const mps_c128* wj = W;
  for (int j = 0; j < count; ++j) {
    const int i = first + j;
    const int cr = h->bond[i + 1], bdim = bonds[j + 1];
    MpoTensor<T> wt;
    for (int e = 0; e < 16; ++e) wt.w[e] = mk<typename real_of<T>::type>(0, 0);
    for (int a = 0; a < adim; ++a)
      for (int b = 0; b < bdim; ++b)
        for (int o = 0; o < 4; ++o) {
          const mps_c128 x = wj[(a * bdim + b) * 4 + o];
          wt.w[(a * 2 + b) * 4 + o] = mk<typename real_of<T>::type>((typename real_of<T>::type)x.re,
                                                                    (typename real_of<T>::type)x.im);
        }
    wj += adim * bdim * 4;
    const T* ysrc = (const T*)h->site[i];
    int64_t yr = 2 * (int64_t)cr, yc = 1;
    int nl = 1;
    hook_before(hk, MPS_KCLASS_THETA, 0, j ? 8.0 * kk * adim * 2.0 * cr * cl : 0);
    if (j > 0) {
      // Y (column-major, (kk adim) x (2 cr)) = C (row-major (kk adim) x cl) . A_i (row-major cl x 2 cr)
      GemmDesc<T> d;
      d.M = kk * adim;
      d.N = 2 * cr;
      d.K = cl;
      d.alpha = mk<typename real_of<T>::type>(1, 0);
      d.beta = mk<typename real_of<T>::type>(0, 0);
      d.A = C;
      d.lda = cl;
      d.a_row = 1;
      d.B = (const T*)h->site[i];
      d.ldb = 2 * cr;
      d.b_row = 1;
      d.C = Y;
      d.ldc = d.M;
      cudaError_t e = gemm_simt<T>(d, h->stream);
      if (e != cudaSuccess) return cuda_fail(h, e, "apply_mpo: carried product");
      nl += gemm_launches(d);
      ysrc = Y;
      yr = 1;
      yc = d.M;
    }
    if (i == last) {
      cudaError_t e = mpo_contract<T>(ysrc, yr, yc, kk, adim, 1, cr, wt, (T*)h->site[i], 0, 1, h->stream);
      hook_after(hk, MPS_KCLASS_THETA, nl);
      if (e != cudaSuccess) return cuda_fail(h, e, "apply_mpo: last site");
      break;
    }
    cudaError_t e = mpo_contract<T>(ysrc, yr, yc, kk, adim, bdim, cr, wt, w.W, w.ldw, 0, h->stream);
    hook_after(hk, MPS_KCLASS_THETA, nl);
    if (e != cudaSuccess) return cuda_fail(h, e, "apply_mpo: contraction");
    const int m = 2 * kk, nn = bdim * cr;
    const int k = std::min(std::min(m, nn), std::min(chi, h->capb[i + 1]));
    double* slot = h->d_disclog + (h->nsplit % kDiscLog);
    QrPlan<T> p = make_plan<T>(w, h->kn, m, nn, k, 1, slot, h->d_scalar + 1);
    e = qr_factor<T>(p, h->stream, hk);
    if (e == cudaSuccess) e = qr_form_q<T>(p, w.Q, w.ldq, h->stream, hk);
    if (e != cudaSuccess) return cuda_fail(h, e, "apply_mpo: split");
    hook_before(hk, MPS_KCLASS_SPLIT, 2.0 * ((double)m * k + (double)k * nn) * sizeof(T), 0);
    e = transpose_copy<T>(w.Q, w.ldq, (T*)h->site[i], k, k, m, 0, h->stream);
    if (e == cudaSuccess) e = split_right<T>(w.W, w.ldw, w.jpvt, w.inv, k, nn, C, h->stream, w.err);
    hook_after(hk, MPS_KCLASS_SPLIT, 3);
    if (e != cudaSuccess) return cuda_fail(h, e, "apply_mpo: split");
    h->bond[i + 1] = k;
    h->nsplit++;
    kk = k;
    adim = bdim;
    cl = cr;
  }
  if (h->policy == MPS_POLICY_CANON) h->centre = last;
  for (int b = last; b > first; --b) {
    if (h->bond[b] <= h->physb[b]) continue;
    rc = apply_2q_t<T>(h, b - 1, kIdentity4, h->physb[b]);
    if (rc) return rc;
  }
  return MPS_OK;
}

// ---------------------------------------------------------------------------
// Layer path (batching of a circuit layer's gates on disjoint bonds): gates
// whose theta is at most kLaneDim x kLaneDim run concurrently on kLanes lanes
// (own stream and workspace each, greedy balance by work), larger ones in order
// on the handle's stream, which then waits for every lane.  Gates touch
// disjoint sites, so the order between them does not matter; the discarded
// weights are logged per gate and added to the total in gate order afterwards,
// so the total is the same sum as on the one-by-one path.
constexpr int kLanes = 8;
constexpr int kLaneDim = 4096;

__global__ void add_slots_kernel(const double* log, int first, int count, double* total) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = *total;
    for (int j = 0; j < count; ++j) t += log[(first + j) % kDiscLog];
    *total = t;
  }
}

int lanes_ready(mps_t h) {
  if (!h->lanes.empty()) return MPS_OK;
  const int dim = std::min(kLaneDim, 2 * h->chicap);
  CUTRY(h, cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming), "layer lanes");
  h->lanes.resize(kLanes);
  for (Lane& ln : h->lanes) {
    CUTRY(h, cudaStreamCreateWithFlags(&ln.stream, cudaStreamNonBlocking), "layer lanes");
    CUTRY(h, cudaEventCreateWithFlags(&ln.done, cudaEventDisableTiming), "layer lanes");
    // same split-K capacity as the handle's workspace: a lane makes the same
    // split choices, so a layer gives exactly the one-by-one result
    ln.L = ws_layout(h->esz, dim, dim, dim, h->kn.nb, h->kn.G, ln.ldw, ln.ldq, 2 * h->chicap);
    ln.ws = (char*)dev_alloc(h, ln.L.total);
    if (!ln.ws) return fail(h, MPS_E_NOMEM, "layer lanes: workspace");
    // the allocation is stream-ordered on the handle's stream; the lane starts after it
    CUTRY(h, cudaMemsetAsync(ln.ws + ln.L.bar, 0, 16, h->stream), "layer lanes");
  }
  // parameters of replayed layers (at most n - 1 gates)
  h->layer_dev = (char*)dev_alloc(h, 16 + (size_t)h->n * 16 * h->esz);
  h->ldisc = (double*)dev_alloc(h, sizeof(double) * (size_t)h->n);
  if (!h->layer_dev || !h->ldisc) return fail(h, MPS_E_NOMEM, "layer parameters");
  CUTRY(h, cudaStreamSynchronize(h->stream), "layer lanes");
  return MPS_OK;
}

// last node of a replayed layer: file the per-gate discarded weights into the log
// at the split counter held in the parameter block, and add them to the total in
// gate order (the same sum as add_slots_kernel's)
__global__ void file_disc_kernel(const double* ldisc, int count, const long long* first, double* log,
                                 double* total) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const long long f = *first;
    double t = *total;
    for (int j = 0; j < count; ++j) {
      log[(f + j) % kDiscLog] = ldisc[j];
      t += ldisc[j];
    }
    *total = t;
  }
}

constexpr size_t kGraphCache = 16;  // executable layer graphs kept per handle

template <typename T>
int layer_t(mps_t h, const int* sites, const mps_c128* gates, int count, int chi) {
  // per-class event timing needs one stream; the SVD split has one scratch per handle
  if (h->prof.enabled || count <= 1 || h->trunc != MPS_TRUNC_QRCP) {
    for (int j = 0; j < count; ++j) {
      int rc = apply_2q_t<T>(h, sites[j], gates + 16 * j, chi);
      if (rc) return rc;
    }
    return MPS_OK;
  }
  int rc = lanes_ready(h);
  if (rc) return rc;
  h->piv_n = 0;
  struct Item {
    int j, cl, cm, cr, k;
    double work;
  };
  std::vector<Item> small, big, tiny;
  for (int j = 0; j < count; ++j) {
    const int i = sites[j];
    Item it;
    it.j = j;
    it.cl = h->bond[i];
    it.cm = h->bond[i + 1];
    it.cr = h->bond[i + 2];
    it.k = std::min(std::min(2 * it.cl, 2 * it.cr), chi);
    const double m = 2.0 * it.cl, n = 2.0 * it.cr;
    it.work = m * n * (it.cm + it.k) + 1e6;  // contraction + factorisation, plus a fixed latency share
    if (h->kn.small && small_gate_fits(it.cl, it.cm, it.cr))
      tiny.push_back(it);  // one CTA each, all in one grouped launch
    else
      (2 * it.cl <= kLaneDim && 2 * it.cr <= kLaneDim ? small : big).push_back(it);
  }
  std::sort(small.begin(), small.end(), [](const Item& a, const Item& b) { return a.work > b.work; });
  // split knobs per gate (autotuned shapes are tuned here, before any lane starts)
  std::vector<Knobs> kj(count);
  for (int j = 0; j < count; ++j) {
    T gt[16];
    gate_to_T<T>(gates + 16 * j, 16, gt);
    rc = tuned_knobs<T>(h, sites[j], gt, chi, nullptr, &kj[j]);
    if (rc) return rc;
  }
  const int64_t first = h->nsplit;
  auto slot_of = [&](int j) { return h->d_disclog + ((first + j) % kDiscLog); };
  const int* err_main = views<T>(h).err;
  // lane gates share the SMs: each panel kernel gets a slice of them, but at
  // least one CTA per 128 rows of theta, with which the per-CTA partial sums of
  // every panel step are those of a full grid, so results do not change.
  const int share = num_sms() / std::max(1, std::min<int>((int)small.size(), kLanes));
  // Every launch of the layer, in order: the lanes' gates, the grouped launches of
  // the small gates, the large gates on the handle's stream, the join and the
  // filing of the discarded weights.  With `staging` (a replayable layer, captured
  // into a CUDA graph) the gates are read from the device parameter block, which the
  // first node copies from the pinned staging buffer, and the discarded weights go
  // through ldisc.  Returns the first failing call's error.
  auto issue = [&](const char* staging, size_t staging_bytes) -> cudaError_t {
    const bool rp = staging != nullptr;
    const T* gbase = rp ? reinterpret_cast<const T*>(h->layer_dev + 16) : nullptr;
    auto disc_of = [&](int j) { return rp ? h->ldisc + j : slot_of(j); };
    auto gdev_of = [&](int j) { return rp ? gbase + 16 * j : nullptr; };
    if (rp) CKE(cudaMemcpyAsync(h->layer_dev, staging, staging_bytes, cudaMemcpyHostToDevice, h->stream));
    CKE(cudaEventRecord(h->ev_fork, h->stream));
    std::vector<double> load(kLanes, 0.0);
    std::vector<char> used(kLanes, 0);
    for (const Item& it : small) {
      const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      Lane& ln = h->lanes[l];
      if (!used[l]) {
        CKE(cudaStreamWaitEvent(ln.stream, h->ev_fork, 0));
        used[l] = 1;
      }
      load[l] += it.work;
      Ws<T> w = ws_views<T>(ln.ws, ln.L, ln.ldw, ln.ldq);
      w.err = const_cast<int*>(err_main);  // one error word per handle
      T gt[16];
      gate_to_T<T>(gates + 16 * it.j, 16, gt);
      const int i = sites[it.j];
      Knobs kl = kj[it.j];
      kl.G = std::min(kl.G, std::max((2 * it.cl + 127) / 128, share));
      CKE(two_site_core<T>(w, kl, it.cl, it.cm, it.cr, chi, (const T*)h->site[i], (const T*)h->site[i + 1], gt,
                           (T*)h->site[i], (T*)h->site[i + 1], disc_of(it.j), nullptr, ln.stream, &h->prof.hooks,
                           nullptr, gdev_of(it.j)));
    }
    // the gates whose theta fits one CTA: one grouped launch per kSmallBatch of them
    for (size_t b0 = 0; b0 < tiny.size(); b0 += kSmallBatch) {
      SmallBatch<T> sb;
      sb.count = (int)std::min<size_t>(kSmallBatch, tiny.size() - b0);
      for (int q = 0; q < sb.count; ++q) {
        const Item& it = tiny[b0 + q];
        T gt[16];
        gate_to_T<T>(gates + 16 * it.j, 16, gt);
        const int i = sites[it.j];
        sb.item[q] = small_item<T>(it.cl, it.cm, it.cr, it.k, (const T*)h->site[i], (const T*)h->site[i + 1], gt,
                                   (T*)h->site[i], (T*)h->site[i + 1], disc_of(it.j), nullptr, nullptr,
                                   gdev_of(it.j));
      }
      CKE(small_gate_launch<T>(sb, h->stream));
    }
    for (const Item& it : big) {
      T gt[16];
      gate_to_T<T>(gates + 16 * it.j, 16, gt);
      const int i = sites[it.j];
      CKE(two_site_core<T>(views<T>(h), kj[it.j], it.cl, it.cm, it.cr, chi, (const T*)h->site[i],
                           (const T*)h->site[i + 1], gt, (T*)h->site[i], (T*)h->site[i + 1], disc_of(it.j), nullptr,
                           h->stream, &h->prof.hooks, nullptr, gdev_of(it.j)));
    }
    for (int l = 0; l < kLanes; ++l) {
      if (!used[l]) continue;
      CKE(cudaEventRecord(h->lanes[l].done, h->lanes[l].stream));
      CKE(cudaStreamWaitEvent(h->stream, h->lanes[l].done, 0));
    }
    if (rp)
      file_disc_kernel<<<1, 32, 0, h->stream>>>(h->ldisc, count, reinterpret_cast<const long long*>(h->layer_dev),
                                                h->d_disclog, h->d_scalar + 1);
    else
      add_slots_kernel<<<1, 32, 0, h->stream>>>(h->d_disclog, (int)(first % kDiscLog), count, h->d_scalar + 1);
    return cudaGetLastError();
  };
  // After the first layer call (which sets every kernel up), each layer shape
  // (precision, bond cap, and per gate the site and its three bond dims) is
  // captured once into a CUDA graph whose parameters (the gates and the split
  // counter) live in device memory; a layer of a known shape is then one graph
  // launch after its parameters are written to the pinned staging buffer that the
  // graph's first node copies.  If the stream cannot be captured, the layer is
  // issued directly and graphs stay off for the handle.
  bool done = false;
  if (h->graphs && h->layer_calls > 0) {
    std::string key = std::to_string(h->prec) + ":" + std::to_string(chi);
    for (int j = 0; j < count; ++j) {
      const int i = sites[j];
      key += ";" + std::to_string(i) + "," + std::to_string(h->bond[i]) + "," + std::to_string(h->bond[i + 1]) + "," +
             std::to_string(h->bond[i + 2]);
    }
    GraphSlot* slot = nullptr;
    for (GraphSlot& g : h->graph_cache)
      if (g.key == key) slot = &g;
    cudaError_t e = cudaSuccess;
    if (!slot) {
      GraphSlot g;
      g.key = key;
      g.staging_bytes = 16 + (size_t)count * 16 * sizeof(T);
      cudaGraph_t graph = nullptr;
      e = cudaMallocHost(&g.staging, g.staging_bytes);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        const cudaError_t ei = issue(g.staging, g.staging_bytes);
        e = cudaStreamEndCapture(h->stream, &graph);
        if (ei != cudaSuccess) e = ei;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (e == cudaSuccess) {
        if (h->graph_cache.size() >= kGraphCache) {
          GraphSlot& old = h->graph_cache.front();
          cudaEventSynchronize(old.done);
          cudaGraphExecDestroy(old.exec);
          cudaEventDestroy(old.done);
          cudaFreeHost(old.staging);
          h->graph_cache.erase(h->graph_cache.begin());
        }
        h->graph_cache.push_back(g);
        slot = &h->graph_cache.back();
      } else {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.done) cudaEventDestroy(g.done);
        if (g.staging) cudaFreeHost(g.staging);
      }
    }
    if (e == cudaSuccess && slot) {
      // the previous launch of this graph has copied its parameters: the staging is free
      e = cudaEventSynchronize(slot->done);
      if (e == cudaSuccess) {
        long long f = first;
        memcpy(slot->staging, &f, sizeof f);
        T* gs = reinterpret_cast<T*>(slot->staging + 16);
        for (int j = 0; j < count; ++j) gate_to_T<T>(gates + 16 * j, 16, gs + 16 * j);
        e = cudaGraphLaunch(slot->exec, h->stream);
      }
      if (e == cudaSuccess) {
        // the layer is enqueued: never issue it a second time
        slot->launches++;
        h->graph_launches++;
        done = true;
        CUTRY(h, cudaEventRecord(slot->done, h->stream), "apply_layer: graph event");
      }
    }
    if (!done) {
      cudaGetLastError();
      h->graphs = false;  // issue directly from now on
    }
  }
  if (!done) {
    cudaError_t e = issue(nullptr, 0);
    if (e != cudaSuccess) return cuda_fail(h, e, "apply_layer");
  }
  h->layer_calls++;
  for (const Item& it : small) h->bond[sites[it.j] + 1] = it.k;
  for (const Item& it : big) h->bond[sites[it.j] + 1] = it.k;
  for (const Item& it : tiny) h->bond[sites[it.j] + 1] = it.k;
  h->nsplit += count;
  return MPS_OK;
}

template <typename T>
int apply_1q_t(mps_t h, int q, const mps_c128* u) {
  T ut[4];
  gate_to_T<T>(u, 4, ut);
  LaunchHooks* hk = &h->prof.hooks;
  hook_before(hk, MPS_KCLASS_OTHER, 2.0 * h->bond[q] * 2 * h->bond[q + 1] * sizeof(T), 0);
  cudaError_t e = apply_1q<T>((T*)h->site[q], h->bond[q], h->bond[q + 1], ut, h->stream);
  hook_after(hk, MPS_KCLASS_OTHER, 1);
  if (e != cudaSuccess) return cuda_fail(h, e, "apply_1q");
  return MPS_OK;
}

template <typename T>
int amplitude_t(mps_t h, const uint8_t* bits, mps_c128* out) {
  c128* v0 = h->d_vec;
  c128* v1 = h->d_vec + h->chicap + 1;
  c128 one = mk<double>(1, 0);
  CUTRY(h, cudaMemcpyAsync(v0, &one, sizeof(c128), cudaMemcpyHostToDevice, h->stream), "amplitude");
  LaunchHooks* hk = &h->prof.hooks;
  for (int i = 0; i < h->n; ++i) {
    const int cl = h->bond[i], cr = h->bond[i + 1];
    const T* M = (const T*)h->site[i] + (bits[i] ? cr : 0);
    hook_before(hk, MPS_KCLASS_OTHER, (double)cl * cr * sizeof(T), 8.0 * cl * cr);
    CUTRY(h, vecmat<T>(v0, M, 2 * cr, cl, cr, v1, h->stream), "amplitude vecmat");
    hook_after(hk, MPS_KCLASS_OTHER, 1);
    std::swap(v0, v1);
  }
  c128 r;
  CUTRY(h, cudaMemcpyAsync(&r, v0, sizeof(c128), cudaMemcpyDeviceToHost, h->stream), "amplitude");
  int rc = check_device_error(h);
  if (rc) return rc;
  out->re = r.re;
  out->im = r.im;
  return MPS_OK;
}

template <typename T>
int centre_norm_t(mps_t h, double* out) {
  const int c = h->centre;
  int64_t cnt = (int64_t)h->bond[c] * 2 * h->bond[c + 1];
  LaunchHooks* hk = &h->prof.hooks;
  hook_before(hk, MPS_KCLASS_OTHER, (double)cnt * sizeof(T), 0);
  CUTRY(h, norm2_sum<T>((const T*)h->site[c], cnt, h->d_partial, kNormParts, h->d_scalar, h->stream), "norm");
  hook_after(hk, MPS_KCLASS_OTHER, 2);
  CUTRY(h, cudaMemcpyAsync(out, h->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, h->stream), "norm");
  return check_device_error(h);
}

// site data of handle x as complex128 (converted into scratch when needed)
const c128* site_c128(mps_t x, int i, c128* scratch, cudaStream_t s) {
  if (x->prec == MPS_PREC_FP64) return (const c128*)x->site[i];
  int64_t cnt = (int64_t)x->bond[i] * 2 * x->bond[i + 1];
  convert<c128, c64>((const c64*)x->site[i], scratch, cnt, s);
  return scratch;
}

int ensure_transfer_scratch(mps_t h, size_t need) {
  if (h->E_elems >= need) return MPS_OK;
  void* p = dev_alloc(h, need * sizeof(c128));
  if (!p) return fail(h, MPS_E_NOMEM, "transfer-matrix scratch allocation failed");
  h->d_E = (c128*)p;
  h->E_elems = need;
  return MPS_OK;
}

// <a|b> by transfer matrices in FP64, computed on a's stream with a's scratch
int overlap_impl(mps_t a, mps_t b, mps_c128* out) {
  const int n = a->n;
  size_t cap = 0;
  for (int i = 0; i < n; ++i) {
    cap = std::max(cap, (size_t)a->capb[i] * 2 * a->capb[i + 1]);
    cap = std::max(cap, (size_t)b->capb[i] * 2 * b->capb[i + 1]);
  }
  size_t eb = 0;
  for (int i = 0; i <= n; ++i) eb = std::max(eb, (size_t)a->capb[i] * b->capb[i]);
  size_t tmpb = 0;
  for (int i = 0; i < n; ++i) tmpb = std::max(tmpb, (size_t)a->capb[i] * b->capb[i + 1]);
  size_t need = 2 * eb + tmpb + 2 * cap + 4;
  int rc = ensure_transfer_scratch(a, need);
  if (rc) return rc;
  c128* E0 = a->d_E;
  c128* E1 = E0 + eb;
  c128* tmp = E1 + eb;
  c128* sa = tmp + tmpb;
  c128* sb = sa + cap;
  cudaStream_t s = a->stream;
  if (b->stream != s) {
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(a, e, "overlap sync");
  }
  c128 one = mk<double>(1, 0);
  CUTRY(a, cudaMemcpyAsync(E0, &one, sizeof(c128), cudaMemcpyHostToDevice, s), "overlap");
  LaunchHooks* hk = &a->prof.hooks;
  for (int i = 0; i < n; ++i) {
    const int la = a->bond[i], ra = a->bond[i + 1], lb = b->bond[i], rb = b->bond[i + 1];
    hook_before(hk, MPS_KCLASS_OTHER, 0, 16.0 * la * lb * rb + 16.0 * ra * la * rb);
    const c128* A = site_c128(a, i, sa, s);
    const c128* B = site_c128(b, i, sb, s);
    int nl = (a->prec == MPS_PREC_MIXED) + (b->prec == MPS_PREC_MIXED);
    for (int sg = 0; sg < 2; ++sg) {
      GemmDesc<c128> d;
      // tmp (la x rb) = E (la x lb) * B^s (lb x rb)
      d.M = la;
      d.N = rb;
      d.K = lb;
      d.alpha = mk<double>(1, 0);
      d.beta = mk<double>(0, 0);
      d.A = E0;
      d.lda = la;
      d.a_row = 0;
      d.a_conj = 0;
      d.a_mask = MASK_NONE;
      d.B = B + sg * rb;
      d.ldb = 2 * rb;
      d.b_row = 1;
      d.b_conj = 0;
      d.b_mask = MASK_NONE;
      d.C = tmp;
      d.ldc = la;
      CUTRY(a, gemm_simt<c128>(d, s), "overlap gemm");
      // E1 (ra x rb) (+)= A^s^H (ra x la) * tmp
      d.M = ra;
      d.N = rb;
      d.K = la;
      d.beta = mk<double>(sg == 0 ? 0 : 1, 0);
      d.A = A + sg * ra;
      d.lda = 2 * ra;
      d.a_row = 0;
      d.a_conj = 1;
      d.B = tmp;
      d.ldb = la;
      d.b_row = 0;
      d.C = E1;
      d.ldc = ra;
      CUTRY(a, gemm_simt<c128>(d, s), "overlap gemm");
    }
    hook_after(hk, MPS_KCLASS_OTHER, 4 + nl);
    std::swap(E0, E1);
  }
  c128 r;
  CUTRY(a, cudaMemcpyAsync(&r, E0, sizeof(c128), cudaMemcpyDeviceToHost, s), "overlap");
  rc = check_device_error(a);
  if (rc) return rc;
  out->re = r.re;
  out->im = r.im;
  return MPS_OK;
}

bool valid_site(mps_t h, int i) { return i >= 0 && i < h->n; }

}  // namespace

// Scratch space of mps_two_site_apply_noalloc.  In host code this name is only
// a stand-in for the device array: its device address comes from
// cudaGetSymbolAddress, looked up once per device with that device current.
static __device__ __align__(256) unsigned char g_noalloc_scratch[MPS_NOALLOC_SCRATCH_BYTES];

namespace {
// waits of the raw-pointer calls (mps_debug_raw_wait changes them for tests)
constexpr unsigned long long kRawTimeoutNs = 10000000000ull;
std::atomic<int> g_raw_barrier_extra{0};
std::atomic<unsigned long long> g_raw_timeout_ns{kRawTimeoutNs};

// after a raw-pointer split: a device-side failure (an expired bounded wait, a
// failed check) leaves the outputs undefined, and the discarded weight becomes NaN
__global__ void raw_status_kernel(const char* err_word, double* disc) {
  if (*reinterpret_cast<const volatile int*>(err_word) != DEV_OK) *disc = __longlong_as_double(0x7ff8000000000000ll);
}

constexpr int kNoallocDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoallocDevices] = {};
}  // namespace

// ===========================================================================
// C ABI
extern "C" {

int mps_version(void) { return 100; }

}  // extern "C"

namespace {
__global__ void fill_random_kernel(c64* p, int64_t n, unsigned seed) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t x = (uint64_t)i * 0x9E3779B97F4A7C15ull + seed;
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdull;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ull;
  x ^= x >> 33;
  p[i] = mk<float>((float)((x & 0xffffff) / 8388608.0 - 1.0), (float)(((x >> 24) & 0xffffff) / 8388608.0 - 1.0));
}
}  // namespace

extern "C" {

int mps_selftest_gemm(int M, int N, int K, int a_row, int a_conj, int a_mask, int b_row, int b_conj, int b_mask,
                      int theta, unsigned seed, double* max_abs_err, double* max_abs_ref) {
  if (M < 1 || N < 1 || K < 1 || !max_abs_err || !max_abs_ref) return MPS_E_ARG;
  const int64_t na = (int64_t)(theta ? 2 * M : M) * K, nb = (int64_t)K * (theta ? 2 * N : N);
  const int64_t nc = theta ? (int64_t)(2 * M) * (2 * N) : (int64_t)M * N;
  c64 *A = nullptr, *B = nullptr, *C1 = nullptr, *C2 = nullptr;
  int* err = nullptr;
  int rc = MPS_OK;
  if (cudaMalloc(&A, sizeof(c64) * na) != cudaSuccess || cudaMalloc(&B, sizeof(c64) * nb) != cudaSuccess ||
      cudaMalloc(&C1, sizeof(c64) * nc) != cudaSuccess || cudaMalloc(&C2, sizeof(c64) * nc) != cudaSuccess ||
      cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
    rc = MPS_E_NOMEM;
  } else {
    cudaMemset(err, 0, sizeof(int));
    fill_random_kernel<<<(unsigned)((na + 255) / 256), 256>>>(A, na, seed);
    fill_random_kernel<<<(unsigned)((nb + 255) / 256), 256>>>(B, nb, seed + 17);
    fill_random_kernel<<<(unsigned)((nc + 255) / 256), 256>>>(C1, nc, seed + 29);
    cudaMemcpy(C2, C1, sizeof(c64) * nc, cudaMemcpyDeviceToDevice);
    cudaError_t e1, e2;
    if (theta) {
      c64 g[16];
      for (int i = 0; i < 16; ++i) g[i] = mk<float>(0.25f * ((i * 7) % 5 - 2), 0.125f * ((i * 3) % 7 - 3));
      e1 = tc_theta(M, K, N, A, B, g, C1, 2 * M, err, 10000000000ull, 0);
      e2 = theta_gemm_simt<c64>(M, K, N, A, B, g, C2, 2 * M, 0);
    } else {
      GemmDesc<c64> d;
      d.M = M;
      d.N = N;
      d.K = K;
      d.alpha = mk<float>(0.7f, 0.2f);
      d.beta = mk<float>(0.3f, -0.5f);
      d.A = A;
      d.lda = a_row ? K : M;
      d.a_row = a_row;
      d.a_conj = a_conj;
      d.a_mask = a_mask;
      d.B = B;
      d.ldb = b_row ? N : K;
      d.b_row = b_row;
      d.b_conj = b_conj;
      d.b_mask = b_mask;
      d.C = C1;
      d.ldc = M;
      e1 = tc_gemm(d, err, 10000000000ull, 0);
      d.C = C2;
      e2 = gemm_simt<c64>(d, 0);
    }
    cudaError_t e3 = cudaDeviceSynchronize();
    int herr = 0;
    cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
      rc = MPS_E_CUDA;
    } else if (herr != 0) {
      rc = MPS_E_TIMEOUT;
    } else {
      std::vector<c64> h1(nc), h2(nc);
      cudaMemcpy(h1.data(), C1, sizeof(c64) * nc, cudaMemcpyDeviceToHost);
      cudaMemcpy(h2.data(), C2, sizeof(c64) * nc, cudaMemcpyDeviceToHost);
      double me = 0, mr = 0;
      for (int64_t i = 0; i < nc; ++i) {
        me = std::max(me, (double)std::fabs(h1[i].re - h2[i].re));
        me = std::max(me, (double)std::fabs(h1[i].im - h2[i].im));
        mr = std::max(mr, (double)std::fabs(h2[i].re));
        mr = std::max(mr, (double)std::fabs(h2[i].im));
      }
      *max_abs_err = me;
      *max_abs_ref = mr;
    }
  }
  cudaFree(A);
  cudaFree(B);
  cudaFree(C1);
  cudaFree(C2);
  cudaFree(err);
  return rc;
}

void mps_config_init(mps_config* cfg) {
  if (!cfg) return;
  memset(cfg, 0, sizeof(*cfg));
  cfg->precision = MPS_PREC_FP64;
  cfg->policy = MPS_POLICY_CANON;
}

int mps_create(mps_t* out, int n, int chi_max) { return mps_create_ex(out, n, chi_max, nullptr); }

int mps_create_ex(mps_t* out, int n, int chi_max, const mps_config* cfg_in) {
  if (!out) return MPS_E_ARG;
  *out = nullptr;
  mps_config cfg;
  if (cfg_in)
    cfg = *cfg_in;
  else
    mps_config_init(&cfg);
  if (n < 1 || n > 4096 || chi_max < 1 || chi_max > 65536) return MPS_E_ARG;
  if (cfg.precision != MPS_PREC_FP64 && cfg.precision != MPS_PREC_MIXED) return MPS_E_ARG;
  if (cfg.policy != MPS_POLICY_CANON && cfg.policy != MPS_POLICY_LOCAL) return MPS_E_ARG;
  if (cfg.panel_width < 0 || cfg.panel_width > kMaxNb) return MPS_E_ARG;
  if ((cfg.alloc == nullptr) != (cfg.free == nullptr)) return MPS_E_ARG;
  if (cfg.wait_timeout_s < 0) return MPS_E_ARG;
  if (cfg.debug_barrier_extra < 0 || cfg.debug_max_ctas < 0) return MPS_E_ARG;
  if (cfg.truncation != MPS_TRUNC_QRCP && cfg.truncation != MPS_TRUNC_SVD && cfg.truncation != MPS_TRUNC_RQRCP)
    return MPS_E_ARG;
  if (cfg.truncation == MPS_TRUNC_SVD && chi_max > kSvdMaxChi) return MPS_E_UNSUPPORTED;
  mps_s* h = new (std::nothrow) mps_s();
  if (!h) return MPS_E_NOMEM;
  h->n = n;
  h->chi_max = chi_max;
  h->prec = cfg.precision;
  h->policy = cfg.policy;
  h->trunc = cfg.truncation;
  h->sketch_seed = (unsigned long long)(unsigned)cfg.sketch_seed;
  h->device = cfg.device;
  h->ualloc = cfg.alloc;
  h->ufree = cfg.free;
  h->actx = cfg.alloc_ctx;
  h->esz = h->prec == MPS_PREC_FP64 ? sizeof(c128) : sizeof(c64);
  h->kn.nb = cfg.panel_width > 0 ? cfg.panel_width : kDefaultNb;
  h->kn.flag_tol = h->prec == MPS_PREC_FP64 ? 1.4901161193847656e-08 : 1e-3;
  double to = cfg.wait_timeout_s > 0 ? cfg.wait_timeout_s : 10.0;
  h->kn.timeout_ns = (unsigned long long)(to * 1e9);
  h->kn.barrier_extra = (unsigned)cfg.debug_barrier_extra;
  h->prof.enabled = (cfg.flags & MPS_FLAG_PROFILE) != 0;
  h->kn.use_tc = h->prec == MPS_PREC_MIXED && (cfg.flags & MPS_FLAG_TENSOR_CORES) != 0;
  h->tune = (cfg.flags & MPS_FLAG_AUTOTUNE) != 0;
  h->graphs = (cfg.flags & MPS_FLAG_NO_GRAPH) == 0;
  // the debug knobs exercise the grid kernels' barriers and row loops, which the
  // one-CTA path of small splits does not have
  h->kn.small = cfg.debug_barrier_extra == 0 && cfg.debug_max_ctas == 0;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
    cudaGetLastError();
    delete h;
    return MPS_E_CUDA;
  }
  if (h->device < 0 || h->device >= ndev) {
    delete h;
    return MPS_E_ARG;
  }
  if (cudaSetDevice(h->device) != cudaSuccess) {
    delete h;
    return MPS_E_CUDA;
  }
  int sms = num_sms();
  h->kn.G = std::min(sms, kMaxCoop);
  if (cfg.debug_max_ctas > 0) h->kn.G = std::min(h->kn.G, cfg.debug_max_ctas);
  if (cfg.stream) {
    h->stream = (cudaStream_t)cfg.stream;
  } else {
    if (cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete h;
      return MPS_E_CUDA;
    }
    h->stream = h->own_stream;
  }
  h->prof.stream = h->stream;
  {
    // the centre moves' look-ahead stream, at the highest priority so that the panels
    // on it get their SMs ahead of the trailing updates; without it the QR runs on
    // the handle's stream alone
    int lo = 0, hi = 0;
    bool ok = cudaDeviceGetStreamPriorityRange(&lo, &hi) == cudaSuccess &&
              cudaStreamCreateWithPriority(&h->la_stream, cudaStreamNonBlocking, hi) == cudaSuccess;
    for (cudaEvent_t& e : h->la_ev) ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      if (h->la_stream) cudaStreamDestroy(h->la_stream);
      h->la_stream = nullptr;
      for (cudaEvent_t& e : h->la_ev) {
        if (e) cudaEventDestroy(e);
        e = nullptr;
      }
    }
  }
  // bond dims and reserved capacities
  h->bond.assign(n + 1, 1);
  h->capb.resize(n + 1);
  int chicap = 1;
  // reserved bonds: twice the chain's bound (at most chi_max), the room an MPO of
  // bond 2 needs while it is zipped up; the outer bonds stay 1
  h->physb.resize(n + 1);
  for (int b = 0; b <= n; ++b) {
    h->physb[b] = max_bond(n, b, chi_max);
    h->capb[b] = (b == 0 || b == n) ? 1 : (int)std::min<int64_t>(2 * (int64_t)h->physb[b], chi_max);
    chicap = std::max(chicap, h->capb[b]);
  }
  h->chicap = chicap;
  // sites: one allocation
  std::vector<size_t> off(n);
  size_t total = 0;
  for (int i = 0; i < n; ++i) {
    off[i] = total;
    total = align_up(total + h->esz * (size_t)h->capb[i] * 2 * h->capb[i + 1]);
  }
  char* sites = (char*)dev_alloc(h, total);
  if (!sites) {
    release(h);
    delete h;
    return MPS_E_NOMEM;
  }
  h->site.resize(n);
  for (int i = 0; i < n; ++i) h->site[i] = sites + off[i];
  // workspace: largest split (m, n <= 2 chicap, k <= chicap)
  h->L = ws_layout(h->esz, 2 * chicap, 2 * chicap, chicap, h->kn.nb, h->kn.G, h->ldw, h->ldq);
  h->ws = (char*)dev_alloc(h, h->L.total);
  h->d_partial = (double*)dev_alloc(h, sizeof(double) * (kNormParts + 8));
  h->d_disclog = (double*)dev_alloc(h, sizeof(double) * kDiscLog);
  h->d_vec = (c128*)dev_alloc(h, sizeof(c128) * (2 * (size_t)chicap + 2));
  if (h->trunc == MPS_TRUNC_SVD) {
    h->SL = svd_layout(h->esz, 2 * chicap);
    h->svd_ws = (char*)dev_alloc(h, h->SL.total);
  }
  if (h->trunc == MPS_TRUNC_RQRCP) {
    h->SKL = sk_layout(h->esz, 2 * chicap, 2 * chicap, h->kn.nb);
    h->sk_ws = (char*)dev_alloc(h, h->SKL.total);
  }
  if (!h->ws || !h->d_partial || !h->d_disclog || !h->d_vec || (h->trunc == MPS_TRUNC_SVD && !h->svd_ws) ||
      (h->trunc == MPS_TRUNC_RQRCP && !h->sk_ws)) {
    release(h);
    delete h;
    return MPS_E_NOMEM;
  }
  h->d_scalar = h->d_partial + kNormParts;
  cudaError_t e = cudaMemsetAsync(h->ws + h->L.bar, 0, 16, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->ws + h->L.err, 0, 16, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_scalar, 0, 8 * sizeof(double), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(sites, 0, total, h->stream);
  if (e == cudaSuccess && h->svd_ws) e = cudaMemsetAsync(h->svd_ws + h->SL.rot, 0, h->SL.part - h->SL.rot, h->stream);
  // |0...0>: every site (1, 2, 1) = [1, 0]
  if (e == cudaSuccess) {
    std::vector<char> one(h->esz, 0);
    if (h->prec == MPS_PREC_FP64) {
      c128 v = mk<double>(1, 0);
      memcpy(one.data(), &v, sizeof v);
    } else {
      c64 v = mk<float>(1, 0);
      memcpy(one.data(), &v, sizeof v);
    }
    for (int i = 0; i < n && e == cudaSuccess; ++i)
      e = cudaMemcpyAsync(h->site[i], one.data(), h->esz, cudaMemcpyHostToDevice, h->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    release(h);
    delete h;
    return e == cudaErrorMemoryAllocation ? MPS_E_NOMEM : MPS_E_CUDA;
  }
  h->centre = 0;
  *out = h;
  return MPS_OK;
}

int mps_destroy(mps_t h) {
  if (!h) return MPS_OK;
  cudaSetDevice(h->device);
  release(h);
  delete h;
  return MPS_OK;
}

const char* mps_last_error(mps_t h) {
  if (!h) return "null handle";
  return h->msg.c_str();
}

int mps_set_stream(mps_t h, void* stream) {
  if (!h) return MPS_E_ARG;
  cudaStream_t ns = stream ? (cudaStream_t)stream : h->own_stream;
  if (!ns) return fail(h, MPS_E_ARG, "no stream to fall back to");
  if (ns != h->stream) {
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "set_stream");
  }
  h->stream = ns;
  h->prof.stream = ns;
  return MPS_OK;
}

int mps_sync(mps_t h) {
  if (!h) return MPS_E_ARG;
  if (h->status != MPS_OK) return h->status;
  cudaSetDevice(h->device);
  return check_device_error(h);
}

int mps_apply_1q(mps_t h, int site, const mps_c128 u[4]) {
  int rc = usable(h);
  if (rc) return rc;
  if (!valid_site(h, site) || !u) return fail(h, MPS_E_ARG, "apply_1q: bad site or gate");
  return h->prec == MPS_PREC_FP64 ? apply_1q_t<c128>(h, site, u) : apply_1q_t<c64>(h, site, u);
}

int mps_apply_2q(mps_t h, int site, const mps_c128 g[16], int chi_max) {
  int rc = usable(h);
  if (rc) return rc;
  if (site < 0 || site + 1 >= h->n || !g) return fail(h, MPS_E_ARG, "apply_2q: bad site or gate");
  if (chi_max > h->chi_max) return fail(h, MPS_E_ARG, "apply_2q: chi_max above the handle's");
  int chi = chi_max <= 0 ? h->chi_max : chi_max;
  return h->prec == MPS_PREC_FP64 ? apply_2q_t<c128>(h, site, g, chi) : apply_2q_t<c64>(h, site, g, chi);
}

// SWAP: g[(2b+a)*4 + (2a+b)] = 1 (output (b, a) from input (a, b)); a constant table, so
// handles on different threads share it without a first-use race
constexpr mps_c128 kSwap4[16] = {{1, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {1, 0}, {0, 0},
                                 {0, 0}, {1, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {1, 0}};

static const mps_c128* swap_gate() { return kSwap4; }

int mps_swap(mps_t h, int site, int chi_max) { return mps_apply_2q(h, site, swap_gate(), chi_max); }

int mps_apply_2q_routed(mps_t h, int q1, int q2, const mps_c128 g[16], int chi_max) {
  int rc = usable(h);
  if (rc) return rc;
  if (q1 < 0 || q2 < 0 || q1 >= h->n || q2 >= h->n || q1 == q2 || !g)
    return fail(h, MPS_E_ARG, "apply_2q_routed: bad positions or gate");
  mps_c128 gg[16];
  memcpy(gg, g, sizeof gg);
  if (q1 > q2) {
    // the same gate with its two qubits listed in the other order: S g S
    const mps_c128* S = swap_gate();
    mps_c128 t[16];
    for (int r = 0; r < 4; ++r)
      for (int c = 0; c < 4; ++c) {
        double re = 0, im = 0;
        for (int x = 0; x < 4; ++x)
          for (int y = 0; y < 4; ++y) {
            double sr = S[r * 4 + x].re * S[y * 4 + c].re;
            if (sr == 0.0) continue;
            re += sr * g[x * 4 + y].re;
            im += sr * g[x * 4 + y].im;
          }
        t[r * 4 + c].re = re;
        t[r * 4 + c].im = im;
      }
    memcpy(gg, t, sizeof gg);
    std::swap(q1, q2);
  }
  for (int b = q1; b < q2 - 1; ++b) {
    rc = mps_swap(h, b, chi_max);
    if (rc) return rc;
  }
  rc = mps_apply_2q(h, q2 - 1, gg, chi_max);
  if (rc) return rc;
  for (int b = q2 - 2; b >= q1; --b) {
    rc = mps_swap(h, b, chi_max);
    if (rc) return rc;
  }
  return MPS_OK;
}

int mps_permute(mps_t h, const int* order, int chi_max, long long* swaps) {
  int rc = usable(h);
  if (rc) return rc;
  if (!order) return fail(h, MPS_E_ARG, "permute: null order");
  if (chi_max > h->chi_max) return fail(h, MPS_E_ARG, "permute: chi_max above the handle's");
  std::vector<int> dest(h->n, -1);  // dest[q] = final position of the site now at q
  for (int p = 0; p < h->n; ++p) {
    const int q = order[p];
    if (q < 0 || q >= h->n || dest[q] >= 0) return fail(h, MPS_E_ARG, "permute: order is not a permutation");
    dest[q] = p;
  }
  long long count = 0;
  for (bool changed = true; changed;) {
    changed = false;
    for (int q = 0; q + 1 < h->n; ++q) {
      if (dest[q] > dest[q + 1]) {
        rc = mps_swap(h, q, chi_max);
        if (rc) return rc;
        std::swap(dest[q], dest[q + 1]);
        ++count;
        changed = true;
      }
    }
  }
  if (swaps) *swaps = count;
  return MPS_OK;
}

int mps_permute_layers(mps_t h, const int* order, int chi_max, long long* swaps, int* passes) {
  int rc = usable(h);
  if (rc) return rc;
  if (!order) return fail(h, MPS_E_ARG, "permute_layers: null order");
  if (chi_max > h->chi_max) return fail(h, MPS_E_ARG, "permute_layers: chi_max above the handle's");
  if (h->policy != MPS_POLICY_LOCAL) return fail(h, MPS_E_STATE, "permute_layers: needs the local policy");
  std::vector<int> dest(h->n, -1);  // dest[q] = final position of the site now at q
  for (int p = 0; p < h->n; ++p) {
    const int q = order[p];
    if (q < 0 || q >= h->n || dest[q] >= 0) return fail(h, MPS_E_ARG, "permute_layers: order is not a permutation");
    dest[q] = p;
  }
  long long count = 0;
  int npass = 0;
  std::vector<int> sites;
  std::vector<mps_c128> gates;
  for (int parity = 0, idle = 0; idle < 2; parity ^= 1) {
    sites.clear();
    for (int q = parity; q + 1 < h->n; q += 2)
      if (dest[q] > dest[q + 1]) {
        sites.push_back(q);
        std::swap(dest[q], dest[q + 1]);
      }
    if (sites.empty()) {
      ++idle;
      continue;
    }
    idle = 0;
    gates.resize(16 * sites.size());
    for (size_t j = 0; j < sites.size(); ++j) memcpy(&gates[16 * j], swap_gate(), 16 * sizeof(mps_c128));
    rc = mps_apply_layer(h, sites.data(), gates.data(), (int)sites.size(), chi_max);
    if (rc) return rc;
    count += (long long)sites.size();
    ++npass;
  }
  if (swaps) *swaps = count;
  if (passes) *passes = npass;
  return MPS_OK;
}

int mps_apply_layer(mps_t h, const int* sites, const mps_c128* gates, int count, int chi_max) {
  int rc = usable(h);
  if (rc) return rc;
  if (count < 0 || (count > 0 && (!sites || !gates))) return fail(h, MPS_E_ARG, "apply_layer: bad arrays");
  if (h->policy != MPS_POLICY_LOCAL) return fail(h, MPS_E_STATE, "apply_layer needs MPS_POLICY_LOCAL");
  std::vector<char> used(h->n, 0);
  for (int j = 0; j < count; ++j) {
    int s = sites[j];
    if (s < 0 || s + 1 >= h->n) return fail(h, MPS_E_ARG, "apply_layer: bad site");
    if (used[s] || used[s + 1]) return fail(h, MPS_E_ARG, "apply_layer: bonds overlap");
    used[s] = used[s + 1] = 1;
  }
  if (chi_max > h->chi_max) return fail(h, MPS_E_ARG, "apply_layer: chi_max above the handle's");
  if (chi_max <= 0) chi_max = h->chi_max;
  return h->prec == MPS_PREC_FP64 ? layer_t<c128>(h, sites, gates, count, chi_max)
                                  : layer_t<c64>(h, sites, gates, count, chi_max);
}

int mps_apply_mpo(mps_t h, int first, int count, const int* bonds, const mps_c128* W, int chi_max) {
  int rc = usable(h);
  if (rc) return rc;
  if (!bonds || !W || count < 1 || first < 0 || first + count > h->n)
    return fail(h, MPS_E_ARG, "apply_mpo: bad range or null pointer");
  if (bonds[0] != 1 || bonds[count] != 1) return fail(h, MPS_E_ARG, "apply_mpo: outer MPO bonds must be 1");
  for (int j = 1; j < count; ++j) {
    if (bonds[j] < 1) return fail(h, MPS_E_ARG, "apply_mpo: MPO bond below 1");
    if (bonds[j] > 2) return fail(h, MPS_E_UNSUPPORTED, "apply_mpo: MPO bonds above 2 are not supported");
  }
  if (chi_max > h->chi_max) return fail(h, MPS_E_ARG, "apply_mpo: chi_max above the handle's");
  int chi = chi_max <= 0 ? h->chi_max : chi_max;
  return h->prec == MPS_PREC_FP64 ? apply_mpo_t<c128>(h, first, count, bonds, W, chi)
                                  : apply_mpo_t<c64>(h, first, count, bonds, W, chi);
}

int mps_amplitude(mps_t h, const uint8_t* bits, mps_c128* out) {
  int rc = usable(h);
  if (rc) return rc;
  if (!bits || !out) return fail(h, MPS_E_ARG, "amplitude: null pointer");
  for (int i = 0; i < h->n; ++i)
    if (bits[i] > 1) return fail(h, MPS_E_ARG, "amplitude: bits must be 0 or 1");
  return h->prec == MPS_PREC_FP64 ? amplitude_t<c128>(h, bits, out) : amplitude_t<c64>(h, bits, out);
}

int mps_fidelity_estimate(mps_t h, double* out) {
  int rc = usable(h);
  if (rc) return rc;
  if (!out) return fail(h, MPS_E_ARG, "fidelity: null pointer");
  if (h->policy == MPS_POLICY_CANON)
    return h->prec == MPS_PREC_FP64 ? centre_norm_t<c128>(h, out) : centre_norm_t<c64>(h, out);
  mps_c128 o;
  rc = overlap_impl(h, h, &o);
  if (rc) return rc;
  *out = o.re;
  return MPS_OK;
}

int mps_overlap(mps_t a, mps_t b, mps_c128* out) {
  int rc = usable(a);
  if (rc) return rc;
  rc = usable(b);
  if (rc) return rc;
  if (!out || a->n != b->n || a->device != b->device) return fail(a, MPS_E_ARG, "overlap: incompatible handles");
  return overlap_impl(a, b, out);
}

int mps_bond_dims(mps_t h, int* out) {
  if (!h || !out) return MPS_E_ARG;
  for (int i = 0; i <= h->n; ++i) out[i] = h->bond[i];
  return MPS_OK;
}

int mps_get_site(mps_t h, int site, int host_fmt, void* host, size_t cap_elems) {
  int rc = usable(h);
  if (rc) return rc;
  if (!valid_site(h, site) || !host || (host_fmt != MPS_HOST_C128 && host_fmt != MPS_HOST_C64))
    return fail(h, MPS_E_ARG, "get_site: bad argument");
  int64_t cnt = (int64_t)h->bond[site] * 2 * h->bond[site + 1];
  if ((size_t)cnt > cap_elems) return fail(h, MPS_E_ARG, "get_site: host buffer too small");
  const bool same = (host_fmt == MPS_HOST_C128) == (h->prec == MPS_PREC_FP64);
  const void* src = h->site[site];
  size_t hsz = host_fmt == MPS_HOST_C128 ? sizeof(c128) : sizeof(c64);
  if (!same) {
    LaunchHooks* hk = &h->prof.hooks;
    hook_before(hk, MPS_KCLASS_OTHER, (double)cnt * (h->esz + hsz), 0);
    cudaError_t e;
    char* stage = h->ws + h->L.W;
    if (host_fmt == MPS_HOST_C128)
      e = convert<c128, c64>((const c64*)src, (c128*)stage, cnt, h->stream);
    else
      e = convert<c64, c128>((const c128*)src, (c64*)stage, cnt, h->stream);
    hook_after(hk, MPS_KCLASS_OTHER, 1);
    if (e != cudaSuccess) return cuda_fail(h, e, "get_site convert");
    src = stage;
  }
  CUTRY(h, cudaMemcpyAsync(host, src, hsz * cnt, cudaMemcpyDeviceToHost, h->stream), "get_site copy");
  return check_device_error(h);
}

int mps_set_site(mps_t h, int site, int chi_l, int chi_r, int host_fmt, const void* host) {
  int rc = usable(h);
  if (rc) return rc;
  if (!valid_site(h, site) || !host || (host_fmt != MPS_HOST_C128 && host_fmt != MPS_HOST_C64))
    return fail(h, MPS_E_ARG, "set_site: bad argument");
  if (chi_l < 1 || chi_r < 1 || chi_l > h->capb[site] || chi_r > h->capb[site + 1])
    return fail(h, MPS_E_ARG, "set_site: bond dims outside the reserved capacity");
  if ((site == 0 && chi_l != 1) || (site == h->n - 1 && chi_r != 1))
    return fail(h, MPS_E_ARG, "set_site: boundary bonds must be 1");
  int64_t cnt = (int64_t)chi_l * 2 * chi_r;
  const bool same = (host_fmt == MPS_HOST_C128) == (h->prec == MPS_PREC_FP64);
  size_t hsz = host_fmt == MPS_HOST_C128 ? sizeof(c128) : sizeof(c64);
  if (same) {
    CUTRY(h, cudaMemcpyAsync(h->site[site], host, hsz * cnt, cudaMemcpyHostToDevice, h->stream), "set_site copy");
  } else {
    char* stage = h->ws + h->L.W;
    CUTRY(h, cudaMemcpyAsync(stage, host, hsz * cnt, cudaMemcpyHostToDevice, h->stream), "set_site copy");
    LaunchHooks* hk = &h->prof.hooks;
    hook_before(hk, MPS_KCLASS_OTHER, (double)cnt * (h->esz + hsz), 0);
    cudaError_t e;
    if (host_fmt == MPS_HOST_C128)
      e = convert<c64, c128>((const c128*)stage, (c64*)h->site[site], cnt, h->stream);
    else
      e = convert<c128, c64>((const c64*)stage, (c128*)h->site[site], cnt, h->stream);
    hook_after(hk, MPS_KCLASS_OTHER, 1);
    if (e != cudaSuccess) return cuda_fail(h, e, "set_site convert");
  }
  h->bond[site] = chi_l;
  h->bond[site + 1] = chi_r;
  return MPS_OK;
}

int mps_set_centre(mps_t h, int centre) {
  if (!h) return MPS_E_ARG;
  if (!valid_site(h, centre)) return fail(h, MPS_E_ARG, "set_centre: bad site");
  h->centre = centre;
  return MPS_OK;
}

int mps_get_centre(mps_t h, int* out) {
  if (!h || !out) return MPS_E_ARG;
  *out = h->centre;
  return MPS_OK;
}

int mps_move_centre(mps_t h, int target) {
  int rc = usable(h);
  if (rc) return rc;
  if (!valid_site(h, target)) return fail(h, MPS_E_ARG, "move_centre: bad site");
  return h->prec == MPS_PREC_FP64 ? move_centre_t<c128>(h, target) : move_centre_t<c64>(h, target);
}

int mps_discarded_weight(mps_t h, double* total, long long* count) {
  int rc = usable(h);
  if (rc) return rc;
  if (!total || !count) return fail(h, MPS_E_ARG, "discarded_weight: null pointer");
  CUTRY(h, cudaMemcpyAsync(total, h->d_scalar + 1, sizeof(double), cudaMemcpyDeviceToHost, h->stream), "discarded");
  rc = check_device_error(h);
  if (rc) return rc;
  *count = h->nsplit;
  return MPS_OK;
}

int mps_svd_last_stats(mps_t h, int* sweeps, long long* rotations) {
  int rc = usable(h);
  if (rc) return rc;
  if (!sweeps || !rotations) return fail(h, MPS_E_ARG, "svd_last_stats: null pointer");
  if (h->trunc != MPS_TRUNC_SVD) return fail(h, MPS_E_STATE, "svd_last_stats: the handle splits by pivoted QR");
  int sw = 0;
  int rot[kSvdMaxSweeps];
  CUTRY(h, cudaMemcpyAsync(&sw, h->svd_ws + h->SL.sweeps, sizeof(int), cudaMemcpyDeviceToHost, h->stream),
        "svd_last_stats");
  CUTRY(h, cudaMemcpyAsync(rot, h->svd_ws + h->SL.rot, sizeof(rot), cudaMemcpyDeviceToHost, h->stream),
        "svd_last_stats");
  rc = check_device_error(h);
  if (rc) return rc;
  long long tot = 0;
  for (int j = 0; j < std::min(std::max(sw, 0), kSvdMaxSweeps); ++j) tot += rot[j];
  *sweeps = sw;
  *rotations = tot;
  return MPS_OK;
}

int mps_last_split_pivots(mps_t h, int* jpvt, int cap, int* n_out, int* k_out) {
  int rc = usable(h);
  if (rc) return rc;
  if (!jpvt || !n_out || !k_out) return fail(h, MPS_E_ARG, "last_split_pivots: null output");
  if (h->piv_n <= 0) return fail(h, MPS_E_STATE, "last_split_pivots: no pivoted split in the workspace");
  if (cap < h->piv_n) return fail(h, MPS_E_ARG, "last_split_pivots: capacity below the column count");
  CUTRY(h, cudaMemcpyAsync(jpvt, views<c64>(h).jpvt, sizeof(int) * (size_t)h->piv_n, cudaMemcpyDeviceToHost,
                           h->stream),
        "last_split_pivots");
  rc = check_device_error(h);
  if (rc) return rc;
  *n_out = h->piv_n;
  *k_out = h->piv_k;
  return MPS_OK;
}

int mps_layer_stats(mps_t h, long long* layers, long long* graph_launches, int* graphs_on) {
  if (!h) return MPS_E_ARG;
  if (layers) *layers = h->layer_calls;
  if (graph_launches) *graph_launches = h->graph_launches;
  if (graphs_on) *graphs_on = h->graphs ? 1 : 0;
  return MPS_OK;
}

int mps_kernel_stats(mps_t h, mps_kstat* out) {
  if (!h || !out) return MPS_E_ARG;
  cudaSetDevice(h->device);
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "kernel_stats");
  h->prof.drain();
  for (int c = 0; c < MPS_KCLASS_COUNT; ++c) out[c] = h->prof.stat[c];
  return MPS_OK;
}

int mps_kernel_stats_reset(mps_t h) {
  if (!h) return MPS_E_ARG;
  cudaSetDevice(h->device);
  cudaStreamSynchronize(h->stream);
  h->prof.drain();
  memset(h->prof.stat, 0, sizeof(h->prof.stat));
  return MPS_OK;
}

// ---- autotuner entry point
int mps_tune_two_site(int precision, int chi_l, int chi_m, int chi_r, int chi_max, int force, mps_tune_result* out) {
  if (!out || chi_l < 1 || chi_m < 1 || chi_r < 1 || chi_max < 1) return MPS_E_ARG;
  if (precision != MPS_PREC_FP64 && precision != MPS_PREC_MIXED) return MPS_E_ARG;
  const int m = 2 * chi_l, n = 2 * chi_r, k = std::min(std::min(m, n), chi_max);
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
    cudaGetLastError();
    return MPS_E_CUDA;
  }
  const int sms = num_sms();
  if (!force) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    if (TuneEntry* hit = tune_find_locked(precision, m, n, k, sms)) {
      out->panel_width = hit->nb;
      out->panel_ctas = hit->ctas;
      out->candidates = 0;
      out->ms = hit->ms;
      out->default_ms = hit->default_ms;
      return MPS_OK;
    }
  }
  const size_t esz = precision == MPS_PREC_FP64 ? sizeof(c128) : sizeof(c64);
  int64_t ldw, ldq;
  WsLayout L = ws_layout(esz, m, n, k, kDefaultNb, kMaxCoop, ldw, ldq);
  const int64_t na = (int64_t)m * chi_m, nbb = (int64_t)chi_m * n, no = (int64_t)std::max(m, n) * k;
  char *ws = nullptr, *bufs = nullptr;
  cudaStream_t s = nullptr;
  int rc = MPS_OK;
  const size_t off_b = align_up(esz * na), off_oa = off_b + align_up(esz * nbb), off_ob = off_oa + align_up(esz * no),
               off_d = off_ob + align_up(esz * no), off_tmp = off_d + kAlign;
  if (cudaMalloc(&ws, L.total) != cudaSuccess ||
      cudaMalloc(&bufs, off_tmp + align_up(sizeof(c64) * std::max(na, nbb))) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    rc = MPS_E_NOMEM;
  }
  TuneEntry e;
  if (rc == MPS_OK) {
    cudaMemsetAsync(ws + L.bar, 0, 16, s);
    cudaMemsetAsync(ws + L.err, 0, 16, s);
    Knobs kn;
    kn.nb = kDefaultNb;
    kn.G = std::min(sms, kMaxCoop);
    kn.flag_tol = precision == MPS_PREC_FP64 ? 1.4901161193847656e-08 : 1e-3;
    kn.timeout_ns = kRawTimeoutNs;
    kn.barrier_extra = 0;
    kn.use_tc = false;
    kn.small = false;  // time the multi-kernel split itself
    mps_c128 gh[16];
    for (int q = 0; q < 16; ++q) gh[q] = {q % 5 == 0 ? 1.0 : 0.0, 0.0};  // the identity gate (any gate times the same)
    c64* tmp = (c64*)(bufs + off_tmp);
    cudaError_t err = cudaSuccess;
    // seeded random sites (the work of a split does not depend on the values)
    for (int which = 0; which < 2 && err == cudaSuccess; ++which) {
      const int64_t cnt = which ? nbb : na;
      fill_random_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(tmp, cnt, 101u + which);
      char* dst = bufs + (which ? off_b : 0);
      err = precision == MPS_PREC_FP64 ? convert<c128, c64>(tmp, (c128*)dst, cnt, s)
                                       : cudaMemcpyAsync(dst, tmp, sizeof(c64) * cnt, cudaMemcpyDeviceToDevice, s);
    }
    if (err == cudaSuccess) {
      if (precision == MPS_PREC_FP64) {
        c128 gt[16];
        gate_to_T<c128>(gh, 16, gt);
        err = tune_split<c128>(ws_views<c128>(ws, L, ldw, ldq), kn, chi_l, chi_m, chi_r, chi_max, (const c128*)bufs,
                               (const c128*)(bufs + off_b), gt, (c128*)(bufs + off_oa), (c128*)(bufs + off_ob),
                               (double*)(bufs + off_d), s, nullptr, &e);
      } else {
        c64 gt[16];
        gate_to_T<c64>(gh, 16, gt);
        err = tune_split<c64>(ws_views<c64>(ws, L, ldw, ldq), kn, chi_l, chi_m, chi_r, chi_max, (const c64*)bufs,
                              (const c64*)(bufs + off_b), gt, (c64*)(bufs + off_oa), (c64*)(bufs + off_ob),
                              (double*)(bufs + off_d), s, nullptr, &e);
      }
    }
    int dev_err = 0;
    if (err == cudaSuccess) err = cudaMemcpyAsync(&dev_err, ws + L.err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    if (err != cudaSuccess) {
      cudaGetLastError();
      rc = MPS_E_CUDA;
    } else if (dev_err != DEV_OK) {
      rc = dev_err == DEV_ERR_TIMEOUT ? MPS_E_TIMEOUT : MPS_E_CUDA;
    }
  }
  if (s) cudaStreamDestroy(s);
  cudaFree(ws);
  cudaFree(bufs);
  if (rc != MPS_OK) return rc;
  e.prec = precision;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_find_locked(precision, m, n, k, sms);  // loads the file's entries first
    tune_store_locked(e);
  }
  out->panel_width = e.nb;
  out->panel_ctas = e.ctas;
  out->candidates = e.candidates;
  out->ms = e.ms;
  out->default_ms = e.default_ms;
  return MPS_OK;
}

// ---- raw-pointer two-site call
int mps_debug_raw_wait(int barrier_extra, double timeout_s) {
  if (barrier_extra < 0 || timeout_s < 0) return MPS_E_ARG;
  g_raw_barrier_extra.store(barrier_extra, std::memory_order_relaxed);
  g_raw_timeout_ns.store(timeout_s > 0 ? (unsigned long long)(timeout_s * 1e9) : kRawTimeoutNs,
                         std::memory_order_relaxed);
  return MPS_OK;
}

int mps_two_site_workspace(int precision, int chi_l, int chi_m, int chi_r, int chi_max, size_t* bytes) {
  if (!bytes || chi_l < 1 || chi_m < 1 || chi_r < 1 || chi_max < 1) return MPS_E_ARG;
  if (precision != MPS_PREC_FP64 && precision != MPS_PREC_MIXED) return MPS_E_ARG;
  size_t esz = precision == MPS_PREC_FP64 ? sizeof(c128) : sizeof(c64);
  int m = 2 * chi_l, n = 2 * chi_r, k = std::min(std::min(m, n), chi_max);
  int64_t ldw, ldq;
  WsLayout L = ws_layout(esz, m, n, k, kDefaultNb, kMaxCoop, ldw, ldq);
  *bytes = L.total;
  return MPS_OK;
}

int mps_two_site_apply(int precision, int chi_l, int chi_m, int chi_r, int chi_max, const void* A, const void* B,
                       const mps_c128 g[16], void* A_out, void* B_out, double* discarded_dev, void* workspace,
                       size_t ws_bytes, void* stream) {
  if (!A || !B || !g || !A_out || !B_out || !workspace) return MPS_E_ARG;
  size_t need = 0;
  int rc = mps_two_site_workspace(precision, chi_l, chi_m, chi_r, chi_max, &need);
  if (rc) return rc;
  if (ws_bytes < need || ((uintptr_t)workspace % kAlign) != 0) return MPS_E_ARG;
  size_t esz = precision == MPS_PREC_FP64 ? sizeof(c128) : sizeof(c64);
  int m = 2 * chi_l, n = 2 * chi_r, k = std::min(std::min(m, n), chi_max);
  int64_t ldw, ldq;
  WsLayout L = ws_layout(esz, m, n, k, kDefaultNb, kMaxCoop, ldw, ldq);
  cudaStream_t s = (cudaStream_t)stream;
  char* base = (char*)workspace;
  if (cudaMemsetAsync(base + L.bar, 0, 16, s) != cudaSuccess) return MPS_E_CUDA;
  if (cudaMemsetAsync(base + L.err, 0, 16, s) != cudaSuccess) return MPS_E_CUDA;
  Knobs kn;
  kn.nb = kDefaultNb;
  kn.G = std::min(num_sms(), kMaxCoop);
  kn.flag_tol = precision == MPS_PREC_FP64 ? 1.4901161193847656e-08 : 1e-3;
  kn.timeout_ns = g_raw_timeout_ns.load(std::memory_order_relaxed);
  kn.barrier_extra = (unsigned)g_raw_barrier_extra.load(std::memory_order_relaxed);
  kn.use_tc = false;
  kn.small = kn.barrier_extra == 0;
  double* slot = discarded_dev ? discarded_dev : (double*)(base + L.disc);
  cudaError_t e;
  if (precision == MPS_PREC_FP64) {
    c128 gt[16];
    gate_to_T<c128>(g, 16, gt);
    e = two_site_core<c128>(ws_views<c128>(base, L, ldw, ldq), kn, chi_l, chi_m, chi_r, chi_max, (const c128*)A,
                            (const c128*)B, gt, (c128*)A_out, (c128*)B_out, slot, nullptr, s, nullptr);
  } else {
    c64 gt[16];
    gate_to_T<c64>(g, 16, gt);
    e = two_site_core<c64>(ws_views<c64>(base, L, ldw, ldq), kn, chi_l, chi_m, chi_r, chi_max, (const c64*)A,
                           (const c64*)B, gt, (c64*)A_out, (c64*)B_out, slot, nullptr, s, nullptr);
  }
  (void)k;
  if (e != cudaSuccess) return MPS_E_CUDA;
  // the call has no handle whose state could carry a device-side failure: a
  // NaN discarded weight reports it, stream-ordered after the split
  raw_status_kernel<<<1, 1, 0, s>>>(base + L.err, slot);
  return cudaGetLastError() == cudaSuccess ? MPS_OK : MPS_E_CUDA;
}

int mps_two_site_apply_noalloc(int precision, int chi_l, int chi_m, int chi_r, int chi_max, const void* A,
                               const void* B, const mps_c128 g[16], void* A_out, void* B_out,
                               double* discarded_dev, void* stream) {
  size_t need = 0;
  int rc = mps_two_site_workspace(precision, chi_l, chi_m, chi_r, chi_max, &need);
  if (rc) return rc;
  if (need > (size_t)MPS_NOALLOC_SCRATCH_BYTES) return MPS_E_UNSUPPORTED;  // beyond the fixed array
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocDevices) return MPS_E_CUDA;
  void* ws = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return MPS_E_CUDA;
      }
      g_noalloc_ptr[dev] = p;
    }
    ws = g_noalloc_ptr[dev];
  }
  return mps_two_site_apply(precision, chi_l, chi_m, chi_r, chi_max, A, B, g, A_out, B_out, discarded_dev, ws,
                            (size_t)MPS_NOALLOC_SCRATCH_BYTES, stream);
}

}  // extern "C"
