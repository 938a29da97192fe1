// Internal interfaces between the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <algorithm>
#include <atomic>
#include <stdint.h>

#include "common.cuh"

namespace mpsg {

// ---------------------------------------------------------------------------
// First-use state kept per device ordinal (kernel attributes, occupancy, SM
// counts).  A CUDA function attribute is set per device, so a process that
// works on two devices needs one entry per device.  Entries are atomics: two
// threads that fill the same entry at once both compute it and store the same
// value, so no caller ever sees a half-made or default entry.
constexpr int kMaxDevices = 64;
struct PerDevice {
  std::atomic<long long> v[kMaxDevices];  // value + 1; 0 = not computed yet
  // The cached value for the current device, or compute() if there is none.
  // compute() returns a value >= 0, or a negative code that is not cached.
  template <typename F>
  long long get(F compute) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
      cudaGetLastError();
      dev = -1;
    }
    if (dev < 0 || dev >= kMaxDevices) return compute();
    long long c = v[dev].load(std::memory_order_acquire);
    if (c > 0) return c - 1;
    const long long r = compute();
    if (r >= 0) v[dev].store(r + 1, std::memory_order_release);
    return r;
  }
};

// ---------------------------------------------------------------------------
// Generic complex GEMM on the CUDA cores:  C = alpha * opA * opB + beta * C.
// C is column-major (ldc).  A is the M x K operand, B the K x N operand, each
// read through a "stored" view: element (i, k) of A is
//     a_row ? A[i*lda + k] : A[i + k*lda]            (conjugated if a_conj)
// and element (k, j) of B is
//     b_row ? B[k*ldb + j] : B[k + j*ldb]            (conjugated if b_conj).
// a_mask selects a structured operand, tested in the stored column-major
// coordinates (r, c) = a_row ? (k, i) : (i, k):
//     MASK_UNIT_LOWER: r > c -> stored, r == c -> 1, r < c -> 0  (reflectors V)
//     MASK_UPPER:      r <= c -> stored, else 0                   (R factor)
enum { MASK_NONE = 0, MASK_UNIT_LOWER = 1, MASK_UPPER = 2 };
constexpr int kMaxSplit = 8;

template <typename T>
struct GemmDesc {
  int M = 0, N = 0, K = 0;
  T alpha{}, beta{};
  const T* A = nullptr;
  int64_t lda = 0;
  int a_row = 0, a_conj = 0, a_mask = MASK_NONE;
  const T* B = nullptr;
  int64_t ldb = 0;
  int b_row = 0, b_conj = 0, b_mask = MASK_NONE;
  T* C = nullptr;
  int64_t ldc = 0;
  // split-K: with splitk > 1 the K range is cut into splitk slices whose
  // products land in wk (splitk * M * N elements) and are summed in a fixed order.
  int splitk = 0;
  T* wk = nullptr;
  // complex64, C-reading variant without split-K (optional): per CTA row tile, the
  // squared norms of the result's columns over the tile's rows, summed in FP32:
  // colsq[tile * ldcs + j], tile = row / 64
  float* colsq = nullptr;
  int64_t ldcs = 0;
};

// Records where a CUDA call first failed on this host thread (file name and line),
// so that the error message of the library call that reports it names the site;
// the report clears the record.
void note_cuda_failure(const char* file, int line);

template <typename T>
cudaError_t gemm_simt(const GemmDesc<T>& d, cudaStream_t s);
// number of kernel launches gemm_simt makes for this descriptor
template <typename T>
int gemm_launches(const GemmDesc<T>& d) {
  return d.splitk > 1 ? 2 : 1;
}
// split count that fills the GPU for a skinny product (few output tiles, long
// K), at most cap_elems / (M N) so the partials fit the workspace
int choose_splitk(int M, int N, int K, int64_t cap_elems, int elem_bytes);

// complex64 GEMM kernels (gemm_c64.cu): same operand views and split-K
// protocol as gemm_simt (the caller runs the reduction); theta contraction
// with the gate epilogue
cudaError_t gemm_c64(const GemmDesc<c64>& d, cudaStream_t s);
cudaError_t theta_c64(int cl, int cm, int cr, const c64* A, const c64* B, const c64* g16, c64* W, int64_t ldw,
                      cudaStream_t s, const c64* gdev = nullptr);
int gemm_c64_tile_rows(int M, int K);

// Tensor-core (tcgen05, 3xTF32) complex64 GEMM with the same operand views
// as gemm_simt (no split-K); a wait that expires sets *err.
bool tc_gemm_applicable(const GemmDesc<c64>& d);
cudaError_t tc_gemm(const GemmDesc<c64>& d, int* err, unsigned long long timeout_ns, cudaStream_t s);
cudaError_t tc_theta(int cl, int cm, int cr, const c64* A, const c64* B, const c64* g16, c64* W, int64_t ldw,
                     int* err, unsigned long long timeout_ns, cudaStream_t s, const c64* gdev = nullptr);

// GEMM dispatch: complex64 products go to the tensor cores when `use_tc` and
// the shape suits them, everything else to gemm_simt.
template <typename T>
cudaError_t gemm_auto(const GemmDesc<T>& d, bool use_tc, int* err, unsigned long long timeout_ns, cudaStream_t s);

// theta contraction with the gate epilogue (Sec. III-B.1 + III-C.2):
//   X[(l,c),(d,r)] = sum_mu A[l,c,mu] B[mu,d,r]
//   W[(b*chi_r + r)*ldw + 2l + a] = sum_{cd} g[2a+b][2c+d] X[(l,c),(d,r)]
// A, B row-major sites; W column-major (2 chi_l) x (2 chi_r).  gdev != NULL: the gate
// is read from device memory there instead of g16 (layers replayed as CUDA graphs).
template <typename T>
cudaError_t theta_gemm_simt(int chi_l, int chi_m, int chi_r, const T* A, const T* B, const T* g16,
                            T* W, int64_t ldw, cudaStream_t s, const T* gdev = nullptr);

// ---------------------------------------------------------------------------
// Elementwise / data movement kernels
template <typename T>
cudaError_t apply_1q(T* site, int chi_l, int chi_r, const T* u4, cudaStream_t s);
// dst (col-major, ldd) = src (row-major rows x cols, lds), optionally conjugated
template <typename T>
cudaError_t transpose_copy(const T* src, int64_t lds, T* dst, int64_t ldd, int rows, int cols,
                           int conj, cudaStream_t s);
// dst[r*ldd + c] = src[r*lds + c] (conj optional): strided 2D copy, same orientation
template <typename T>
cudaError_t copy2d(const T* src, int64_t lds, T* dst, int64_t ldd, int rows, int cols, int conj,
                   cudaStream_t s);
// Left split: site (row-major m x k, ld k) = Q (col-major m x k, ldq)
// Right split: site[kk*n + c] = R[kk, pos(c)] with pos = inverse of jpvt
// (R: first k rows of column-major W, upper trapezoidal; zero below).
// err: the device error word for the bounds-checking build's checks of jpvt (may be NULL)
template <typename T>
cudaError_t split_right(const T* W, int64_t ldw, const int* jpvt, int* inv_scratch, int k, int n,
                        T* site, cudaStream_t s, int* err = nullptr);
template <typename T>
cudaError_t set_identity(T* Q, int64_t ldq, int m, int k, cudaStream_t s);
template <typename TO, typename TI>
cudaError_t convert(const TI* src, TO* dst, int64_t count, cudaStream_t s);
// sum |x_i|^2 in FP64, deterministic, result to *out (device)
template <typename T>
cudaError_t norm2_sum(const T* x, int64_t count, double* partial, int npart, double* out,
                      cudaStream_t s);
// out (1 x cols) = v (1 x rows) * M (row-major rows x cols, ld), T accumulation in FP64
template <typename T>
cudaError_t vecmat(const c128* v, const T* M, int64_t ld, int rows, int cols, c128* out,
                   cudaStream_t s);

// ---------------------------------------------------------------------------
// Pivoted / plain blocked Householder QR of a column-major m x n matrix W.

template <typename T>
struct QrPlan {
  int m, n, k;     // k reflectors
  int nb;          // panel width
  int pivot;       // 1 = column-pivoted (QP3), 0 = plain QR
  T* W;
  int64_t ldw;
  // outputs / scratch (device)
  T* tau;          // k
  int* jpvt;       // n
  T* Tfac;         // ceil(k/nb) * nb * nb, per-panel triangular factors (column-major nb x nb)
  c128* Wg;        // ceil(k/nb) * nb * nb, per-step w = V^H v saved by the panel kernel
  T* F;            // n x nb row-major (ld nb): conj of the QP3 matrix F, so W -= V F^H reads it plainly
  double* vn1;     // n
  double* vn2;     // n
  // reduction scratch for the cooperative panel kernel
  double* red_norm;   // G
  c128* red_w;        // G * nb
  double* red_argv;   // G
  int* red_argi;      // G
  c128* alpha_slot;   // 1
  unsigned* bar;      // 2 (zeroed once)
  int* err;           // device error word
  double* discarded;  // out: ||W[k:m, k:n]||_F^2 (pivot mode)
  double* disc_total; // optional: discarded is also added here
  T* Tblk;            // ceil(npanels/2) * (2nb)^2: factors of outer blocks of two panels
  T* G12;             // nb * nb Gram block V1^H V2
  T* Y;               // 2nb * max(n, k) scratch for block-reflector GEMMs
  T* Z;               // 2nb * max(n, k)
  T* SK;              // split-K partials: kMaxSplit * 2nb * max(n, k)
  int64_t sk_cap = 0; // elements of SK
  int G;              // cooperative grid size cap
  double flag_tol;    // norm-downdate recompute threshold
  unsigned long long timeout_ns;
  unsigned barrier_extra;  // 0 normally; >0 only to exercise the timeout path
  int kclass = -1;         // >= 0: attribute every launch to this kernel class
  bool use_tc = false;     // complex64 GEMMs on the tensor cores
  // pivot == 2: pivots chosen on a random sketch (blocked randomized QRCP); the
  // sketch scratch below is then required
  int lsk = 0;              // sketch rows (2 nb + oversampling)
  int64_t ldy = 0;          // leading dimension of Om, Ys, Yw, Ssk (>= lsk, multiple of 4)
  T* Om = nullptr;          // ldy x m: sketching matrix (+-1)
  T* Ys = nullptr;          // ldy x n: sketch, columns in the current order of W
  T* Yw = nullptr;          // ldy x n: copy factored to choose one block's pivots
  T* Ssk = nullptr;         // ldy x 2 nb: Y_sel R11^{-1}
  T* sk_tau = nullptr;      // nb: reflector scalars of the sketch panel
  c128* sk_Wg = nullptr;    // nb x nb: w vectors of the sketch panel
  int* sk_jpvt = nullptr;   // n: column order of the sketch panel
  int* piv_seq = nullptr;   // 2 nb: position taken at each step of a block's pivot choice
  unsigned long long seed = 0;  // generator state of the sketching matrix
  // pivot == 0 with look-ahead (optional): the panels, their T factors and the
  // updates of the next outer block run on s2 (a high-priority stream) while the
  // rest of each trailing update runs on the caller's stream with its own scratch
  // (Y2, Z2: 2nb * max(n, k); SK2: sk_cap elements); la_ev: three events
  cudaStream_t s2 = nullptr;
  cudaEvent_t* la_ev = nullptr;
  T* Y2 = nullptr;
  T* Z2 = nullptr;
  T* SK2 = nullptr;
};

// randomized QRCP: a block of pivots is two panels (2 nb, at most kSketchBlockMax
// columns) and the sketch has the block size plus kSketchOversample rows
constexpr int kSketchOversample = 8;
constexpr int kSketchBlockMax = 64;

// ---------------------------------------------------------------------------
// Small two-site gates (small_gate.cu): theta of at most kSmallDim x kSmallDim
// split entirely in one CTA; a batch is one grouped launch, one CTA per gate.
constexpr int kSmallDim = 64;
constexpr int kSmallMaxCm = 256;
constexpr int kSmallBatch = 32;

template <typename T>
struct SmallGate {
  const T* A;          // site i, row-major (cl, 2, cm)
  const T* B;          // site i+1, row-major (cm, 2, cr)
  T* Aout;             // (cl, 2, k); may alias A
  T* Bout;             // (k, 2, cr); may alias B
  double* disc;        // discarded weight of this split
  double* disc_total;  // optional: the discarded weight is also added here
  int* jpvt_out;       // optional: the pivot order (2 cr entries)
  int cl, cm, cr, k;
  T g[16];             // gate, g[(2a+b)*4 + (2c+d)]
  const T* gdev;       // the gate in device memory instead (graph replay); NULL: g
};

template <typename T>
struct SmallBatch {
  int count;
  SmallGate<T> item[kSmallBatch];
};

bool small_gate_fits(int cl, int cm, int cr);
template <typename T>
cudaError_t small_gate_launch(const SmallBatch<T>& b, cudaStream_t s);

struct LaunchHooks;  // profiling hooks (engine.cu)

template <typename T>
cudaError_t qr_factor(const QrPlan<T>& p, cudaStream_t s, LaunchHooks* hooks);
// Q (column-major m x k, ldq) = H_0 ... H_{k-1} I[:, :k]
template <typename T>
cudaError_t qr_form_q(const QrPlan<T>& p, T* Q, int64_t ldq, cudaStream_t s, LaunchHooks* hooks);

int num_sms();

// Profiling hooks: the engine passes these so every launch is counted and,
// when profiling, bracketed by CUDA events.
// Every kernel launch of the library sits between hook_before and
// hook_after; `nlaunch` is the number of kernels launched in between.
struct LaunchHooks {
  void (*before)(LaunchHooks* h, int kclass, double bytes, double flops);
  void (*after)(LaunchHooks* h, int kclass, int nlaunch);
  void* ctx;
};

inline void hook_before(LaunchHooks* h, int kclass, double bytes, double flops) {
  if (h && h->before) h->before(h, kclass, bytes, flops);
}
inline void hook_after(LaunchHooks* h, int kclass, int nlaunch) {
  if (h && h->after) h->after(h, kclass, nlaunch);
}

// ---------------------------------------------------------------------------
// MPO zip-up contraction (mpo.cu; Sec. III-C.3): tensor W[a][b][out][in] with
// a, b < 2, element ((a*2 + b)*2 + out)*2 + in; unused bond entries are zero.
template <typename T>
struct MpoTensor {
  T w[16];
};
// Z[(kk,out),(b,r)] = sum_{a,in} W[a][b][out][in] Y[(kk*adim + a)*ys_row + (in*cr + r)*ys_col];
// Z column-major (ldz), or, with to_site (bdim == 1), the row-major site (kk, 2, cr)
template <typename T>
cudaError_t mpo_contract(const T* Y, int64_t ys_row, int64_t ys_col, int kk, int adim, int bdim, int cr,
                         const MpoTensor<T>& W, T* Z, int64_t ldz, int to_site, cudaStream_t s);

// ---------------------------------------------------------------------------
// Truncated SVD split by one-sided Jacobi (svd.cu; Sec. III-B.2 Table III).
constexpr int kSvdMaxSweeps = 40;
constexpr int kSvdParts = 256;

template <typename T>
struct SvdPlan {
  int m, n, k;        // theta m x n, k kept singular values (k <= min(m, n))
  const T* W;         // theta, column-major, ldw
  int64_t ldw;
  T* X;               // n * m scratch: theta^H, rotated in place
  T* V;               // m * m scratch: accumulated rotations
  double* sig2;       // m
  double* tail;       // m
  int* perm;          // m
  int* rot;           // kSvdMaxSweeps
  int* sweeps;        // 1: sweeps run (kSvdMaxSweeps + 1 = stopped unconverged)
  double* part;       // kSvdParts
  double* fro2;       // 1
  unsigned* bar;      // grid barrier words (shared with the QR panels; stream-ordered)
  int* err;           // device error word
  unsigned long long timeout_ns;
  unsigned barrier_extra;
  double* discarded;  // out: sum of the discarded squared singular values
  double* disc_total; // optional: discarded is also added here
};

// left site (row-major m x k) = V[:, kept]; right site (row-major k x n) = (theta^H V)[:, kept]^H
template <typename T>
cudaError_t svd_split(const SvdPlan<T>& p, T* Aout, T* Bout, cudaStream_t s, LaunchHooks* hooks);

}  // namespace mpsg
