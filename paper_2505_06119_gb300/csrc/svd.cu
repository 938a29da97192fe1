// Truncated SVD split of a two-site block: the SVD alternative to pivoted QR
// (Sec. III-B.2 Table III, compared with it for bond truncation in Sec. IV-A.1).
//
// One-sided (Hestenes) Jacobi on X = theta^H (n x m, column j = conj of row j
// of theta).  Plane rotations of pairs of columns of X, applied alike to the
// columns of V (which starts as I_m), make the columns of X mutually
// orthogonal: X V = Y, hence theta = V Y^H with V unitary, and the squared
// column norms of Y are the squared singular values of theta.  Keeping the k
// columns of largest norm gives
//   left site  = V[:, kept]      (an isometry whatever the rank of theta),
//   right site = Y[:, kept]^H    (diag(S) V^dagger of the kept part),
//   discarded  = sum of the other squared column norms.
//
// Rotation of columns (x, y) with a = x^H x, b = y^H y, c = x^H y = |c| e^{i phi}:
//   zeta = (b - a) / (2|c|),  t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
//   cs = 1 / sqrt(1 + t^2),   sn = cs t,
//   x <- cs x - sn e^{-i phi} y,   y <- sn e^{i phi} x + cs y,
// which is unitary and leaves x^H y = 0 (the 2 x 2 Hermitian eigenproblem of
// the pair's Gram matrix).  A pair is rotated only if |c| > tol sqrt(a b),
// tol = sqrt(n) eps, and neither column is below the zero level
// (sqrt(n) eps)^2 ||theta||_F^2: without that level the columns that must
// vanish when m > n (or when theta is rank deficient) keep trading rounding
// noise and the sweeps never end.
//
// Parallel order: round-robin (circle method) over the m columns, m/2 disjoint
// pairs per round, m-1 rounds per sweep, so every pair meets once per sweep.
// One persistent cooperative kernel runs all sweeps, one warp per pair and one
// bounded grid barrier per round; a sweep without any rotation ends it.  The
// pair sums are reduced in a fixed order (per-lane chunks, then an xor
// butterfly whose result is the same in every lane), so runs are reproducible
// and every lane derives the same rotation.
//
// Precision: the data (X, V), the pair sums and the rotation parameters are in
// the handle's precision; in complex64 the rotation (cs, sn e^{i phi}) is scaled
// to unit norm in FP64 before it is rounded, which keeps the accumulated V
// orthonormal to FP32 rounding (without it the FP32 parameter chain leaves
// rotations off unitary by several ulps and V drifts ten times further).  The
// squared singular values, their order and the discarded weight are FP64.
//
// Grid: one warp per pair; warps per CTA are chosen so that the m/2 pairs of a
// round spread over all SMs (the FP64 work of a pair competes for the few FP64
// units of an SM sub-partition).  The two V columns of a pair are prefetched
// into L1 while the pair sums are formed, so their rotation does not wait on L2.
#include <atomic>

#include "internal.h"

namespace mpsg {

namespace {

constexpr int kJMaxWarps = 8;  // warps (pairs in flight) per CTA, at most
constexpr int kChunk = 8;  // elements per lane summed (and loaded) together before the running sum

template <typename T>
struct JacobiArgs {
  T* X;
  int64_t ldx;
  int len;  // rows of X (n)
  T* V;
  int64_t ldv;
  int M;           // columns of X and order of V (m)
  const double* fro2;  // ||theta||_F^2
  int* rot;        // [max_sweeps] rotations per sweep, zeroed before the launch
  int* sweeps;     // out: sweeps run (max_sweeps + 1 if the last one still rotated)
  unsigned* bar;
  int* err;
  unsigned long long timeout_ns;
  unsigned barrier_extra;
  double tol;
  int max_sweeps;
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// pair j of round r of the circle method over Mp (even) players
__device__ __forceinline__ void round_pair(int r, int j, int Mp, int& p, int& q) {
  const int L = Mp - 1;
  int a, b;
  if (j == 0) {
    a = r;
    b = L;
  } else {
    a = (r + j) % L;
    b = (r - j + L) % L;
  }
  p = min(a, b);
  q = max(a, b);
}

// x <- c x - s1 y,  y <- s2 x + c y  over `len` elements, one warp; kChunk
// elements per lane are loaded before any is used, so their latencies overlap
template <typename T, typename R>
__device__ __forceinline__ void rotate_cols(T* __restrict__ xp, T* __restrict__ xq, int len, R c, T s1, T s2,
                                            int lane) {
  for (int t0 = 0; t0 < len; t0 += 32 * kChunk) {
    T x[kChunk], y[kChunk];
#pragma unroll
    for (int u = 0; u < kChunk; ++u) {
      const int t = t0 + u * 32 + lane;
      if (t < len) {
        x[u] = xp[t];
        y[u] = xq[t];
      }
    }
#pragma unroll
    for (int u = 0; u < kChunk; ++u) {
      const int t = t0 + u * 32 + lane;
      if (t < len) {
        T xn, yn;
        xn.re = c * x[u].re - (s1.re * y[u].re - s1.im * y[u].im);
        xn.im = c * x[u].im - (s1.re * y[u].im + s1.im * y[u].re);
        yn.re = (s2.re * x[u].re - s2.im * x[u].im) + c * y[u].re;
        yn.im = (s2.re * x[u].im + s2.im * x[u].re) + c * y[u].im;
        xp[t] = xn;
        xq[t] = yn;
      }
    }
  }
}

__device__ __forceinline__ void prefetch_l1(const void* ptr) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(ptr));
}

// lanes prefetch the 128-byte lines of one column of `len` elements
template <typename T>
__device__ __forceinline__ void prefetch_col(const T* col, int len, int lane) {
  constexpr int per_line = 128 / (int)sizeof(T);
  for (int t = lane * per_line; t < len; t += 32 * per_line) prefetch_l1(col + t);
}

template <typename R>
__device__ __forceinline__ R warp_sum_r(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// one pair (p < q) by one warp; returns 1 if it rotated
template <typename T>
__device__ int jacobi_pair(const JacobiArgs<T>& a, int p, int q, int lane, typename real_of<T>::type zero_level) {
  using R = typename real_of<T>::type;
  T* xp = a.X + (int64_t)p * a.ldx;
  T* xq = a.X + (int64_t)q * a.ldx;
  T* vp = a.V + (int64_t)p * a.ldv;
  T* vq = a.V + (int64_t)q * a.ldv;
  prefetch_col(vp, a.M, lane);
  prefetch_col(vq, a.M, lane);
  R saa = 0, sbb = 0, scr = 0, sci = 0;
  for (int t0 = 0; t0 < a.len; t0 += 32 * kChunk) {
    R caa = 0, cbb = 0, ccr = 0, cci = 0;
#pragma unroll
    for (int u = 0; u < kChunk; ++u) {
      const int t = t0 + u * 32 + lane;
      if (t < a.len) {
        const T x = xp[t], y = xq[t];
        caa = fma(x.re, x.re, fma(x.im, x.im, caa));
        cbb = fma(y.re, y.re, fma(y.im, y.im, cbb));
        ccr = fma(x.re, y.re, fma(x.im, y.im, ccr));    // Re conj(x) y
        cci = fma(x.re, y.im, fma(-x.im, y.re, cci));   // Im conj(x) y
      }
    }
    saa += caa;
    sbb += cbb;
    scr += ccr;
    sci += cci;
  }
  saa = warp_sum_r(saa);
  sbb = warp_sum_r(sbb);
  scr = warp_sum_r(scr);
  sci = warp_sum_r(sci);
  if (!(saa > zero_level) || !(sbb > zero_level)) return 0;
  const R ac = hypot(scr, sci);
  if (!(ac > (R)a.tol * sqrt(saa) * sqrt(sbb))) return 0;
  const R zeta = (sbb - saa) / (R(2) * ac);
  const R az = fabs(zeta);
  const R big = sizeof(R) == 4 ? R(1e15) : R(1e150);
  const R t = az > big ? R(0.5) / zeta : (zeta >= R(0) ? R(1) : R(-1)) / (az + sqrt(R(1) + zeta * zeta));
  R cs = R(1) / sqrt(R(1) + t * t);
  R sr = cs * t * (scr / ac), si = cs * t * (sci / ac);  // sn e^{i phi}
  if constexpr (sizeof(R) == 4) {
    const double nn = (double)cs * cs + (double)sr * sr + (double)si * si;
    const double sc = rsqrt(nn);
    cs = (R)(cs * sc);
    sr = (R)(sr * sc);
    si = (R)(si * sc);
  }
  const T s1 = mk<R>(sr, -si);  // sn e^{-i phi}
  const T s2 = mk<R>(sr, si);   // sn e^{+i phi}
  rotate_cols<T, R>(xp, xq, a.len, cs, s1, s2, lane);
  rotate_cols<T, R>(vp, vq, a.M, cs, s1, s2, lane);
  return 1;
}

template <typename T>
__global__ void __launch_bounds__(32 * kJMaxWarps) jacobi_kernel(JacobiArgs<T> a) {
  using R = typename real_of<T>::type;
  const int lane = threadIdx.x & 31;
  const int wpc = blockDim.x >> 5;
  const int gw = blockIdx.x * wpc + (threadIdx.x >> 5);
  const int nw = gridDim.x * wpc;
  const int Mp = a.M + (a.M & 1);
  const int P = Mp / 2;
  const unsigned expected = gridDim.x + a.barrier_extra;
  const double eps = sizeof(R) == 4 ? 1.1920928955078125e-07 : 2.220446049250313e-16;
  const double zl = eps * sqrt((double)a.len);
  const R zero_level = (R)(zl * zl * (*a.fro2));
  for (int sweep = 0; sweep < a.max_sweeps; ++sweep) {
    int rotated = 0;
    for (int r = 0; r < Mp - 1; ++r) {
      for (int j = gw; j < P; j += nw) {
        int p, q;
        round_pair(r, j, Mp, p, q);
        if (q < a.M) rotated += jacobi_pair<T>(a, p, q, lane, zero_level);
      }
      if (!grid_barrier(a.bar, expected, a.err, a.timeout_ns)) return;
    }
    if (lane == 0 && rotated) atomicAdd(&a.rot[sweep], rotated);
    if (!grid_barrier(a.bar, expected, a.err, a.timeout_ns)) return;
    if (ld_relaxed_i32(&a.rot[sweep]) == 0) {
      if (blockIdx.x == 0 && threadIdx.x == 0) *a.sweeps = sweep + 1;
      return;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.sweeps = a.max_sweeps + 1;
}

// sig2[j] = ||X[:, j]||^2 in FP64, one warp per column, fixed order
template <typename T>
__global__ void col_norm2_kernel(const T* X, int64_t ldx, int len, int M, double* sig2, int* err) {
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= M) return;
  const T* x = X + (int64_t)j * ldx;
  double acc = 0.0;
  for (int t = lane; t < len; t += 32) acc += (double)x[t].re * x[t].re + (double)x[t].im * x[t].im;
  acc = warp_sum(acc);
  if (lane == 0) {
    if (!isfinite(acc)) atomicCAS(err, DEV_OK, DEV_ERR_NONFINITE);
    sig2[j] = acc;
  }
}

// rank of column j in non-increasing sig2 (lower index first on ties; a
// non-finite value ranks last), perm[rank] = j for the k kept columns, and
// tail[j] = sig2[j] for the discarded ones (0 for kept)
__global__ void sv_rank_kernel(const double* sig2, int M, int k, int* perm, double* tail) {
  __shared__ double s[1024];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const double mine = j < M ? (isfinite(sig2[j]) ? sig2[j] : -1.0) : 0.0;
  int rank = 0;
  for (int base = 0; base < M; base += 1024) {
    __syncthreads();
    for (int i = threadIdx.x; i < 1024; i += blockDim.x)
      s[i] = base + i < M ? (isfinite(sig2[base + i]) ? sig2[base + i] : -1.0) : -2.0;
    __syncthreads();
    const int lim = min(1024, M - base);
    if (j < M)
      for (int i = 0; i < lim; ++i) {
        const double v = s[i];
        rank += (v > mine) || (v == mine && base + i < j);
      }
  }
  if (j < M) {
    if (rank < k) perm[rank] = j;
    tail[j] = rank < k ? 0.0 : fmax(mine, 0.0);
  }
}

// discarded = sum_j tail[j] (one block, fixed order); also added to *total
__global__ void sv_discarded_kernel(const double* tail, int M, double* out, double* total) {
  __shared__ double s[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < M; i += 256) acc += tail[i];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (out) *out = s[0];
    if (total) *total += s[0];
  }
}

// left site (row-major m x k): site[r*k + t] = V[r + perm[t]*ldv], 32 x 32 tiles
template <typename T>
__global__ void svd_left_kernel(const T* V, int64_t ldv, const int* perm, int m, int k, T* site, int* err) {
  __shared__ T tile[32][33];
  const int r0 = blockIdx.x * 32, t0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int i = ty; i < 32; i += 8) {
    const int t = t0 + i, r = r0 + tx;
    if (t < k && r < m) {
      const int c = perm[t];
      if (c < 0 || c >= m) {
        atomicCAS(err, DEV_OK, DEV_ERR_BOUNDS);
        continue;
      }
      tile[i][tx] = V[r + (int64_t)c * ldv];
    }
  }
  __syncthreads();
  for (int i = ty; i < 32; i += 8) {
    const int r = r0 + i, t = t0 + tx;
    if (t < k && r < m) {
      const int c = perm[t];
      if (c >= 0 && c < m) site[(int64_t)r * k + t] = tile[tx][i];
    }
  }
}

// right site (row-major k x n): site[t*n + c] = conj(X[c + perm[t]*ldx])
template <typename T>
__global__ void svd_right_kernel(const T* X, int64_t ldx, const int* perm, int M, int k, int n, T* site,
                                 int* err) {
  const int t = blockIdx.y;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= k || c >= n) return;
  const int j = perm[t];
  if (j < 0 || j >= M) {
    if (c == 0) atomicCAS(err, DEV_OK, DEV_ERR_BOUNDS);
    return;
  }
  site[(int64_t)t * n + c] = cconj(X[c + (int64_t)j * ldx]);
}

// launch shape of the Jacobi kernel for `pairs` pairs per round: warps per CTA so
// that the pairs spread over every SM, CTAs capped by co-residency (cached per
// device and block size)
template <typename T>
void jacobi_shape(int pairs, int& G, int& warps) {
  static PerDevice cap[2][kJMaxWarps + 1];
  const int sms = num_sms();
  warps = std::max(1, std::min(kJMaxWarps, (pairs + sms - 1) / sms));
  const int w = warps;
  const long long c = cap[sizeof(T) == 8 ? 0 : 1][warps].get([w, sms]() -> long long {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_kernel<T>, 32 * w, 0) != cudaSuccess ||
        per_sm < 1) {
      cudaGetLastError();
      per_sm = 1;
    }
    return (long long)per_sm * sms;
  });
  G = std::max(1, std::min((int)c, (pairs + warps - 1) / warps));
}

}  // namespace

template <typename T>
cudaError_t svd_split(const SvdPlan<T>& p, T* Aout, T* Bout, cudaStream_t s, LaunchHooks* hk) {
  const int m = p.m, n = p.n, k = p.k;
  if (m < 1 || n < 1 || k < 1 || k > std::min(m, n)) return cudaErrorInvalidValue;
  hook_before(hk, MPS_KCLASS_SVD, 0, 0);
  // X = theta^H (n x m, ldx = n), V = I_m, ||theta||_F^2
  cudaError_t e = transpose_copy<T>(p.W, p.ldw, p.X, n, n, m, 1, s);
  if (e == cudaSuccess) e = set_identity<T>(p.V, m, m, m, s);
  if (e == cudaSuccess) e = norm2_sum<T>(p.X, (int64_t)n * m, p.part, kSvdParts, p.fro2, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(p.rot, 0, sizeof(int) * kSvdMaxSweeps, s);
  if (e != cudaSuccess) return e;
  JacobiArgs<T> a;
  a.X = p.X;
  a.ldx = n;
  a.len = n;
  a.V = p.V;
  a.ldv = m;
  a.M = m;
  a.fro2 = p.fro2;
  a.rot = p.rot;
  a.sweeps = p.sweeps;
  a.bar = p.bar;
  a.err = p.err;
  a.timeout_ns = p.timeout_ns;
  a.barrier_extra = p.barrier_extra;
  a.tol = (sizeof(T) == 8 ? 1.1920928955078125e-07 : 2.220446049250313e-16) * sqrt((double)n);
  a.max_sweeps = kSvdMaxSweeps;
  int G = 1, warps = 1;
  jacobi_shape<T>((m + 1) / 2, G, warps);
  void* args[] = {&a};
  e = cudaLaunchCooperativeKernel((const void*)jacobi_kernel<T>, dim3(G), dim3(32 * warps), args, 0, s);
  if (e != cudaSuccess) return e;
  col_norm2_kernel<T><<<(m + 7) / 8, 256, 0, s>>>(p.X, n, n, m, p.sig2, p.err);
  sv_rank_kernel<<<(m + 255) / 256, 256, 0, s>>>(p.sig2, m, k, p.perm, p.tail);
  sv_discarded_kernel<<<1, 256, 0, s>>>(p.tail, m, p.discarded, p.disc_total);
  svd_left_kernel<T><<<dim3((m + 31) / 32, (k + 31) / 32), dim3(32, 8), 0, s>>>(p.V, m, p.perm, m, k, Aout, p.err);
  svd_right_kernel<T><<<dim3((n + 127) / 128, k), 128, 0, s>>>(p.X, n, p.perm, m, k, n, Bout, p.err);
  e = cudaGetLastError();
  hook_after(hk, MPS_KCLASS_SVD, 10);
  return e;
}

template cudaError_t svd_split<c64>(const SvdPlan<c64>&, c64*, c64*, cudaStream_t, LaunchHooks*);
template cudaError_t svd_split<c128>(const SvdPlan<c128>&, c128*, c128*, cudaStream_t, LaunchHooks*);

}  // namespace mpsg
