// Blocked Householder QR with column pivoting (QP3 formulation) on one GPU.
//
// Computes theta P = Q R stopped after k pivots (Sec. III-B.2, QR with
// pivoting; truncation of Sec. III-C.2).  The matrix W (m x n, column-major)
// is factored in panels of nb columns:
//
//   panel kernel (persistent, cooperative, one CTA per SM at most), for each
//   step J of the panel:
//     A. pivot p = argmax_t vn1[t] over trailing columns (vn1 = squared column
//        norms in FP64; lowest index on ties), from per-CTA partial maxima;
//     B. swap columns J and p; bring column J up to date with the panel's
//        earlier reflectors, x = W[J:m, J] - V F[p,:]^H; partial sums of
//        ||x_{J+1:}||^2 (FP64) and V^H x;
//     C. reflector: beta = -sign(Re alpha) ||x||, tau = (beta - alpha)/beta,
//        v = (1, x_{J+1:} / (alpha - beta)), in FP64 (one warp, overlapped
//        with D1, which needs only x);
//     D. for every trailing column t (columns split across CTAs):
//        D1: y_t = W[J:m, t]^H x, the BLAS-2 sweep over the trailing matrix,
//            streamed in 4 KB (column, row-chunk) pieces by bulk asynchronous
//            copies into shared memory (cp.async.bulk + mbarrier);
//        D2: F[t, k] = tau (y_t - F[t, :k] w) with w = V^H v,
//            row update W[J, t] -= W[J, panel] F[t, :]^H (this row is final R),
//            FP64 downdate of the squared norm, vn1[t] -= |W[J, t]|^2, with an
//            exact recompute when vn1[t] <= tol * vn2[t] (vn2 = the last exact
//            value), the accuracy criterion of LAPACK's xLAQPS.
//   The data path (F, the row update, V^H v) runs in the data precision;
//   FP64 carries the norms, the reflector norm / beta / tau and the pivots.
//   F is stored conjugated.  Two grid barriers per step, every wait bounded.
//
//   trailing update: W[J1:m, J1:n] -= V F^H (rank-nb GEMM), then an exact
//   recompute of every trailing column norm.
//
// Without pivoting (centre moves, Sec. III-C.1) the panel only touches its own
// columns; when it fits, it runs on one 16-CTA thread-block cluster with the
// panel resident in shared memory (qr_cpanel_kernel).  Pairs of panels form
// 64-column blocks whose compact-WY reflector C -= V T^H V^H C updates the rest
// of the matrix.
//
// Q[:, :k] = H_0 ... H_{k-1} I is formed backwards block by block (64 columns,
// T of each block merged from its two panels' factors, which are built by
// recursive doubling from the w vectors the panel kernel saves).
#include <algorithm>

#include "internal.h"

namespace mpsg {

namespace {

constexpr int PNT = 512;  // threads of the panel kernel
constexpr int PNW = PNT / 32;
constexpr int kPanelNbMax = 32;  // widest panel the kernel supports
constexpr int kDBatch = 32;      // trailing columns per phase-D batch
constexpr int kDChMax = 32;      // row chunks per column in phase D (about 8 KB each)
constexpr int kDpCap = kDBatch * kDChMax;  // phase-D chunk sums held at once
constexpr int kSlot = 4096;      // bytes of one bulk-copy slot (phase D, bulk mode)
constexpr int kRing = PNW * 2 * kSlot;  // two slots per warp
constexpr int kNSW = 1;                 // warps on the reflector scalars in bulk mode
constexpr int kNDW = PNW - kNSW;        // warps on the trailing sweep in bulk mode

template <typename T>
struct PanelArgs {
  T* W;
  int64_t ldw;
  int m, n;
  int j0, kb, nend, nb;
  int pivot;
  T* F;
  double* vn1;  // squared column norms (current)
  double* vn2;  // squared column norms at the last exact computation
  int* jpvt;
  T* tau;
  T* Tp;  // this panel's T factor, column-major nb x nb
  c128* Wg;  // this panel's w vectors, nb x nb (column kk = w of step kk)
  double* red_norm;
  T* red_w;
  long long* red_argv;
  int* red_argi;
  c128* alpha_slot;
  unsigned* bar;
  int* err;
  unsigned expected;
  unsigned long long timeout_ns;
  double flag_tol;
  int xcap;    // elements of x that fit in dynamic shared memory
  int xs_off;  // byte offset of the x vector in dynamic shared memory
  int bulk;    // phase D streams column chunks with bulk asynchronous copies
  int keep;    // bulk mode: chunks per CTA and step read under the L2 keep policy
  int* piv_seq;  // optional: the pivot position p taken at each step
};

// Squared column norm below which a reflector is the identity (tau = 0): the
// smallest normal number of the data type's real part squared (complex64: FLT_MIN^2,
// complex128: DBL_MIN).  Such a column holds rounding residue of exact zeros; its
// entries' squares underflow, so ||x|| and alpha - beta would round to zero and
// 1/(alpha - beta) to infinity, and v would turn into NaN.
template <typename T>
__device__ __forceinline__ double zero_column_level() {
  return sizeof(T) == 8 ? 1.3814317e-76 : 2.2250738585072014e-308;
}

// Pivot key of a squared norm: for a non-negative double (or +inf) its bit
// pattern orders like its value, so pivots are compared as 64-bit integers
// (exact, and off the FP64 pipe); NaN or negative values map to -1 and never win.
__device__ __forceinline__ long long pkey(double v) {
  const long long b = __double_as_longlong(v);
  return (b >= 0 && b <= 0x7FF0000000000000LL) ? b : -1LL;
}

__device__ __forceinline__ bool better(long long v, int i, long long bv, int bi) {
  return (v > bv) || (v == bv && i < bi);
}

// Block-wide argmax of (key, index) pairs; result valid in thread 0.
__device__ void block_argmax(long long& v, int& i) {
  __shared__ long long sv[PNW];
  __shared__ int si[PNW];
  for (int o = 16; o > 0; o >>= 1) {
    long long ov = __shfl_xor_sync(0xffffffffu, v, o);
    int oi = __shfl_xor_sync(0xffffffffu, i, o);
    if (better(ov, oi, v, i)) {
      v = ov;
      i = oi;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    sv[warp] = v;
    si[warp] = i;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < PNW; ++w)
      if (better(sv[w], si[w], v, i)) {
        v = sv[w];
        i = si[w];
      }
  }
  __syncthreads();
}

__device__ double block_sum(double v) {
  __shared__ double s[PNW];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) s[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {  // butterfly over the warp sums: 4 dependent FP64 adds instead of 16
    t = lane < PNW ? s[lane] : 0.0;
    for (int o = 1; o < PNW; o <<= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  __syncthreads();
  return t;  // valid in thread 0
}

__device__ __forceinline__ void split_range(int lo, int hi, int parts, int idx, int& a, int& b) {
  int len = hi - lo;
  if (len <= 0) {
    a = b = lo;
    return;
  }
  a = lo + (int)((int64_t)len * idx / parts);
  b = lo + (int)((int64_t)len * (idx + 1) / parts);
}

// Dot product sum_{r in [r0, r1)} conj(col[r]) * xb[r - base] by one warp
// (base even, xb 16-byte aligned), 16-byte vector loads of the column and of
// x, eight column loads in flight per lane.
template <typename T>
__device__ __forceinline__ T warp_dot_conj(const T* __restrict__ col, const T* __restrict__ xb, int base, int r0,
                                           int r1, int lane);

__device__ __forceinline__ void dot_pair(float4 v, float4 x, float& ar, float& ai, float& br, float& bi) {
  // (v.x + i v.y)^* (x.x + i x.y) and (v.z + i v.w)^* (x.z + i x.w)
  ar = fmaf(v.x, x.x, ar);
  ar = fmaf(v.y, x.y, ar);
  ai = fmaf(v.x, x.y, ai);
  ai = fmaf(-v.y, x.x, ai);
  br = fmaf(v.z, x.z, br);
  br = fmaf(v.w, x.w, br);
  bi = fmaf(v.z, x.w, bi);
  bi = fmaf(-v.w, x.z, bi);
}

template <>
__device__ __forceinline__ c64 warp_dot_conj<c64>(const c64* __restrict__ col, const c64* __restrict__ xb, int base,
                                                  int r0, int r1, int lane) {
  float ar = 0.f, ai = 0.f, br = 0.f, bi = 0.f;
  // an odd first row (the only possible one: chunks end on even rows, m is even)
  // is taken by lane 0; its load is issued now and consumed after the sweep
  const bool peel = (r0 & 1) && r0 < r1;
  const int r = peel ? r0 + 1 : r0;
  c64 pc = mk<float>(0.f, 0.f), px = mk<float>(0.f, 0.f);
  if (peel && lane == 0) {
    pc = col[r0];
    px = xb[r0 - base];
  }
  const int npairs = (r1 - r) >> 1;
  const float4* c4 = reinterpret_cast<const float4*>(col + r);
  const float4* x4 = reinterpret_cast<const float4*>(xb + (r - base));
  constexpr int UN = 8;
  // lane-uniform trip count, predicated loads: no lane ever runs a tail alone
  for (int q0 = 0; q0 < npairs; q0 += 32 * UN) {
    float4 vv[UN];
#pragma unroll
    for (int u = 0; u < UN; ++u) {
      const int q = q0 + lane + 32 * u;
      vv[u] = q < npairs ? c4[q] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < UN; ++u) {
      const int q = q0 + lane + 32 * u;
      if (q < npairs) dot_pair(vv[u], x4[q], ar, ai, br, bi);
    }
  }
  if (((r1 - r) & 1) && lane == 0) {  // odd last row: cannot happen with even chunk ends
    c64 c = col[r1 - 1], v = xb[r1 - 1 - base];
    br = fmaf(c.re, v.re, br);
    br = fmaf(c.im, v.im, br);
    bi = fmaf(c.re, v.im, bi);
    bi = fmaf(-c.im, v.re, bi);
  }
  ar = fmaf(pc.re, px.re, ar);
  ar = fmaf(pc.im, px.im, ar);
  ai = fmaf(pc.re, px.im, ai);
  ai = fmaf(-pc.im, px.re, ai);
  c64 s;
  s.re = warp_sum(ar + br);
  s.im = warp_sum(ai + bi);
  return s;
}

template <>
__device__ __forceinline__ c128 warp_dot_conj<c128>(const c128* __restrict__ col, const c128* __restrict__ xb,
                                                    int base, int r0, int r1, int lane) {
  double ar = 0.0, ai = 0.0, br = 0.0, bi = 0.0;
  const double2* c2 = reinterpret_cast<const double2*>(col);
  const double2* x2 = reinterpret_cast<const double2*>(xb) - base;
  constexpr int UN = 8;
  for (int r00 = r0; r00 < r1; r00 += 32 * UN) {
    double2 vv[UN];
#pragma unroll
    for (int u = 0; u < UN; ++u) {
      const int r = r00 + lane + 32 * u;
      vv[u] = r < r1 ? c2[r] : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int u = 0; u < UN; ++u) {
      const int r = r00 + lane + 32 * u;
      if (r < r1) {
        const double2 xv = x2[r];
        const double2 v = vv[u];
        if (u & 1) {
          br = fma(v.x, xv.x, br);
          br = fma(v.y, xv.y, br);
          bi = fma(v.x, xv.y, bi);
          bi = fma(-v.y, xv.x, bi);
        } else {
          ar = fma(v.x, xv.x, ar);
          ar = fma(v.y, xv.y, ar);
          ai = fma(v.x, xv.y, ai);
          ai = fma(-v.y, xv.x, ai);
        }
      }
    }
  }
  c128 s;
  s.re = warp_sum(ar + br);
  s.im = warp_sum(ai + bi);
  return s;
}

// y = sum_r conj(c[r]) x[r] over one column chunk held in shared memory (c)
// and x in shared or global memory; rows [0, nrows), row 0 left out when
// skip0.  Result warp-reduced (every lane).  For complex64 nrows is even and
// both pointers 16-byte aligned.
template <typename T>
__device__ __forceinline__ T chunk_dot(const T* c, const T* x, int nrows, bool skip0, int lane);

template <>
__device__ __forceinline__ c64 chunk_dot<c64>(const c64* c, const c64* x, int nrows, bool skip0, int lane) {
  float ar = 0.f, ai = 0.f, br = 0.f, bi = 0.f;
  const float4* c4 = reinterpret_cast<const float4*>(c);
  const float4* x4 = reinterpret_cast<const float4*>(x);
  const int nq = nrows >> 1;
#pragma unroll 4
  for (int q = lane; q < nq; q += 32) {
    float4 v = c4[q];
    const float4 xv = x4[q];
    if (q == 0 && skip0) {
      v.x = 0.f;
      v.y = 0.f;
    }
    dot_pair(v, xv, ar, ai, br, bi);
  }
  c64 s;
  s.re = warp_sum(ar + br);
  s.im = warp_sum(ai + bi);
  return s;
}

template <>
__device__ __forceinline__ c128 chunk_dot<c128>(const c128* c, const c128* x, int nrows, bool skip0, int lane) {
  double ar = 0.0, ai = 0.0;
  const double2* c2 = reinterpret_cast<const double2*>(c);
  const double2* x2 = reinterpret_cast<const double2*>(x);
#pragma unroll 4
  for (int r = lane; r < nrows; r += 32) {
    double2 v = c2[r];
    const double2 xv = x2[r];
    if (r == 0 && skip0) {
      v.x = 0.0;
      v.y = 0.0;
    }
    ar = fma(v.x, xv.x, ar);
    ar = fma(v.y, xv.y, ar);
    ai = fma(v.x, xv.y, ai);
    ai = fma(-v.y, xv.x, ai);
  }
  c128 s;
  s.re = warp_sum(ar);
  s.im = warp_sum(ai);
  return s;
}

template <typename T>
__global__ void __launch_bounds__(PNT, 1) qr_panel_kernel(PanelArgs<T> a) {
  using R = typename real_of<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* xs = reinterpret_cast<T*>(smem_raw + a.xs_off);
  __shared__ __align__(8) unsigned long long s_mbar[PNW][2];  // bulk mode: one barrier per slot
  __shared__ T s_wacc[kPanelNbMax];   // sum over CTAs of V_i^H x below row J
  __shared__ __align__(8) unsigned long long s_xbar;  // bulk mode: x staging copy
  __shared__ T s_vrow[kPanelNbMax];   // W[J, j0+i]
  __shared__ T s_wp[PNW][kPanelNbMax];  // per-warp partials of V^H x (phase B)
  __shared__ T s_dp[kDpCap];  // phase-D chunk sums
  __shared__ T s_wn[kDBatch];                         // D2: updated row-J entries of the batch
  __shared__ T s_wJ[kDBatch];                         // D2: row-J entries before the update
  __shared__ T s_fi[kDBatch][kPanelNbMax];            // D2: conj(F) rows of the batch's columns
  __shared__ double s_v1[kDBatch], s_v2[kDBatch];    // D2: squared norms (current, last exact)
  __shared__ int s_need[kDBatch];                     // D2: exact recompute flags
  __shared__ int s_bi;
  __shared__ c128 s_scal[3];  // tau, 1/(alpha-beta), beta

  const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int m = a.m, nb = a.nb;
  T* W = a.W;
  const int64_t ldw = a.ldw;
  // an earlier bounded wait expired: the factorisation is void, leave at once
  // (decided once for the whole CTA)
  __shared__ int s_skip;
  unsigned bgen = 0;  // thread 0: generation of the grid barrier (grid_barrier_g)
  if (tid == 0) {
    s_skip = ld_relaxed_i32(a.err) != DEV_OK;
    bgen = ld_acquire_u32(&a.bar[1]);
  }
  if (a.bulk && lane == 0) {
    mbar_init(smem_u32(&s_mbar[warp][0]), 1);
    mbar_init(smem_u32(&s_mbar[warp][1]), 1);
    if (warp == 0) mbar_init(smem_u32(&s_xbar), 1);
  }
  const uint64_t pol_keep = l2_policy_keep(), pol_stream = l2_policy_stream();
  unsigned ph = 0;   // bulk mode: parity of the next completion of this warp's slots
  unsigned xph = 0;  // bulk mode: parity of the next completion of the x copy
  __syncthreads();
  if (s_skip) return;

  // Phase 0: partial argmax over this CTA's share of [j0, nend)
  if (a.pivot) {
    int c0, c1;
    split_range(a.j0, a.nend, G, b, c0, c1);
    long long bv = -1;
    int bi = 0x7fffffff;
    for (int t = c0 + tid; t < c1; t += PNT) {
      long long v = pkey(a.vn1[t]);
      if (better(v, t, bv, bi)) {
        bv = v;
        bi = t;
      }
    }
    block_argmax(bv, bi);
    if (tid == 0) {
      a.red_argv[b] = bv;
      a.red_argi[b] = bi;
    }
    if (!grid_barrier_g(a.bar, a.expected, a.err, a.timeout_ns, bgen)) return;
  }

  c128 s_prev = mk<double>(0, 0);
  for (int kk = 0; kk < a.kb; ++kk) {
    const int J = a.j0 + kk;
    // rows J..m-1 of the phase-B work: at most 128 per CTA
    const int gb = max(1, min(G, (m - J + 127) / 128));
    // ---------------- A: pivot
    int p = J;
    if (a.pivot) {
      if (warp == 0) {
        long long bv = -1;
        int bi = 0x7fffffff;
        long long v[5];
        int ix[5];
#pragma unroll
        for (int u = 0; u < 5; ++u) {
          const int g = lane + 32 * u;
          v[u] = -1;
          ix[u] = 0x7fffffff;
          if (g < G) {
            v[u] = a.red_argv[g];
            ix[u] = a.red_argi[g];
          }
        }
#pragma unroll
        for (int u = 0; u < 5; ++u)
          if (better(v[u], ix[u], bv, bi)) {
            bv = v[u];
            bi = ix[u];
          }
        for (int g = lane + 160; g < G; g += 32) {  // more than 160 CTAs
          long long vv = a.red_argv[g];
          int ii = a.red_argi[g];
          if (better(vv, ii, bv, bi)) {
            bv = vv;
            bi = ii;
          }
        }
        for (int o = 16; o > 0; o >>= 1) {
          long long ov = __shfl_xor_sync(0xffffffffu, bv, o);
          int oi = __shfl_xor_sync(0xffffffffu, bi, o);
          if (better(ov, oi, bv, bi)) {
            bv = ov;
            bi = oi;
          }
        }
        if (lane == 0) s_bi = bi;
      }
      __syncthreads();
      p = s_bi;
      if (p < J || p >= a.nend) {  // only reachable with non-finite norms
        if (tid == 0) atomicCAS(a.err, DEV_OK, DEV_ERR_NONFINITE);
        p = J;
      }
    }
    T* colJ = W + (int64_t)J * ldw;
    T* colP = W + (int64_t)p * ldw;
    // ---------------- B1: swap rows above J (any CTA).  The first PNT rows of this
    // CTA's share are loaded here and stored after the B2 row loop, so that their
    // round trip overlaps B2's loads (the rows are disjoint from B2's).
    int s0 = 0, s1 = 0;
    if (p != J) split_range(0, J, G, b, s0, s1);
    const bool b1 = s0 + tid < s1;
    T b1j = mk<R>(0, 0), b1p = mk<R>(0, 0);
    if (b1) {
      b1j = colJ[s0 + tid];
      b1p = colP[s0 + tid];
    }
    // ---------------- B2: rows [u0, u1) of J..m-1: swap, deferred scaling of the
    // previous reflector, column update x = W[:,J] - V F[p,:]^H, partial sums.
    // 4 threads per row; thread `sub` owns panel columns i = sub + 4u.
    if (b < gb) {
      int u0, u1;
      split_range(J, m, gb, b, u0, u1);
      const int sub = tid & 3;
      constexpr int U = kPanelNbMax / 4;
      T fp[U], cs[U];  // fp: conj(F[p, :]), loaded with the first pass's loads
#pragma unroll
      for (int u = 0; u < U; ++u) {
        fp[u] = mk<R>(0, 0);
        cs[u] = mk<R>(0, 0);
      }
      double nrm = 0.0;
      bool wrote = false;  // this thread stored rows >= J of columns J / p (read later by bulk copies)
      // 128 rows per pass (more than one pass only when m - J > 128 G)
      for (int rb = u0; rb < u1; rb += PNT / 4) {
        const int r = rb + (tid >> 2);
        const bool act = r < u1;
        T vr[U];
        // issue every load of this pass before using any
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int i = sub + 4 * u;
          vr[u] = mk<R>(0, 0);
          if (i < kk && act) vr[u] = W[r + (int64_t)(a.j0 + i) * ldw];
        }
        T cj = mk<R>(0, 0), cp = mk<R>(0, 0);
        if (act && sub == 0) {
          cj = colJ[r];
          cp = colP[r];
        }
        if (rb == u0) {
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int i = sub + 4 * u;
            if (i < kk) fp[u] = a.F[(int64_t)p * nb + i];
          }
        }
        if (kk > 0 && act && sub == ((kk - 1) & 3)) {  // previous reflector: rows > J-1, scaled once
          const int u = (kk - 1) >> 2;
          const T scp = ccast<R>(s_prev);
#pragma unroll
          for (int uu = 0; uu < U; ++uu)
            if (uu == u) {
              vr[uu] = vr[uu] * scp;
              W[r + (int64_t)(J - 1) * ldw] = vr[uu];
            }
        }
        T x = (sub == 0) ? ((p != J) ? cp : cj) : mk<R>(0, 0);
#pragma unroll
        for (int u = 0; u < U; ++u) x = x - vr[u] * fp[u];  // F stored conjugated
        x.re += __shfl_xor_sync(0xffffffffu, x.re, 1);
        x.im += __shfl_xor_sync(0xffffffffu, x.im, 1);
        x.re += __shfl_xor_sync(0xffffffffu, x.re, 2);
        x.im += __shfl_xor_sync(0xffffffffu, x.im, 2);
        if (act && sub == 0) {
          colJ[r] = x;
          if (p != J) colP[r] = cj;
          wrote = true;
          if (r > J) nrm += (double)x.re * (double)x.re + (double)x.im * (double)x.im;
          if (r == J) *a.alpha_slot = ccast<double>(x);
        }
        // partial w_i = sum_{rows > J} conj(V[r, i]) x_r
        if (act && r > J) {
#pragma unroll
          for (int u = 0; u < U; ++u) cs[u] = cs[u] + cconj(vr[u]) * x;
        }
      }
      if (b1) {
        colJ[s0 + tid] = b1p;
        colP[s0 + tid] = b1j;
      }
      if (a.bulk && wrote) fence_proxy_async();  // these stores before the bulk reads of phase C/D
      // reduce over the 8 rows of the warp
#pragma unroll
      for (int u = 0; u < U; ++u) {
        T c = cs[u];
        c.re += __shfl_xor_sync(0xffffffffu, c.re, 4);
        c.im += __shfl_xor_sync(0xffffffffu, c.im, 4);
        c.re += __shfl_xor_sync(0xffffffffu, c.re, 8);
        c.im += __shfl_xor_sync(0xffffffffu, c.im, 8);
        c.re += __shfl_xor_sync(0xffffffffu, c.re, 16);
        c.im += __shfl_xor_sync(0xffffffffu, c.im, 16);
        if (lane < 4) s_wp[warp][sub + 4 * u] = c;
      }
      nrm = block_sum(nrm);  // contains __syncthreads: s_wp complete afterwards
      if (tid == 0) a.red_norm[b] = nrm;
      if (tid < kk) {
        T w = s_wp[0][tid];
        for (int q = 1; q < PNW; ++q) w = w + s_wp[q][tid];
        a.red_w[(int64_t)b * nb + tid] = w;
      }
    }
    if (b >= gb && b1) {
      colJ[s0 + tid] = b1p;
      colP[s0 + tid] = b1j;
    }
    for (int r = s0 + PNT + tid; r < s1; r += PNT) {  // shares of more than PNT rows (small grids)
      T t0 = colJ[r];
      colJ[r] = colP[r];
      colP[r] = t0;
    }
    if (b == 0 && tid == 0 && p != J) {
      int t0 = a.jpvt[J];
      a.jpvt[J] = a.jpvt[p];
      a.jpvt[p] = t0;
    }
    if (b == 0 && tid == 0 && a.piv_seq) a.piv_seq[kk] = p;
    if (!grid_barrier_g(a.bar, a.expected, a.err, a.timeout_ns, bgen)) return;

    // ---------------- C: reflector (every CTA, identical FP64 arithmetic).
    // Warp 0 computes beta, tau and 1/(alpha - beta) in FP64, then combines the
    // CTAs' partial sums of V^H x.  In bulk mode x is staged by one bulk copy and
    // the other warps go straight on to the trailing sweep (phase D1), which needs
    // only x; the reflector scalars are first used in the D2 epilogue.
    const int L = m - J - 1;  // rows below the pivot row
    // x = W[J+1:m, J] staged from the even row xbase (16-byte aligned vectors)
    const int xbase = (sizeof(T) == 8) ? ((J + 1) & ~1) : (J + 1);
    const bool staged = (m - xbase <= a.xcap);
    const bool xcopy = a.bulk && staged && m > xbase;  // x arrives by bulk copy this step
    if (xcopy && tid == 0) {
      const uint32_t bytes = (uint32_t)((m - xbase) * sizeof(T));
      fence_proxy_async();  // phase-B writes of column J, and last step's reads of xs
      mbar_expect_tx(smem_u32(&s_xbar), bytes);
      bulk_g2s(smem_u32(xs), colJ + xbase, bytes, smem_u32(&s_xbar));
    }
    if (!a.bulk && staged)
      for (int r = tid; r < m - xbase; r += PNT) xs[r] = colJ[xbase + r];
    if (warp == 0) {
      double nv[5];
      c128 al = mk<double>(0, 0);
#pragma unroll
      for (int u = 0; u < 5; ++u) {
        const int g = lane + 32 * u;
        nv[u] = g < gb ? a.red_norm[g] : 0.0;
      }
      if (lane == 0) al = *a.alpha_slot;
      double xn = 0.0;
#pragma unroll
      for (int u = 0; u < 5; ++u) xn += nv[u];
      for (int g = lane + 160; g < gb; g += 32) xn += a.red_norm[g];
      xn = warp_sum(xn);
      if (lane == 0) {
        c128 tau, sc, beta;
        if ((xn == 0.0 && al.im == 0.0) || al.re * al.re + al.im * al.im + xn < zero_column_level<T>()) {
          tau = mk<double>(0, 0);
          sc = mk<double>(0, 0);
          beta = al;
        } else {
          double nrm = sqrt(al.re * al.re + al.im * al.im + xn);
          double bt = al.re >= 0.0 ? -nrm : nrm;
          tau = mk<double>((bt - al.re) / bt, -al.im / bt);
          c128 dnm = mk<double>(al.re - bt, al.im);
          double dd = dnm.re * dnm.re + dnm.im * dnm.im;
          sc = mk<double>(dnm.re / dd, -dnm.im / dd);  // 1 / (alpha - beta)
          beta = mk<double>(bt, 0.0);
        }
        s_scal[0] = tau;
        s_scal[1] = sc;
        s_scal[2] = beta;
      }
    }
    if (warp == 0 && lane < kk) {
      // lane i: sum over the CTAs of V_i^H x (below row J), in CTA order; row J of V
      T acc = mk<R>(0, 0);
      int g = 0;
      for (; g + 4 <= gb; g += 4) {
        const T p0 = a.red_w[(int64_t)g * nb + lane], p1 = a.red_w[(int64_t)(g + 1) * nb + lane];
        const T p2 = a.red_w[(int64_t)(g + 2) * nb + lane], p3 = a.red_w[(int64_t)(g + 3) * nb + lane];
        acc = acc + p0;
        acc = acc + p1;
        acc = acc + p2;
        acc = acc + p3;
      }
      for (; g < gb; ++g) acc = acc + a.red_w[(int64_t)g * nb + lane];
      s_wacc[lane] = acc;
      s_vrow[lane] = W[J + (int64_t)(a.j0 + lane) * ldw];
    }
    if (!a.bulk) __syncthreads();

    // ---------------- D: trailing columns in batches of up to kDBatch; each column's
    // sweep y_t = W[J+1:m, t]^H x is cut into row chunks of about 8 KB so that
    // the items (column, chunk) spread evenly over the warps; chunk sums are
    // combined in a fixed order, then one warp per column finishes F, the row
    // update and the norm downdate.
    const T* xsrc = staged ? xs : colJ + xbase;
    // chunks on even absolute rows: [xbase + ch*chr, xbase + (ch+1)*chr) clipped to [J+1, m)
    const int Lx = m - xbase;
    const int nch = max(1, min(kDChMax, (int)(((int64_t)Lx * sizeof(T) + 8191) / 8192)));
    const int chr = (((Lx + nch - 1) / nch) + 1) & ~1;  // rows per chunk (even)
    int c0, c1;
    split_range(J + 1, a.nend, G, b, c0, c1);
    long long bv = -1;
    int bi = 0x7fffffff;
    // bulk mode: chunks of kSlot bytes from row xbase, each copied by the TMA
    // unit into one of the consuming warp's two slots (double buffering)
    constexpr int CR = kSlot / (int)sizeof(T);
    const int nchb = a.bulk ? (Lx + CR - 1) / CR : nch;  // chunks per column
    const int nbc = a.bulk ? max(1, min(kDBatch, kDpCap / max(nchb, 1))) : kDBatch;
    if (a.bulk && lane == 0) fence_proxy_async();  // generic writes before the barrier -> async reads
    bool xseen = false;
    bool pre = false;  // bulk mode: this batch's first two items were issued during the previous one
    // The sweep direction alternates from step to step (batches, and the (column,
    // chunk) items inside a batch): the columns one step reads last are still in L2
    // when the next step starts, so part of each sweep is served from L2.  Every
    // chunk sum lands in its own slot and is combined in a fixed order, so the
    // results do not depend on the direction.  In bulk mode the last a.keep chunks
    // of this CTA's traversal (the first ones of the next step's) are read under the
    // L2 keep policy and the others under the stream policy, so that the lines the
    // next step will read first are the last to be evicted.
    const bool rev = (kk & 1) != 0;
    const int nbat = c1 > c0 ? (c1 - c0 + nbc - 1) / nbc : 0;
    const int bfull = nbc * nchb;                                             // chunks of a full batch
    const int blast = nbat > 0 ? (c1 - c0 - (nbat - 1) * nbc) * nchb : 0;  // of the last (first when rev)
    const int keep_from = (c1 - c0) * nchb - a.keep;  // traversal position of the first kept chunk
    // chunks of the batches before traversal position q
    auto before = [&](int q) { return rev ? (q == 0 ? 0 : blast + (q - 1) * bfull) : q * bfull; };
    for (int bq = 0; bq < nbat; ++bq) {
      const int cb = c0 + (rev ? nbat - 1 - bq : bq) * nbc;
      const int nc = min(nbc, c1 - cb);
      // warp 0 stages the D2 epilogue's operands of the batch in shared memory while
      // the other warps sweep (written before barrier 1 or in earlier steps; F row J
      // stands in for the pivot column's row)
      if (warp == 0) {
        for (int c8 = 0; c8 < nc; c8 += 8) {
          T fv[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int t = cb + c8 + u;
            fv[u] = (c8 + u < nc && lane < kk) ? a.F[(int64_t)((t == p) ? J : t) * nb + lane] : mk<R>(0, 0);
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) s_fi[c8 + u][lane] = fv[u];
        }
        if (lane < nc) {
          const int t = cb + lane;
          const int src = (t == p) ? J : t;
          s_wJ[lane] = W[J + (int64_t)t * ldw];
          if (a.pivot) {
            s_v1[lane] = a.vn1[src];
            s_v2[lane] = a.vn2[src];
          }
        }
      }
      // D1: chunk sums
      if (a.bulk) {
        // items (column, chunk) dealt round-robin to the sweep warps kNSW..PNW-1
        const int dw = warp - kNSW;
        const int nit = nc * nchb;
        const int nli = (dw >= 0 && nit > dw) ? (nit - dw + kNDW - 1) / kNDW : 0;  // this warp's items
        unsigned char* slot0 = smem_raw + warp * 2 * kSlot;
        // first two items of batch cb0 (nc0 columns) into slots 0 and 1
        auto prologue = [&](int cb0, int nc0, int base0) {
          const int nit0 = nc0 * nchb;
          const int nli0 = (dw >= 0 && nit0 > dw) ? (nit0 - dw + kNDW - 1) / kNDW : 0;
          for (int li = 0; li < min(2, nli0); ++li) {
            const int ir = dw + kNDW * li, it = rev ? nit0 - 1 - ir : ir, cl = it / nchb, ch = it - cl * nchb;
            const int cs = xbase + ch * CR, ce = min(m, cs + CR);
            const uint32_t mb = smem_u32(&s_mbar[warp][li]);
            mbar_expect_tx(mb, (uint32_t)((ce - cs) * sizeof(T)));
            bulk_g2s_hint(smem_u32(slot0 + li * kSlot), W + (int64_t)(cb0 + cl) * ldw + cs,
                          (uint32_t)((ce - cs) * sizeof(T)), mb, base0 + ir >= keep_from ? pol_keep : pol_stream);
          }
        };
        const int base = before(bq);
        if (lane == 0 && !pre) prologue(cb, nc, base);
        pre = false;
        // x (staged by the bulk copy of phase C) is waited for after the first chunk
        // copies were issued, so that the two round trips overlap
        if (nli > 0 && xcopy && !xseen) {
          if (!mbar_wait(smem_u32(&s_xbar), xph, a.err, a.timeout_ns))
            mbar_wait_plain(smem_u32(&s_xbar), xph, a.timeout_ns);
          xseen = true;
        }
        for (int li = 0; li < nli; ++li) {
          const int q = li & 1;
          const int ir = dw + kNDW * li, it = rev ? nit - 1 - ir : ir, cl = it / nchb, ch = it - cl * nchb;
          const int cs = xbase + ch * CR, ce = min(m, cs + CR);
          const uint32_t mb = smem_u32(&s_mbar[warp][q]);
          const uint32_t par = (ph >> q) & 1u;
          // on expiry (error word set) the copy in flight still lands before the slot is reused
          if (!mbar_wait(mb, par, a.err, a.timeout_ns)) mbar_wait_plain(mb, par, a.timeout_ns);
          ph ^= 1u << q;
          const T s = chunk_dot<T>(reinterpret_cast<const T*>(slot0 + q * kSlot), xsrc + (cs - xbase), ce - cs,
                                   cs <= J, lane);
          if (lane == 0) s_dp[cl * nchb + ch] = s;
          __syncwarp();
          if (lane == 0 && li + 2 < nli) {
            const int ir2 = ir + 2 * kNDW, it2 = rev ? nit - 1 - ir2 : ir2, cl2 = it2 / nchb, ch2 = it2 - cl2 * nchb;
            const int cs2 = xbase + ch2 * CR, ce2 = min(m, cs2 + CR);
            // the slot's previous contents were consumed above (values in registers,
            // __syncwarp passed), so the copy cannot overtake those reads
            mbar_expect_tx(mb, (uint32_t)((ce2 - cs2) * sizeof(T)));
            bulk_g2s_hint(smem_u32(slot0 + q * kSlot), W + (int64_t)(cb + cl2) * ldw + cs2,
                          (uint32_t)((ce2 - cs2) * sizeof(T)), mb, base + ir2 >= keep_from ? pol_keep : pol_stream);
          }
        }
        // every slot of this warp is free again: start the next batch's copies now,
        // so they are in flight during this batch's epilogue
        if (bq + 1 < nbat) {
          const int cbn = c0 + (rev ? nbat - 2 - bq : bq + 1) * nbc;
          if (lane == 0) prologue(cbn, min(nbc, c1 - cbn), before(bq + 1));
          pre = true;
        }
      } else {
        for (int ir = warp; ir < nc * nch; ir += PNW) {
          const int it = rev ? nc * nch - 1 - ir : ir, cl = it / nch, ch = it - cl * nch;
          const int t = cb + cl;
          const int r0 = max(J + 1, xbase + ch * chr), r1 = min(m, xbase + (ch + 1) * chr);
          const T* col = W + (int64_t)t * ldw;
          T s = mk<R>(0, 0);
          if (r0 < r1) s = warp_dot_conj<T>(col, xsrc, xbase, r0, r1, lane);
          if (lane == 0) s_dp[cl * nch + ch] = s;
        }
      }
      __syncthreads();
      // D2: per-column epilogue; operands of all of this warp's columns fetched first.
      // tau and 1/(alpha-beta) are FP64 results; the data path uses them rounded.
      const T tau = ccast<R>(s_scal[0]), sc = ccast<R>(s_scal[1]);
      const T w_l = lane < kk ? cconj(s_vrow[lane]) + sc * s_wacc[lane] : mk<R>(0, 0);  // V_l^H v
      constexpr int CPW = kDBatch / PNW;  // columns per warp
      T fT[CPW];
#pragma unroll
      for (int q = 0; q < CPW; ++q) {
        const int cl = warp + PNW * q;
        fT[q] = mk<R>(0, 0);
        if (cl >= nc) continue;  // warp-uniform
        const int t = cb + cl;
        T* Ft = a.F + (int64_t)t * nb;
        // chunk sums in chunk order; eight shared-memory loads in flight at a time
        T acc = mk<R>(0, 0);
        for (int c8 = 0; c8 < nchb; c8 += 8) {
          T dv[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) dv[u] = c8 + u < nchb ? s_dp[cl * nchb + c8 + u] : mk<R>(0, 0);
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (c8 + u < nchb) acc = acc + dv[u];
        }
        const T wJt = s_wJ[cl];
        const T y = cconj(wJt) + sc * acc;
        // F[t, kk] = tau * (y - sum_i F[src, i] w_i); row update of W[J, t]
        // (the array holds conj(F): the trailing update reads it as F^H directly)
        T fw = mk<R>(0, 0), rowu = mk<R>(0, 0);
        if (lane < kk) {
          const T fi = s_fi[cl][lane];  // conj(F[src, lane])
          cfma(fw, cconj(fi), w_l);
          cfma(rowu, s_vrow[lane], fi);
          if (t == p) Ft[lane] = fi;
        }
        fw.re = warp_sum(fw.re);
        fw.im = warp_sum(fw.im);
        rowu.re = warp_sum(rowu.re);
        rowu.im = warp_sum(rowu.im);
        const T f = tau * (y - fw);
        const T wnew = wJt - rowu - cconj(f);
        fT[q] = f;
        if (lane == 0) {
          Ft[kk] = cconj(f);
          W[J + (int64_t)t * ldw] = wnew;
          s_wn[cl] = wnew;
        }
      }
      // FP64 downdate of the squared norms, one column per lane of warp 0, so that the
      // batch's FP64 arithmetic takes a handful of warp instructions; a column whose
      // downdated norm has lost accuracy is flagged for an exact recompute
      if (a.pivot) {
        __syncthreads();
        if (warp == 0 && lane < nc) {
          double v1 = s_v1[lane];
          int need = 0;
          if (L <= 0) {
            v1 = 0.0;
          } else if (v1 > 0.0) {
            const T wn = s_wn[lane];
            const double r2 = (double)wn.re * (double)wn.re + (double)wn.im * (double)wn.im;
            const double c = fmax(v1 - r2, 0.0);
            if (c <= a.flag_tol * s_v2[lane])
              need = 1;
            else
              v1 = c;
          }
          s_v1[lane] = v1;
          s_need[lane] = need;
        }
        __syncthreads();
      }
#pragma unroll
      for (int q = 0; q < CPW; ++q) {
        const int cl = warp + PNW * q;
        if (cl >= nc) continue;  // warp-uniform
        const int t = cb + cl;
        const int src = (t == p) ? J : t;
        const T* col = W + (int64_t)t * ldw;
        const T* Fs = a.F + (int64_t)src * nb;
        const T f = fT[q];
        double v1 = 0.0, v2 = a.pivot ? s_v2[cl] : 0.0;
        int need = 0;
        if (a.pivot) {
          v1 = s_v1[cl];
          need = s_need[cl];
        }
        if (need) {
          // exact squared norm of the column after step J: rows > J of
          // W[:, t] - V[:, 0:kk] F[t, 0:kk]^H - (s x) conj(f)
          double nr = 0.0;
          const c128 cf = cconj(ccast<double>(f));
          const c128 scd = ccast<double>(sc);
          for (int r = J + 1 + lane; r < m; r += 32) {
            c128 z = ccast<double>(col[r]);
            for (int i = 0; i < kk; ++i) {
              c128 vv = ccast<double>(W[r + (int64_t)(a.j0 + i) * ldw]);
              z = z - vv * ccast<double>(Fs[i]);  // Fs holds conj(F)
            }
            c128 vx = scd * ccast<double>(colJ[r]);
            z = z - vx * cf;
            nr += z.re * z.re + z.im * z.im;
          }
          nr = warp_sum(nr);
          v1 = nr;
          v2 = nr;
        }
        if (lane == 0 && a.pivot) {
          a.vn1[t] = v1;
          a.vn2[t] = v2;
          const long long k1 = pkey(v1);
          if (better(k1, t, bv, bi)) {
            bv = k1;
            bi = t;
          }
        }
      }
      __syncthreads();  // s_dp reused by the next batch
    }
    if (a.pivot) {
      block_argmax(bv, bi);
      if (tid == 0) {
        a.red_argv[b] = bv;
        a.red_argi[b] = bi;
      }
    }
    __syncthreads();  // reflector scalars complete even where this CTA had no trailing columns
    if (b == 0) {
      // w of this step, for the triangular factor T of the panel (tfactor_kernel)
      const T scd = ccast<R>(s_scal[1]);
      if (tid < kk) a.Wg[(int64_t)kk * nb + tid] = ccast<double>(cconj(s_vrow[tid]) + scd * s_wacc[tid]);
      if (tid == 32) {
        a.tau[J] = ccast<R>(s_scal[0]);
        W[J + (int64_t)J * ldw] = ccast<R>(s_scal[2]);
      }
    }
    if (xcopy) {
      // the x copy has landed before xs is staged again or the CTA leaves
      if (tid == 0 && !mbar_wait(smem_u32(&s_xbar), xph, a.err, a.timeout_ns))
        mbar_wait_plain(smem_u32(&s_xbar), xph, a.timeout_ns);
      xph ^= 1u;
    }
    s_prev = s_scal[1];
    // (no proxy fence here: what this step wrote with plain stores, row J and the
    // panel's own columns, is not read by a bulk copy before the next phase-B fence)
    if (!grid_barrier_g(a.bar, a.expected, a.err, a.timeout_ns, bgen)) return;
  }
  // final deferred scaling of the panel's last reflector, rows > Jl
  if (a.kb > 0) {
    const int Jl = a.j0 + a.kb - 1;
    int u0, u1;
    split_range(Jl + 1, m, G, b, u0, u1);
    T* prev = W + (int64_t)Jl * ldw;
    T sc = ccast<R>(s_prev);
    for (int r = u0 + tid; r < u1; r += PNT) prev[r] = prev[r] * sc;
  }
}

// ---------------------------------------------------------------------------
// Unpivoted panel on one thread-block cluster (centre moves, Sec. III-C.1).
// The panel W[j0:m, j0:j0+kb] is spread over the cluster's CTAs by rows and
// stays in their shared memory for the whole factorisation; each step needs
// two cluster-wide reductions (the reflector norm with alpha, then v^H of
// every panel column), exchanged through distributed shared memory between
// hardware cluster barriers instead of grid barriers in global memory.
// Per step J = j0 + kk (right-looking inside the panel):
//   beta = -sign(Re alpha) ||x||, tau = (beta - alpha)/beta, v = (1, x/(alpha-beta))
//   d_c = v^H W[J:m, c] for every panel column c;
//   c > kk: W[J:m, c] -= conj(tau) v d_c;   c < kk: w_kk[c] = conj(d_c) (T factor)
// Control flow is identical in every CTA (no early exit), so every cluster
// barrier is reached by all of them; FP64 carries the norm, beta and tau.
constexpr int CPT = 512;             // threads of the cluster panel kernel
constexpr int CPW = CPT / 32;
constexpr int kClusterMax = 16;

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t map_cta(const void* p, unsigned rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ double ld_dsmem_f64(uint32_t a) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ c64 ld_dsmem(const c64*, uint32_t a) {
  float x, y;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(x), "=f"(y) : "r"(a) : "memory");
  return mk<float>(x, y);
}
__device__ __forceinline__ c128 ld_dsmem(const c128*, uint32_t a) {
  double x, y;
  asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];" : "=d"(x), "=d"(y) : "r"(a) : "memory");
  return mk<double>(x, y);
}

template <typename T>
struct CPanelArgs {
  T* W;
  int64_t ldw;
  int m, j0, kb, nb;
  int rb;        // panel rows held by each CTA
  T* tau;
  c128* Wg;      // this panel's w vectors (column kk = w of step kk)
};

// Block-wide FP64 sum, the result in thread 0.  The threads' values go through
// shared memory and four warps (one per scheduler) add 128 each before a warp
// reduction: four times fewer FP64 warp instructions than a shuffle reduction in
// every warp, and FP64 instructions are slow on this GPU.
static_assert(CPT == 512, "cp_block_sum assumes 512 threads");
__device__ __forceinline__ double cp_block_sum(double v, double* s_part, double* s_red) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  s_part[tid] = v;
  __syncthreads();
  if (warp < 4) {
    const double* p = s_part + warp * 128 + lane;
    double t = (p[0] + p[32]) + (p[64] + p[96]);
    t = warp_sum(t);
    if (lane == 0) s_red[warp] = t;
  }
  __syncthreads();
  return tid == 0 ? (s_red[0] + s_red[1]) + (s_red[2] + s_red[3]) : 0.0;
}

// Per step J = j0 + kk, with x = column kk below row J:
//   partials of this CTA (computed at the end of the previous step):
//     ||x||^2 (FP64), alpha = W[J, kk] (its owner), e_c = sum_{r > J} conj(x_r) W[r, c],
//     W[J, c] (the owner of row J), for every panel column c;
//   one cluster barrier; every CTA combines all partials in the same fixed order;
//   beta, tau, sc = 1/(alpha - beta) in FP64 (warp 0) while the other warps combine e, W[J, :];
//   d_c = v^H W[:, c] = W[J, c] + conj(sc) e_c;  c > kk: W[J:m, c] -= v conj(tau) d_c;
//   c < kk: w_kk[c] = conj(d_c);  then the partials of step kk + 1.
template <typename T>
__global__ void __launch_bounds__(CPT, 1) qr_cpanel_kernel(CPanelArgs<T> a) {
  using R = typename real_of<T>::type;
  extern __shared__ __align__(16) unsigned char cp_raw[];
  T* P = reinterpret_cast<T*>(cp_raw);   // [kb][rb], column c at P + c * rb
  __shared__ double s_r1[2][3];           // per step: ||x||^2 partial, alpha (re, im)
  __shared__ T s_e[2][kPanelNbMax];       // per step: partial e_c
  __shared__ T s_j[2][kPanelNbMax];       // per step: W[J, c] (owner) or 0
  __shared__ T s_pe[kPanelNbMax][kClusterMax + 1];  // gathered partials, combined in rank order
  __shared__ T s_pj[kPanelNbMax][kClusterMax + 1];
  __shared__ T s_f[kPanelNbMax];          // conj(tau) d_c
  __shared__ T s_d[kPanelNbMax];          // d_c
  __shared__ double s_red[CPW];
  __shared__ double s_part[CPT];          // cp_block_sum: one value per thread
  __shared__ c128 s_sc[3];                // tau, 1/(alpha-beta), beta
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned cs = gridDim.x;           // CTAs in the cluster (one cluster)
  const unsigned rank = cluster_rank();
  const int m = a.m, kb = a.kb, rb = a.rb;
  const int r0 = a.j0 + (int)rank * rb, r1 = min(m, r0 + rb);
  const int nr = max(0, r1 - r0);
  // partials of the step on column c (row J): norm and alpha from `part`, e and W[J, :]
  auto partials = [&](int c, int J, double part) {
    const int pr = c & 1;
    const T* x = P + c * rb;
    const int rs = max(0, J + 1 - r0);  // first local row > J
    for (int q = warp; q < kb; q += CPW) {
      const T* col = P + q * rb;
      T acc = mk<R>(0, 0);
      for (int rr = rs + lane; rr < nr; rr += 32) cfma(acc, cconj(x[rr]), col[rr]);
      acc.re = warp_sum(acc.re);
      acc.im = warp_sum(acc.im);
      if (lane == 0) {
        s_e[pr][q] = acc;
        s_j[pr][q] = (J >= r0 && J < r1) ? col[J - r0] : mk<R>(0, 0);
      }
    }
    const double t = cp_block_sum(part, s_part, s_red);
    if (tid == 0) {
      const bool own = J >= r0 && J < r1;
      const T al = own ? x[J - r0] : mk<R>(0, 0);
      s_r1[pr][0] = t;
      s_r1[pr][1] = (double)al.re;
      s_r1[pr][2] = (double)al.im;
    }
  };
  for (int c = 0; c < kb; ++c)
    for (int rr = tid; rr < nr; rr += CPT) P[c * rb + rr] = a.W[(r0 + rr) + (int64_t)(a.j0 + c) * a.ldw];
  __syncthreads();
  {
    double part = 0.0;
    for (int rr = max(0, a.j0 + 1 - r0) + tid; rr < nr; rr += CPT) {
      const T v = P[rr];
      part += (double)v.re * (double)v.re + (double)v.im * (double)v.im;
    }
    partials(0, a.j0, part);
  }

  for (int kk = 0; kk < kb; ++kk) {
    const int J = a.j0 + kk, par = kk & 1;
    T* x = P + kk * rb;
    cluster_sync();
    if (warp == 0) {
      // reflector, identical in every CTA (partials combined in the same order)
      // the norm partials of every CTA; alpha from the CTA that owns row J (the
      // others hold zero), read directly instead of summed
      const unsigned own = (unsigned)((J - a.j0) / rb);
      double v0 = 0.0, v1 = 0.0, v2 = 0.0;
      if (lane < (int)cs) v0 = ld_dsmem_f64(map_cta(&s_r1[par][0], lane));
      if (lane == 0) {
        v1 = ld_dsmem_f64(map_cta(&s_r1[par][1], own));
        v2 = ld_dsmem_f64(map_cta(&s_r1[par][2], own));
      }
      for (int o = 1; o < kClusterMax; o <<= 1) v0 += __shfl_xor_sync(0xffffffffu, v0, o);
      if (lane == 0) {
        const double xn = v0;
        const c128 al = mk<double>(v1, v2);
        c128 tau, sc, beta;
        if ((xn == 0.0 && al.im == 0.0) || al.re * al.re + al.im * al.im + xn < zero_column_level<T>()) {
          tau = mk<double>(0, 0);
          sc = mk<double>(0, 0);
          beta = al;
        } else {
          // two FP64 divisions (1/beta, 1/|alpha - beta|^2) instead of four: on this
          // GPU every FP64 operation of this single-lane chain is on the step's
          // critical path
          const double nv = sqrt(al.re * al.re + al.im * al.im + xn);
          const double bt = al.re >= 0.0 ? -nv : nv;
          const double ibt = 1.0 / bt;
          tau = mk<double>((bt - al.re) * ibt, -al.im * ibt);
          const c128 dnm = mk<double>(al.re - bt, al.im);
          const double idd = 1.0 / (dnm.re * dnm.re + dnm.im * dnm.im);
          sc = mk<double>(dnm.re * idd, -dnm.im * idd);  // 1 / (alpha - beta)
          beta = mk<double>(bt, 0.0);
        }
        s_sc[0] = tau;
        s_sc[1] = sc;
        s_sc[2] = beta;
      }
    } else {
      // gather e_c and W[J, c] of every CTA (warps 1..)
      for (int idx = tid - 32; idx < 2 * kb * (int)cs; idx += CPT - 32) {
        const int arr = idx / (kb * (int)cs), rem = idx - arr * kb * (int)cs;
        const int c = rem / (int)cs, q = rem - c * (int)cs;
        const T* src = arr == 0 ? &s_e[par][c] : &s_j[par][c];
        const T v = ld_dsmem(static_cast<const T*>(nullptr), map_cta(src, q));
        if (arr == 0)
          s_pe[c][q] = v;
        else
          s_pj[c][q] = v;
      }
    }
    __syncthreads();
    const T tau = ccast<R>(s_sc[0]), sc = ccast<R>(s_sc[1]);
    if (tid < kb) {
      T e = mk<R>(0, 0), wj = mk<R>(0, 0);
      for (int q = 0; q < (int)cs; ++q) {
        e = e + s_pe[tid][q];
        wj = wj + s_pj[tid][q];
      }
      const T d = wj + cconj(sc) * e;  // v^H W[:, c]
      s_d[tid] = d;
      s_f[tid] = cconj(tau) * d;
    }
    __syncthreads();
    if (rank == 0) {
      if (tid < kk) a.Wg[(int64_t)kk * a.nb + tid] = ccast<double>(cconj(s_d[tid]));
      if (tid == 32) a.tau[J] = tau;
    }
    // v stored in place of x; trailing panel columns W[J:m, c] -= v conj(tau) d_c;
    // the next column's norm below row J+1 is accumulated on the way
    const int rs = max(0, J - r0);  // first local row >= J
    double part = 0.0;
    for (int rr = rs + tid; rr < nr; rr += CPT) {
      const int r = r0 + rr;
      T v = mk<R>(1, 0);
      if (r > J) {
        v = x[rr] * sc;
        x[rr] = v;
      }
      for (int c = kk + 1; c < kb; ++c) {
        T* col = P + c * rb;
        const T nv = col[rr] - v * s_f[c];
        col[rr] = nv;
        if (c == kk + 1 && r > J + 1) part += (double)nv.re * (double)nv.re + (double)nv.im * (double)nv.im;
      }
    }
    if (J >= r0 && J < r1 && tid == 0) x[J - r0] = ccast<R>(s_sc[2]);  // R diagonal
    __syncthreads();
    if (kk + 1 < kb) partials(kk + 1, J + 1, part);  // contains __syncthreads
  }
  cluster_sync();  // no CTA leaves while another may still read its shared memory
  for (int c = 0; c < kb; ++c)
    for (int rr = tid; rr < nr; rr += CPT) a.W[(r0 + rr) + (int64_t)(a.j0 + c) * a.ldw] = P[c * rb + rr];
}

// Triangular factor of each panel's block reflector (H_j0 ... H_j0+kb-1 =
// I - V T V^H, forward columnwise), built by recursive doubling: the factor
// of [V1 V2] is [[T1, -T1 (V1^H V2) T2], [0, T2]], so starting from the
// 1 x 1 factors tau_i, log2(nb) rounds merge neighbouring blocks of width h
// into blocks of width 2h.  The Gram entries V_j^H v_i (j < i) are the w
// vectors the panel kernel saved (FP64); the arithmetic runs in the data
// precision.  One CTA of 1024 threads per panel, thread (i, j) owns T[i, j].
template <typename T>
__global__ void __launch_bounds__(1024) tfactor_kernel(const c128* Wg, const T* tau, int pan0, int k, int nb,
                                                       T* Tfac) {
  using R = typename real_of<T>::type;
  __shared__ T Ts[kPanelNbMax][kPanelNbMax + 1];
  __shared__ T Gs[kPanelNbMax][kPanelNbMax + 1];
  const int pan = pan0 + blockIdx.x;
  const int j0 = pan * nb, kb = min(nb, k - j0);
  const c128* w = Wg + (size_t)pan * nb * nb;
  const int i = threadIdx.x % 32, j = threadIdx.x / 32;
  const T z = mk<R>(0, 0);
  Ts[i][j] = (i == j && i < kb) ? tau[j0 + i] : z;
  Gs[i][j] = (i < j && j < kb) ? ccast<R>(w[(size_t)j * nb + i]) : z;  // V_i^H v_j
  __syncthreads();
  for (int h = 1; h < kb; h *= 2) {
    const int s0 = i / (2 * h) * (2 * h);
    const bool mine = (j / (2 * h) == i / (2 * h)) && (i - s0 < h) && (j - s0 >= h);
    // X = T1 G12 into the (still empty) upper-right block
    if (mine) {
      T x = z;
      for (int l = i; l < s0 + h; ++l) cfma(x, Ts[i][l], Gs[l][j]);
      Ts[i][j] = x;
    }
    __syncthreads();
    // T12 = -X T2
    T y = z;
    if (mine)
      for (int l = s0 + h; l <= j; ++l) cfma(y, Ts[i][l], Ts[l][j]);
    __syncthreads();
    if (mine) Ts[i][j] = z - y;
    __syncthreads();
  }
  if (i < nb && j < nb) Tfac[(size_t)pan * nb * nb + i + (size_t)j * nb] = Ts[i][j];
}

// Squared norm of col[r0:r1) by one warp.  complex128: FP64 throughout.
// complex64: FP32 squares summed per lane with Kahan compensation (error of
// order the FP32 unit roundoff, independent of the length), lanes combined in
// FP64; 16-byte vector loads.
template <typename T>
__device__ __forceinline__ double warp_norm2(const T* __restrict__ col, int r0, int r1, int lane);

template <>
__device__ __forceinline__ double warp_norm2<c64>(const c64* __restrict__ col, int r0, int r1, int lane) {
  float s = 0.f, c = 0.f;
  auto add = [&](float v) {
    float y = v - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
  };
  int r = r0;
  if ((r & 1) && r < r1) {
    if (lane == 0) add(cabs2(col[r]));
    ++r;
  }
  const int npairs = (r1 - r) >> 1;
  const float4* c4 = reinterpret_cast<const float4*>(col + r);
  for (int q0 = 0; q0 < npairs; q0 += 256) {
    float4 vv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int q = q0 + lane + 32 * u;
      vv[u] = q < npairs ? c4[q] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) add(vv[u].x * vv[u].x + vv[u].y * vv[u].y + vv[u].z * vv[u].z + vv[u].w * vv[u].w);
  }
  if (((r1 - r) & 1) && lane == 0) add(cabs2(col[r1 - 1]));
  return warp_sum((double)s - (double)c);
}

template <>
__device__ __forceinline__ double warp_norm2<c128>(const c128* __restrict__ col, int r0, int r1, int lane) {
  double a = 0.0, b = 0.0;
  const double2* c2 = reinterpret_cast<const double2*>(col);
  for (int r00 = r0; r00 < r1; r00 += 256) {
    double2 vv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int r = r00 + lane + 32 * u;
      vv[u] = r < r1 ? c2[r] : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int u = 0; u < 8; u += 2) {
      a = fma(vv[u].x, vv[u].x, a);
      a = fma(vv[u].y, vv[u].y, a);
      b = fma(vv[u + 1].x, vv[u + 1].x, b);
      b = fma(vv[u + 1].y, vv[u + 1].y, b);
    }
  }
  return warp_sum(a + b);
}

// Triangular factor of two consecutive panels as one block reflector:
// (I - V1 T1 V1^H)(I - V2 T2 V2^H) = I - V T V^H with V = [V1 V2] and
// T = [[T1, -T1 (V1^H V2) T2], [0, T2]].  T1 (k1 x k1), T2 (k2 x k2) and
// G12 = V1^H V2 (k1 x k2) are column-major with leading dims ld1, ld2, ldg;
// T is written column-major with leading dim ldT.  One CTA of 1024 threads.
template <typename T>
__global__ void tmerge_kernel(const T* T1, int ld1, int k1, const T* T2, int ld2, int k2, const T* G12, int ldg,
                              T* Tout, int ldT) {
  using R = typename real_of<T>::type;
  __shared__ T s_t1[32][33], s_t2[32][33], s_g[32][33], s_x[32][33];
  const int i = threadIdx.x % 32, j = threadIdx.x / 32;
  const T z = mk<R>(0, 0);
  s_t1[i][j] = (i < k1 && j < k1) ? T1[i + (int64_t)j * ld1] : z;
  s_t2[i][j] = (i < k2 && j < k2) ? T2[i + (int64_t)j * ld2] : z;
  s_g[i][j] = (i < k1 && j < k2) ? G12[i + (int64_t)j * ldg] : z;
  __syncthreads();
  T acc = z;  // (T1 G12)[i][j]
  for (int l = 0; l < 32; ++l) cfma(acc, s_t1[i][l], s_g[l][j]);
  s_x[i][j] = acc;
  __syncthreads();
  acc = z;  // (T1 G12 T2)[i][j]
  for (int l = 0; l < 32; ++l) cfma(acc, s_x[i][l], s_t2[l][j]);
  const int kt = k1 + k2;
  if (i < k1 && j < k1) Tout[i + (int64_t)j * ldT] = s_t1[i][j];
  if (i < k2 && j < k2) Tout[k1 + i + (int64_t)(k1 + j) * ldT] = s_t2[i][j];
  if (i < k1 && j < k2) Tout[i + (int64_t)(k1 + j) * ldT] = z - acc;
  if (i < k2 && j < k1) Tout[k1 + i + (int64_t)j * ldT] = z;
  (void)kt;
}

// vn1[t] = vn2[t] = ||W[r0:m, t]||^2 for t in [c0, n): one warp per column.
template <typename T>
__global__ void col_norms_kernel(const T* W, int64_t ldw, int m, int r0, int c0, int n, double* vn1,
                                 double* vn2) {
  const int lane = threadIdx.x & 31;
  const int t = c0 + (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  if (t >= n) return;
  double s = warp_norm2<T>(W + (int64_t)t * ldw, r0, m, lane);
  if (lane == 0) {
    vn1[t] = s;
    vn2[t] = s;
  }
}

// vn1 = vn2 = squared column norms of a trailing block, from the per-tile partial
// sums (FP32, 64 rows each) that the block's update GEMM produced in its epilogue,
// added in FP64 in tile order; column j of the block is column c0 + j of W
__global__ void colsq_reduce_kernel(const float* P, int64_t ldp, int ntile, int N, int c0, double* vn1,
                                    double* vn2) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  double s = 0.0;
  for (int t = 0; t < ntile; ++t) s += (double)P[(int64_t)t * ldp + j];
  vn1[c0 + j] = s;
  vn2[c0 + j] = s;
}

// discarded = sum_{t in [c0, n)} vn1[t] (squared norms), one block, fixed order
__global__ void discarded_kernel(const double* vn1, int c0, int n, double* out, double* total) {
  __shared__ double s[256];
  double acc = 0.0;
  for (int t = c0 + threadIdx.x; t < n; t += 256) acc += vn1[t];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *out = s[0];
    if (total) *total += s[0];
  }
}

__global__ void iota_kernel(int* p, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = i;
}

PerDevice g_sms;  // zero-initialised (static storage)

}  // namespace

int num_sms() {
  return (int)g_sms.get([]() -> long long {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return 1;  // not cached: the next call asks again
    }
    return std::max(n, 1);
  });
}

// L2 capacity of the current device in bytes (0 when it cannot be read)
static PerDevice g_l2;
static int l2_bytes() {
  return (int)g_l2.get([]() -> long long {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrL2CacheSize, dev) != cudaSuccess) {
      cudaGetLastError();
      return -1;  // not cached: the next call asks again
    }
    return std::max(n, 0);
  });
}

constexpr int kPanelSmem = 200 * 1024;  // dynamic shared memory of the sketch-pivot kernel
// dynamic shared memory of the panel kernel: static + dynamic stays within the 227 KB
// a CTA may use (its static part holds the D2 staging arrays, twice as large in complex128)
template <typename T>
constexpr int panel_smem() {
  return sizeof(T) == 8 ? 200 * 1024 : 176 * 1024;
}

constexpr int kCPanelSmem = 200 * 1024;

// Cluster size usable for the unpivoted panel kernel on this device (16 when
// non-portable clusters of 16 CTAs with the full shared-memory carve-out can
// be resident, else 8, else 0 = not available).
template <typename T>
static int cpanel_cluster_size() {
  static PerDevice cache;
  return (int)cache.get([]() -> long long {
    if (cudaFuncSetAttribute(qr_cpanel_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kCPanelSmem) !=
        cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    cudaFuncSetAttribute(qr_cpanel_kernel<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaGetLastError();
    for (int cs : {16, 8}) {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = cs;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3(cs);
      cfg.blockDim = dim3(CPT);
      cfg.dynamicSmemBytes = kCPanelSmem;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int n = 0;
      if (cudaOccupancyMaxActiveClusters(&n, qr_cpanel_kernel<T>, &cfg) == cudaSuccess && n >= 1) return cs;
      cudaGetLastError();
    }
    return 0;
  });
}

template <typename T>
static cudaError_t panel_setup(int& max_blocks) {
  static PerDevice cache;
  cudaError_t err = cudaSuccess;
  const long long r = cache.get([&err]() -> long long {
    int smem = panel_smem<T>();
    err = cudaFuncSetAttribute(qr_panel_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (err != cudaSuccess) return -1;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, qr_panel_kernel<T>, PNT, smem);
    if (err != cudaSuccess) return -1;
    if (per_sm * num_sms() < 1) {
      err = cudaErrorInvalidConfiguration;
      return -1;
    }
    return per_sm * num_sms();
  });
  if (r < 0) return err != cudaSuccess ? err : cudaErrorInvalidConfiguration;
  max_blocks = (int)r;
  return cudaSuccess;
}

#define CK(x)                                  \
  do {                                         \
    cudaError_t e_ = (x);                      \
    if (e_ != cudaSuccess) {                   \
      note_cuda_failure(__FILE__, __LINE__);   \
      return e_;                               \
    }                                          \
  } while (0)

// Launch accounting of one QR: either by kernel class, or everything under
// the plan's override class (centre moves).
struct ClassMap {
  int over;
  int operator()(int c) const { return over >= 0 ? over : c; }
};

// Block reflector of the outer block starting at panel `pi` (panels pi and
// pi+1 when both exist): T (kbb x kbb, leading dim 2 nb) into p.Tblk[pi / 2],
// from the per-panel factors and the Gram block V1^H V2.  Returns the block
// width kbb.  Launch count added to *nl.
template <typename T>
static cudaError_t outer_tfactor(const QrPlan<T>& p, int pi, int* kbb_out, int* nl, cudaStream_t s) {
  using R = typename real_of<T>::type;
  const int nb = p.nb, k = p.k, m = p.m, ob = 2 * nb;
  const int j0 = pi * nb;
  const int k1 = std::min(nb, k - j0);
  const int k2 = std::max(0, std::min(nb, k - j0 - nb));
  T* Tb = p.Tblk + (size_t)(pi / 2) * ob * ob;
  const T* T1 = p.Tfac + (size_t)pi * nb * nb;
  const T* T2 = p.Tfac + (size_t)(pi + 1) * nb * nb;
  if (k2 > 0) {
    // G12 = V1^H V2 over the rows where V2 is nonzero (rows >= j0 + nb)
    GemmDesc<T> d;
    d.M = k1;
    d.N = k2;
    d.K = m - (j0 + nb);
    d.alpha = mk<R>(1, 0);
    d.beta = mk<R>(0, 0);
    d.A = p.W + (j0 + nb) + (int64_t)j0 * p.ldw;  // V1 rows >= j0+nb: plain (below V1's diagonal)
    d.lda = p.ldw;
    d.a_row = 1;
    d.a_conj = 1;
    d.a_mask = MASK_NONE;
    d.B = p.W + (j0 + nb) + (int64_t)(j0 + nb) * p.ldw;  // V2, unit lower
    d.ldb = p.ldw;
    d.b_row = 0;
    d.b_conj = 0;
    d.b_mask = MASK_UNIT_LOWER;
    d.C = p.G12;
    d.ldc = nb;
    d.splitk = choose_splitk(k1, k2, d.K, p.sk_cap, (int)sizeof(T));
    d.wk = p.SK;
    *nl += gemm_launches(d);
    CK(gemm_simt<T>(d, s));
  }
  tmerge_kernel<T><<<1, 1024, 0, s>>>(T1, nb, k1, T2, nb, k2, p.G12, nb, Tb, ob);
  CK(cudaGetLastError());
  *nl += 1;
  *kbb_out = k1 + k2;
  return cudaSuccess;
}

// Apply (I - V Tb V^H)^H (trans = 1) or (I - V Tb V^H) (trans = 0) to
// C = X[j0:m, c0:c0+N] (column-major, ldx), V = W[j0:m, j0:j0+kbb] unit lower:
//   Y = V^H C,  Z = Tb^H Y (or Tb Y),  C -= V Z.
template <typename T>
static cudaError_t apply_block(const QrPlan<T>& p, int j0, int kbb, const T* Tb, int ldT, int trans, T* X,
                               int64_t ldx, int c0, int N, int* nl, cudaStream_t s) {
  using R = typename real_of<T>::type;
  if (N <= 0 || kbb <= 0) return cudaSuccess;
  const int M = p.m - j0;
  GemmDesc<T> d;
  d.M = kbb;
  d.N = N;
  d.K = M;
  d.alpha = mk<R>(1, 0);
  d.beta = mk<R>(0, 0);
  d.A = p.W + j0 + (int64_t)j0 * p.ldw;  // V^H
  d.lda = p.ldw;
  d.a_row = 1;
  d.a_conj = 1;
  d.a_mask = MASK_UNIT_LOWER;
  d.B = X + j0 + (int64_t)c0 * ldx;
  d.ldb = ldx;
  d.b_row = 0;
  d.b_conj = 0;
  d.b_mask = MASK_NONE;
  d.C = p.Y;
  d.ldc = kbb;
  d.splitk = choose_splitk(kbb, N, M, p.sk_cap, (int)sizeof(T));
  d.wk = p.SK;
  *nl += gemm_launches(d);
  CK(gemm_simt<T>(d, s));
  d.splitk = 0;
  d.wk = nullptr;
  d.M = kbb;
  d.N = N;
  d.K = kbb;
  d.A = Tb;
  d.lda = ldT;
  d.a_row = trans ? 1 : 0;
  d.a_conj = trans ? 1 : 0;
  d.a_mask = MASK_NONE;
  d.B = p.Y;
  d.ldb = kbb;
  d.C = p.Z;
  d.ldc = kbb;
  *nl += 1;
  CK(gemm_simt<T>(d, s));
  d.M = M;
  d.N = N;
  d.K = kbb;
  d.alpha = mk<R>(-1, 0);
  d.beta = mk<R>(1, 0);
  d.A = p.W + j0 + (int64_t)j0 * p.ldw;  // V
  d.lda = p.ldw;
  d.a_row = 0;
  d.a_conj = 0;
  d.a_mask = MASK_UNIT_LOWER;
  d.B = p.Z;
  d.ldb = kbb;
  d.C = X + j0 + (int64_t)c0 * ldx;
  d.ldc = ldx;
  *nl += 1;
  return gemm_auto<T>(d, p.use_tc, p.err, p.timeout_ns, s);
}

// Launch one panel (pivoted or not) described by `a` (every data field set):
// chooses bulk copies, the grid size and the shared memory; an unpivoted panel
// whose rows fit the shared memory of one cluster runs on qr_cpanel_kernel when
// `cluster_ok`.
template <typename T>
static cudaError_t launch_panel(PanelArgs<T>& a, unsigned barrier_extra, int gcap, bool cluster_ok, cudaStream_t s) {
  const int m = a.m, j0 = a.j0, kb = a.kb;
  const int smem = panel_smem<T>();
  // bulk copies need 16-byte aligned column chunks: an aligned base, a
  // 16-byte multiple column stride and (complex64) chunks of whole row pairs
  a.bulk = (reinterpret_cast<uintptr_t>(a.W) % 16 == 0) && ((a.ldw * (int64_t)sizeof(T)) % 16 == 0) &&
           (sizeof(T) == 16 || m % 2 == 0);
  const int ncols = a.nend - j0;
  // enough CTAs for both the per-step row work (phase B) and the trailing columns
  int G = std::max(1, std::min(gcap, std::max((ncols + 7) / 8, (m - j0 + 63) / 64)));
  a.expected = (unsigned)G + barrier_extra;
  int dyn;
  if (a.bulk) {
    // bulk mode: the copy slots, then x when it fits beside them (else x is
    // read from global memory, where it stays in L2)
    const int64_t xb = ((int64_t)(m - j0 + 2) * sizeof(T) + 15) / 16 * 16;
    const bool fits = kRing + xb <= smem;
    dyn = kRing + (fits ? (int)xb : 0);
    a.xs_off = kRing;
    a.xcap = fits ? (int)(xb / (int64_t)sizeof(T)) : 0;
    // three quarters of L2 hold the chunks each step reads last (the rest keeps
    // x, F and the reduction slots)
    a.keep = (int)std::min<int64_t>(1 << 30, (int64_t)std::max(0, l2_bytes()) * 3 / 4 / ((int64_t)G * kSlot));
  } else {
    // dynamic shared memory sized to the x vector this panel stages (rounded
    // to 16 KB): the rest of the SM's unified L1/shared storage stays L1,
    // which holds the trailing sweep's loads in flight
    const int need = (int)std::min<int64_t>((int64_t)(m - j0 + 2) * sizeof(T), smem);
    dyn = std::min(smem, (need + 16383) / 16384 * 16384);
    a.keep = 0;
    a.xs_off = 0;
    a.xcap = dyn / (int)sizeof(T);
  }
  void* args[] = {&a};
  // unpivoted panels whose rows fit the shared memory of one cluster run on it
  const int ccs = (a.pivot || !cluster_ok) ? 0 : cpanel_cluster_size<T>();
  const int crb = ccs > 0 ? ((m - j0 + ccs - 1) / ccs + 1) / 2 * 2 : 0;
  if (ccs > 0 && (int64_t)kb * crb * (int64_t)sizeof(T) <= kCPanelSmem) {
    CPanelArgs<T> ca;
    ca.W = a.W;
    ca.ldw = a.ldw;
    ca.m = m;
    ca.j0 = j0;
    ca.kb = kb;
    ca.nb = a.nb;
    ca.rb = crb;
    ca.tau = a.tau;
    ca.Wg = a.Wg;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = ccs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(ccs);
    cfg.blockDim = dim3(CPT);
    cfg.dynamicSmemBytes = (size_t)kb * crb * sizeof(T);
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, qr_cpanel_kernel<T>, ca);
  }
  return cudaLaunchCooperativeKernel((const void*)qr_panel_kernel<T>, dim3(G), dim3(PNT), args, (size_t)dyn, s);
}

template <typename T>
cudaError_t qr_factor_sketched(const QrPlan<T>& p, cudaStream_t s, LaunchHooks* hooks);

// Plain QR (pivot == 0) with look-ahead, for panels that run on one thread-block
// cluster (16 SMs): while the cluster factors the panels of outer block q + 1, the
// other SMs apply outer block q's reflector to the columns beyond block q + 1.
// Per outer block q (panels 2q, 2q + 1), in this order:
//   s2: panel 2q, its T factor, its update of panel 2q + 1's columns, panel 2q + 1,
//       its T factor, the outer T factor of the pair;
//   s2: (after the main stream's update of block q - 1) the pair's reflector on the
//       columns of block q + 1;
//   s:  (after the outer factor) the pair's reflector on the columns beyond block q + 1.
// The two streams use separate GEMM scratch; every column sees the reflectors in
// order (block q - 1's main-stream update before block q's look-ahead update).
// Launches are accounted as one bracket on the caller's stream.
template <typename T>
static cudaError_t qr_factor_lookahead(const QrPlan<T>& p, cudaStream_t s, LaunchHooks* hooks) {
  const ClassMap K{p.kclass};
  const int m = p.m, n = p.n, k = p.k, nb = p.nb;
  const int npanels = (k + nb - 1) / nb;
  cudaStream_t s2 = p.s2;
  cudaEvent_t ev_fork = p.la_ev[0], ev_vt = p.la_ev[1], ev_b = p.la_ev[2];
  QrPlan<T> pm = p;  // the main stream's scratch
  pm.Y = p.Y2;
  pm.Z = p.Z2;
  pm.SK = p.SK2;
  int maxb = 1;
  CK(panel_setup<T>(maxb));
  const int gcap = std::max(1, std::min(p.G > 0 ? p.G : maxb, maxb));
  double alg = 0.0;
  for (int j = 0; j < k; ++j) alg += 8.0 * (m - j) * (std::min(n, (j / nb + 1) * nb) - j);
  hook_before(hooks, K(MPS_KCLASS_PANEL), 0.0, alg);
  int nl = 1;
  CK(cudaMemsetAsync(p.Tfac, 0, sizeof(T) * (size_t)npanels * nb * nb, s));
  iota_kernel<<<(n + 255) / 256, 256, 0, s>>>(p.jpvt, n);
  CK(cudaGetLastError());
  CK(cudaEventRecord(ev_fork, s));
  CK(cudaStreamWaitEvent(s2, ev_fork, 0));
  bool b_issued = false;  // ev_b holds a main-stream update not yet waited for by s2
  cudaError_t err = cudaSuccess;
  auto panel = [&](int pi) -> cudaError_t {
    const int j0 = pi * nb, kb = std::min(nb, k - j0);
    PanelArgs<T> a;
    a.W = p.W;
    a.ldw = p.ldw;
    a.m = m;
    a.n = n;
    a.j0 = j0;
    a.kb = kb;
    a.nend = std::min(n, j0 + kb);
    a.nb = nb;
    a.pivot = 0;
    a.F = p.F;
    a.vn1 = p.vn1;
    a.vn2 = p.vn2;
    a.jpvt = p.jpvt;
    a.tau = p.tau;
    a.Tp = p.Tfac + (size_t)pi * nb * nb;
    a.Wg = p.Wg + (size_t)pi * nb * nb;
    a.red_norm = p.red_norm;
    a.red_w = reinterpret_cast<T*>(p.red_w);
    a.red_argv = reinterpret_cast<long long*>(p.red_argv);
    a.red_argi = p.red_argi;
    a.alpha_slot = p.alpha_slot;
    a.bar = p.bar;
    a.err = p.err;
    a.timeout_ns = p.timeout_ns;
    a.flag_tol = p.flag_tol;
    a.piv_seq = nullptr;
    CK(launch_panel<T>(a, p.barrier_extra, gcap, true, s2));
    tfactor_kernel<T><<<1, 1024, 0, s2>>>(p.Wg, p.tau, pi, k, nb, p.Tfac);
    nl += 2;
    return cudaGetLastError();
  };
  for (int pb = 0; pb < npanels && err == cudaSuccess; pb += 2) {
    const int jb = pb * nb;
    const int kb0 = std::min(nb, k - jb);
    err = panel(pb);
    if (err != cudaSuccess) break;
    if (pb + 1 < npanels) {
      // the first panel's reflector on its partner's columns, then the partner
      err = apply_block<T>(p, jb, kb0, p.Tfac + (size_t)pb * nb * nb, nb, 1, p.W, p.ldw, jb + kb0,
                           std::min(nb, k - jb - kb0), &nl, s2);
      if (err == cudaSuccess) err = panel(pb + 1);
      if (err != cudaSuccess) break;
    }
    int kbb = 0;
    err = outer_tfactor<T>(p, pb, &kbb, &nl, s2);
    if (err != cudaSuccess) break;
    const T* Tb = p.Tblk + (size_t)(pb / 2) * 4 * nb * nb;
    const int c0 = std::min(k, jb + 2 * nb);         // first column after the pair
    const int la_end = std::min(n, c0 + 2 * nb);     // end of the next pair's columns
    if (c0 >= n) continue;
    if ((err = cudaEventRecord(ev_vt, s2)) != cudaSuccess) break;
    if (b_issued && (err = cudaStreamWaitEvent(s2, ev_b, 0)) != cudaSuccess) break;
    b_issued = false;
    // look-ahead: the next pair's columns, on the critical path
    err = apply_block<T>(p, jb, kbb, Tb, 2 * nb, 1, p.W, p.ldw, c0, la_end - c0, &nl, s2);
    if (err != cudaSuccess) break;
    if (la_end < n) {
      if ((err = cudaStreamWaitEvent(s, ev_vt, 0)) != cudaSuccess) break;
      err = apply_block<T>(pm, jb, kbb, Tb, 2 * nb, 1, p.W, p.ldw, la_end, n - la_end, &nl, s);
      if (err != cudaSuccess) break;
      if ((err = cudaEventRecord(ev_b, s)) != cudaSuccess) break;
      b_issued = true;
    }
  }
  // join: the caller's stream continues once the critical-path stream is done
  cudaError_t e2 = cudaEventRecord(ev_fork, s2);
  if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(s, ev_fork, 0);
  hook_after(hooks, K(MPS_KCLASS_PANEL), nl);
  if (err != cudaSuccess) {
    note_cuda_failure(__FILE__, __LINE__);
    return err;
  }
  CK(e2);
  return cudaSuccess;
}

// Whether a plain QR of this plan can run with look-ahead: every panel on the
// cluster kernel (the first panel, the tallest, fits its shared memory), the
// caller gave a second stream and the second scratch set, and the plan attributes
// all its launches to one kernel class (they are timed as one bracket).
template <typename T>
static bool lookahead_ok(const QrPlan<T>& p) {
  if (p.pivot != 0 || !p.s2 || !p.la_ev || !p.Y2 || !p.Z2 || !p.SK2 || p.kclass < 0) return false;
  const int ccs = cpanel_cluster_size<T>();
  if (ccs <= 0) return false;
  const int crb = ((p.m + ccs - 1) / ccs + 1) / 2 * 2;
  return (int64_t)std::min(p.nb, p.k) * crb * (int64_t)sizeof(T) <= kCPanelSmem;
}

template <typename T>
cudaError_t qr_factor(const QrPlan<T>& p, cudaStream_t s, LaunchHooks* hooks) {
  using R = typename real_of<T>::type;
  const ClassMap K{p.kclass};
  const int m = p.m, n = p.n, k = p.k, nb = p.nb;
  if (k <= 0) {
    if (p.pivot && p.discarded) {
      // nothing factored: discarded = ||W||_F^2
      hook_before(hooks, K(MPS_KCLASS_NORMS), (double)m * n * sizeof(T), 0);
      int threads = 256, warps = threads / 32;
      if (n > 0) {
        col_norms_kernel<T><<<(n + warps - 1) / warps, threads, 0, s>>>(p.W, p.ldw, m, 0, 0, n, p.vn1, p.vn2);
        CK(cudaGetLastError());
      }
      discarded_kernel<<<1, 256, 0, s>>>(p.vn1, 0, n, p.discarded, p.disc_total);
      CK(cudaGetLastError());
      hook_after(hooks, K(MPS_KCLASS_NORMS), n > 0 ? 2 : 1);
    }
    return cudaSuccess;
  }
  if (p.pivot == 2) return qr_factor_sketched<T>(p, s, hooks);
  if (lookahead_ok<T>(p)) return qr_factor_lookahead<T>(p, s, hooks);
  int maxb = 1;
  CK(panel_setup<T>(maxb));
  const int gcap = std::max(1, std::min(p.G > 0 ? p.G : maxb, maxb));
  const int npanels = (k + nb - 1) / nb;
  CK(cudaMemsetAsync(p.Tfac, 0, sizeof(T) * (size_t)npanels * nb * nb, s));
  hook_before(hooks, K(MPS_KCLASS_OTHER), 4.0 * n, 0);
  iota_kernel<<<(n + 255) / 256, 256, 0, s>>>(p.jpvt, n);
  CK(cudaGetLastError());
  hook_after(hooks, K(MPS_KCLASS_OTHER), 1);
  if (p.pivot) {
    hook_before(hooks, K(MPS_KCLASS_NORMS), (double)m * n * sizeof(T), 3.0 * m * n);
    int warps = 8;
    col_norms_kernel<T><<<(n + warps - 1) / warps, warps * 32, 0, s>>>(p.W, p.ldw, m, 0, 0, n, p.vn1, p.vn2);
    CK(cudaGetLastError());
    hook_after(hooks, K(MPS_KCLASS_NORMS), 1);
  }
  int tblk_done = 0;  // outer blocks whose factor the unpivoted trailing updates already built
  for (int pi = 0; pi < npanels; ++pi) {
    const int j0 = pi * nb;
    const int kb = std::min(nb, k - j0);
    const int J1 = j0 + kb;
    PanelArgs<T> a;
    a.W = p.W;
    a.ldw = p.ldw;
    a.m = m;
    a.n = n;
    a.j0 = j0;
    a.kb = kb;
    a.nend = p.pivot ? n : std::min(n, j0 + kb);
    a.nb = nb;
    a.pivot = p.pivot;
    a.F = p.F;
    a.vn1 = p.vn1;
    a.vn2 = p.vn2;
    a.jpvt = p.jpvt;
    a.tau = p.tau;
    a.Tp = p.Tfac + (size_t)pi * nb * nb;
    a.Wg = p.Wg + (size_t)pi * nb * nb;
    a.red_norm = p.red_norm;
    a.red_w = reinterpret_cast<T*>(p.red_w);
    a.red_argv = reinterpret_cast<long long*>(p.red_argv);
    a.red_argi = p.red_argi;
    a.alpha_slot = p.alpha_slot;
    a.bar = p.bar;
    a.err = p.err;
    a.timeout_ns = p.timeout_ns;
    a.flag_tol = p.flag_tol;
    a.piv_seq = nullptr;
    double bytes = 0.0, flops = 0.0;
    for (int j = j0; j < J1; ++j) {  // algorithmic: per step one read of the trailing block rows J..m
      double rows = (double)(m - j), cols = (double)(a.nend - j);
      bytes += rows * cols * sizeof(T);
      flops += 8.0 * rows * cols;
    }
    hook_before(hooks, K(MPS_KCLASS_PANEL), bytes, flops);
    CK(launch_panel<T>(a, p.barrier_extra, gcap, !p.pivot, s));
    hook_after(hooks, K(MPS_KCLASS_PANEL), 1);
    if (p.pivot) {
      // complex64: the update's epilogue also sums the squared column norms of the
      // block it writes (per 64-row tile, into the split-K scratch, which this
      // update does not use), so the norms need no second pass over the block
      bool fused = false;
      int ntile = 0;
      if (J1 < n && J1 < m) {
        GemmDesc<T> d;
        d.M = m - J1;
        d.N = n - J1;
        d.K = kb;
        d.alpha = mk<R>(-1, 0);
        d.beta = mk<R>(1, 0);
        d.A = p.W + J1 + (int64_t)j0 * p.ldw;
        d.lda = p.ldw;
        d.a_row = 0;
        d.a_conj = 0;
        d.a_mask = MASK_NONE;
        d.B = p.F + (int64_t)J1 * nb;  // B(k, j) = conj(F[J1 + j, k]): the array holds conj(F), col-major, ld nb
        d.ldb = nb;
        d.b_row = 0;
        d.b_conj = 0;
        d.b_mask = MASK_NONE;
        d.C = p.W + J1 + (int64_t)J1 * p.ldw;
        d.ldc = p.ldw;
        if constexpr (sizeof(T) == 8) {
          ntile = (d.M + 63) / 64;
          if (!p.use_tc && gemm_c64_tile_rows(d.M, d.K) == 64 && (int64_t)ntile * d.N <= 2 * p.sk_cap) {
            d.colsq = reinterpret_cast<float*>(p.SK);
            d.ldcs = d.N;
            fused = true;
          }
        }
        double M = d.M, N = d.N;
        hook_before(hooks, K(MPS_KCLASS_UPDATE), (2.0 * M * N + (M + N) * kb) * sizeof(T), 8.0 * M * N * kb);
        CK(gemm_auto<T>(d, p.use_tc, p.err, p.timeout_ns, s));
        hook_after(hooks, K(MPS_KCLASS_UPDATE), 1);
      }
      if (J1 < n && fused) {
        hook_before(hooks, K(MPS_KCLASS_NORMS), 4.0 * ntile * (n - J1) + 16.0 * (n - J1), (double)ntile * (n - J1));
        colsq_reduce_kernel<<<(n - J1 + 255) / 256, 256, 0, s>>>(reinterpret_cast<const float*>(p.SK), n - J1, ntile,
                                                                n - J1, J1, p.vn1, p.vn2);
        CK(cudaGetLastError());
        hook_after(hooks, K(MPS_KCLASS_NORMS), 1);
      } else if (J1 < n) {
        hook_before(hooks, K(MPS_KCLASS_NORMS), (double)std::max(0, m - J1) * (n - J1) * sizeof(T),
                    3.0 * std::max(0, m - J1) * (n - J1));
        int warps = 8;
        col_norms_kernel<T><<<(n - J1 + warps - 1) / warps, warps * 32, 0, s>>>(p.W, p.ldw, m, J1, J1, n, p.vn1,
                                                                               p.vn2);
        CK(cudaGetLastError());
        hook_after(hooks, K(MPS_KCLASS_NORMS), 1);
      }
    } else if (J1 < n) {
      // two-level blocking: panels are paired into outer blocks of 2 nb columns;
      // the first panel of a pair updates only its partner's columns, the pair's
      // combined block reflector then updates everything to the right.
      int nl = 1;
      const bool first_of_pair = (pi % 2 == 0) && (pi + 1 < npanels);
      const int pb = pi - (pi % 2);  // first panel of this outer block
      const int jb = first_of_pair ? j0 : pb * nb;
      const int c0 = first_of_pair ? J1 : std::min(k, jb + 2 * nb);
      const int c1 = first_of_pair ? std::min(k, j0 + 2 * nb) : n;  // partner columns only
      const double M = m - jb, N = c1 - c0, kr = first_of_pair ? kb : c0 - jb;
      hook_before(hooks, K(MPS_KCLASS_UPDATE), (2.0 * M * kr + 3.0 * M * N) * sizeof(T), 16.0 * M * N * kr);
      tfactor_kernel<T><<<1, 1024, 0, s>>>(p.Wg, p.tau, pi, k, nb, p.Tfac);
      CK(cudaGetLastError());
      if (first_of_pair) {
        CK(apply_block<T>(p, j0, kb, p.Tfac + (size_t)pi * nb * nb, nb, 1, p.W, p.ldw, c0, c1 - c0, &nl, s));
      } else {
        int kbb = 0;
        CK(outer_tfactor<T>(p, pb, &kbb, &nl, s));
        tblk_done = pb / 2 + 1;
        CK(apply_block<T>(p, jb, kbb, p.Tblk + (size_t)(pb / 2) * 4 * nb * nb, 2 * nb, 1, p.W, p.ldw, c0, c1 - c0,
                          &nl, s));
      }
      hook_after(hooks, K(MPS_KCLASS_UPDATE), nl);
    }
  }
  {
    // triangular factors for Q formation: every panel's own factor (the
    // unpivoted path already has all but the last), then the outer blocks
    const int first = p.pivot ? 0 : npanels - 1;
    const int cnt = p.pivot ? npanels : 1;
    int nl = 1;
    hook_before(hooks, K(MPS_KCLASS_FORMQ), 0, 0);
    tfactor_kernel<T><<<cnt, 1024, 0, s>>>(p.Wg, p.tau, first, k, nb, p.Tfac);
    CK(cudaGetLastError());
    for (int pb = 2 * tblk_done; pb < npanels; pb += 2) {
      int kbb = 0;
      CK(outer_tfactor<T>(p, pb, &kbb, &nl, s));
    }
    hook_after(hooks, K(MPS_KCLASS_FORMQ), nl);
  }
  if (p.pivot && p.discarded) {
    hook_before(hooks, K(MPS_KCLASS_NORMS), 8.0 * (n - k), 0);
    discarded_kernel<<<1, 256, 0, s>>>(p.vn1, k, n, p.discarded, p.disc_total);
    CK(cudaGetLastError());
    hook_after(hooks, K(MPS_KCLASS_NORMS), 1);
  }
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Truncated QR with randomized column pivoting (pivot == 2): blocked RQRCP of
// Duersch and Gu / Martinsson et al.  The pivots of each block of nb columns are
// chosen by nb steps of the pivoted panel kernel on a small sketch Y = Omega W
// (lsk = nb + oversampling rows) instead of on W itself; the block is then
// factored without pivoting (the centre-move panel kernels) and applied to the
// whole trailing matrix as one block reflector (GEMMs), and the sketch of the
// trailing columns is updated as Y2 -= (Y1 R11^{-1}) R12.  The per-pivot pass
// over the trailing matrix of QP3 is gone; what remains per pivot is the panel's
// own column work and a pass over the short sketch.

// Omega (ldy x m, column-major, rows < lsk): entry (i, r) = -1 when the top bit of
// SplitMix64 output number i*m + r is set, else +1.  SplitMix64 (Steele, Lea and
// Flood, OOPSLA 2014) as a counter-based generator: the output for counter c is
// the mixing function applied to seed + (c + 1) * 0x9E3779B97F4A7C15 (mod 2^64).
__device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long seed, unsigned long long c) {
  unsigned long long z = seed + (c + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <typename T>
__global__ void sketch_omega_kernel(T* Om, int64_t ldy, int lsk, int m, unsigned long long seed) {
  using R = typename real_of<T>::type;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= ldy * (int64_t)m) return;
  const int i = (int)(idx % ldy);
  const int64_t r = idx / ldy;
  R v = 0;
  if (i < lsk) v = (splitmix64_at(seed, (unsigned long long)i * (unsigned long long)m + (unsigned long long)r) >> 63)
                       ? R(-1)
                       : R(1);
  Om[idx] = mk<R>(v, 0);
}

// The column swaps a sketch panel made, applied to another matrix: for t < kb, in
// order, swap columns j0 + t and j0 + seq[t] of A (rows [0, rows)); with jpvt the
// same swaps are made on jpvt (block 0).
template <typename T>
__global__ void apply_swaps_kernel(T* A, int64_t lda, int rows, int j0, const int* seq, int kb, int* jpvt, int nc,
                                   int* err) {
  __shared__ int s_seq[kSketchBlockMax];
  if (threadIdx.x < kb) {
    const int q = seq[threadIdx.x];
    // a position outside [t, nc) would be an out-of-range column: the swap is skipped
    s_seq[threadIdx.x] = index_ok(q >= (int)threadIdx.x && q < nc, err) ? q : (int)threadIdx.x;
  }
  __syncthreads();
  if (jpvt && blockIdx.x == 0 && threadIdx.x == 0) {
    for (int t = 0; t < kb; ++t) {
      const int q = j0 + s_seq[t];
      const int x = jpvt[j0 + t];
      jpvt[j0 + t] = jpvt[q];
      jpvt[q] = x;
    }
  }
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
    for (int t = 0; t < kb; ++t) {
      const int q = j0 + s_seq[t];
      if (q == j0 + t) continue;
      T* a = A + r + (int64_t)(j0 + t) * lda;
      T* b = A + r + (int64_t)q * lda;
      const T x = *a;
      *a = *b;
      *b = x;
    }
  }
}

// S (ldy x kb, rows < lsk) with S R11 = Y[:, j0:j0+kb], R11 = W[j0:j0+kb, j0:j0+kb]
// upper triangular (read from W: every thread reads the same entries), by forward
// substitution per sketch row; a diagonal entry whose squared modulus is below the
// smallest normal number of the data type (a column with no residual) contributes
// nothing (its column of S is zero).
template <typename T>
__global__ void sketch_solve_kernel(const T* Ys, int64_t ldy, int lsk, int j0, int kb, const T* W, int64_t ldw,
                                    T* S) {
  using R = typename real_of<T>::type;
  const double tiny = sizeof(R) == 8 ? 2.2250738585072014e-308 : 1.1754943508222875e-38;
  for (int i = threadIdx.x; i < lsk; i += blockDim.x) {
    T sv[kSketchBlockMax];
    for (int c = 0; c < kb; ++c) {
      T rhs = Ys[i + (int64_t)(j0 + c) * ldy];
      const T* rc = W + j0 + (int64_t)(j0 + c) * ldw;  // column c of R11
      for (int t = 0; t < c; ++t) rhs = rhs - sv[t] * rc[t];
      const T d = rc[c];
      const double d2 = (double)d.re * (double)d.re + (double)d.im * (double)d.im;
      T q = mk<R>(0, 0);
      if (d2 >= tiny) {
        const R inv = (R)(1.0 / d2);
        q = rhs * mk<R>(d.re * inv, -d.im * inv);  // rhs / d
      }
      sv[c] = q;
      S[i + (int64_t)c * ldy] = q;
    }
  }
}

// Pivots of one block from the sketch: kb steps of column-pivoted Householder QR
// on the l x nc matrix Y (column-major, ld ldy), writing at step j the position p
// that was swapped with j (the contract of PanelArgs::piv_seq).  As in the panel
// kernel, the squared column norms are FP64, downdated after every step
// (vn1 -= |y_j|^2) and recomputed exactly when vn1 <= flag_tol * vn2 (vn2 = the last
// exact value); exact ties of squared norms go to the lowest original column.
// Cooperative grid, one grid barrier per step: every CTA keeps its share of the
// columns in shared memory, row-major so that one thread per column reads and
// updates it without bank conflicts, publishes its best candidate (norm, column and
// the column's entries) in a double-buffered global slot, and after the barrier all
// CTAs pick the same winner and build the same reflector in FP64.  CTA 0 keeps the
// position map.
constexpr int SKT = 256;  // threads of the sketch-pivot kernel
constexpr int SKW = SKT / 32;

template <typename T>
struct SketchPivArgs {
  const T* Y;
  int64_t ldy;
  int l, nc, kb;
  int* piv_seq;
  int* col_at;   // nc: CTA 0's position map
  int* pos_of;   // nc
  T* pub;        // 2 * G * (l + 2) published candidates
  unsigned* bar;
  int* err;
  unsigned expected;
  unsigned long long timeout_ns;
  double flag_tol;
};

template <typename T>
__device__ __forceinline__ double sk_col_norm2(const T* ys, int nl, int c, int r0, int l) {
  double s2 = 0.0;
  for (int r = r0; r < l; ++r) {
    const T x = ys[r * nl + c];
    s2 += (double)x.re * (double)x.re + (double)x.im * (double)x.im;
  }
  return s2;
}

template <typename T>
__global__ void __launch_bounds__(SKT) sketch_pivots_kernel(SketchPivArgs<T> a) {
  using R = typename real_of<T>::type;
  extern __shared__ __align__(16) unsigned char sk_smem[];
  const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int l = a.l;
  int c0, c1;
  split_range(0, a.nc, G, b, c0, c1);
  const int nl = c1 - c0;
  // carve-up of the dynamic shared memory, every part starting on a 16-byte boundary
  // (l * nl * sizeof(T) is a multiple of 16 for the even sketch heights used; each
  // norm array is rounded up to an even count of doubles)
  const int nl2 = (nl + 1) & ~1;
  T* ys = reinterpret_cast<T*>(sk_smem);                          // l x nl, row-major (row r at ys + r nl)
  double* vn1 = reinterpret_cast<double*>(ys + (int64_t)l * nl);  // nl squared norms (< 0: consumed)
  double* vn2 = vn1 + nl2;                                        // nl: the last exact values
  T* xw = reinterpret_cast<T*>(vn2 + nl2);                        // the winner's column, l entries
  __shared__ double s_bv[SKW];
  __shared__ int s_bi[SKW];
  __shared__ int s_win, s_wb;
  __shared__ c128 s_tau, s_sc;
  __shared__ int s_skip;
  unsigned bgen = 0;  // thread 0: generation of the grid barrier (grid_barrier_g)
  if (tid == 0) {
    s_skip = ld_relaxed_i32(a.err) != DEV_OK;
    bgen = ld_acquire_u32(&a.bar[1]);
  }
  for (int e = tid; e < l * nl; e += SKT) {
    const int c = e / l, r = e - c * l;  // coalesced reads along each column
    ys[r * nl + c] = a.Y[r + (int64_t)(c0 + c) * a.ldy];
  }
  if (b == 0)
    for (int c = tid; c < a.nc; c += SKT) {
      a.col_at[c] = c;
      a.pos_of[c] = c;
    }
  __syncthreads();
  if (s_skip) return;
  for (int c = tid; c < nl; c += SKT) {
    const double s2 = sk_col_norm2(ys, nl, c, 0, l);
    vn1[c] = s2;
    vn2[c] = s2;
  }
  __syncthreads();
  const int slot = l + 2;  // published entries per CTA: norm, column index, the column
  for (int j = 0; j < a.kb; ++j) {
    // local candidate: the largest norm, the lowest column on ties
    double bv = -1.0;
    int bi = 0x7fffffff;
    for (int c = tid; c < nl; c += SKT)
      if (vn1[c] > bv) {  // ascending c per thread
        bv = vn1[c];
        bi = c0 + c;
      }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi < bi)) {
        bv = ov;
        bi = oi;
      }
    }
    if (lane == 0) {
      s_bv[warp] = bv;
      s_bi[warp] = bi;
    }
    __syncthreads();
    T* pub = a.pub + ((int64_t)(j & 1) * G + b) * slot;
    if (tid == 0) {
      for (int w = 1; w < SKW; ++w)
        if (s_bv[w] > s_bv[0] || (s_bv[w] == s_bv[0] && s_bi[w] < s_bi[0])) {
          s_bv[0] = s_bv[w];
          s_bi[0] = s_bi[w];
        }
      pub[0] = mk<R>((R)0, (R)0);
      reinterpret_cast<double*>(pub)[0] = s_bv[0];  // the norm travels as FP64 bits
      reinterpret_cast<int*>(pub + 1)[0] = s_bi[0];
    }
    __syncthreads();
    if (s_bi[0] >= c0 && s_bi[0] < c1) {
      const int c = s_bi[0] - c0;
      for (int r = tid; r < l; r += SKT) pub[2 + r] = ys[r * nl + c];
    }
    if (!grid_barrier_g(a.bar, a.expected, a.err, a.timeout_ns, bgen)) return;
    // the winner over all CTAs (identical in every CTA)
    const T* pset = a.pub + (int64_t)(j & 1) * G * slot;
    if (warp == 0) {
      double wv = -1.0;
      int wi = 0x7fffffff, wb = 0;
      for (int g = lane; g < G; g += 32) {
        const double v = reinterpret_cast<const volatile double*>(pset + (int64_t)g * slot)[0];
        const int i = reinterpret_cast<const volatile int*>(pset + (int64_t)g * slot + 1)[0];
        if (v > wv || (v == wv && i < wi)) {
          wv = v;
          wi = i;
          wb = g;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, wv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, wi, o);
        const int ob = __shfl_xor_sync(0xffffffffu, wb, o);
        if (ov > wv || (ov == wv && oi < wi)) {
          wv = ov;
          wi = oi;
          wb = ob;
        }
      }
      if (lane == 0) {
        s_win = wi;
        s_wb = wb;
      }
    }
    __syncthreads();
    const int win = s_win, wb = s_wb;
    if (win < 0 || win >= a.nc) {  // only reachable with non-finite norms
      if (tid == 0) atomicCAS(a.err, DEV_OK, DEV_ERR_NONFINITE);
      return;
    }
    for (int r = tid; r < l; r += SKT) xw[r] = pset[(int64_t)wb * slot + 2 + r];
    __syncthreads();
    // reflector of x = winner[j:l] in FP64 (warp 0; the same arithmetic in every CTA)
    if (warp == 0) {
      double tail = 0.0;
      for (int r = j + 1 + lane; r < l; r += 32) {
        const T x = xw[r];
        tail += (double)x.re * (double)x.re + (double)x.im * (double)x.im;
      }
      tail = warp_sum(tail);
      if (lane == 0) {
        const c128 al = ccast<double>(xw[j]);
        c128 tau, sc;
        if ((tail == 0.0 && al.im == 0.0) || al.re * al.re + al.im * al.im + tail < zero_column_level<T>()) {
          tau = mk<double>(0, 0);
          sc = mk<double>(0, 0);
        } else {
          const double nr = sqrt(al.re * al.re + al.im * al.im + tail);
          const double bt = al.re >= 0.0 ? -nr : nr;
          tau = mk<double>((bt - al.re) / bt, -al.im / bt);
          const c128 dnm = mk<double>(al.re - bt, al.im);
          const double dd = dnm.re * dnm.re + dnm.im * dnm.im;
          sc = mk<double>(dnm.re / dd, -dnm.im / dd);
        }
        s_tau = tau;
        s_sc = sc;
        if (b == 0) {
          // sequential swap semantics: the winner's current position p is swapped with j
          const int p = a.pos_of[win], cj = a.col_at[j];
          a.piv_seq[j] = p;
          a.col_at[p] = cj;
          a.pos_of[cj] = p;
          a.col_at[j] = win;
          a.pos_of[win] = j;
        }
      }
    }
    __syncthreads();
    const T sc = ccast<R>(s_sc), ctau = cconj(ccast<R>(s_tau));
    for (int r = j + 1 + tid; r < l; r += SKT) xw[r] = xw[r] * sc;  // v (v_j = 1 implicit)
    if (win >= c0 && win < c1 && tid == 0) vn1[win - c0] = -1.0;    // consumed
    __syncthreads();
    const bool apply = !(s_tau.re == 0.0 && s_tau.im == 0.0);
    // one thread per remaining column: H^H applied, then the FP64 norm downdate
    for (int c = tid; c < nl; c += SKT) {
      if (vn1[c] < 0.0) continue;
      T yj = ys[j * nl + c];
      if (apply) {
        T d = yj;
        for (int r = j + 1; r < l; ++r) cfma_conj(d, xw[r], ys[r * nl + c]);
        const T f = ctau * d;
        yj = yj - f;
        ys[j * nl + c] = yj;
        for (int r = j + 1; r < l; ++r) ys[r * nl + c] = ys[r * nl + c] - xw[r] * f;
      }
      const double r2 = (double)yj.re * (double)yj.re + (double)yj.im * (double)yj.im;
      const double v1 = fmax(vn1[c] - r2, 0.0);
      if (v1 <= a.flag_tol * vn2[c]) {
        const double e2 = sk_col_norm2(ys, nl, c, j + 1, l);
        vn1[c] = e2;
        vn2[c] = e2;
      } else {
        vn1[c] = v1;
      }
    }
    __syncthreads();
  }
}

template <typename T>
static size_t sketch_piv_smem(int l, int nl) {
  return (size_t)l * nl * sizeof(T) + 2 * (size_t)((nl + 1) & ~1) * 8 + (size_t)l * sizeof(T);
}

// Launch sketch_pivots_kernel for the l x nc sketch Y (pub: 2 G (l + 2) elements of
// scratch, maps: 2 nc ints).
template <typename T>
static cudaError_t launch_sketch_pivots(const T* Y, int64_t ldy, int l, int nc, int kb, int* piv_seq, int* maps,
                                        T* pub, int64_t pub_cap, unsigned* bar, int* err, unsigned barrier_extra,
                                        unsigned long long timeout_ns, double flag_tol, cudaStream_t s) {
  static PerDevice once;
  cudaError_t attr = cudaSuccess;
  once.get([&attr]() -> long long {
    attr = cudaFuncSetAttribute(sketch_pivots_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPanelSmem);
    return attr == cudaSuccess ? 1 : -1;
  });
  if (attr != cudaSuccess) return attr;
  // about 128 columns per CTA (one thread per column does a step's work in a few
  // hundred cycles, so the grid barrier sets the pace); more CTAs where the columns
  // do not fit one CTA's shared memory (one CTA per SM at most)
  int G = std::max(1, std::min(num_sms(), (nc + 127) / 128));
  while (G < num_sms() && sketch_piv_smem<T>(l, (nc + G - 1) / G) > (size_t)(160 * 1024)) ++G;
  const size_t smem = sketch_piv_smem<T>(l, (nc + G - 1) / G);
  if (smem > (size_t)kPanelSmem || 2 * (int64_t)G * (l + 2) > pub_cap) return cudaErrorInvalidConfiguration;
  if (sizeof(T) == 8 && (l & 1)) return cudaErrorInvalidValue;  // the norm arrays must start 16-byte aligned
  SketchPivArgs<T> a;
  a.Y = Y;
  a.ldy = ldy;
  a.l = l;
  a.nc = nc;
  a.kb = kb;
  a.piv_seq = piv_seq;
  a.col_at = maps;
  a.pos_of = maps + nc;
  a.pub = pub;
  a.bar = bar;
  a.err = err;
  a.expected = (unsigned)G + barrier_extra;
  a.timeout_ns = timeout_ns;
  a.flag_tol = flag_tol;
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel((const void*)sketch_pivots_kernel<T>, dim3(G), dim3(SKT), args, smem, s);
}

template <typename T>
cudaError_t qr_factor_sketched(const QrPlan<T>& p, cudaStream_t s, LaunchHooks* hooks) {
  using R = typename real_of<T>::type;
  const ClassMap K{p.kclass};
  const int m = p.m, n = p.n, k = p.k, nb = p.nb, l = p.lsk;
  const int64_t ldy = p.ldy;
  if (!p.Om || !p.Ys || !p.Ssk || !p.piv_seq || l < 2 * nb || ldy < l || 2 * nb > kSketchBlockMax)
    return cudaErrorInvalidValue;
  int maxb = 1;
  CK(panel_setup<T>(maxb));
  const int gcap = std::max(1, std::min(p.G > 0 ? p.G : maxb, maxb));
  const int npanels = (k + nb - 1) / nb;
  CK(cudaMemsetAsync(p.Tfac, 0, sizeof(T) * (size_t)npanels * nb * nb, s));
  // Y = Omega W
  hook_before(hooks, K(MPS_KCLASS_OTHER), (double)m * n * sizeof(T), 8.0 * l * m * n);
  iota_kernel<<<(n + 255) / 256, 256, 0, s>>>(p.jpvt, n);
  CK(cudaGetLastError());
  {
    const int64_t tot = ldy * (int64_t)m;
    sketch_omega_kernel<T><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(p.Om, ldy, l, m, p.seed);
    CK(cudaGetLastError());
    GemmDesc<T> d;
    d.M = l;
    d.N = n;
    d.K = m;
    d.alpha = mk<R>(1, 0);
    d.beta = mk<R>(0, 0);
    d.A = p.Om;
    d.lda = ldy;
    d.a_row = 0;
    d.B = p.W;
    d.ldb = p.ldw;
    d.b_row = 0;
    d.C = p.Ys;
    d.ldc = ldy;
    d.splitk = choose_splitk(l, n, m, p.sk_cap, (int)sizeof(T));
    d.wk = p.SK;
    CK(gemm_simt<T>(d, s));
    hook_after(hooks, K(MPS_KCLASS_OTHER), 2 + gemm_launches(d));
  }
  const int bw = 2 * nb;  // pivots per sketch block: two panels, one block reflector
  for (int j0 = 0; j0 < k; j0 += bw) {
    const int kbb = std::min(bw, k - j0);
    const int kb0 = std::min(nb, kbb), kb1 = kbb - kb0;
    const int pi0 = j0 / nb;
    const int J1 = j0 + kbb;
    const int nr = n - j0;
    // a. the block's pivots from the sketch's remaining columns (sketch_pivots_kernel),
    //    then the same column swaps on W, on the sketch and on jpvt
    hook_before(hooks, K(MPS_KCLASS_PANEL), (double)l * nr * sizeof(T), 8.0 * l * nr * kbb);
    CK(launch_sketch_pivots<T>(p.Ys + (int64_t)j0 * ldy, ldy, l, nr, kbb, p.piv_seq, reinterpret_cast<int*>(p.vn1),
                               p.SK, p.sk_cap, p.bar, p.err, p.barrier_extra, p.timeout_ns, p.flag_tol, s));
    apply_swaps_kernel<T><<<std::max(1, std::min(1024, (m + 255) / 256)), 256, 0, s>>>(p.W, p.ldw, m, j0, p.piv_seq,
                                                                                      kbb, p.jpvt, nr, p.err);
    CK(cudaGetLastError());
    apply_swaps_kernel<T><<<1, 256, 0, s>>>(p.Ys, ldy, l, j0, p.piv_seq, kbb, nullptr, nr, p.err);
    CK(cudaGetLastError());
    hook_after(hooks, K(MPS_KCLASS_PANEL), 3);
    // b. the block's two panels without pivoting (as a centre move's): the first
    //    panel's reflector is applied to the second panel's columns only
    PanelArgs<T> b;
    b.F = p.F;
    b.vn1 = p.vn1;
    b.vn2 = p.vn2;
    b.red_norm = p.red_norm;
    b.red_w = reinterpret_cast<T*>(p.red_w);
    b.red_argv = reinterpret_cast<long long*>(p.red_argv);
    b.red_argi = p.red_argi;
    b.alpha_slot = p.alpha_slot;
    b.bar = p.bar;
    b.err = p.err;
    b.timeout_ns = p.timeout_ns;
    b.flag_tol = p.flag_tol;
    b.nb = nb;
    b.W = p.W;
    b.ldw = p.ldw;
    b.m = m;
    b.n = n;
    b.pivot = 0;
    b.jpvt = p.jpvt;
    b.tau = p.tau;
    b.piv_seq = nullptr;
    for (int h = 0; h < 2; ++h) {
      const int kbh = h == 0 ? kb0 : kb1;
      if (kbh <= 0) break;
      const int jh = j0 + h * nb, pih = pi0 + h;
      b.j0 = jh;
      b.kb = kbh;
      b.nend = jh + kbh;
      b.Tp = p.Tfac + (size_t)pih * nb * nb;
      b.Wg = p.Wg + (size_t)pih * nb * nb;
      double bytes = 0.0, flops = 0.0;
      for (int j = jh; j < jh + kbh; ++j) {
        bytes += (double)(m - j) * (jh + kbh - j) * sizeof(T);
        flops += 8.0 * (m - j) * (jh + kbh - j);
      }
      hook_before(hooks, K(MPS_KCLASS_PANEL), bytes, flops);
      CK(launch_panel<T>(b, p.barrier_extra, gcap, true, s));
      hook_after(hooks, K(MPS_KCLASS_PANEL), 1);
      int nl = 1;
      hook_before(hooks, K(MPS_KCLASS_UPDATE), 0, 0);
      tfactor_kernel<T><<<1, 1024, 0, s>>>(p.Wg, p.tau, pih, k, nb, p.Tfac);
      CK(cudaGetLastError());
      if (h == 0 && kb1 > 0)
        CK(apply_block<T>(p, j0, kb0, p.Tfac + (size_t)pi0 * nb * nb, nb, 1, p.W, p.ldw, j0 + kb0, kb1, &nl, s));
      hook_after(hooks, K(MPS_KCLASS_UPDATE), nl);
    }
    // the block's reflector: both panels' T factors merged into one (the outer
    // factor, also used to form Q), applied to every column to the right
    {
      int nl = 0, kbm = 0;
      const double M = m - j0, N = n - J1;
      hook_before(hooks, K(MPS_KCLASS_UPDATE), (2.0 * M * kbb + 3.0 * M * N) * sizeof(T), 16.0 * M * N * kbb);
      CK(outer_tfactor<T>(p, pi0, &kbm, &nl, s));
      CK(apply_block<T>(p, j0, kbm, p.Tblk + (size_t)(pi0 / 2) * 4 * nb * nb, 2 * nb, 1, p.W, p.ldw, J1, n - J1, &nl,
                        s));
      hook_after(hooks, K(MPS_KCLASS_UPDATE), nl);
    }
    if (J1 < n) {
      // c. sketch update Y[:, J1:] -= (Y[:, j0:J1] R11^{-1}) R12
      const double N = n - J1;
      hook_before(hooks, K(MPS_KCLASS_OTHER), (double)(l + kbb) * N * sizeof(T) * 2, 8.0 * l * kbb * N);
      sketch_solve_kernel<T><<<1, 128, 0, s>>>(p.Ys, ldy, l, j0, kbb, p.W, p.ldw, p.Ssk);
      CK(cudaGetLastError());
      GemmDesc<T> d;
      d.M = l;
      d.N = n - J1;
      d.K = kbb;
      d.alpha = mk<R>(-1, 0);
      d.beta = mk<R>(1, 0);
      d.A = p.Ssk;
      d.lda = ldy;
      d.a_row = 0;
      d.B = p.W + j0 + (int64_t)J1 * p.ldw;
      d.ldb = p.ldw;
      d.b_row = 0;
      d.C = p.Ys + (int64_t)J1 * ldy;
      d.ldc = ldy;
      CK(gemm_simt<T>(d, s));
      hook_after(hooks, K(MPS_KCLASS_OTHER), 2);
    }
  }
  if (p.discarded) {
    // discarded = ||W[k:m, k:n]||_F^2
    hook_before(hooks, K(MPS_KCLASS_NORMS), (double)std::max(0, m - k) * (n - k) * sizeof(T), 0);
    if (k < n)
      col_norms_kernel<T><<<(n - k + 7) / 8, 256, 0, s>>>(p.W, p.ldw, m, k, k, n, p.vn1, p.vn2);
    CK(cudaGetLastError());
    discarded_kernel<<<1, 256, 0, s>>>(p.vn1, k, n, p.discarded, p.disc_total);
    CK(cudaGetLastError());
    hook_after(hooks, K(MPS_KCLASS_NORMS), k < n ? 2 : 1);
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t qr_form_q(const QrPlan<T>& p, T* Q, int64_t ldq, cudaStream_t s, LaunchHooks* hooks) {
  using R = typename real_of<T>::type;
  const ClassMap K{p.kclass};
  const int m = p.m, k = p.k, nb = p.nb;
  if (k <= 0) return cudaSuccess;
  hook_before(hooks, K(MPS_KCLASS_FORMQ), (double)m * k * sizeof(T), 0);
  CK(set_identity<T>(Q, ldq, m, k, s));
  hook_after(hooks, K(MPS_KCLASS_FORMQ), 1);
  const int npanels = (k + nb - 1) / nb;
  const int ob = 2 * nb;
  const int nblk = (npanels + 1) / 2;
  for (int bi = nblk - 1; bi >= 0; --bi) {
    const int j0 = bi * ob;
    const int kbb = std::min(ob, k - j0);
    const int M = m - j0, N = k - j0;
    int nl = 0;
    hook_before(hooks, K(MPS_KCLASS_FORMQ), (2.0 * M * N + 2.0 * M * kbb) * sizeof(T), 16.0 * M * N * kbb);
    CK(apply_block<T>(p, j0, kbb, p.Tblk + (size_t)bi * ob * ob, ob, 0, Q, ldq, j0, N, &nl, s));
    hook_after(hooks, K(MPS_KCLASS_FORMQ), nl);
  }
  return cudaSuccess;
}

template cudaError_t qr_factor<c64>(const QrPlan<c64>&, cudaStream_t, LaunchHooks*);
template cudaError_t qr_factor<c128>(const QrPlan<c128>&, cudaStream_t, LaunchHooks*);
template cudaError_t qr_form_q<c64>(const QrPlan<c64>&, c64*, int64_t, cudaStream_t, LaunchHooks*);
template cudaError_t qr_form_q<c128>(const QrPlan<c128>&, c128*, int64_t, cudaStream_t, LaunchHooks*);

}  // namespace mpsg
