// Blocked Householder QR with column pivoting (QP3 formulation) on one GPU.
//
// Computes theta P = Q R stopped after k pivots (Sec. III-B.2, QR with
// pivoting; truncation of Sec. III-C.2).  The matrix W (m x n, column-major)
// is factored in panels of nb columns:
//
//   panel kernel (persistent, cooperative, one CTA per SM at most), for each
//   step J of the panel:
//     A. pivot p = argmax_t vn1[t] over trailing columns (FP64, lowest index
//        on ties), from per-CTA partial maxima;
//     B. swap columns J and p; bring column J up to date with the panel's
//        earlier reflectors, x = W[J:m, J] - V F[p,:]^H; partial sums of
//        ||x_{J+1:}||^2 (FP64) and V^H x;
//     C. reflector: beta = -sign(Re alpha) ||x||, tau = (beta - alpha)/beta,
//        v = (1, x_{J+1:} / (alpha - beta)), in FP64;
//     D. for every trailing column t (split across CTAs, one warp per column):
//        y_t = W[J:m, t]^H v (the BLAS-2 sweep over the trailing matrix),
//        F[t, k] = tau (y_t - F[t, :k] w) with w = V^H v,
//        row update W[J, t] -= W[J, panel] F[t, :]^H (this row is final R),
//        FP64 norm downdate of vn1[t] with an exact recompute when the
//        downdate loses accuracy (|vn1|/|vn2| below a threshold).
//   Two grid barriers per step, every wait bounded.
//
//   trailing update: W[J1:m, J1:n] -= V F^H (rank-nb GEMM), then an exact FP64
//   recompute of every trailing column norm.
//
// Without pivoting (centre moves, Sec. III-C.1) the panel kernel only touches
// the panel's own columns and the rest of the matrix receives the compact-WY
// block reflector, C -= V T^H V^H C.
//
// Q[:, :k] = H_0 ... H_{k-1} I is formed backwards panel by panel with the
// triangular factors T accumulated by the panel kernel (H_j0..H_j0+kb-1 =
// I - V T V^H).
#include <algorithm>

#include "internal.h"

namespace mpsg {

namespace {

constexpr int PNT = 512;  // threads of the panel kernel
constexpr int PNW = PNT / 32;

template <typename T>
struct PanelArgs {
  T* W;
  int64_t ldw;
  int m, n;
  int j0, kb, nend, nb;
  int pivot;
  int gb;  // CTAs taking part in phase B
  T* F;
  double* vn1;
  double* vn2;
  int* jpvt;
  T* tau;
  T* Tp;  // this panel's T factor, column-major nb x nb
  double* red_norm;
  c128* red_w;
  double* red_argv;
  int* red_argi;
  c128* alpha_slot;
  unsigned* bar;
  int* err;
  unsigned expected;
  unsigned long long timeout_ns;
  double flag_tol;
  int xcap;  // elements of x that fit in dynamic shared memory
};

__device__ __forceinline__ bool better(double v, int i, double bv, int bi) {
  return (v > bv) || (v == bv && i < bi);
}

// Block-wide argmax of (value, index) pairs; result valid in thread 0.
__device__ void block_argmax(double& v, int& i) {
  __shared__ double sv[PNW];
  __shared__ int si[PNW];
  for (int o = 16; o > 0; o >>= 1) {
    double ov = __shfl_xor_sync(0xffffffffu, v, o);
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
  if (threadIdx.x == 0)
    for (int w = 0; w < PNW; ++w) t += s[w];
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

template <typename T>
__global__ void __launch_bounds__(PNT, 1) qr_panel_kernel(PanelArgs<T> a) {
  using R = typename real_of<T>::type;
  extern __shared__ unsigned char smem_raw[];
  T* xs = reinterpret_cast<T*>(smem_raw);
  __shared__ c128 s_w[64];        // w_i = V_i^H v
  __shared__ T s_fp[64];          // F[p, :kk] (phase B)
  __shared__ T s_vrow[64];        // W[J, j0+i], i < kk
  __shared__ double s_bv;
  __shared__ int s_bi;
  __shared__ c128 s_scal[3];  // tau, s, beta

  const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int m = a.m;
  T* W = a.W;
  const int64_t ldw = a.ldw;
  // an earlier bounded wait expired: the factorisation is void, leave at once
  if (ld_relaxed_i32(a.err) != DEV_OK) return;

  // Phase 0: partial argmax over this CTA's share of [j0, nend)
  if (a.pivot) {
    int c0, c1;
    split_range(a.j0, a.nend, G, b, c0, c1);
    double bv = -1.0;
    int bi = 0x7fffffff;
    for (int t = c0 + tid; t < c1; t += PNT) {
      double v = a.vn1[t];
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
    if (!grid_barrier(a.bar, a.expected, a.err, a.timeout_ns)) return;
  }

  c128 s_prev = mk<double>(0, 0);
  int rb0, rb1;  // phase-B row range of this CTA
  if (b < a.gb)
    split_range(0, m, a.gb, b, rb0, rb1);
  else
    rb0 = rb1 = 0;

  for (int kk = 0; kk < a.kb; ++kk) {
    const int J = a.j0 + kk;
    // ---------------- A: pivot
    int p = J;
    if (a.pivot) {
      if (tid < 32) {
        double bv = -1.0;
        int bi = 0x7fffffff;
        for (int g = lane; g < G; g += 32) {
          double v = a.red_argv[g];
          int i = a.red_argi[g];
          if (better(v, i, bv, bi)) {
            bv = v;
            bi = i;
          }
        }
        for (int o = 16; o > 0; o >>= 1) {
          double ov = __shfl_xor_sync(0xffffffffu, bv, o);
          int oi = __shfl_xor_sync(0xffffffffu, bi, o);
          if (better(ov, oi, bv, bi)) {
            bv = ov;
            bi = oi;
          }
        }
        if (lane == 0) {
          s_bv = bv;
          s_bi = bi;
        }
      }
      __syncthreads();
      p = s_bi;
      if (p < J || p >= a.nend) {  // cannot happen with finite norms
        if (tid == 0) atomicCAS(a.err, DEV_OK, DEV_ERR_NONFINITE);
        p = J;
      }
    }
    // ---------------- B: swap, column update, partial sums
    if (b < a.gb) {
      for (int i = tid; i < kk; i += PNT) s_fp[i] = a.F[(int64_t)p * a.nb + i];
      __syncthreads();
      T* colJ = W + (int64_t)J * ldw;
      T* colP = W + (int64_t)p * ldw;
      if (kk > 0) {  // deferred scaling of the previous reflector (rows > J-1)
        T* prev = W + (int64_t)(J - 1) * ldw;
        T sc = ccast<R>(s_prev);
        for (int r = max(rb0, J) + tid; r < rb1; r += PNT) prev[r] = prev[r] * sc;
      }
      if (p != J)
        for (int r = rb0 + tid; r < rb1; r += PNT) {
          T t0 = colJ[r];
          colJ[r] = colP[r];
          colP[r] = t0;
        }
      __syncthreads();
      double nrm = 0.0;
      for (int r = max(rb0, J) + tid; r < rb1; r += PNT) {
        T x = colJ[r];
        for (int i = 0; i < kk; ++i) {
          T v = W[r + (int64_t)(a.j0 + i) * ldw];
          // x -= v * conj(F[p, i])
          x = x - v * cconj(s_fp[i]);
        }
        colJ[r] = x;
        if (r > J) nrm += (double)cabs2(x);
        if (r == J) *a.alpha_slot = ccast<double>(x);
      }
      nrm = block_sum(nrm);
      if (tid == 0) a.red_norm[b] = nrm;
      __syncthreads();
      // partial w_i = sum_{r > J} conj(V[r, i]) x_r over this CTA's rows
      for (int i = warp; i < kk; i += PNW) {
        c128 acc = mk<double>(0, 0);
        const T* vc = W + (int64_t)(a.j0 + i) * ldw;
        for (int r = max(rb0, J + 1) + lane; r < rb1; r += 32) cfma_conj(acc, ccast<double>(vc[r]), ccast<double>(colJ[r]));
        acc.re = warp_sum(acc.re);
        acc.im = warp_sum(acc.im);
        if (lane == 0) a.red_w[(int64_t)b * a.nb + i] = acc;
      }
      if (b == 0 && tid == 0 && p != J) {
        int t0 = a.jpvt[J];
        a.jpvt[J] = a.jpvt[p];
        a.jpvt[p] = t0;
      }
    }
    if (!grid_barrier(a.bar, a.expected, a.err, a.timeout_ns)) return;

    // ---------------- C: reflector (every CTA, identical FP64 arithmetic)
    if (tid < 32) {
      double xn = 0.0;
      if (lane == 0)
        for (int g = 0; g < a.gb; ++g) xn += a.red_norm[g];
      if (lane == 0) {
        c128 al = *a.alpha_slot;
        c128 tau, sc, beta;
        if (xn == 0.0 && al.im == 0.0) {
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
    __syncthreads();
    const c128 tau = s_scal[0], sc = s_scal[1];
    for (int i = warp; i < kk; i += PNW) {
      c128 acc = mk<double>(0, 0);
      for (int g = lane; g < a.gb; g += 32) {
        c128 v = a.red_w[(int64_t)g * a.nb + i];
        acc.re += v.re;
        acc.im += v.im;
      }
      // fixed-order lane tree: identical in every CTA
      acc.re = warp_sum(acc.re);
      acc.im = warp_sum(acc.im);
      if (lane == 0) {
        c128 vr = ccast<double>(W[J + (int64_t)(a.j0 + i) * ldw]);
        s_w[i] = cconj(vr) + sc * acc;  // V_i^H v
      }
    }
    for (int i = tid; i < kk; i += PNT) s_vrow[i] = W[J + (int64_t)(a.j0 + i) * ldw];
    __syncthreads();
    if (b == 0 && tid == 0) {
      a.tau[J] = ccast<R>(tau);
      W[J + (int64_t)J * ldw] = ccast<R>(s_scal[2]);
      // T[0:kk, kk] = -tau T[0:kk, 0:kk] w ;  T[kk, kk] = tau
      T* Tc = a.Tp + (int64_t)kk * a.nb;
      for (int i = 0; i < kk; ++i) {
        c128 acc = mk<double>(0, 0);
        for (int j = i; j < kk; ++j) cfma(acc, ccast<double>(a.Tp[i + (int64_t)j * a.nb]), s_w[j]);
        Tc[i] = ccast<R>(mk<double>(0, 0) - tau * acc);
      }
      Tc[kk] = ccast<R>(tau);
    }

    // ---------------- D: trailing columns
    const int L = m - J - 1;  // rows below the pivot row
    const bool staged = (L <= a.xcap);
    const T* colJ = W + (int64_t)J * ldw;
    if (staged) {
      for (int r = tid; r < L; r += PNT) xs[r] = colJ[J + 1 + r];
      __syncthreads();
    }
    int c0, c1;
    split_range(J + 1, a.nend, G, b, c0, c1);
    double bv = -1.0;
    int bi = 0x7fffffff;
    for (int t = c0 + warp; t < c1; t += PNW) {
      const int src = (t == p) ? J : t;
      const T* col = W + (int64_t)t * ldw;
      // y_t = sum_{r > J} conj(W[r,t]) x_r   (accumulated in the data precision)
      T acc = mk<R>(0, 0);
      if (staged) {
        for (int r = lane; r < L; r += 32) cfma_conj(acc, col[J + 1 + r], xs[r]);
      } else {
        for (int r = lane; r < L; r += 32) cfma_conj(acc, col[J + 1 + r], colJ[J + 1 + r]);
      }
      acc.re = warp_sum(acc.re);
      acc.im = warp_sum(acc.im);
      c128 wJt = ccast<double>(col[J]);
      c128 y = cconj(wJt) + sc * ccast<double>(acc);
      // F[t, kk] = tau * (y - sum_i F[src, i] w_i)
      c128 fw = mk<double>(0, 0), rowu = mk<double>(0, 0);
      const T* Fs = a.F + (int64_t)src * a.nb;
      for (int i = lane; i < kk; i += 32) {
        c128 fi = ccast<double>(Fs[i]);
        cfma(fw, fi, s_w[i]);
        cfma(rowu, ccast<double>(s_vrow[i]), cconj(fi));
      }
      fw.re = warp_sum(fw.re);
      fw.im = warp_sum(fw.im);
      rowu.re = warp_sum(rowu.re);
      rowu.im = warp_sum(rowu.im);
      c128 f = tau * (y - fw);
      T* Ft = a.F + (int64_t)t * a.nb;
      if (t == p)
        for (int i = lane; i < kk; i += 32) Ft[i] = Fs[i];
      __syncwarp();
      c128 wnew = wJt - rowu - cconj(f);
      double v1 = 0.0, v2 = 0.0;
      int need = 0;
      if (lane == 0) {
        Ft[kk] = ccast<R>(f);
        W[J + (int64_t)t * ldw] = ccast<R>(wnew);
        if (a.pivot) {
          v1 = a.vn1[src];
          v2 = a.vn2[src];
          if (L <= 0) {
            v1 = 0.0;
          } else if (v1 != 0.0) {
            double tt = sqrt(wnew.re * wnew.re + wnew.im * wnew.im) / v1;
            tt = fmax(0.0, (1.0 + tt) * (1.0 - tt));
            double t2 = tt * (v1 / v2) * (v1 / v2);
            if (t2 <= a.flag_tol)
              need = 1;
            else
              v1 = v1 * sqrt(tt);
          }
        }
      }
      need = __shfl_sync(0xffffffffu, need, 0);
      if (need) {
        // exact norm of the column after step J: rows > J of
        // W[:, t] - V[:, 0:kk] F[t, 0:kk]^H - (s x) conj(f)
        double nr = 0.0;
        c128 cf = cconj(f);
        for (int r = J + 1 + lane; r < m; r += 32) {
          c128 z = ccast<double>(col[r]);
          for (int i = 0; i < kk; ++i) {
            c128 vv = ccast<double>(W[r + (int64_t)(a.j0 + i) * ldw]);
            z = z - vv * cconj(ccast<double>(Fs[i]));
          }
          c128 vx = sc * ccast<double>(colJ[r]);
          z = z - vx * cf;
          nr += z.re * z.re + z.im * z.im;
        }
        nr = warp_sum(nr);
        v1 = sqrt(nr);
        v2 = v1;
      }
      if (lane == 0 && a.pivot) {
        a.vn1[t] = v1;
        a.vn2[t] = v2;
        if (better(v1, t, bv, bi)) {
          bv = v1;
          bi = t;
        }
      }
    }
    if (a.pivot) {
      block_argmax(bv, bi);
      if (tid == 0) {
        a.red_argv[b] = bv;
        a.red_argi[b] = bi;
      }
    }
    s_prev = sc;
    if (!grid_barrier(a.bar, a.expected, a.err, a.timeout_ns)) return;
  }
  // final deferred scaling of the panel's last reflector
  if (b < a.gb && a.kb > 0) {
    const int Jl = a.j0 + a.kb - 1;
    T* prev = W + (int64_t)Jl * ldw;
    T sc = ccast<R>(s_prev);
    for (int r = max(rb0, Jl + 1) + tid; r < rb1; r += PNT) prev[r] = prev[r] * sc;
  }
}

// vn1[t] = vn2[t] = ||W[r0:m, t]|| for t in [c0, n): one warp per column, FP64.
template <typename T>
__global__ void col_norms_kernel(const T* W, int64_t ldw, int m, int r0, int c0, int n, double* vn1,
                                 double* vn2) {
  const int lane = threadIdx.x & 31;
  const int t = c0 + (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  if (t >= n) return;
  const T* col = W + (int64_t)t * ldw;
  double s = 0.0;
  for (int r = r0 + lane; r < m; r += 32) s += (double)cabs2(col[r]);
  s = warp_sum(s);
  if (lane == 0) {
    double v = sqrt(s);
    vn1[t] = v;
    vn2[t] = v;
  }
}

// discarded = sum_{t in [c0, n)} vn1[t]^2, one block, fixed order
__global__ void discarded_kernel(const double* vn1, int c0, int n, double* out, double* total) {
  __shared__ double s[256];
  double acc = 0.0;
  for (int t = c0 + threadIdx.x; t < n; t += 256) acc += vn1[t] * vn1[t];
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

int g_sms = 0;

}  // namespace

int num_sms() {
  if (g_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_sms <= 0) g_sms = 1;
  }
  return g_sms;
}

template <typename T>
static int panel_xcap() {
  return (200 * 1024) / (int)sizeof(T);
}

template <typename T>
static cudaError_t panel_setup(int& max_blocks) {
  static int cached = -1;
  if (cached < 0) {
    int smem = panel_xcap<T>() * (int)sizeof(T);
    cudaError_t e = cudaFuncSetAttribute(qr_panel_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, qr_panel_kernel<T>, PNT, smem);
    if (e != cudaSuccess) return e;
    cached = per_sm * num_sms();
    if (cached < 1) return cudaErrorInvalidConfiguration;
  }
  max_blocks = cached;
  return cudaSuccess;
}

#define CK(x)                                  \
  do {                                         \
    cudaError_t e_ = (x);                      \
    if (e_ != cudaSuccess) return e_;          \
  } while (0)

template <typename T>
cudaError_t qr_factor(const QrPlan<T>& p, cudaStream_t s, LaunchHooks* hooks) {
  using R = typename real_of<T>::type;
  const int m = p.m, n = p.n, k = p.k, nb = p.nb;
  if (k <= 0) {
    if (p.pivot && p.discarded) {
      // nothing factored: discarded = ||W||_F^2
      hook_before(hooks, MPS_KCLASS_NORMS, (double)m * n * sizeof(T), 0);
      int threads = 256, warps = threads / 32;
      if (n > 0) {
        col_norms_kernel<T><<<(n + warps - 1) / warps, threads, 0, s>>>(p.W, p.ldw, m, 0, 0, n, p.vn1, p.vn2);
        CK(cudaGetLastError());
      }
      discarded_kernel<<<1, 256, 0, s>>>(p.vn1, 0, n, p.discarded, p.disc_total);
      CK(cudaGetLastError());
      hook_after(hooks, MPS_KCLASS_NORMS, n > 0 ? 2 : 1);
    }
    return cudaSuccess;
  }
  int maxb = 1;
  CK(panel_setup<T>(maxb));
  const int gcap = std::max(1, std::min(p.G > 0 ? p.G : maxb, maxb));
  const int npanels = (k + nb - 1) / nb;
  CK(cudaMemsetAsync(p.Tfac, 0, sizeof(T) * (size_t)npanels * nb * nb, s));
  hook_before(hooks, MPS_KCLASS_OTHER, 4.0 * n, 0);
  iota_kernel<<<(n + 255) / 256, 256, 0, s>>>(p.jpvt, n);
  CK(cudaGetLastError());
  hook_after(hooks, MPS_KCLASS_OTHER, 1);
  if (p.pivot) {
    hook_before(hooks, MPS_KCLASS_NORMS, (double)m * n * sizeof(T), 3.0 * m * n);
    int warps = 8;
    col_norms_kernel<T><<<(n + warps - 1) / warps, warps * 32, 0, s>>>(p.W, p.ldw, m, 0, 0, n, p.vn1, p.vn2);
    CK(cudaGetLastError());
    hook_after(hooks, MPS_KCLASS_NORMS, 1);
  }
  const int smem = panel_xcap<T>() * (int)sizeof(T);
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
    a.red_norm = p.red_norm;
    a.red_w = p.red_w;
    a.red_argv = p.red_argv;
    a.red_argi = p.red_argi;
    a.alpha_slot = p.alpha_slot;
    a.bar = p.bar;
    a.err = p.err;
    a.timeout_ns = p.timeout_ns;
    a.flag_tol = p.flag_tol;
    a.xcap = panel_xcap<T>();
    const int ncols = a.nend - j0;
    int G = std::max(1, std::min(gcap, (ncols + 7) / 8));
    a.gb = std::max(1, std::min(G, (m - j0 + 255) / 256));
    a.expected = (unsigned)G + p.barrier_extra;
    // algorithmic bytes: per step one read of the trailing block rows J..m
    double bytes = 0.0, flops = 0.0;
    for (int j = j0; j < J1; ++j) {
      double rows = (double)(m - j), cols = (double)(a.nend - j);
      bytes += rows * cols * sizeof(T);
      flops += 8.0 * rows * cols;
    }
    void* args[] = {&a};
    hook_before(hooks, MPS_KCLASS_PANEL, bytes, flops);
    CK(cudaLaunchCooperativeKernel((const void*)qr_panel_kernel<T>, dim3(G), dim3(PNT), args, (size_t)smem, s));
    hook_after(hooks, MPS_KCLASS_PANEL, 1);
    if (p.pivot) {
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
        d.B = p.F + (int64_t)J1 * nb;  // B(k, j) = conj(F[J1 + j, k]) -> stored col-major, ld nb
        d.ldb = nb;
        d.b_row = 0;
        d.b_conj = 1;
        d.b_mask = MASK_NONE;
        d.C = p.W + J1 + (int64_t)J1 * p.ldw;
        d.ldc = p.ldw;
        double M = d.M, N = d.N;
        hook_before(hooks, MPS_KCLASS_UPDATE, (2.0 * M * N + (M + N) * kb) * sizeof(T), 8.0 * M * N * kb);
        CK(gemm_simt<T>(d, s));
        hook_after(hooks, MPS_KCLASS_UPDATE, 1);
      }
      if (J1 < n) {
        hook_before(hooks, MPS_KCLASS_NORMS, (double)std::max(0, m - J1) * (n - J1) * sizeof(T),
                    3.0 * std::max(0, m - J1) * (n - J1));
        int warps = 8;
        col_norms_kernel<T><<<(n - J1 + warps - 1) / warps, warps * 32, 0, s>>>(p.W, p.ldw, m, J1, J1, n, p.vn1,
                                                                               p.vn2);
        CK(cudaGetLastError());
        hook_after(hooks, MPS_KCLASS_NORMS, 1);
      }
    } else if (J1 < n) {
      // C = W[j0:m, J1:n] <- (I - V T V^H)^H C = C - V T^H (V^H C)
      const int M = m - j0, N = n - J1;
      GemmDesc<T> d;
      d.M = kb;
      d.N = N;
      d.K = M;
      d.alpha = mk<R>(1, 0);
      d.beta = mk<R>(0, 0);
      d.A = p.W + j0 + (int64_t)j0 * p.ldw;  // V^H
      d.lda = p.ldw;
      d.a_row = 1;
      d.a_conj = 1;
      d.a_mask = MASK_UNIT_LOWER;
      d.B = p.W + j0 + (int64_t)J1 * p.ldw;
      d.ldb = p.ldw;
      d.b_row = 0;
      d.b_conj = 0;
      d.b_mask = MASK_NONE;
      d.C = p.Y;
      d.ldc = nb;
      hook_before(hooks, MPS_KCLASS_UPDATE, ((double)M * N + (double)M * kb) * sizeof(T), 8.0 * M * N * kb);
      CK(gemm_simt<T>(d, s));
      d.M = kb;
      d.N = N;
      d.K = kb;
      d.A = a.Tp;  // T^H
      d.lda = nb;
      d.a_row = 1;
      d.a_conj = 1;
      d.a_mask = MASK_NONE;
      d.B = p.Y;
      d.ldb = nb;
      d.C = p.Z;
      d.ldc = nb;
      CK(gemm_simt<T>(d, s));
      d.M = M;
      d.N = N;
      d.K = kb;
      d.alpha = mk<R>(-1, 0);
      d.beta = mk<R>(1, 0);
      d.A = p.W + j0 + (int64_t)j0 * p.ldw;  // V
      d.lda = p.ldw;
      d.a_row = 0;
      d.a_conj = 0;
      d.a_mask = MASK_UNIT_LOWER;
      d.B = p.Z;
      d.ldb = nb;
      d.C = p.W + j0 + (int64_t)J1 * p.ldw;
      d.ldc = p.ldw;
      CK(gemm_simt<T>(d, s));
      hook_after(hooks, MPS_KCLASS_UPDATE, 3);
    }
  }
  if (p.pivot && p.discarded) {
    hook_before(hooks, MPS_KCLASS_NORMS, 8.0 * (n - k), 0);
    discarded_kernel<<<1, 256, 0, s>>>(p.vn1, k, n, p.discarded, p.disc_total);
    CK(cudaGetLastError());
    hook_after(hooks, MPS_KCLASS_NORMS, 1);
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t qr_form_q(const QrPlan<T>& p, T* Q, int64_t ldq, cudaStream_t s, LaunchHooks* hooks) {
  using R = typename real_of<T>::type;
  const int m = p.m, k = p.k, nb = p.nb;
  if (k <= 0) return cudaSuccess;
  hook_before(hooks, MPS_KCLASS_FORMQ, (double)m * k * sizeof(T), 0);
  CK(set_identity<T>(Q, ldq, m, k, s));
  hook_after(hooks, MPS_KCLASS_FORMQ, 1);
  const int npanels = (k + nb - 1) / nb;
  for (int pi = npanels - 1; pi >= 0; --pi) {
    const int j0 = pi * nb;
    const int kb = std::min(nb, k - j0);
    const int M = m - j0, N = k - j0;
    const T* Tp = p.Tfac + (size_t)pi * nb * nb;
    GemmDesc<T> d;
    // Y = V^H Q[j0:m, j0:k]
    d.M = kb;
    d.N = N;
    d.K = M;
    d.alpha = mk<R>(1, 0);
    d.beta = mk<R>(0, 0);
    d.A = p.W + j0 + (int64_t)j0 * p.ldw;
    d.lda = p.ldw;
    d.a_row = 1;
    d.a_conj = 1;
    d.a_mask = MASK_UNIT_LOWER;
    d.B = Q + j0 + (int64_t)j0 * ldq;
    d.ldb = ldq;
    d.b_row = 0;
    d.b_conj = 0;
    d.b_mask = MASK_NONE;
    d.C = p.Y;
    d.ldc = nb;
    hook_before(hooks, MPS_KCLASS_FORMQ, (2.0 * M * N + 2.0 * M * kb) * sizeof(T), 16.0 * M * N * kb);
    CK(gemm_simt<T>(d, s));
    // Z = T Y
    d.M = kb;
    d.N = N;
    d.K = kb;
    d.A = Tp;
    d.lda = nb;
    d.a_row = 0;
    d.a_conj = 0;
    d.a_mask = MASK_NONE;
    d.B = p.Y;
    d.ldb = nb;
    d.C = p.Z;
    d.ldc = nb;
    CK(gemm_simt<T>(d, s));
    // Q[j0:m, j0:k] -= V Z
    d.M = M;
    d.N = N;
    d.K = kb;
    d.alpha = mk<R>(-1, 0);
    d.beta = mk<R>(1, 0);
    d.A = p.W + j0 + (int64_t)j0 * p.ldw;
    d.lda = p.ldw;
    d.a_row = 0;
    d.a_conj = 0;
    d.a_mask = MASK_UNIT_LOWER;
    d.B = p.Z;
    d.ldb = nb;
    d.C = Q + j0 + (int64_t)j0 * ldq;
    d.ldc = ldq;
    CK(gemm_simt<T>(d, s));
    hook_after(hooks, MPS_KCLASS_FORMQ, 3);
  }
  return cudaSuccess;
}

template cudaError_t qr_factor<c64>(const QrPlan<c64>&, cudaStream_t, LaunchHooks*);
template cudaError_t qr_factor<c128>(const QrPlan<c128>&, cudaStream_t, LaunchHooks*);
template cudaError_t qr_form_q<c64>(const QrPlan<c64>&, c64*, int64_t, cudaStream_t, LaunchHooks*);
template cudaError_t qr_form_q<c128>(const QrPlan<c128>&, c128*, int64_t, cudaStream_t, LaunchHooks*);

}  // namespace mpsg
