// Two-site gates whose theta fits one CTA (Sec. III-C.2 with the split of
// Sec. III-B.2), for the bonds near the ends of a chain, where a gate is a few
// microseconds of arithmetic and the multi-kernel pipeline would be bound by its
// launches and grid barriers.  One CTA does the whole gate in shared memory:
//
//   1. X = A B (the bond contraction), theta = the gate contracted into X's
//      physical indices, theta as the (2 chi_l) x (2 chi_r) matrix with row (l, a)
//      and column (b, r);
//   2. k = min(m, n, chi_max) steps of column-pivoted Householder QR: exact FP64
//      squared norms of the remaining columns every step, the largest taken (the
//      lowest index on ties), beta = -sign(Re alpha) ||x||, tau = (beta - alpha) /
//      beta, v = (1, x_1.. / (alpha - beta)) with FP64 scalars, H^H applied to the
//      columns to the right; the identity reflector for a column without a tail
//      or one whose squared norm is below the smallest normal number (as the grid
//      kernels);
//   3. the discarded weight ||theta[k:, k:]||_F^2 in FP64;
//   4. Q[:, :k] = H_0 ... H_{k-1} I, then the left site Q and the right site R P^T.
//
// A layer's small gates run as one grouped launch (one CTA per gate, the gates
// passed by value); a single gate is the same launch with one item, so a layer
// gives the one-by-one result bit for bit.
#include "internal.h"

namespace mpsg {

namespace {

constexpr int SNT = 256;        // threads per CTA
constexpr int SNW = SNT / 32;
constexpr int LD = kSmallDim;   // leading dimension of theta and Q in shared memory

// squared column norm below which the reflector is the identity: FLT_MIN^2 for
// complex64, DBL_MIN for complex128 (rounding residue whose squares underflow)
template <typename T>
__device__ __forceinline__ double small_zero_level() {
  return sizeof(T) == 8 ? 1.3814317e-76 : 2.2250738585072014e-308;
}

template <typename T>
__global__ void __launch_bounds__(SNT) small_gate_kernel(const __grid_constant__ SmallBatch<T> batch) {
  using R = typename real_of<T>::type;
  const SmallGate<T>& G = batch.item[blockIdx.x];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* th = reinterpret_cast<T*>(smem_raw);  // m x n, column-major, ld LD
  T* Qs = th + LD * LD;                    // X, then Q (m x k), column-major, ld LD
  __shared__ double s_norm[kSmallDim];
  __shared__ T s_tau[kSmallDim];
  __shared__ int s_piv[kSmallDim];
  __shared__ T s_g[16];
  __shared__ int s_p;
  __shared__ c128 s_sc, s_beta, s_taud;
  __shared__ double s_disc[SNW];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int cl = G.cl, cm = G.cm, cr = G.cr, k = G.k;
  const int m = 2 * cl, n = 2 * cr;
  if (tid < 16) s_g[tid] = G.gdev ? G.gdev[tid] : G.g[tid];
  // 1. X = A B (m x n), then theta with the gate epilogue
  for (int e = tid; e < m * n; e += SNT) {
    const int i = e % m, j = e / m;
    const T* a = G.A + (int64_t)i * cm;
    const T* b = G.B + j;
    T acc = mk<R>(0, 0);
    for (int mu = 0; mu < cm; ++mu) cfma(acc, a[mu], b[(int64_t)mu * n]);
    Qs[i + j * LD] = acc;
  }
  for (int t = tid; t < n; t += SNT) s_piv[t] = t;
  __syncthreads();
  for (int e = tid; e < m * n; e += SNT) {
    const int row = e % m, col = e / m;
    const int l = row >> 1, a = row & 1, b = col / cr, r = col - b * cr;
    T acc = mk<R>(0, 0);
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int d = 0; d < 2; ++d) cfma(acc, s_g[(2 * a + b) * 4 + 2 * c + d], Qs[(2 * l + c) + (d * cr + r) * LD]);
    th[row + col * LD] = acc;
  }
  __syncthreads();

  // 2. k pivoted Householder steps
  for (int j = 0; j < k; ++j) {
    // exact squared norms of the remaining columns (rows j..m-1), one warp per column
    for (int t = j + warp; t < n; t += SNW) {
      double s = 0.0;
      for (int r = j + lane; r < m; r += 32) {
        const T x = th[r + t * LD];
        s += (double)x.re * (double)x.re + (double)x.im * (double)x.im;
      }
      s = warp_sum(s);
      if (lane == 0) s_norm[t] = s;
    }
    __syncthreads();
    // argmax, the lowest index on ties
    if (warp == 0) {
      double bv = -1.0;
      int bi = n;
      for (int t = j + lane; t < n; t += 32)
        if (s_norm[t] > bv) {  // ascending t per lane: the first maximum is kept
          bv = s_norm[t];
          bi = t;
        }
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) {
          bv = ov;
          bi = oi;
        }
      }
      if (lane == 0) s_p = bi < n ? bi : j;
    }
    __syncthreads();
    const int p = s_p;
    if (p != j) {
      for (int r = tid; r < m; r += SNT) {
        const T x = th[r + j * LD];
        th[r + j * LD] = th[r + p * LD];
        th[r + p * LD] = x;
      }
      if (tid == 0) {
        const int x = s_piv[j];
        s_piv[j] = s_piv[p];
        s_piv[p] = x;
      }
      __syncthreads();
    }
    // reflector scalars in FP64 (warp 0)
    if (warp == 0) {
      double tail = 0.0;
      for (int r = j + 1 + lane; r < m; r += 32) {
        const T x = th[r + j * LD];
        tail += (double)x.re * (double)x.re + (double)x.im * (double)x.im;
      }
      tail = warp_sum(tail);
      if (lane == 0) {
        const c128 al = ccast<double>(th[j + j * LD]);
        c128 tau, sc, beta;
        if ((tail == 0.0 && al.im == 0.0) || al.re * al.re + al.im * al.im + tail < small_zero_level<T>()) {
          tau = mk<double>(0, 0);
          sc = mk<double>(0, 0);
          beta = al;
        } else {
          const double nrm = sqrt(al.re * al.re + al.im * al.im + tail);
          const double bt = al.re >= 0.0 ? -nrm : nrm;
          tau = mk<double>((bt - al.re) / bt, -al.im / bt);
          const c128 dnm = mk<double>(al.re - bt, al.im);
          const double dd = dnm.re * dnm.re + dnm.im * dnm.im;
          sc = mk<double>(dnm.re / dd, -dnm.im / dd);
          beta = mk<double>(bt, 0.0);
        }
        s_taud = tau;
        s_sc = sc;
        s_beta = beta;
        s_tau[j] = ccast<R>(tau);
      }
    }
    __syncthreads();
    const T sc = ccast<R>(s_sc);
    for (int r = j + 1 + tid; r < m; r += SNT) th[r + j * LD] = th[r + j * LD] * sc;  // v below the diagonal
    __syncthreads();
    const T ctau = cconj(ccast<R>(s_taud));
    if (!(s_taud.re == 0.0 && s_taud.im == 0.0)) {
      // H^H = I - conj(tau) v v^H on the columns right of j, one warp per column
      for (int t = j + 1 + warp; t < n; t += SNW) {
        const T top = th[j + t * LD];  // read by every lane before lane 0 rewrites it
        T d = mk<R>(0, 0);
        for (int r = j + 1 + lane; r < m; r += 32) cfma_conj(d, th[r + j * LD], th[r + t * LD]);
        d.re = warp_sum(d.re);
        d.im = warp_sum(d.im);
        d = d + top;
        const T f = ctau * d;
        __syncwarp();
        if (lane == 0) th[j + t * LD] = top - f;
        for (int r = j + 1 + lane; r < m; r += 32) th[r + t * LD] = th[r + t * LD] - th[r + j * LD] * f;
      }
    }
    __syncthreads();
    if (tid == 0) th[j + j * LD] = ccast<R>(s_beta);  // R_jj
    __syncthreads();
  }

  // 3. discarded weight ||theta[k:, k:]||_F^2
  double dsum = 0.0;
  for (int t = k + warp; t < n; t += SNW)
    for (int r = k + lane; r < m; r += 32) {
      const T x = th[r + t * LD];
      dsum += (double)x.re * (double)x.re + (double)x.im * (double)x.im;
    }
  dsum = warp_sum(dsum);
  if (lane == 0) s_disc[warp] = dsum;
  // 4. Q[:, :k] = H_0 ... H_{k-1} I, backwards
  for (int e = tid; e < m * k; e += SNT) {
    const int r = e % m, t = e / m;
    Qs[r + t * LD] = mk<R>(r == t ? 1 : 0, 0);
  }
  __syncthreads();
  if (tid == 0) {
    double tot = 0.0;
    for (int w = 0; w < SNW; ++w) tot += s_disc[w];
    *G.disc = tot;
    if (G.disc_total) *G.disc_total += tot;
  }
  for (int j = k - 1; j >= 0; --j) {
    const T tau = s_tau[j];
    if (!(tau.re == 0 && tau.im == 0)) {
      for (int t = j + warp; t < k; t += SNW) {
        const T top = Qs[j + t * LD];
        T d = mk<R>(0, 0);
        for (int r = j + 1 + lane; r < m; r += 32) cfma_conj(d, th[r + j * LD], Qs[r + t * LD]);
        d.re = warp_sum(d.re);
        d.im = warp_sum(d.im);
        d = d + top;
        const T f = tau * d;
        __syncwarp();
        if (lane == 0) Qs[j + t * LD] = top - f;
        for (int r = j + 1 + lane; r < m; r += 32) Qs[r + t * LD] = Qs[r + t * LD] - th[r + j * LD] * f;
      }
    }
    __syncthreads();
  }
  // 5. left site (row-major m x k) = Q, right site (row-major k x n) = R P^T
  for (int e = tid; e < m * k; e += SNT) {
    const int row = e / k, t = e - row * k;
    G.Aout[e] = Qs[row + t * LD];
  }
  for (int e = tid; e < k * n; e += SNT) {
    const int t = e / n, c = e - t * n;
    G.Bout[(int64_t)t * n + s_piv[c]] = t <= c ? th[t + c * LD] : mk<R>(0, 0);
  }
  if (G.jpvt_out)
    for (int t = tid; t < n; t += SNT) G.jpvt_out[t] = s_piv[t];
}

template <typename T>
constexpr int small_smem() {
  return 2 * LD * LD * (int)sizeof(T);
}

}  // namespace

bool small_gate_fits(int cl, int cm, int cr) {
  return 2 * cl <= kSmallDim && 2 * cr <= kSmallDim && cm >= 1 && cm <= kSmallMaxCm;
}

template <typename T>
cudaError_t small_gate_launch(const SmallBatch<T>& b, cudaStream_t s) {
  if (b.count <= 0) return cudaSuccess;
  if (b.count > kSmallBatch) return cudaErrorInvalidValue;
  static PerDevice once;
  cudaError_t attr = cudaSuccess;
  once.get([&attr]() -> long long {
    attr = cudaFuncSetAttribute(small_gate_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, small_smem<T>());
    return attr == cudaSuccess ? 1 : -1;
  });
  if (attr != cudaSuccess) return attr;
  small_gate_kernel<T><<<b.count, SNT, small_smem<T>(), s>>>(b);
  return cudaGetLastError();
}

template cudaError_t small_gate_launch<c64>(const SmallBatch<c64>&, cudaStream_t);
template cudaError_t small_gate_launch<c128>(const SmallBatch<c128>&, cudaStream_t);

}  // namespace mpsg
