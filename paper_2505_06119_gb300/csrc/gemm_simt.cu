// Complex GEMMs on the CUDA cores: the generic GEMM used by the block-reflector
// updates, centre moves and contractions, and the theta contraction with its
// fused gate epilogue (Sec. III-B.1 bond contraction, Sec. III-C.2 tensor
// application).  The kernels here serve complex128 (FP64 DFMA); complex64
// products go to the wider-tile kernels of gemm_c64.cu.
#include <algorithm>
#include <type_traits>

#include "internal.h"

namespace mpsg {

namespace {

constexpr int BM = 64, BN = 64, BK = 8, NT = 256;

template <typename T>
__device__ __forceinline__ T load_a(const GemmDesc<T>& d, int i, int k, int kend) {
  using R = typename real_of<T>::type;
  if (i >= d.M || k >= kend) return mk<R>(0, 0);
  int r = d.a_row ? k : i, c = d.a_row ? i : k;
  if (d.a_mask == MASK_UNIT_LOWER) {
    if (r < c) return mk<R>(0, 0);
    if (r == c) return mk<R>(1, 0);
  } else if (d.a_mask == MASK_UPPER) {
    if (r > c) return mk<R>(0, 0);
  }
  T v = d.a_row ? d.A[(int64_t)i * d.lda + k] : d.A[i + (int64_t)k * d.lda];
  return d.a_conj ? cconj(v) : v;
}

template <typename T>
__device__ __forceinline__ T load_b(const GemmDesc<T>& d, int k, int j, int kend) {
  using R = typename real_of<T>::type;
  if (k >= kend || j >= d.N) return mk<R>(0, 0);
  int r = d.b_row ? j : k, c = d.b_row ? k : j;
  if (d.b_mask == MASK_UNIT_LOWER) {
    if (r < c) return mk<R>(0, 0);
    if (r == c) return mk<R>(1, 0);
  } else if (d.b_mask == MASK_UPPER) {
    if (r > c) return mk<R>(0, 0);
  }
  T v = d.b_row ? d.B[(int64_t)k * d.ldb + j] : d.B[k + (int64_t)j * d.ldb];
  return d.b_conj ? cconj(v) : v;
}

// One CTA computes a 64 x 64 tile of C; each thread a 4 x 4 micro-tile.
// Tiles of A and B are staged through shared memory with a register
// prefetch of the next K-slice; the global load pattern follows whichever
// index is contiguous in memory.
template <typename T>
__global__ void __launch_bounds__(NT) gemm_simt_kernel(GemmDesc<T> d) {
  using R = typename real_of<T>::type;
  __shared__ T As[2][BK][BM];
  __shared__ T Bs[2][BK][BN];
  const int tid = threadIdx.x;
  const int i0 = blockIdx.x * BM, j0 = blockIdx.y * BN;
  // split-K: this CTA covers K-slice blockIdx.z (whole multiples of BK)
  int kbeg = 0, kend = d.K;
  if (d.splitk > 1) {
    int per = ((d.K + d.splitk - 1) / d.splitk + BK - 1) / BK * BK;
    kbeg = blockIdx.z * per;
    kend = min(d.K, kbeg + per);
  }
  const int tm = tid % 16, tn = tid / 16;

  // global->smem mapping (2 elements of A and 2 of B per thread per slice)
  int ai[2], ak[2], bk[2], bj[2];
  for (int e = 0; e < 2; ++e) {
    int t = tid + e * NT;  // 0..511
    if (d.a_row) {         // contiguous along k
      ai[e] = t / BK;
      ak[e] = t % BK;
    } else {  // contiguous along i
      ai[e] = t % BM;
      ak[e] = t / BM;
    }
    if (d.b_row) {  // contiguous along j
      bj[e] = t % BN;
      bk[e] = t / BN;
    } else {
      bj[e] = t / BK;
      bk[e] = t % BK;
    }
  }

  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = mk<R>(0, 0);

  T ra[2], rb[2];
  const int nslices = kend > kbeg ? (kend - kbeg + BK - 1) / BK : 0;
  for (int e = 0; e < 2; ++e) {
    ra[e] = load_a(d, i0 + ai[e], kbeg + ak[e], kend);
    rb[e] = load_b(d, kbeg + bk[e], j0 + bj[e], kend);
  }
  for (int e = 0; e < 2; ++e) {
    As[0][ak[e]][ai[e]] = ra[e];
    Bs[0][bk[e]][bj[e]] = rb[e];
  }
  __syncthreads();
  for (int s = 0; s < nslices; ++s) {
    const int buf = s & 1;
    if (s + 1 < nslices) {
      const int kb = kbeg + (s + 1) * BK;
      for (int e = 0; e < 2; ++e) {
        ra[e] = load_a(d, i0 + ai[e], kb + ak[e], kend);
        rb[e] = load_b(d, kb + bk[e], j0 + bj[e], kend);
      }
    }
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[buf][kk][tm * 4 + a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[buf][kk][tn * 4 + b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) cfma(acc[a][b], av[a], bv[b]);
    }
    if (s + 1 < nslices) {
      for (int e = 0; e < 2; ++e) {
        As[buf ^ 1][ak[e]][ai[e]] = ra[e];
        Bs[buf ^ 1][bk[e]][bj[e]] = rb[e];
      }
    }
    __syncthreads();
  }
  if (d.splitk > 1) {
    T* P = d.wk + (int64_t)blockIdx.z * d.M * d.N;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int j = j0 + tn * 4 + b;
      if (j >= d.N) continue;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        int i = i0 + tm * 4 + a;
        if (i < d.M) P[i + (int64_t)j * d.M] = acc[a][b];
      }
    }
    return;
  }
  const bool beta_zero = (d.beta.re == (R)0 && d.beta.im == (R)0);
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    int j = j0 + tn * 4 + b;
    if (j >= d.N) continue;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      int i = i0 + tm * 4 + a;
      if (i >= d.M) continue;
      T* c = d.C + i + (int64_t)j * d.ldc;
      T v = d.alpha * acc[a][b];
      if (!beta_zero) v = v + d.beta * (*c);
      *c = v;
    }
  }
}

// C = alpha * sum_z P[z] + beta * C, summed in z order
template <typename T>
__global__ void splitk_reduce_kernel(GemmDesc<T> d) {
  using R = typename real_of<T>::type;
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t total = (int64_t)d.M * d.N;
  if (idx >= total) return;
  int64_t i = idx % d.M, j = idx / d.M;
  T acc = d.wk[idx];
  for (int z = 1; z < d.splitk; ++z) acc = acc + d.wk[(int64_t)z * total + idx];
  T* c = d.C + i + j * d.ldc;
  T v = d.alpha * acc;
  if (!(d.beta.re == (R)0 && d.beta.im == (R)0)) v = v + d.beta * (*c);
  *c = v;
}

// theta tile: 32 values of l (64 rows of A) x 32 values of r (both halves d=0,1).
constexpr int TL = 32, TR = 32;

template <typename T>
struct ThetaArgs {
  int cl, cm, cr;
  const T* A;
  const T* B;
  T g[16];
  const T* gdev;  // the gate in device memory instead (layers replayed as CUDA graphs); NULL: g
  T* W;
  int64_t ldw;
};

template <typename T>
__global__ void __launch_bounds__(NT) theta_kernel(ThetaArgs<T> p) {
  using R = typename real_of<T>::type;
  __shared__ T As[2][BK][2 * TL];  // index 2*(l-l0)+c
  __shared__ T Bs[2][BK][2 * TR];  // index d*TR + (r-r0)
  const int tid = threadIdx.x;
  const int l0 = blockIdx.x * TL, r0 = blockIdx.y * TR;
  const int tl = tid % 16, tr = tid / 16;
  const int m = 2 * p.cl, n = 2 * p.cr;
  const int64_t lda = p.cm, ldb = n;

  // A tile: rows 2*l0 .. 2*l0+63 (row-major, contiguous along mu)
  int arow[2], ak[2], bk[2], bcol[2];
  for (int e = 0; e < 2; ++e) {
    int t = tid + e * NT;
    arow[e] = t / BK;  // 0..63
    ak[e] = t % BK;
    bcol[e] = t % (2 * TR);  // 0..63 -> (d, r)
    bk[e] = t / (2 * TR);    // 0..7
  }
  auto ldA = [&](int e, int k) -> T {
    int row = 2 * l0 + arow[e];
    if (row >= m || k >= p.cm) return mk<R>(0, 0);
    return p.A[(int64_t)row * lda + k];
  };
  auto ldB = [&](int e, int k) -> T {
    int dd = bcol[e] / TR, r = r0 + bcol[e] % TR;
    if (r >= p.cr || k >= p.cm) return mk<R>(0, 0);
    return p.B[(int64_t)k * ldb + dd * p.cr + r];
  };

  T acc[2][2][2][2];  // [li][ri][c][d]
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int dd = 0; dd < 2; ++dd) acc[a][b][c][dd] = mk<R>(0, 0);

  T ra[2], rb[2];
  const int nslices = (p.cm + BK - 1) / BK;
  for (int e = 0; e < 2; ++e) {
    ra[e] = ldA(e, ak[e]);
    rb[e] = ldB(e, bk[e]);
  }
  for (int e = 0; e < 2; ++e) {
    As[0][ak[e]][arow[e]] = ra[e];
    Bs[0][bk[e]][bcol[e]] = rb[e];
  }
  __syncthreads();
  for (int s = 0; s < nslices; ++s) {
    const int buf = s & 1;
    if (s + 1 < nslices) {
      const int kb = (s + 1) * BK;
      for (int e = 0; e < 2; ++e) {
        ra[e] = ldA(e, kb + ak[e]);
        rb[e] = ldB(e, kb + bk[e]);
      }
    }
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T av[2][2], bv[2][2];
#pragma unroll
      for (int li = 0; li < 2; ++li)
#pragma unroll
        for (int c = 0; c < 2; ++c) av[li][c] = As[buf][kk][2 * (tl + 16 * li) + c];
#pragma unroll
      for (int ri = 0; ri < 2; ++ri)
#pragma unroll
        for (int dd = 0; dd < 2; ++dd) bv[ri][dd] = Bs[buf][kk][dd * TR + tr + 16 * ri];
#pragma unroll
      for (int li = 0; li < 2; ++li)
#pragma unroll
        for (int ri = 0; ri < 2; ++ri)
#pragma unroll
          for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int dd = 0; dd < 2; ++dd) cfma(acc[li][ri][c][dd], av[li][c], bv[ri][dd]);
    }
    if (s + 1 < nslices) {
      for (int e = 0; e < 2; ++e) {
        As[buf ^ 1][ak[e]][arow[e]] = ra[e];
        Bs[buf ^ 1][bk[e]][bcol[e]] = rb[e];
      }
    }
    __syncthreads();
  }
  // gate epilogue: theta[l,a,b,r] = sum_{c,d} g[2a+b][2c+d] X[l,c,d,r]
#pragma unroll
  for (int li = 0; li < 2; ++li) {
    int l = l0 + tl + 16 * li;
    if (l >= p.cl) continue;
#pragma unroll
    for (int ri = 0; ri < 2; ++ri) {
      int r = r0 + tr + 16 * ri;
      if (r >= p.cr) continue;
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          T v = mk<R>(0, 0);
#pragma unroll
          for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int dd = 0; dd < 2; ++dd) {
              const int gi = (2 * a + b) * 4 + 2 * c + dd;
              cfma(v, p.gdev ? p.gdev[gi] : p.g[gi], acc[li][ri][c][dd]);
            }
          p.W[(int64_t)(b * p.cr + r) * p.ldw + 2 * l + a] = v;
        }
    }
  }
}

}  // namespace

int choose_splitk(int M, int N, int K, int64_t cap_elems, int elem_bytes) {
  const int bm = elem_bytes == 8 ? gemm_c64_tile_rows(M, K) : BM, bn = elem_bytes == 8 ? 128 : BN;
  const int64_t tiles = (int64_t)((M + bm - 1) / bm) * ((N + bn - 1) / bn);
  const int64_t want = (2 * 152 + tiles - 1) / tiles;
  const int64_t by_k = K / 64;
  const int64_t by_cap = cap_elems / std::max<int64_t>(1, (int64_t)M * N);
  const int64_t s = std::min(std::min(want, by_k), std::min<int64_t>(by_cap, 256));
  return s < 1 ? 1 : (int)s;
}

template <typename T>
cudaError_t gemm_simt(const GemmDesc<T>& d, cudaStream_t s) {
  if (d.M <= 0 || d.N <= 0) return cudaSuccess;
  const int sk = (d.splitk > 1 && d.wk) ? d.splitk : 1;
  GemmDesc<T> dd = d;
  dd.splitk = sk;
  cudaError_t e;
  if constexpr (std::is_same<T, c64>::value) {
    e = gemm_c64(dd, s);
  } else {
    dim3 grid((d.M + BM - 1) / BM, (d.N + BN - 1) / BN, sk);
    if (grid.y > 65535) return cudaErrorInvalidConfiguration;
    gemm_simt_kernel<T><<<grid, NT, 0, s>>>(dd);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess || sk == 1) return e;
  int64_t total = (int64_t)d.M * d.N;
  splitk_reduce_kernel<T><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(dd);
  return cudaGetLastError();
}

template <typename T>
cudaError_t theta_gemm_simt(int chi_l, int chi_m, int chi_r, const T* A, const T* B, const T* g16,
                            T* W, int64_t ldw, cudaStream_t s, const T* gdev) {
  if constexpr (std::is_same<T, c64>::value) {
    return theta_c64(chi_l, chi_m, chi_r, A, B, g16, W, ldw, s, gdev);
  } else {
    ThetaArgs<T> p;
    p.cl = chi_l;
    p.cm = chi_m;
    p.cr = chi_r;
    p.A = A;
    p.B = B;
    for (int i = 0; i < 16; ++i) p.g[i] = g16[i];
    p.gdev = gdev;
    p.W = W;
    p.ldw = ldw;
    dim3 grid((chi_l + TL - 1) / TL, (chi_r + TR - 1) / TR);
    if (grid.y > 65535) return cudaErrorInvalidConfiguration;
    theta_kernel<T><<<grid, NT, 0, s>>>(p);
    return cudaGetLastError();
  }
}

template <typename T>
cudaError_t gemm_auto(const GemmDesc<T>& d, bool use_tc, int* err, unsigned long long timeout_ns, cudaStream_t s) {
  if constexpr (std::is_same<T, c64>::value) {
    if (use_tc && tc_gemm_applicable(d)) return tc_gemm(d, err, timeout_ns, s);
  }
  return gemm_simt<T>(d, s);
}

template cudaError_t gemm_auto<c64>(const GemmDesc<c64>&, bool, int*, unsigned long long, cudaStream_t);
template cudaError_t gemm_auto<c128>(const GemmDesc<c128>&, bool, int*, unsigned long long, cudaStream_t);
template cudaError_t gemm_simt<c64>(const GemmDesc<c64>&, cudaStream_t);
template cudaError_t gemm_simt<c128>(const GemmDesc<c128>&, cudaStream_t);
template cudaError_t theta_gemm_simt<c64>(int, int, int, const c64*, const c64*, const c64*, c64*,
                                          int64_t, cudaStream_t, const c64*);
template cudaError_t theta_gemm_simt<c128>(int, int, int, const c128*, const c128*, const c128*,
                                           c128*, int64_t, cudaStream_t, const c128*);

}  // namespace mpsg
