// Bandwidth kernels: one-qubit gates, site split / reshape / un-pivot,
// layout changes, precision conversion, reductions and the amplitude chain.
#include "internal.h"

namespace mpsg {

namespace {

// A[l, s, r] <- sum_s' u[s][s'] A[l, s', r]   (Sec. II-A.2)
template <typename T>
__global__ void apply_1q_kernel(T* site, int cl, int cr, T u00, T u01, T u10, T u11) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t total = (int64_t)cl * cr;
  if (idx >= total) return;
  int64_t l = idx / cr, r = idx % cr;
  T* p0 = site + l * 2 * cr + r;
  T* p1 = p0 + cr;
  T x0 = *p0, x1 = *p1;
  *p0 = u00 * x0 + u01 * x1;
  *p1 = u10 * x0 + u11 * x1;
}

// dst[r + c*ldd] = src[r*lds + c]  (optionally conjugated), 32x32 tiles
template <typename T>
__global__ void transpose_kernel(const T* src, int64_t lds, T* dst, int64_t ldd, int rows, int cols, int conj) {
  __shared__ T tile[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int i = ty; i < 32; i += 8) {
    int r = r0 + i, c = c0 + tx;
    if (r < rows && c < cols) {
      T v = src[(int64_t)r * lds + c];
      tile[i][tx] = conj ? cconj(v) : v;
    }
  }
  __syncthreads();
  for (int i = ty; i < 32; i += 8) {
    int c = c0 + i, r = r0 + tx;
    if (r < rows && c < cols) dst[r + (int64_t)c * ldd] = tile[tx][i];
  }
}

template <typename T>
__global__ void copy2d_kernel(const T* src, int64_t lds, T* dst, int64_t ldd, int rows, int cols, int conj) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t total = (int64_t)rows * cols;
  if (idx >= total) return;
  int64_t r = idx / cols, c = idx % cols;
  T v = src[r * lds + c];
  dst[r * ldd + c] = conj ? cconj(v) : v;
}

__global__ void invert_perm_kernel(const int* jpvt, int* inv, int n, int* err) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) {
    const int q = jpvt[t];
    if (index_ok(q >= 0 && q < n, err)) inv[q] = t;
  }
}

// site[kk*n + c] = R(kk, inv[c]),  R(kk, t) = kk <= t ? W[kk + t*ldw] : 0
template <typename T>
__global__ void split_right_kernel(const T* W, int64_t ldw, const int* inv, int k, int n, T* site, int* err) {
  using R = typename real_of<T>::type;
  __shared__ T tile[32][33];  // [c][kk]
  const int k0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int i = ty; i < 32; i += 8) {
    int c = c0 + i, kk = k0 + tx;
    T v = mk<R>(0, 0);
    if (c < n && kk < k) {
      int t = inv[c];
      if (kk <= t && index_ok(t < n, err)) v = W[kk + (int64_t)t * ldw];
    }
    tile[i][tx] = v;
  }
  __syncthreads();
  for (int i = ty; i < 32; i += 8) {
    int kk = k0 + i, c = c0 + tx;
    if (kk < k && c < n) site[(int64_t)kk * n + c] = tile[tx][i];
  }
}

template <typename T>
__global__ void identity_kernel(T* Q, int64_t ldq, int m, int k) {
  using R = typename real_of<T>::type;
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t total = (int64_t)m * k;
  if (idx >= total) return;
  int64_t c = idx / m, r = idx % m;
  Q[r + c * ldq] = mk<R>(r == c ? 1 : 0, 0);
}

template <typename TO, typename TI>
__global__ void convert_kernel(const TI* src, TO* dst, int64_t count) {
  using RO = typename real_of<TO>::type;
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx < count) dst[idx] = ccast<RO>(src[idx]);
}

template <typename T>
__global__ void norm2_partial_kernel(const T* x, int64_t count, double* partial) {
  __shared__ double s[256];
  const int64_t per = (count + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * per, hi = min(count, lo + per);
  double acc = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += 256) acc += (double)cabs2(x[i]);
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = s[0];
}

__global__ void sum_partials_kernel(const double* partial, int npart, double* out) {
  __shared__ double s[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < npart; i += 256) acc += partial[i];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0];
}

// out[j] = sum_l v[l] M[l*ld + j]; block = 32 columns x 8 row groups
template <typename T>
__global__ void vecmat_kernel(const c128* v, const T* M, int64_t ld, int rows, int cols, c128* out) {
  __shared__ c128 s[8][32];
  const int j = blockIdx.x * 32 + threadIdx.x;
  c128 acc = mk<double>(0, 0);
  if (j < cols)
    for (int l = threadIdx.y; l < rows; l += 8) cfma(acc, v[l], ccast<double>(M[(int64_t)l * ld + j]));
  s[threadIdx.y][threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.y == 0 && j < cols) {
    c128 t = s[0][threadIdx.x];
    for (int g = 1; g < 8; ++g) t = t + s[g][threadIdx.x];
    out[j] = t;
  }
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

template <typename T>
cudaError_t apply_1q(T* site, int chi_l, int chi_r, const T* u, cudaStream_t s) {
  int64_t total = (int64_t)chi_l * chi_r;
  if (total == 0) return cudaSuccess;
  apply_1q_kernel<T><<<blocks_for(total, 256), 256, 0, s>>>(site, chi_l, chi_r, u[0], u[1], u[2], u[3]);
  return cudaGetLastError();
}

template <typename T>
cudaError_t transpose_copy(const T* src, int64_t lds, T* dst, int64_t ldd, int rows, int cols, int conj,
                           cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  dim3 grid((cols + 31) / 32, (rows + 31) / 32);
  if (grid.y > 65535) return cudaErrorInvalidConfiguration;
  transpose_kernel<T><<<grid, dim3(32, 8), 0, s>>>(src, lds, dst, ldd, rows, cols, conj);
  return cudaGetLastError();
}

template <typename T>
cudaError_t copy2d(const T* src, int64_t lds, T* dst, int64_t ldd, int rows, int cols, int conj, cudaStream_t s) {
  int64_t total = (int64_t)rows * cols;
  if (total <= 0) return cudaSuccess;
  copy2d_kernel<T><<<blocks_for(total, 256), 256, 0, s>>>(src, lds, dst, ldd, rows, cols, conj);
  return cudaGetLastError();
}

template <typename T>
cudaError_t split_right(const T* W, int64_t ldw, const int* jpvt, int* inv, int k, int n, T* site, cudaStream_t s,
                        int* err) {
  if (k <= 0 || n <= 0) return cudaSuccess;
  invert_perm_kernel<<<blocks_for(n, 256), 256, 0, s>>>(jpvt, inv, n, err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dim3 grid((n + 31) / 32, (k + 31) / 32);
  if (grid.y > 65535) return cudaErrorInvalidConfiguration;
  split_right_kernel<T><<<grid, dim3(32, 8), 0, s>>>(W, ldw, inv, k, n, site, err);
  return cudaGetLastError();
}

template <typename T>
cudaError_t set_identity(T* Q, int64_t ldq, int m, int k, cudaStream_t s) {
  int64_t total = (int64_t)m * k;
  if (total <= 0) return cudaSuccess;
  identity_kernel<T><<<blocks_for(total, 256), 256, 0, s>>>(Q, ldq, m, k);
  return cudaGetLastError();
}

template <typename TO, typename TI>
cudaError_t convert(const TI* src, TO* dst, int64_t count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  convert_kernel<TO, TI><<<blocks_for(count, 256), 256, 0, s>>>(src, dst, count);
  return cudaGetLastError();
}

template <typename T>
cudaError_t norm2_sum(const T* x, int64_t count, double* partial, int npart, double* out, cudaStream_t s) {
  if (npart < 1) npart = 1;
  norm2_partial_kernel<T><<<npart, 256, 0, s>>>(x, count, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  sum_partials_kernel<<<1, 256, 0, s>>>(partial, npart, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t vecmat(const c128* v, const T* M, int64_t ld, int rows, int cols, c128* out, cudaStream_t s) {
  if (cols <= 0) return cudaSuccess;
  vecmat_kernel<T><<<(cols + 31) / 32, dim3(32, 8), 0, s>>>(v, M, ld, rows, cols, out);
  return cudaGetLastError();
}

#define INST(T)                                                                                      \
  template cudaError_t apply_1q<T>(T*, int, int, const T*, cudaStream_t);                            \
  template cudaError_t transpose_copy<T>(const T*, int64_t, T*, int64_t, int, int, int, cudaStream_t); \
  template cudaError_t copy2d<T>(const T*, int64_t, T*, int64_t, int, int, int, cudaStream_t);        \
  template cudaError_t split_right<T>(const T*, int64_t, const int*, int*, int, int, T*, cudaStream_t, int*); \
  template cudaError_t set_identity<T>(T*, int64_t, int, int, cudaStream_t);                         \
  template cudaError_t norm2_sum<T>(const T*, int64_t, double*, int, double*, cudaStream_t);         \
  template cudaError_t vecmat<T>(const c128*, const T*, int64_t, int, int, c128*, cudaStream_t);
INST(c64)
INST(c128)
template cudaError_t convert<c64, c128>(const c128*, c64*, int64_t, cudaStream_t);
template cudaError_t convert<c128, c64>(const c64*, c128*, int64_t, cudaStream_t);
template cudaError_t convert<c128, c128>(const c128*, c128*, int64_t, cudaStream_t);
template cudaError_t convert<c64, c64>(const c64*, c64*, int64_t, cudaStream_t);

}  // namespace mpsg
