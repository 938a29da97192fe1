// MPO application by zip-up (Sec. III-C.3): the per-site contraction of the MPO
// tensor with the carried block.  The carried block times the site is a plain
// GEMM (gemm_simt); this kernel then contracts the MPO tensor
// W[a][b][out][in] (bond dims <= 2, passed by value) into it:
//
//   Z[(kk, out), (b, r)] = sum_{a, in} W[a][b][out][in] Y[(kk, a), (in, r)]
//
// Y is read through (row, column) strides, so it can be the GEMM's
// column-major output or, on the first site, the row-major site itself.  Z goes
// either to the column-major QR workspace (rows 2 kk, columns b chi_r) or, on
// the last site (b = 1), straight into the row-major site (kk, 2, chi_r).
#include "internal.h"

namespace mpsg {

namespace {

template <typename T>
__global__ void mpo_z_kernel(const T* __restrict__ Y, int64_t ys_row, int64_t ys_col, int kk, int adim, int bdim,
                             int cr, MpoTensor<T> W, T* __restrict__ Z, int64_t ldz, int to_site) {
  using R = typename real_of<T>::type;
  const int64_t rows = 2 * (int64_t)kk;
  const int64_t total = rows * bdim * cr;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = idx % rows, col = idx / rows;
    const int kq = (int)(row >> 1), t = (int)(row & 1);
    const int bb = (int)(col / cr), r = (int)(col % cr);
    T acc = mk<R>(0, 0);
    for (int a = 0; a < adim; ++a)
      for (int s = 0; s < 2; ++s) {
        const T w = W.w[((a * 2 + bb) * 2 + t) * 2 + s];
        const T y = Y[((int64_t)kq * adim + a) * ys_row + ((int64_t)s * cr + r) * ys_col];
        cfma(acc, w, y);
      }
    if (to_site)
      Z[row * cr + r] = acc;  // bdim == 1: site (kk, 2, cr), row = 2 kq + t
    else
      Z[row + col * ldz] = acc;
  }
}

}  // namespace

template <typename T>
cudaError_t mpo_contract(const T* Y, int64_t ys_row, int64_t ys_col, int kk, int adim, int bdim, int cr,
                         const MpoTensor<T>& W, T* Z, int64_t ldz, int to_site, cudaStream_t s) {
  const int64_t total = 2 * (int64_t)kk * bdim * cr;
  if (total <= 0) return cudaSuccess;
  if (adim < 1 || adim > 2 || bdim < 1 || bdim > 2 || (to_site && bdim != 1)) return cudaErrorInvalidValue;
  const int64_t blocks = std::min<int64_t>((total + 255) / 256, 152 * 16);
  mpo_z_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(Y, ys_row, ys_col, kk, adim, bdim, cr, W, Z, ldz, to_site);
  return cudaGetLastError();
}

template cudaError_t mpo_contract<c64>(const c64*, int64_t, int64_t, int, int, int, int, const MpoTensor<c64>&, c64*,
                                       int64_t, int, cudaStream_t);
template cudaError_t mpo_contract<c128>(const c128*, int64_t, int64_t, int, int, int, int, const MpoTensor<c128>&,
                                        c128*, int64_t, int, cudaStream_t);

}  // namespace mpsg
