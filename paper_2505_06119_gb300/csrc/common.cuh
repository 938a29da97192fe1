// Shared device/host definitions of the GB300 MPS library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mps.h"

namespace mpsg {

// ---------------------------------------------------------------------------
// complex element types: c64 = cplx<float>, c128 = cplx<double>
template <typename R>
struct __align__(sizeof(R) * 2) cplx {
  R re, im;
};
using c64 = cplx<float>;
using c128 = cplx<double>;

template <typename R>
__host__ __device__ __forceinline__ cplx<R> mk(R re, R im) {
  cplx<R> c;
  c.re = re;
  c.im = im;
  return c;
}
template <typename R>
__host__ __device__ __forceinline__ cplx<R> operator+(cplx<R> a, cplx<R> b) {
  return mk<R>(a.re + b.re, a.im + b.im);
}
template <typename R>
__host__ __device__ __forceinline__ cplx<R> operator-(cplx<R> a, cplx<R> b) {
  return mk<R>(a.re - b.re, a.im - b.im);
}
template <typename R>
__host__ __device__ __forceinline__ cplx<R> operator*(cplx<R> a, cplx<R> b) {
  return mk<R>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename R>
__host__ __device__ __forceinline__ cplx<R> cconj(cplx<R> a) {
  return mk<R>(a.re, -a.im);
}
template <typename R>
__host__ __device__ __forceinline__ R cabs2(cplx<R> a) {
  return a.re * a.re + a.im * a.im;
}
// acc += a * b
template <typename R>
__host__ __device__ __forceinline__ void cfma(cplx<R>& acc, cplx<R> a, cplx<R> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}
// acc += conj(a) * b
template <typename R>
__host__ __device__ __forceinline__ void cfma_conj(cplx<R>& acc, cplx<R> a, cplx<R> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
}
template <typename RO, typename RI>
__host__ __device__ __forceinline__ cplx<RO> ccast(cplx<RI> a) {
  return mk<RO>((RO)a.re, (RO)a.im);
}

template <typename T>
struct real_of;
template <>
struct real_of<c64> {
  using type = float;
};
template <>
struct real_of<c128> {
  using type = double;
};

// ---------------------------------------------------------------------------
// device error word values (written by kernels, read by the host)
enum : int {
  DEV_OK = 0,
  DEV_ERR_TIMEOUT = 1,   // a bounded wait gave up
  DEV_ERR_BOUNDS = 2,    // an index check failed
  DEV_ERR_NONFINITE = 3  // a NaN/Inf reached a pivot decision
};

// Index checks of the bounds-checking build (compiled with -DMPS_BOUNDS_CHECK): where
// an index comes from device data (a permutation, a pivot sequence), a value outside
// its range records DEV_ERR_BOUNDS in the device error word (when one is given) and
// the access is skipped.  The ordinary build compiles the check to `true`.
#ifdef MPS_BOUNDS_CHECK
__device__ __forceinline__ bool index_ok(bool in_range, int* err) {
  if (!in_range && err) atomicCAS(err, 0, 2);  // DEV_OK -> DEV_ERR_BOUNDS
  return in_range;
}
#else
__device__ __forceinline__ bool index_ok(bool, int*) { return true; }
#endif

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed_i32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned atom_add_acqrel_u32(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_u32(unsigned* p, unsigned v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier for a cooperative launch of `expected` CTAs.
//   bar[0] = arrival count (returns to 0 after every barrier),
//   bar[1] = generation (monotonic).
// Every wait is bounded: after `timeout_ns` of spinning, or as soon as another
// CTA has raised *err, the CTA records DEV_ERR_TIMEOUT (first writer wins) and
// the call returns false.  Callers leave the kernel when it returns false.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned expected, int* err,
                                             unsigned long long timeout_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned gen = ld_acquire_u32(&bar[1]);
    unsigned arrived = atom_add_acqrel_u32(&bar[0], 1u);
    if (arrived == expected - 1) {
      st_relaxed_u32(&bar[0], 0u);
      st_release_u32(&bar[1], gen + 1);
    } else {
      unsigned long long t0 = globaltimer_ns();
      unsigned spins = 0;
      while (ld_acquire_u32(&bar[1]) == gen) {
        if (ld_relaxed_i32(err) != DEV_OK) {
          ok = 0;
          break;
        }
        if ((++spins & 63u) == 0u && globaltimer_ns() - t0 > timeout_ns) {
          atomicCAS(err, DEV_OK, DEV_ERR_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// The same barrier for a kernel that read the generation word once at its start
// (thread 0, before its first arrival; the word only advances once every CTA has
// arrived, so that value is current) and tracks it in `gen` (thread 0's copy):
// one round trip to global memory less per barrier.
__device__ __forceinline__ bool grid_barrier_g(unsigned* bar, unsigned expected, int* err,
                                               unsigned long long timeout_ns, unsigned& gen) {
  __shared__ int s_okg;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned arrived = atom_add_acqrel_u32(&bar[0], 1u);
    if (arrived == expected - 1) {
      st_relaxed_u32(&bar[0], 0u);
      st_release_u32(&bar[1], gen + 1);
    } else {
      unsigned long long t0 = globaltimer_ns();
      unsigned spins = 0;
      while (ld_acquire_u32(&bar[1]) == gen) {
        if (ld_relaxed_i32(err) != DEV_OK) {
          ok = 0;
          break;
        }
        if ((++spins & 63u) == 0u && globaltimer_ns() - t0 > timeout_ns) {
          atomicCAS(err, DEV_OK, DEV_ERR_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    gen += 1;
    s_okg = ok;
  }
  __syncthreads();
  return s_okg != 0;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
__device__ __forceinline__ uint32_t mbar_try(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok;
}
// Bounded wait for the phase of the given parity; false (and the error word set)
// on expiry or when another thread has already failed.
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, int* err, unsigned long long timeout_ns) {
  if (mbar_try(a, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  for (unsigned it = 1;; ++it) {
    if (mbar_try(a, parity)) return true;
    if ((it & 255u) == 0u) {
      if (ld_relaxed_i32(err) != DEV_OK) return false;
      if (globaltimer_ns() - t0 > timeout_ns) {
        atomicCAS(err, DEV_OK, DEV_ERR_TIMEOUT);
        return false;
      }
    }
  }
}

// Bounded wait that ignores the error word: lets an asynchronous copy that is
// already in flight land before its buffer is reused or the CTA leaves.
__device__ __forceinline__ bool mbar_wait_plain(uint32_t a, uint32_t parity, unsigned long long timeout_ns) {
  if (mbar_try(a, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  for (unsigned it = 1;; ++it) {
    if (mbar_try(a, parity)) return true;
    if ((it & 255u) == 0u && globaltimer_ns() - t0 > timeout_ns) return false;
  }
}
// Arrive on the barrier and add `bytes` to the transaction count of its phase.
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
// Bulk asynchronous copy global -> shared (TMA, untiled): src and dst 16-byte
// aligned, bytes a multiple of 16; completion is signalled on `mbar`.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}
// The same copy with an L2 cache policy (from l2_policy_keep / l2_policy_stream).
__device__ __forceinline__ void bulk_g2s_hint(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar,
                                              uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(mbar), "l"(policy)
      : "memory");
}
// L2 policies: lines read under `keep` are evicted after the others, lines read
// under `stream` first.
__device__ __forceinline__ uint64_t l2_policy_keep() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_policy_stream() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// Order this thread's generic-proxy accesses with later async-proxy ones.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async;" ::: "memory"); }

template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace mpsg
