// Complex64 GEMM on the 5th-generation tensor cores (tcgen05, TMEM accumulators).
//
//   C[i, j] = alpha * sum_k A(i, k) B(j, k) + beta * C[i, j]        (general)
//   theta[l,a,b,r] = sum_{cd} g[2a+b][2c+d] sum_mu A[l,c,mu] B[mu,d,r] (theta:
//   the bond contraction of Sec. III-B.1 with the gate of Sec. III-C.2 applied
//   in the epilogue)
//
// Precision: each FP32 component x is split into big = tf32(x) (round to
// nearest) and small = x - big; a real product is big*big + big*small +
// small*big ("3xTF32"), which keeps FP32-level products on the tensor cores.  A
// complex product is four real ones, so one K-step of 8 issues 12 MMAs:
// re += ArBr - AiBi, im += ArBi + AiBr (the minus via the instruction's
// negate-A bit).  The tensor cores' FP32 accumulation does not round to nearest,
// and over a long K its error grows with K; so the MMAs of every kPromoteKs
// K-steps go into a fresh TMEM accumulator (two buffers, alternating) that
// accumulator warps read and add, rounding to nearest, into FP32 registers while
// the MMAs go on into the other buffer.  The error then stays that of FP32 sums.
//
// CTA = 9 warps.  Warps 0-3 convert operand tiles (any layout, optional
// conjugation / triangular mask) from global memory into the 128-byte-swizzled
// K-major shared-memory layout the MMA reads: four planar parts (re big, im
// big, re small, im small) per operand.  Warp 4 owns the TMEM allocation and one
// of its threads issues the MMAs.  Warps 5-8 hold the register accumulators (one
// row each per thread) and run the epilogue.  Two-stage mbarrier pipeline for the
// operands, two TMEM buffers for the partial sums; every wait is bounded and
// records DEV_ERR_TIMEOUT in the device error word on expiry.
//
// Tile: 128 rows (M) x 64 complex columns (N) x 32 K per stage.  TMEM buffer q:
// real parts in columns [128 q, 128 q + 64), imaginary parts in the next 64.
#include <algorithm>
#include <cstring>

#include "internal.h"

namespace mpsg {

namespace {

constexpr int TM = 128, TN = 64, TK = 32;
constexpr int A_PART = TM * TK * 4;            // bytes of one planar part of an A tile (16 KB)
constexpr int B_PART = TN * TK * 4;            // 8 KB
constexpr int STAGE = 4 * A_PART + 4 * B_PART; // 96 KB
constexpr int NSTAGE = 2;
constexpr int TC_THREADS = 288;
constexpr int TC_SMEM = NSTAGE * STAGE + 1024;  // + alignment slack
constexpr int TMEM_COLS = 256;                  // two accumulator buffers of 2 x TN columns
constexpr int kPromoteKs = 1;                   // K-steps of 8 per TMEM partial sum
constexpr int kBlocksPerStage = (TK / 8) / kPromoteKs;

struct TcOperand {
  const c64* p;
  int64_t ld;
  int rows, K;
  int kcontig;     // element (row, k) at p[row*ld + k] (1) or p[row + k*ld] (0)
  int conj;
  int mask;        // MASK_* in stored coordinates (r, c) = kcontig ? (k, row) : (row, k)
  int theta_cr;    // > 0: packed row u of tile t is logical row (u/32)*theta_cr + 32t + u%32
};

struct TcArgs {
  TcOperand A, B;
  int M, N, K;
  c64 alpha, beta;
  c64* C;
  int64_t ldc;
  int theta;  // 1: theta epilogue into W
  c64 g[16];
  const c64* gdev;  // the gate in device memory instead (graph replay); NULL: g
  int cl, cr;
  c64* W;
  int64_t ldw;
  int* err;
  unsigned long long timeout_ns;
};

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms of
// 1024 bytes (stride byte offset), SM100 descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;                    // leading byte offset (unused with swizzle)
  d |= (uint64_t)(1024u >> 4) << 32;          // stride byte offset
  d |= (uint64_t)1u << 46;                    // descriptor version
  d |= (uint64_t)2u << 61;                    // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::tf32: F32 accumulate, TF32 A and B, both
// K-major, M = 128, N = 64; bit 13 negates A.
__device__ __forceinline__ uint32_t idesc_tf32(int neg_a) {
  uint32_t d = 0;
  d |= 1u << 4;               // D format F32
  d |= 2u << 7;               // A format TF32
  d |= 2u << 10;              // B format TF32
  d |= (uint32_t)neg_a << 13;
  d |= (uint32_t)(TN >> 3) << 17;
  d |= (uint32_t)(TM >> 4) << 24;
  return d;
}

__device__ __forceinline__ void umma(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          dtmem),
      "l"(ad), "l"(bd), "r"(id), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ float tf32_big(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Element (row, k) of an operand, zero outside and honouring conj / mask.
__device__ __forceinline__ c64 op_elem(const TcOperand& o, int row, int k) {
  c64 z = mk<float>(0.f, 0.f);
  if (row < 0 || k >= o.K) return z;
  int rr = o.kcontig ? k : row, cc = o.kcontig ? row : k;
  if (o.mask == MASK_UNIT_LOWER) {
    if (rr < cc) return z;
    if (rr == cc) return mk<float>(1.f, 0.f);
  } else if (o.mask == MASK_UPPER) {
    if (rr > cc) return z;
  }
  c64 v = o.kcontig ? o.p[(int64_t)row * o.ld + k] : o.p[row + (int64_t)k * o.ld];
  return o.conj ? cconj(v) : v;
}

// Logical row of packed row u of tile t (-1 = padding).
__device__ __forceinline__ int op_row(const TcOperand& o, int tile_rows, int t, int u) {
  if (o.theta_cr > 0) {
    const int r = 32 * t + (u & 31);
    if (r >= o.theta_cr) return -1;
    return (u >> 5) * o.theta_cr + r;
  }
  const int row = t * tile_rows + u;
  return row < o.rows ? row : -1;
}

// Convert the rows x 32 tile (t, kb) of an operand into its four planar,
// 128-byte-swizzled parts at `base` (part stride part_bytes).  128 threads.
template <int ROWS>
__device__ __forceinline__ void convert_tile(const TcOperand& o, int t, int kb, unsigned char* base, int part_bytes,
                                             int tid) {
  constexpr int ITEMS = ROWS * 8;  // (row, 16-byte chunk of 4 k values)
#pragma unroll 2
  for (int e = tid; e < ITEMS; e += 128) {
    int u, c;
    if (o.kcontig) {  // lanes along k: 8 lanes read one row's 32 k values
      u = e >> 3;
      c = e & 7;
    } else {  // lanes along rows: each k column is read contiguously
      u = e % ROWS;
      c = e / ROWS;
    }
    const int row = op_row(o, ROWS, t, u);
    const int k0 = kb * TK + 4 * c;
    float4 rb, ib, rs, is;
    float* prb = &rb.x;
    float* pib = &ib.x;
    float* prs = &rs.x;
    float* pis = &is.x;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const c64 v = op_elem(o, row, k0 + q);
      const float br = tf32_big(v.re), bi = tf32_big(v.im);
      prb[q] = br;
      pib[q] = bi;
      prs[q] = v.re - br;
      pis[q] = v.im - bi;
    }
    const int off = u * 128 + ((c ^ (u & 7)) << 4);
    *reinterpret_cast<float4*>(base + off) = rb;
    *reinterpret_cast<float4*>(base + part_bytes + off) = ib;
    *reinterpret_cast<float4*>(base + 2 * part_bytes + off) = rs;
    *reinterpret_cast<float4*>(base + 3 * part_bytes + off) = is;
  }
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__global__ void __launch_bounds__(TC_THREADS, 1) tc_gemm_kernel(const __grid_constant__ TcArgs a) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long bar_full[NSTAGE], bar_empty[NSTAGE], acc_full[2], acc_empty[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_skip;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // an earlier bounded wait expired: nothing to do (decided once for the whole CTA)
  if (tid == 0) s_skip = ld_relaxed_i32(a.err) != DEV_OK;
  __syncthreads();
  if (s_skip) return;
  unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int tm = blockIdx.x, tn = blockIdx.y;
  const int nkb = (a.K + TK - 1) / TK;
  const int nblk = nkb * kBlocksPerStage;  // TMEM partial sums of the whole K range

  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      mbar_init(smem_u32(&bar_full[s]), 128);
      mbar_init(smem_u32(&bar_empty[s]), 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(smem_u32(&acc_full[q]), 1);
      mbar_init(smem_u32(&acc_empty[q]), 128);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 4) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;

  bool ok = true;
  float accr[TN], acci[TN];  // accumulator warps: row (warp % 4) * 32 + lane, every column of the tile
  if (warp < 4) {
    // ---- converters
    for (int kb = 0; kb < nkb && ok; ++kb) {
      const int s = kb & 1;
      if (kb >= NSTAGE) ok = mbar_wait(smem_u32(&bar_empty[s]), ((kb >> 1) - 1) & 1, a.err, a.timeout_ns);
      if (!ok) break;
      unsigned char* st = sm + s * STAGE;
      convert_tile<TM>(a.A, tm, kb, st, A_PART, tid);
      convert_tile<TN>(a.B, tn, kb, st + 4 * A_PART, B_PART, tid);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(smem_u32(&bar_full[s]));
    }
  } else if (warp == 4) {
    if (lane == 0) {
      // ---- MMA issuer
      const uint32_t id_pos = idesc_tf32(0), id_neg = idesc_tf32(1);
      int blk = 0;
      for (int kb = 0; kb < nkb && ok; ++kb) {
        const int s = kb & 1;
        if (!mbar_wait(smem_u32(&bar_full[s]), (kb >> 1) & 1, a.err, a.timeout_ns)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t st = smem_u32(sm + s * STAGE);
        for (int ks = 0; ks < TK / 8 && ok; ++ks) {
          const int q = blk & 1;
          const bool opens = ks % kPromoteKs == 0;
          if (opens && blk >= 2) {
            // the accumulator warps have read this buffer's previous partial sum
            if (!mbar_wait(smem_u32(&acc_empty[q]), ((blk >> 1) - 1) & 1, a.err, a.timeout_ns)) {
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          }
          const uint32_t dre = tmem + q * 2 * TN, dim = dre + TN;
          const uint32_t ko = ks * 32;  // 8 tf32 = 32 bytes along K inside the swizzle atom
          const uint64_t arb = sdesc(st + 0 * A_PART + ko), aib = sdesc(st + 1 * A_PART + ko);
          const uint64_t ars = sdesc(st + 2 * A_PART + ko), ais = sdesc(st + 3 * A_PART + ko);
          const uint32_t bst = st + 4 * A_PART;
          const uint64_t brb = sdesc(bst + 0 * B_PART + ko), bib = sdesc(bst + 1 * B_PART + ko);
          const uint64_t brs = sdesc(bst + 2 * B_PART + ko), bis = sdesc(bst + 3 * B_PART + ko);
          const uint32_t first = opens ? 0u : 1u;
          // re += Ar Br - Ai Bi
          umma(dre, arb, brb, id_pos, first);
          umma(dre, arb, brs, id_pos, 1);
          umma(dre, ars, brb, id_pos, 1);
          umma(dre, aib, bib, id_neg, 1);
          umma(dre, aib, bis, id_neg, 1);
          umma(dre, ais, bib, id_neg, 1);
          // im += Ar Bi + Ai Br
          umma(dim, arb, bib, id_pos, first);
          umma(dim, arb, bis, id_pos, 1);
          umma(dim, ars, bib, id_pos, 1);
          umma(dim, aib, brb, id_pos, 1);
          umma(dim, aib, brs, id_pos, 1);
          umma(dim, ais, brb, id_pos, 1);
          if (ks % kPromoteKs == kPromoteKs - 1) {
            umma_commit(smem_u32(&acc_full[q]));  // fires when this partial sum is complete
            ++blk;
          }
        }
        umma_commit(smem_u32(&bar_empty[s]));
      }
    }
  } else {
    // ---- accumulator warps: add every TMEM partial sum into registers (round to nearest)
#pragma unroll
    for (int c = 0; c < TN; ++c) {
      accr[c] = 0.f;
      acci[c] = 0.f;
    }
    const uint32_t trow = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    for (int blk = 0; blk < nblk; ++blk) {
      const int q = blk & 1;
      if (!mbar_wait(smem_u32(&acc_full[q]), (blk >> 1) & 1, a.err, a.timeout_ns)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int c0 = 0; c0 < TN; c0 += 16) {
        float re[16], im[16];
        tmem_ld16(trow + q * 2 * TN + c0, re);
        tmem_ld16(trow + q * 2 * TN + TN + c0, im);
        tmem_wait_ld();
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          accr[c0 + c] += re[c];
          acci[c0 + c] += im[c];
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(smem_u32(&acc_empty[q]));
    }
    // ---- epilogue from the registers
    const bool store = ok && ld_relaxed_i32(a.err) == DEV_OK;
    const int i = tm * TM + 32 * (warp & 3) + lane;
    if (!a.theta) {
      if (store && i < a.M) {
        const bool bz = (a.beta.re == 0.f && a.beta.im == 0.f);
#pragma unroll
        for (int c = 0; c < TN; ++c) {  // fully unrolled: the accumulators stay in registers
          const int j = tn * TN + c;
          if (j < a.N) {
            c64* cp = a.C + i + (int64_t)j * a.ldc;
            c64 v = a.alpha * mk<float>(accr[c], acci[c]);
            if (!bz) v = v + a.beta * (*cp);
            *cp = v;
          }
        }
      }
    } else {
      // theta: row i = (l, c) = 2l + c, column u = (d, r) = 32d + (r - 32 tn)
      const int ca = i & 1, l = i >> 1;
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        // X[(l, c'), (d, r)] for both c' (own row and partner row i^1)
        const c64 own0 = mk<float>(accr[q], acci[q]), own1 = mk<float>(accr[32 + q], acci[32 + q]);
        c64 oth0, oth1;
        oth0.re = __shfl_xor_sync(0xffffffffu, own0.re, 1);
        oth0.im = __shfl_xor_sync(0xffffffffu, own0.im, 1);
        oth1.re = __shfl_xor_sync(0xffffffffu, own1.re, 1);
        oth1.im = __shfl_xor_sync(0xffffffffu, own1.im, 1);
        const c64 xc0d0 = ca ? oth0 : own0, xc0d1 = ca ? oth1 : own1;
        const c64 xc1d0 = ca ? own0 : oth0, xc1d1 = ca ? own1 : oth1;
        const int r = 32 * tn + q;
        if (store && l < a.cl && r < a.cr) {
#pragma unroll
          for (int bb = 0; bb < 2; ++bb) {
            const c64* gr = (a.gdev ? a.gdev : a.g) + (2 * ca + bb) * 4;
            c64 v = gr[0] * xc0d0;
            cfma(v, gr[1], xc0d1);
            cfma(v, gr[2], xc1d0);
            cfma(v, gr[3], xc1d1);
            a.W[(int64_t)(bb * a.cr + r) * a.ldw + i] = v;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 4) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

PerDevice g_tc_init;  // kernel attribute set once per device

cudaError_t tc_setup() {
  cudaError_t e = cudaSuccess;
  g_tc_init.get([&e]() -> long long {
    e = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    return e == cudaSuccess ? 1 : -1;
  });
  return e;
}

TcOperand operand_a(const GemmDesc<c64>& d) {
  TcOperand o;
  o.p = d.A;
  o.ld = d.lda;
  o.rows = d.M;
  o.K = d.K;
  o.kcontig = d.a_row ? 1 : 0;  // A(i,k) = A[i*lda + k] or A[i + k*lda]
  o.conj = d.a_conj;
  o.mask = d.a_mask;
  o.theta_cr = 0;
  return o;
}

TcOperand operand_b(const GemmDesc<c64>& d) {
  // the MMA's B is N x K: row j, column k = B(k, j)
  TcOperand o;
  o.p = d.B;
  o.ld = d.ldb;
  o.rows = d.N;
  o.K = d.K;
  o.kcontig = d.b_row ? 0 : 1;  // B(k,j) = B[k*ldb + j] (row j contiguous across j) or B[k + j*ldb]
  o.conj = d.b_conj;
  o.mask = d.b_mask;
  o.theta_cr = 0;
  return o;
}

}  // namespace

// Only long contractions gain from the tensor cores here; rank-nb updates
// (K = panel width) stay on the CUDA cores.
bool tc_gemm_applicable(const GemmDesc<c64>& d) { return d.M >= 64 && d.N >= 32 && d.K >= 128 && d.splitk <= 1; }

cudaError_t tc_gemm(const GemmDesc<c64>& d, int* err, unsigned long long timeout_ns, cudaStream_t s) {
  if (d.M <= 0 || d.N <= 0) return cudaSuccess;
  cudaError_t e = tc_setup();
  if (e != cudaSuccess) return e;
  TcArgs a;
  memset(&a, 0, sizeof(a));
  a.A = operand_a(d);
  a.B = operand_b(d);
  a.M = d.M;
  a.N = d.N;
  a.K = d.K;
  a.alpha = d.alpha;
  a.beta = d.beta;
  a.C = d.C;
  a.ldc = d.ldc;
  a.theta = 0;
  a.err = err;
  a.timeout_ns = timeout_ns;
  dim3 grid((d.M + TM - 1) / TM, (d.N + TN - 1) / TN);
  if (grid.y > 65535) return cudaErrorInvalidConfiguration;
  tc_gemm_kernel<<<grid, TC_THREADS, TC_SMEM, s>>>(a);
  return cudaGetLastError();
}

cudaError_t tc_theta(int cl, int cm, int cr, const c64* A, const c64* B, const c64* g16, c64* W, int64_t ldw,
                     int* err, unsigned long long timeout_ns, cudaStream_t s, const c64* gdev) {
  cudaError_t e = tc_setup();
  if (e != cudaSuccess) return e;
  TcArgs a;
  memset(&a, 0, sizeof(a));
  // A: site i as a (2 cl) x cm row-major matrix
  a.A.p = A;
  a.A.ld = cm;
  a.A.rows = 2 * cl;
  a.A.K = cm;
  a.A.kcontig = 1;
  a.A.conj = 0;
  a.A.mask = MASK_NONE;
  a.A.theta_cr = 0;
  // B: site i+1 as cm x (2 cr) row-major; MMA row j = column (d, r) of it
  a.B.p = B;
  a.B.ld = 2 * (int64_t)cr;
  a.B.rows = 2 * cr;
  a.B.K = cm;
  a.B.kcontig = 0;
  a.B.conj = 0;
  a.B.mask = MASK_NONE;
  a.B.theta_cr = cr;
  a.M = 2 * cl;
  a.N = 2 * cr;
  a.K = cm;
  a.theta = 1;
  for (int i = 0; i < 16; ++i) a.g[i] = g16[i];
  a.gdev = gdev;
  a.cl = cl;
  a.cr = cr;
  a.W = W;
  a.ldw = ldw;
  a.err = err;
  a.timeout_ns = timeout_ns;
  dim3 grid((2 * cl + TM - 1) / TM, (cr + 31) / 32);
  if (grid.y > 65535) return cudaErrorInvalidConfiguration;
  tc_gemm_kernel<<<grid, TC_THREADS, TC_SMEM, s>>>(a);
  return cudaGetLastError();
}

}  // namespace mpsg
