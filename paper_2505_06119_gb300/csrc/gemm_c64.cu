// Complex64 GEMM on the CUDA cores (FP32 FFMA), the workhorse of the mixed
// path: block-reflector updates and Q formation of the QR factorisations
// (Sec. III-B.2, III-C.1), the absorption of R/L factors in centre moves, and
// the theta contraction with its fused gate epilogue (Sec. III-B.1, III-C.2).
//
// CTA tile BM x 128 (BM = 128 or 64), K slices of 16, 256 threads; thread
// (tm, tn) of a 16 x 16 grid owns rows 32g + 2tm + {0,1} and columns
// 32h + 2tn + {0,1}, so its operand fragments are 16-byte shared-memory
// vectors read without bank conflicts.
//
// Operand slices reach shared memory through a ring of kStages buffers filled
// by asynchronous 8-byte copies (any alignment, any leading dimension); the
// copies of slice s + kStages - 1 are in flight while slice s is multiplied,
// and no register holds staged data.  Elements outside the matrix or zero
// under the operand mask are zero-filled by the copy; what a plain copy cannot
// express (conjugation, the unit diagonal of a reflector block) is applied by
// each thread to the elements it copied, after they land and before the slice
// is published to the CTA.
//
// The product sum is accumulated from zero and rounded on its own before the
// epilogue forms C = alpha * sum + beta * C (C read only by the C-reading
// variant of the kernel), which keeps a small update from being rounded at the
// scale of C once per K step.  With split-K the raw partial products go to the
// workspace and a reduction applies alpha and beta.
//
// Theta mode: A is the row-major site A_i ((l,c) x mu), B the row-major site
// A_{i+1} (mu x (d,r)); the tile's 128 columns are 64 values of r for both d,
// arranged so that every thread holds, for each of its (l, r), all four
// X[(l,c),(d,r)]; the 4 x 4 gate is applied in registers and theta is written
// column-major into the factorisation workspace.
#include <algorithm>

#include "internal.h"

namespace mpsg {

namespace {

constexpr int G_NT = 256;
constexpr int G_BN = 128;
constexpr int G_BK = 16;
constexpr int G_PAD = 2;  // complex elements of padding per shared-memory row
constexpr int kStages = 3;

template <int BM>
constexpr int g_smem_bytes() {
  return kStages * G_BK * ((BM + G_PAD) + (G_BN + G_PAD)) * (int)sizeof(c64);
}

struct ThetaEpi {
  int cr;      // chi_r
  c64 g[16];   // gate, g[(2a+b)*4 + 2c+d]
  const c64* gdev;  // the gate in device memory instead (layers replayed as CUDA graphs); NULL: g
  c64* W;      // theta, column-major, leading dimension ldw
  int64_t ldw;
};

__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Classification of one operand element under its mask, in the stored
// column-major coordinates (r, c): 0 = zero, 1 = stored value, 2 = unit.
__device__ __forceinline__ int mask_kind(int mask, int r, int c) {
  if (mask == MASK_UNIT_LOWER) return r > c ? 1 : (r == c ? 2 : 0);
  if (mask == MASK_UPPER) return r <= c ? 1 : 0;
  return 1;
}

// BM = 64 tiles run two CTAs per SM (at most 128 registers a thread) so one
// CTA's C traffic overlaps the other's arithmetic in short contractions.
// BETA: C is read (beta != 0, no split-K); compiled separately so the long
// contractions, which never read C, keep the register allocation of a kernel
// without that code.
template <int BM, bool THETA, bool BETA>
__global__ void __launch_bounds__(G_NT, BM == 64 ? 2 : 1) gemm_c64_kernel(GemmDesc<c64> d, ThetaEpi te) {
  constexpr int RG = BM / 32;             // row pairs per thread
  constexpr int EA = BM * G_BK / G_NT;    // A elements copied per thread and slice
  constexpr int EB = G_BN * G_BK / G_NT;  // B elements copied per thread and slice
  constexpr int LAS = BM + G_PAD, LBS = G_BN + G_PAD;
  extern __shared__ __align__(16) unsigned char g_sm[];
  c64* As = reinterpret_cast<c64*>(g_sm);  // [kStages][G_BK][LAS]
  c64* Bs = As + kStages * G_BK * LAS;     // [kStages][G_BK][LBS]
  const int tid = threadIdx.x, tm = tid % 16, tn = tid / 16;
  const int i0 = blockIdx.x * BM;
  const int j0 = blockIdx.y * (THETA ? G_BN / 2 : G_BN);  // theta: first r of the tile
  int kbeg = 0, kend = d.K;
  const bool split = d.splitk > 1;
  if (split) {
    const int per = ((d.K + d.splitk - 1) / d.splitk + G_BK - 1) / G_BK * G_BK;
    kbeg = blockIdx.z * per;
    kend = min(d.K, kbeg + per);
  }
  // triangular operands: K ranges where the mask zeroes the whole tile row/column
  // block contribute nothing and are skipped (the sums are unchanged: only exact
  // zero products are left out)
  if (d.a_mask == MASK_UPPER) {
    if (d.a_row) kend = min(kend, i0 + BM);
    else kbeg = max(kbeg, i0);
  } else if (d.a_mask == MASK_UNIT_LOWER) {
    if (d.a_row) kbeg = max(kbeg, i0);
    else kend = min(kend, i0 + BM);
  }
  if (!THETA) {
    if (d.b_mask == MASK_UPPER) {
      if (d.b_row) kbeg = max(kbeg, j0);
      else kend = min(kend, j0 + G_BN);
    } else if (d.b_mask == MASK_UNIT_LOWER) {
      if (d.b_row) kend = min(kend, j0 + G_BN);
      else kbeg = max(kbeg, j0);
    }
  }
  constexpr bool beta_nz = BETA && !THETA;  // the host launches BETA only without split-K
  const bool fix_a = d.a_conj || d.a_mask == MASK_UNIT_LOWER;
  const bool fix_b = d.b_conj || d.b_mask == MASK_UNIT_LOWER;

  // this thread's copy slots: element e of A sits at tile (ia + e*dia, ka + e*dka),
  // element e of B at (kb_ + e*dkb, jb + e*djb)
  const int ia = d.a_row ? tid / G_BK : tid % BM;
  const int ka = d.a_row ? tid % G_BK : tid / BM;
  const int dia = d.a_row ? G_NT / G_BK : 0;
  const int dka = d.a_row ? 0 : G_NT / BM;
  const int jb = d.b_row ? tid % G_BN : tid / G_BK;
  const int kb_ = d.b_row ? tid / G_BN : tid % G_BK;
  const int djb = d.b_row ? 0 : G_NT / G_BK;
  const int dkb = d.b_row ? G_NT / G_BN : 0;
  // theta: local column -> (d, r) -> global column (d.N when r is out of range)
  auto bcol = [&](int jj) -> int {
    if (THETA) {
      const int r = j0 + 16 * (jj >> 5) + ((jj >> 1) & 15);
      return r < te.cr ? (jj & 1) * te.cr + r : d.N;
    }
    return j0 + jj;
  };

  auto issue = [&](int slice) {
    const int stage = slice % kStages;
    const int k0 = kbeg + slice * G_BK;
    c64* as = As + stage * G_BK * LAS;
    c64* bs = Bs + stage * G_BK * LBS;
#pragma unroll
    for (int e = 0; e < EA; ++e) {
      const int ii = ia + e * dia, kk = ka + e * dka;
      const int i = i0 + ii, k = k0 + kk;
      int kind = 0;
      const c64* src = d.A;
      if (i < d.M && k < kend) {
        kind = d.a_row ? mask_kind(d.a_mask, k, i) : mask_kind(d.a_mask, i, k);
        src = d.a_row ? d.A + ((int64_t)i * d.lda + k) : d.A + (i + (int64_t)k * d.lda);
      }
      cp_async8(smem_u32(as + kk * LAS + ii), src, kind == 1 ? 8 : 0);
    }
#pragma unroll
    for (int e = 0; e < EB; ++e) {
      const int jj = jb + e * djb, kk = kb_ + e * dkb;
      const int j = bcol(jj), k = k0 + kk;
      int kind = 0;
      const c64* src = d.B;
      if (j < d.N && k < kend) {
        kind = d.b_row ? mask_kind(d.b_mask, j, k) : mask_kind(d.b_mask, k, j);
        src = d.b_row ? d.B + ((int64_t)k * d.ldb + j) : d.B + (k + (int64_t)j * d.ldb);
      }
      cp_async8(smem_u32(bs + kk * LBS + jj), src, kind == 1 ? 8 : 0);
    }
  };
  // after this thread's copies of `slice` have landed: unit diagonals,
  // conjugation and alpha on the elements it copied
  auto fixup = [&](int slice) {
    const int stage = slice % kStages;
    const int k0 = kbeg + slice * G_BK;
    if (fix_a) {
      c64* as = As + stage * G_BK * LAS;
#pragma unroll
      for (int e = 0; e < EA; ++e) {
        const int ii = ia + e * dia, kk = ka + e * dka;
        const int i = i0 + ii, k = k0 + kk;
        if (i >= d.M || k >= kend) continue;
        const int kind = d.a_row ? mask_kind(d.a_mask, k, i) : mask_kind(d.a_mask, i, k);
        c64* p = as + kk * LAS + ii;
        c64 v = kind == 2 ? mk<float>(1.f, 0.f) : *p;
        if (d.a_conj) v = cconj(v);
        *p = v;
      }
    }
    if (fix_b) {
      c64* bs = Bs + stage * G_BK * LBS;
#pragma unroll
      for (int e = 0; e < EB; ++e) {
        const int jj = jb + e * djb, kk = kb_ + e * dkb;
        const int j = bcol(jj), k = k0 + kk;
        if (j >= d.N || k >= kend) continue;
        const int kind = d.b_row ? mask_kind(d.b_mask, j, k) : mask_kind(d.b_mask, k, j);
        c64* p = bs + kk * LBS + jj;
        c64 v = kind == 2 ? mk<float>(1.f, 0.f) : *p;
        if (d.b_conj) v = cconj(v);
        *p = v;
      }
    }
  };

  const int nslices = kend > kbeg ? (kend - kbeg + G_BK - 1) / G_BK : 0;
#pragma unroll
  for (int s = 0; s < kStages - 1; ++s) {
    if (s < nslices) issue(s);
    cp_async_commit();
  }

  float acc[2 * RG][8][2];
  {
#pragma unroll
    for (int a = 0; a < 2 * RG; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) acc[a][b][0] = acc[a][b][1] = 0.f;
  }

  for (int s = 0; s < nslices; ++s) {
    cp_async_wait<kStages - 2>();  // this thread's copies of slice s have landed
    if (fix_a || fix_b) fixup(s);
    __syncthreads();  // slice s visible to all; slice s-1's buffer free
    if (s + kStages - 1 < nslices) issue(s + kStages - 1);
    cp_async_commit();
    const c64* Ab = As + (s % kStages) * G_BK * LAS + 2 * tm;
    const c64* Bb = Bs + (s % kStages) * G_BK * LBS + 2 * tn;
    // partially unrolled: a fully unrolled slice overflows the instruction cache
#pragma unroll 4
    for (int kk = 0; kk < G_BK; ++kk) {
      float4 av[RG], bv[4];
#pragma unroll
      for (int g = 0; g < RG; ++g) av[g] = *reinterpret_cast<const float4*>(Ab + kk * LAS + 32 * g);
#pragma unroll
      for (int h = 0; h < 4; ++h) bv[h] = *reinterpret_cast<const float4*>(Bb + kk * LBS + 32 * h);
#pragma unroll
      for (int g = 0; g < RG; ++g)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const float ar = e ? av[g].z : av[g].x, ai = e ? av[g].w : av[g].y;
#pragma unroll
          for (int h = 0; h < 4; ++h)
#pragma unroll
            for (int f = 0; f < 2; ++f) {
              const float br = f ? bv[h].z : bv[h].x, bi = f ? bv[h].w : bv[h].y;
              float* c = acc[2 * g + e][2 * h + f];
              c[0] = fmaf(ar, br, c[0]);
              c[0] = fmaf(-ai, bi, c[0]);
              c[1] = fmaf(ar, bi, c[1]);
              c[1] = fmaf(ai, br, c[1]);
            }
        }
    }
  }
  cp_async_wait<0>();  // nothing may be in flight when the CTA leaves

  if constexpr (THETA) {
    // theta[(l,a),(b,r)] = sum_{c,d} g[2a+b][2c+d] X[(l,c),(d,r)]
#pragma unroll
    for (int g = 0; g < RG; ++g) {
      const int l = i0 / 2 + 16 * g + tm;
      if (2 * l >= d.M) continue;
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const int r = j0 + 16 * h + tn;
        if (r >= te.cr) continue;
        c64 X[2][2];
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
          for (int dd = 0; dd < 2; ++dd)
            X[c][dd] = mk<float>(acc[2 * g + c][2 * h + dd][0], acc[2 * g + c][2 * h + dd][1]);
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          c64 v[2];
#pragma unroll
          for (int a = 0; a < 2; ++a) {
            c64 s = mk<float>(0.f, 0.f);
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
              for (int dd = 0; dd < 2; ++dd) {
                const int gi = (2 * a + b) * 4 + 2 * c + dd;
                cfma(s, te.gdev ? te.gdev[gi] : te.g[gi], X[c][dd]);
              }
            v[a] = s;
          }
          c64* dst = te.W + (int64_t)(b * te.cr + r) * te.ldw + 2 * l;
          dst[0] = v[0];
          dst[1] = v[1];
        }
      }
    }
  } else {
    // destination: C, or this split's slice of the workspace (leading dimension M)
    c64* dst = split ? d.wk + (int64_t)blockIdx.z * d.M * d.N : d.C;
    const int64_t ldd = split ? d.M : d.ldc;
    // 16-byte accesses where allowed (the 128-row kernel without C reads keeps
    // scalar stores: measured faster there)
    const bool dvec = (BETA || BM == 64) && ((reinterpret_cast<uintptr_t>(dst) & 15) == 0) && ((ldd & 1) == 0);
    const bool alpha_one = split || (d.alpha.re == 1.f && d.alpha.im == 0.f);
    float sq[4][2] = {};  // colsq: this thread's rows of each of its columns
#pragma unroll
    for (int g = 0; g < RG; ++g) {
      const int i = i0 + 32 * g + 2 * tm;
      if (i >= d.M) continue;
      const bool pair = i + 1 < d.M;
      // C of this row group, all loads issued before the group's first store (a
      // store to C could alias a later load, so the compiler would otherwise keep
      // each load behind the previous store and pay one memory latency per pair)
      float4 cin[4][2];
      if constexpr (beta_nz) {
#pragma unroll
        for (int h = 0; h < 4; ++h)
#pragma unroll
          for (int f = 0; f < 2; ++f) {
            const int j = j0 + 32 * h + 2 * tn + f;
            cin[h][f] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (j >= d.N) continue;
            const c64* cp = dst + i + (int64_t)j * ldd;
            if (dvec && pair) {
              cin[h][f] = *reinterpret_cast<const float4*>(cp);
            } else {
              cin[h][f].x = cp[0].re;
              cin[h][f].y = cp[0].im;
              if (pair) {
                cin[h][f].z = cp[1].re;
                cin[h][f].w = cp[1].im;
              }
            }
          }
      }
#pragma unroll
      for (int h = 0; h < 4; ++h)
#pragma unroll
        for (int f = 0; f < 2; ++f) {
          const int j = j0 + 32 * h + 2 * tn + f;
          if (j >= d.N) continue;
          c64* cp = dst + i + (int64_t)j * ldd;
          c64 v0 = mk<float>(acc[2 * g][2 * h + f][0], acc[2 * g][2 * h + f][1]);
          c64 v1 = mk<float>(acc[2 * g + 1][2 * h + f][0], acc[2 * g + 1][2 * h + f][1]);
          if (!alpha_one) {
            v0 = d.alpha * v0;
            v1 = d.alpha * v1;
          }
          if constexpr (beta_nz) {  // C = alpha sum + beta C, the sum rounded on its own first
            v0 = v0 + d.beta * mk<float>(cin[h][f].x, cin[h][f].y);
            v1 = v1 + d.beta * mk<float>(cin[h][f].z, cin[h][f].w);
          }
          if (dvec && pair) {
            *reinterpret_cast<float4*>(cp) = make_float4(v0.re, v0.im, v1.re, v1.im);
          } else {
            cp[0] = v0;
            if (pair) cp[1] = v1;
          }
          if constexpr (beta_nz) {
            sq[h][f] += fmaf(v0.re, v0.re, v0.im * v0.im);
            if (pair) sq[h][f] += fmaf(v1.re, v1.re, v1.im * v1.im);
          }
        }
    }
    if constexpr (beta_nz && BM == 64) {
      // column sums over the tile's 64 rows: the 16 threads of a column (tm, the
      // lane's low four bits) combine theirs, the first writes
      if (d.colsq) {
#pragma unroll
        for (int h = 0; h < 4; ++h)
#pragma unroll
          for (int f = 0; f < 2; ++f) {
            float v = sq[h][f];
#pragma unroll
            for (int o = 1; o < 16; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            const int j = j0 + 32 * h + 2 * tn + f;
            if (tm == 0 && j < d.N) d.colsq[(int64_t)blockIdx.x * d.ldcs + j] = v;
          }
      }
    }
  }
}

template <int BM, bool THETA, bool BETA>
cudaError_t launch(const GemmDesc<c64>& d, const ThetaEpi& te, dim3 grid, cudaStream_t s) {
  // the attribute is set once per device and instantiation
  static PerDevice once;
  cudaError_t attr = cudaSuccess;
  once.get([&attr]() -> long long {
    attr = cudaFuncSetAttribute(gemm_c64_kernel<BM, THETA, BETA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                g_smem_bytes<BM>());
    return attr == cudaSuccess ? 1 : -1;
  });
  if (attr != cudaSuccess) return attr;
  gemm_c64_kernel<BM, THETA, BETA><<<grid, G_NT, g_smem_bytes<BM>(), s>>>(d, te);
  return cudaGetLastError();
}

}  // namespace

// 128-row tiles for long contractions; 64-row tiles (two CTAs per SM) for
// short ones, whose time goes into reading and writing C
int gemm_c64_tile_rows(int M, int K) { return (M > 64 && K > 64) ? 128 : 64; }

cudaError_t gemm_c64(const GemmDesc<c64>& d, cudaStream_t s) {
  ThetaEpi te{};
  const int BM = gemm_c64_tile_rows(d.M, d.K);
  dim3 grid((d.M + BM - 1) / BM, (d.N + G_BN - 1) / G_BN, d.splitk > 1 ? d.splitk : 1);
  if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidConfiguration;
  const bool beta = d.splitk <= 1 && !(d.beta.re == 0.f && d.beta.im == 0.f);
  if (BM == 128) return beta ? launch<128, false, true>(d, te, grid, s) : launch<128, false, false>(d, te, grid, s);
  return beta ? launch<64, false, true>(d, te, grid, s) : launch<64, false, false>(d, te, grid, s);
}

cudaError_t theta_c64(int cl, int cm, int cr, const c64* A, const c64* B, const c64* g16, c64* W, int64_t ldw,
                      cudaStream_t s, const c64* gdev) {
  GemmDesc<c64> d;
  d.M = 2 * cl;
  d.N = 2 * cr;
  d.K = cm;
  d.alpha = mk<float>(1.f, 0.f);
  d.beta = mk<float>(0.f, 0.f);
  d.A = A;
  d.lda = cm;
  d.a_row = 1;
  d.B = B;
  d.ldb = 2 * cr;
  d.b_row = 1;
  ThetaEpi te;
  te.cr = cr;
  for (int q = 0; q < 16; ++q) te.g[q] = g16[q];
  te.gdev = gdev;
  te.W = W;
  te.ldw = ldw;
  dim3 grid((d.M + 127) / 128, (cr + G_BN / 2 - 1) / (G_BN / 2), 1);
  if (grid.y > 65535) return cudaErrorInvalidConfiguration;
  return launch<128, true, false>(d, te, grid, s);
}

}  // namespace mpsg
