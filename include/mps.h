/*
 * mps.h — C ABI of the GB300 matrix-product-state two-site gate engine.
 *
 * The engine evolves a matrix product state (MPS) of n qubits under one- and
 * two-qubit gates (Sec. II-B.1 MPS definition; Sec. III-C tensor application
 * and site permutation).  A two-qubit gate on neighbouring sites (i, i+1):
 *
 *   1. contracts A_i (chi_l x 2 x chi_m) and A_{i+1} (chi_m x 2 x chi_r) over
 *      their shared bond (Sec. III-B.1 bond contraction) and the 4x4 gate into
 *      the physical indices, giving theta as a (2 chi_l) x (2 chi_r) matrix
 *      with row (l, a) and column (b, r);
 *   2. splits theta by a column-pivoted Householder QR, theta P = Q R
 *      (Sec. III-B.2, Table of decomposition routines: QR with pivoting),
 *      stopped after k = min(2 chi_l, 2 chi_r, chi_max) pivots;
 *   3. stores Q[:, :k] as the new A_i (chi_l x 2 x k) and R[:k, :] P^T as the
 *      new A_{i+1} (k x 2 x chi_r).  The state is not renormalised: its squared
 *      norm is the norm fidelity F = <psi|psi> of Sec. III-E.
 *   A handle created with truncation = MPS_TRUNC_SVD splits theta by its SVD
 *   theta = U S V^dagger instead (the same table's SVD row, compared with
 *   pivoted QR in Sec. IV-A.1): A_i = U[:, :k], A_{i+1} = diag(S[:k]) V^dagger[:k, :].
 *
 * Conventions
 *   - Site layout: row-major (chi_l, 2, chi_r), the flat row-major layout of
 *     Sec. III-A.1.  Site 0 holds the most significant bit of a basis index
 *     (tensor-product order of Sec. II-A.1).  chi_0 = chi_n = 1.
 *   - One-qubit gate u[out*2 + in].  Two-qubit gate g[(2a+b)*4 + (2c+d)],
 *     row = output; a/c label the first listed qubit, b/d the second.
 *   - Bond dimensions grow structurally: a split always keeps
 *     k = min(2 chi_l, 2 chi_r, chi_max) columns, with no rank tolerance.
 *   - Policies: MPS_POLICY_CANON keeps one orthogonality centre and moves it to
 *     site i (QR rightward / LQ leftward, no truncation; Sec. III-C.1) before a
 *     gate on (i, i+1); afterwards the centre is i+1.  MPS_POLICY_LOCAL never
 *     moves the centre (each split truncates its own theta).
 *   - Precisions: MPS_PREC_FP64 stores complex128 and computes in FP64.
 *     MPS_PREC_MIXED stores complex64, runs the contractions and the QR bulk in
 *     FP32-class arithmetic, and keeps column norms, reflector norms/beta/tau
 *     and pivot comparisons in FP64.
 *
 * Ownership and errors
 *   - Host arrays passed in are read before the call returns; host arrays
 *     passed out are written before it returns.  The library owns all device
 *     memory of a handle (allocated at create, sized for the largest bond
 *     dims the chain and chi_max allow), except in the raw-pointer calls
 *     (mps_two_site_*), where the caller owns every buffer.
 *   - Every call returns MPS_OK (0) or a negative MPS_E_* code.  Mutating calls
 *     are asynchronous on the handle's stream; device-side failures (a bounded
 *     wait that expired, a failed index check) surface at the next synchronous
 *     call (mps_sync, mps_amplitude, mps_fidelity_estimate, mps_overlap,
 *     mps_get_site, mps_discarded_weight).  After such a failure the handle
 *     rejects further mutation with MPS_E_STATE; mps_last_error() describes it.
 *     Index checks: the kernels that take indices from device data (the pivot
 *     permutation of a split, the column swaps of randomized pivoting) check
 *     them in the library built with -DMPS_BOUNDS_CHECK, and a value out of
 *     range then records the failure (MPS_E_CUDA, "device-side check failed")
 *     instead of an access out of range; the ordinary build leaves them out.
 *   - A handle is not thread-safe; distinct handles may be used from distinct
 *     threads, and on distinct devices.  What the library sets up at first use
 *     (kernel attributes, occupancy, cluster sizes) is kept per device. */
#ifndef MPS_GB300_H
#define MPS_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* The library is built with hidden symbol visibility; the declarations of this header
 * are its only exports. */
#if defined(__GNUC__)
#pragma GCC visibility push(default)
#endif

#define MPS_OK 0
#define MPS_E_ARG (-1)         /* invalid argument (checked on the host, nothing launched) */
#define MPS_E_NOMEM (-2)       /* a device or pinned-host allocation failed */
#define MPS_E_CUDA (-3)        /* a CUDA runtime call failed (message in mps_last_error) */
#define MPS_E_TIMEOUT (-4)     /* a bounded device-side wait expired */
#define MPS_E_STATE (-5)       /* handle is in an error state, or call invalid in this state */
#define MPS_E_UNSUPPORTED (-6) /* request outside what this build supports */

#define MPS_PREC_FP64 0
#define MPS_PREC_MIXED 1

#define MPS_POLICY_CANON 0
#define MPS_POLICY_LOCAL 1

/* mps_config.truncation: how a two-site block is split and truncated */
#define MPS_TRUNC_QRCP 0 /* truncated column-pivoted Householder QR (default; Sec. III-B.2) */
#define MPS_TRUNC_SVD 1  /* truncated SVD by one-sided Jacobi (Sec. III-B.2 Table III, Sec. IV-A.1):
                            the k largest singular values are kept, so the discarded weight is the
                            least any rank-k split can reach.  Needs 2 (2 chi)^2 more elements of
                            device memory, limits the handle to chi_max <= 4096, and is much slower
                            than QRCP: every sweep of the Jacobi iteration touches all column pairs. */

#define MPS_TRUNC_RQRCP 2 /* truncated QR with randomized column pivoting (blocked RQRCP of Duersch-Gu and
                            Martinsson et al.; one of the QR improvements Sec. IV-A.1 points to): the
                            pivots of each block of twice the panel width (64 columns by default)
                            come from a pivoted QR of a small random sketch Y = Omega theta (block
                            width + 8 rows, entries +-1
                            from SplitMix64 with state sketch_seed + s for the s-th two-site split of
                            the handle), the block itself is factored without pivoting and applied as
                            one block reflector, and the sketch is updated as Y2 -= Y1 R11^{-1} R12.
                            Pivots, and so the truncated state, differ from MPS_TRUNC_QRCP's; the
                            kept rank and the norm identity are the same.  Layers run gate by gate. */

/* host element formats for mps_get_site / mps_set_site */
#define MPS_HOST_C128 0
#define MPS_HOST_C64 1

/* mps_config.flags */
#define MPS_FLAG_PROFILE 1          /* time the tracked kernels with CUDA events (mps_kernel_stats) */
#define MPS_FLAG_AUTOTUNE 4         /* choose the QR panel width and the pivoted panel kernel's CTA count of
                                       every two-site split shape (precision, 2 chi_l, 2 chi_r, k) by timing
                                       the candidates on the first split of that shape (see
                                       mps_tune_two_site); layers use the choice too.  Off by default: the
                                       choice can change the rounding, though not the bars of the results. */
#define MPS_FLAG_NO_GRAPH 8         /* issue every mps_apply_layer call directly instead of capturing
                                       it into a CUDA graph (see mps_apply_layer) */
#define MPS_FLAG_TENSOR_CORES 2     /* mixed precision: long-K complex products (theta, centre-move
                                       absorption) on the tcgen05 tensor cores with 3xTF32 splitting.
                                       Off by default: the tensor cores' FP32 accumulation drifts
                                       linearly with K (about 6e-5 relative at K = 4096 on GB300),
                                       above the CUDA-core path's 1e-7. */

typedef struct mps_s* mps_t;
typedef struct {
  double re, im;
} mps_c128;
typedef struct {
  float re, im;
} mps_c64;

typedef void* (*mps_alloc_fn)(size_t bytes, void* ctx);
typedef void (*mps_free_fn)(void* ptr, void* ctx);

typedef struct {
  int precision;          /* MPS_PREC_FP64 (default) or MPS_PREC_MIXED */
  int policy;             /* MPS_POLICY_CANON (default) or MPS_POLICY_LOCAL */
  int device;             /* CUDA device ordinal; default 0 */
  void* stream;           /* cudaStream_t to run on; NULL = the library creates one */
  int panel_width;        /* QR panel width nb in [1, 32]; 0 = default (32) */
  double wait_timeout_s;  /* limit of every device-side wait; 0 = default (10 s) */
  mps_alloc_fn alloc;     /* optional device allocator; NULL = cudaMalloc */
  mps_free_fn free;       /* must be given together with alloc */
  void* alloc_ctx;        /* passed to alloc/free */
  int flags;              /* MPS_FLAG_* */
  int debug_barrier_extra; /* testing only, normally 0: a grid barrier waits for this many
                              arrivals that never come, so every bounded wait expires and
                              the call fails with MPS_E_TIMEOUT instead of hanging */
  int debug_max_ctas;     /* testing only, normally 0: caps the CTAs of the cooperative QR
                             panel kernel so that small matrices take the paths of large
                             ones (more than 128 rows per CTA); negative: MPS_E_ARG */
  int truncation;         /* MPS_TRUNC_QRCP (default), MPS_TRUNC_SVD or MPS_TRUNC_RQRCP */
  int sketch_seed;        /* MPS_TRUNC_RQRCP: generator state of the first split's sketch (default 0) */
  int reserved[4];
} mps_config;

/* Fill *cfg with the defaults listed above. */
void mps_config_init(mps_config* cfg);

/* Create the state |0...0> of n qubits (every site [1,0], all bonds 1;
 * Sec. II-B.1), FP64 path, canonical policy, centre at site 0.
 * n >= 1, chi_max >= 1.  Device memory for every site is reserved up front
 * for bond dims min(2^b, 2^(n-b), chi_max). */
int mps_create(mps_t* out, int n, int chi_max);
/* As mps_create with an explicit configuration (NULL = defaults). */
int mps_create_ex(mps_t* out, int n, int chi_max, const mps_config* cfg);
/* Release the handle and all its device memory.  NULL is accepted. */
int mps_destroy(mps_t h);

/* One-qubit gate on `site` (Sec. II-A.2): A[l,s,r] <- sum_s' u[s*2+s'] A[l,s',r]. */
int mps_apply_1q(mps_t h, int site, const mps_c128 u[4]);

/* Two-qubit gate g on (site, site+1), split by truncated pivoted QR as in the
 * header comment (Sec. III-C.2, III-B.2), or by the truncated SVD when the handle
 * was created with truncation = MPS_TRUNC_SVD (left site U[:, :k], right site
 * diag(S[:k]) V^dagger[:k, :], same k).  chi_max (<= the handle's) caps the
 * new bond; chi_max <= 0 means the handle's value. */
int mps_apply_2q(mps_t h, int site, const mps_c128 g[16], int chi_max);

/* SWAP of the qubits on (site, site+1): the two-site path with the SWAP gate,
 * theta[l,a,b,r] = X[l,b,a,r] (Sec. III-C.4 site permutation). */
int mps_swap(mps_t h, int site, int chi_max);

/* Two-qubit gate on the ordered pair of positions (q1, q2), not necessarily
 * adjacent (Sec. III-C.4, Sec. III-D.2 SWAP approach).  With lo < hi the
 * qubit at lo is moved right by SWAPs on bonds (lo,lo+1) .. (hi-2,hi-1), the
 * gate is applied on (hi-1, hi), and the SWAPs are undone in reverse order. */
int mps_apply_2q_routed(mps_t h, int q1, int q2, const mps_c128 g[16], int chi_max);

/* Site permutation by nearest-neighbour SWAPs in bubble-sort order (Sec. III-C,
 * "Site permutation"; the re-embedding between horizontal and vertical nearest
 * neighbours of Sec. III-D.2).  order[p] (a permutation of 0..n-1) is the current
 * position of the site that must end at position p.  Each pass walks the chain
 * left to right and applies mps_swap(p, chi_max) where the target positions of
 * sites p and p+1 are out of order, until none is: the number of SWAPs is the
 * number of inversions of the permutation, written to *swaps when swaps != NULL.
 * Every SWAP truncates like a gate.  Host-side validation (MPS_E_ARG for a bad
 * order) happens before any SWAP; asynchronous otherwise. */
int mps_permute(mps_t h, const int* order, int chi_max, long long* swaps);

/* The site permutation of mps_permute as a pipeline of layers: odd-even
 * transposition sort, the parallel form of that bubble sort (Sec. III-C site
 * permutation; the re-embeddings of Sec. III-D.2).  Pass t takes the pairs
 * (q, q+1) with q of the parity of t whose target positions are out of order;
 * those SWAPs act on disjoint bonds and run as one mps_apply_layer call (its
 * concurrent lanes).  Passes alternate until an even and an odd pass in a row
 * find nothing to swap (at most n passes).  The SWAP count is again the number
 * of inversions (*swaps), *passes the number of layers run (either may be
 * NULL).  Requires MPS_POLICY_LOCAL (MPS_E_STATE otherwise); every SWAP
 * truncates like a gate, so the state equals applying the passes' SWAPs one by
 * one in pass order, which differs from mps_permute's order once truncation
 * acts.  Host-side validation first; asynchronous otherwise. */
int mps_permute_layers(mps_t h, const int* order, int chi_max, long long* swaps, int* passes);

/* All two-qubit gates of one circuit layer, on pairwise disjoint bonds
 * sites[j], sites[j]+1 (gates[16*j .. 16*j+15]) (the gates of a brick-wall
 * layer, Sec. III-D; network parallelism, Sec. I).  Requires MPS_POLICY_LOCAL
 * (no centre moves, so the gates commute exactly).  Gates whose two-site block
 * fits one CTA (at most 64 x 64) run together as one grouped launch, one CTA
 * per gate (32 gates per launch); gates whose block is at most 4096 x 4096 run
 * concurrently on eight internal streams, each with its own workspace
 * (allocated through the handle's allocator at the first call, about 8 x the
 * workspace of a chi = 2048 split); larger ones run in order on the handle's
 * stream, which waits for all of them before returning.  From the second call
 * on, the layer's launches are captured into a CUDA graph and replayed; a
 * layer of the same shape (sites, bond dims, bond cap) reuses the handle's
 * executable graph, updated with the new gates (MPS_FLAG_NO_GRAPH: direct
 * launches; a stream that cannot be captured turns graphs off for the handle).
 * The result equals applying the gates one by one, bit for bit; with
 * MPS_FLAG_PROFILE the gates run one by one.  Asynchronous; errors as for
 * mps_apply_2q.  chi_max as for mps_apply_2q. */
int mps_apply_layer(mps_t h, const int* sites, const mps_c128* gates, int count, int chi_max);

/* Matrix product operator on sites first .. first+count-1, applied by zip-up
 * (Sec. III-C.3; the IQFT's controlled-phase MPOs of Sec. III-D.1 have bond 2).
 * bonds[0..count] are the MPO's bond dims: bonds[0] = bonds[count] = 1 and
 * 1 <= bonds[j] <= 2 (larger: MPS_E_UNSUPPORTED).  W holds the site tensors one
 * after another, site j as W_j[a][b][out][in] (a < bonds[j], b < bonds[j+1],
 * row-major, bonds[j] * bonds[j+1] * 4 entries).  Left to right, the carried block
 * times site j and W_j form Z[(kk, out), (b, r)], which the truncated pivoted QR
 * splits (Q to the site, R P^T carried on; k = min(rows, columns, chi_max, room));
 * the last Z is the last site.  The room reserved for a bond is twice the chain's
 * bound min(2^b, 2^(n-b), chi_max) (at most chi_max), so one MPO of bond 2 is never
 * truncated for lack of room; bonds left above the chain's bound are then brought
 * back to it by splitting the identity two-site gate, right to left (exact under
 * the canonical policy).  Under MPS_POLICY_CANON the centre is moved to `first`
 * before and is at the last recompressed site (or `last`) after.  The zip-up splits
 * are pivoted QRs whatever the handle's truncation setting; the recompression splits
 * follow it.  count = 1 applies W_0[0][0] as a one-qubit gate.  chi_max <= 0: the
 * handle's.  Asynchronous. */
int mps_apply_mpo(mps_t h, int first, int count, const int* bonds, const mps_c128* W, int chi_max);

/* <bits|psi> = A_0[:, b_0, :] A_1[:, b_1, :] ... (bits[i] in {0,1} for site i).
 * Synchronous. */
int mps_amplitude(mps_t h, const uint8_t* bits, mps_c128* out);

/* Norm fidelity F = <psi|psi> (Sec. III-E).  Canonical policy: the squared
 * norm of the centre site; local policy: full transfer-matrix contraction.
 * Synchronous; accumulated in FP64 for both precisions. */
int mps_fidelity_estimate(mps_t h, double* out);

/* <a|b> by transfer-matrix contraction in FP64 (both handles must have the
 * same n; precisions may differ).  Synchronous. */
int mps_overlap(mps_t a, mps_t b, mps_c128* out);

/* Copy the n+1 bond dimensions into out[0..n]. */
int mps_bond_dims(mps_t h, int* out);

/* Copy site `site` (chi_l*2*chi_r elements, row-major) to host memory in
 * format host_fmt (MPS_HOST_C128 / MPS_HOST_C64).  cap_elems = capacity of
 * `host` in elements; MPS_E_ARG if too small.  Synchronous. */
int mps_get_site(mps_t h, int site, int host_fmt, void* host, size_t cap_elems);

/* Overwrite site `site` with a host array of shape (chi_l, 2, chi_r).  The
 * bond dims must agree with the neighbours once all sites of a change are set;
 * mps_set_site itself only checks chi_l/chi_r against the reserved capacity.
 * Stream-ordered: `host` is read before return (pinned or pageable). */
int mps_set_site(mps_t h, int site, int chi_l, int chi_r, int host_fmt, const void* host);

/* Declare that the state is in mixed-canonical form with centre `centre`
 * (caller's guarantee, e.g. after loading sites).  No data is touched. */
int mps_set_centre(mps_t h, int centre);
int mps_get_centre(mps_t h, int* out);
/* Move the orthogonality centre to `target` (QR / LQ without truncation,
 * Sec. III-C.1). */
int mps_move_centre(mps_t h, int target);

/* Sum and count of the discarded weights ||theta_trailing||_F^2 of all
 * two-site splits so far.  Synchronous. */
int mps_discarded_weight(mps_t h, double* total, long long* count);

/* Iteration record of the most recent SVD split (handles created with
 * truncation = MPS_TRUNC_SVD): *sweeps = Jacobi sweeps run (the last one found
 * every pair orthogonal; kSvdMaxSweeps + 1 = stopped at the sweep limit), and
 * *rotations = plane rotations applied over all sweeps.  0 and 0 before the first
 * split.  MPS_E_STATE on a QRCP handle.  Synchronous. */
int mps_svd_last_stats(mps_t h, int* sweeps, long long* rotations);

/* Column order of the most recent two-site split by pivoted QR that
 * mps_apply_2q, mps_swap or mps_apply_2q_routed made on this handle
 * (Sec. III-B.2, theta P = Q R): jpvt[t] for t < n is the column of theta,
 * numbered b*chi_r + r for column (b, r), at pivot position t; the first k are
 * the kept pivots in the order they were taken.  *n_out = n = 2 chi_r and
 * *k_out = k of that split.  MPS_E_STATE when the workspace has been used for
 * anything else since (a centre move, a layer, an MPO, an SVD split) or no
 * such split was made; MPS_E_ARG when cap < n.  Synchronous.  A diagnostic: it
 * lets a test check each pivot choice against an independent factorisation. */
int mps_last_split_pivots(mps_t h, int* jpvt, int cap, int* n_out, int* k_out);

/* Use `stream` (a cudaStream_t) for all further work; NULL = the handle's own. */
int mps_set_stream(mps_t h, void* stream);
/* Wait for all queued work; surfaces device-side errors. */
int mps_sync(mps_t h);
/* Last error message of the handle ("" if none).  Valid until the next call. */
const char* mps_last_error(mps_t h);

/* Layer calls so far, how many of them ran as a CUDA graph launch, and whether
 * graphs are still on for the handle (any pointer may be NULL). */
int mps_layer_stats(mps_t h, long long* layers, long long* graph_launches, int* graphs_on);

/* Kernel classes tracked by mps_kernel_stats. */
#define MPS_KCLASS_THETA 0  /* theta contraction + gate epilogue */
#define MPS_KCLASS_PANEL 1  /* pivoted-QR panel (per-step GEMV, pivots, reflectors) */
#define MPS_KCLASS_UPDATE 2 /* trailing / block-reflector GEMM updates */
#define MPS_KCLASS_NORMS 3  /* column-norm recompute */
#define MPS_KCLASS_FORMQ 4  /* Q formation */
#define MPS_KCLASS_SPLIT 5  /* site split / reshape / un-pivot */
#define MPS_KCLASS_OTHER 6  /* 1q gates, conversions, observables */
#define MPS_KCLASS_CANON 7  /* centre moves: plain QR / LQ, Q formation, absorption */
#define MPS_KCLASS_SVD 8    /* SVD split: Jacobi sweeps, singular values, split (MPS_TRUNC_SVD) */
#define MPS_KCLASS_COUNT 9

typedef struct {
  long long launches;   /* kernel launches of this class since the last reset */
  double ms;            /* summed CUDA-event time (only with MPS_FLAG_PROFILE) */
  double alg_bytes;     /* algorithmic HBM bytes of those launches */
  double alg_flops;     /* algorithmic real flops of those launches */
} mps_kstat;

/* Per-class launch counts (always) and event timings (MPS_FLAG_PROFILE).
 * out must hold MPS_KCLASS_COUNT entries.  Synchronous. */
int mps_kernel_stats(mps_t h, mps_kstat* out);
int mps_kernel_stats_reset(mps_t h);

/* ---------------------------------------------------------------------------
 * Raw-pointer two-site call (no handle).  The caller owns every buffer.
 *
 * Applies gate g to the two sites A (chi_l x 2 x chi_m) and B (chi_m x 2 x
 * chi_r), device arrays in the precision's element type (complex128 for
 * MPS_PREC_FP64, complex64 for MPS_PREC_MIXED), row-major, and writes
 * A_out (chi_l x 2 x k) and B_out (k x 2 x chi_r), k = min(2chi_l, 2chi_r,
 * chi_max) (Sec. III-C.2 with the split of Sec. III-B.2).  A_out may alias A
 * and B_out may alias B.  *discarded_dev (device double) receives the
 * discarded weight.  `workspace` must hold mps_two_site_workspace() bytes,
 * 256-byte aligned.  Asynchronous on `stream` (cudaStream_t, NULL = default).
 * The return code covers the host-side checks and the launches only.  These
 * calls have no handle to carry a device-side failure (a bounded wait that
 * expired, a failed check), so they report one by writing NaN to
 * *discarded_dev, stream-ordered after the split; A_out and B_out are then
 * undefined.  Callers that need to detect such failures pass discarded_dev. */
int mps_two_site_workspace(int precision, int chi_l, int chi_m, int chi_r, int chi_max,
                           size_t* bytes);
int mps_two_site_apply(int precision, int chi_l, int chi_m, int chi_r, int chi_max,
                       const void* A, const void* B, const mps_c128 g[16], void* A_out,
                       void* B_out, double* discarded_dev, void* workspace, size_t ws_bytes,
                       void* stream);

/* Autotuner of the two-site split (the paper tunes its block size chi_b by a sweep,
 * Sec. IV-A.3; here the knobs are GB300's): times one split of the shape
 * (chi_l, chi_m, chi_r, chi_max) in the given precision on seeded random sites with
 * every candidate QR panel width {32, 16, 8} x CTA count of the pivoted panel kernel
 * {all, 3/4, 1/2 of the SMs} and keeps the fastest, in a process-wide cache keyed by
 * (precision, 2 chi_l, 2 chi_r, k, SM count).  When the environment variable
 * MPS_TUNE_CACHE names a file, the cache is first filled from it and every new
 * entry is appended to it as one JSON object per line.  force = 0 returns a cached
 * entry without timing (out->candidates = 0).  Handles created with
 * MPS_FLAG_AUTOTUNE consult the same cache.  Allocates its own device memory on the
 * current device and synchronises.  MPS_E_ARG for bad sizes, MPS_E_NOMEM, MPS_E_CUDA. */
typedef struct {
  int panel_width;   /* chosen QR panel width nb */
  int panel_ctas;    /* chosen CTA count of the pivoted panel kernel */
  int candidates;    /* configurations timed (0: taken from the cache) */
  double ms;         /* one split with the chosen configuration (CUDA events, best of the runs) */
  double default_ms; /* one split with the defaults (panel width 32, every SM) */
} mps_tune_result;
int mps_tune_two_site(int precision, int chi_l, int chi_m, int chi_r, int chi_max, int force, mps_tune_result* out);

/* Testing only: every later raw-pointer call (mps_two_site_apply and
 * mps_two_site_apply_noalloc) bounds its device-side waits by timeout_s
 * (0 = the default, 10 s) and makes its grid barriers wait for barrier_extra
 * arrivals that never come (0 = normal operation), so a test can make a wait
 * expire and see the NaN discarded weight.  Process-wide; MPS_E_ARG for
 * negative values. */
int mps_debug_raw_wait(int barrier_extra, double timeout_s);

/* Workspace size of mps_two_site_apply_noalloc: 16 MiB. */
#define MPS_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)

/* mps_two_site_apply for callers that must not allocate device memory at all:
 * code that runs inside someone else's memory manager (an allocator callback,
 * a framework that owns every byte of the GPU), or a loop with a fixed memory
 * budget where a cudaMalloc could fail or synchronise the device at the wrong
 * moment.  The paper has no counterpart; this is a convenience of the library.
 *
 * Arguments and results are those of mps_two_site_apply minus the workspace:
 * the scratch space is one fixed device array inside the library,
 * MPS_NOALLOC_SCRATCH_BYTES long, which every GPU that loads the library keeps
 * until the process exits.  The call returns MPS_E_UNSUPPORTED, doing nothing,
 * when mps_two_site_workspace reports more than that (complex128 bonds of a
 * few hundred, complex64 ones somewhat larger).  The caller still owns and
 * passes A, B, A_out, B_out and discarded_dev.
 * All calls share that one array and it keeps whatever the last call left in
 * it (every call clears the parts that must start at zero itself): two calls
 * whose GPU work overlaps, on different streams or from threads the caller
 * does not order, race on it and must be serialised by the caller.
 * The first call on a device looks up the array's device address with that
 * device current (cudaGetSymbolAddress); make that first call before any
 * stream capture begins.  A device-side failure shows as a NaN discarded
 * weight, as for mps_two_site_apply; the array's error word is cleared by the
 * next call, so pass discarded_dev to see it. */
int mps_two_site_apply_noalloc(int precision, int chi_l, int chi_m, int chi_r, int chi_max, const void* A,
                               const void* B, const mps_c128 g[16], void* A_out, void* B_out,
                               double* discarded_dev, void* stream);

/* Built-in self-test of the tensor-core complex64 GEMM against the CUDA-core
 * one on seeded random operands (diagnostic; allocates its own device memory
 * on the current device and synchronises it).  theta = 0: C = alpha*op(A)op(B)
 * + beta*C, M x N x K, with the operand views of the library's GEMM: a_row
 * (A(i,k) = A[i*K + k], else A[i + k*M]), b_row (B(k,j) = B[k*N + j], else
 * B[k + j*K]), conj flags and masks (0 none, 1 unit lower, 2 upper).
 * theta = 1: the theta contraction with a fixed gate, chi_l = M, chi_r = N,
 * chi_m = K.  Outputs the largest absolute difference and the largest
 * absolute reference entry. */
int mps_selftest_gemm(int M, int N, int K, int a_row, int a_conj, int a_mask, int b_row, int b_conj, int b_mask,
                      int theta, unsigned seed, double* max_abs_err, double* max_abs_ref);

/* Library version (major*10000 + minor*100 + patch). */
int mps_version(void);

#if defined(__GNUC__)
#pragma GCC visibility pop
#endif

#ifdef __cplusplus
}
#endif

#endif /* MPS_GB300_H */
