// CPU oracle: plain Householder QR with (optional) column pivoting, complex FP64.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the GPU library links or calls this
// file; it exists so that tests and the benchmark's CPU-baseline leg can check
// and time the GPU path against a slow, obviously correct restatement.
//
// What it computes (Sec. III-B.2, Table "Tensor decomposition routines": QR with
// pivoting, M = Q R P^T; truncation of the bond as in Sec. III-C.2/III-C.4):
//
//   for j = 0 .. k-1  (k = min(m, n, kmax)):
//     1. c_t = || A[j:m, t] ||^2 for every t >= j, recomputed exactly from the
//        current matrix (no norm downdating);
//     2. p = argmax_t c_t, the lowest index on exact ties;
//     3. swap columns j and p of A and of jpvt;
//     4. build the reflector H_j = I - tau v v^H that maps x = A[j:m, j] to
//        (beta, 0, ..., 0) under H_j^H:  alpha = x_0,
//        beta = -sign(Re alpha) * ||x|| (sign(0) = +1),
//        tau = (beta - alpha) / beta,  v = (1, x_1.. / (alpha - beta));
//        when ||x_1..|| = 0 and Im alpha = 0, tau = 0 and H_j = I; also when
//        ||x||^2 is below the smallest normal double (the formula is undefined
//        there: the squares underflow and alpha - beta rounds to zero);
//     5. apply H_j^H = I - conj(tau) v v^H to A[j:m, j+1:n].
//   After k steps the first k rows of A hold R (upper trapezoidal), the
//   columns below the diagonal hold v (unit leading entry implicit) and the
//   discarded weight is || A[k:m, k:n] ||_F^2.
//
// With pivot = 0 steps 1-3 are skipped (plain QR, used to move the
// orthogonality centre, Sec. III-C.1).
//
// oracle_cpqr_replay runs the same steps with the pivot of every step given
// instead of chosen, and reports the chosen and the largest exact residual norm
// of each step.  The paper leaves ties between equal column norms open; with
// the replay a test can check that a pivot sequence chosen by another
// implementation is greedy at every step and compare its factors with those of
// that same sequence.
//
// Q[:, :k] = H_0 H_1 ... H_{k-1} I[:, :k] is formed by applying the reflectors
// one at a time from the last to the first.
//
// Matrices are column-major.  Per-column work may run on several OpenMP
// threads; every element is computed by one thread in a fixed order, so the
// result does not depend on the thread count.

#include <cfloat>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

struct cd {
  double re, im;
};

inline cd add(cd a, cd b) { return {a.re + b.re, a.im + b.im}; }
inline cd sub(cd a, cd b) { return {a.re - b.re, a.im - b.im}; }
inline cd mul(cd a, cd b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
inline cd conj(cd a) { return {a.re, -a.im}; }
inline cd scale(cd a, double s) { return {a.re * s, a.im * s}; }
inline double abs2(cd a) { return a.re * a.re + a.im * a.im; }
// a / b, textbook formula (the oracle's inputs keep |b| far from overflow).
inline cd divide(cd a, cd b) {
  double d = abs2(b);
  return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}

// Squared norm of column t, rows r0..m-1.
double col_norm2(const cd* A, int64_t lda, int m, int r0, int t) {
  const cd* c = A + (int64_t)t * lda;
  double s = 0.0;
  for (int r = r0; r < m; ++r) s += abs2(c[r]);
  return s;
}

// The factorisation of oracle_cpqr.  With `order` given (pivot mode only), step
// 2 takes the column whose original index is order[j] instead of the argmax and
// records its exact squared norm in chosen2[j] and the step's largest one in
// max2[j]: a replay of a pivot sequence chosen elsewhere.  Every other operation
// is the same as without `order`.
int cpqr_impl(int m, int n, int kmax, int pivot, cd* A, int64_t lda, cd* tau, int* jpvt, int* k_out,
              double* discarded, const int* order, double* chosen2, double* max2) {
  if (m < 0 || n < 0 || kmax < 0 || lda < (m > 1 ? m : 1)) return -1;
  int k = m < n ? m : n;
  if (kmax < k) k = kmax;
  for (int t = 0; t < n; ++t) jpvt[t] = t;
  std::vector<double> c(n > 0 ? n : 1);
  for (int j = 0; j < k; ++j) {
    if (pivot) {
      // 1. exact norms of the remaining columns
#pragma omp parallel for schedule(static)
      for (int t = j; t < n; ++t) c[t] = col_norm2(A, lda, m, j, t);
      // 2. pivot: largest norm, lowest index on ties
      int p = j;
      for (int t = j + 1; t < n; ++t)
        if (c[t] > c[p]) p = t;
      if (order) {  // replay: the given column, wherever it is now
        max2[j] = c[p];
        p = -1;
        for (int t = j; t < n; ++t)
          if (jpvt[t] == order[j]) p = t;
        if (p < 0) return -1;  // order[j] is not among the remaining columns
        chosen2[j] = c[p];
      }
      // 3. swap columns j and p
      if (p != j) {
        cd* a = A + (int64_t)j * lda;
        cd* b = A + (int64_t)p * lda;
        for (int r = 0; r < m; ++r) {
          cd tmp = a[r];
          a[r] = b[r];
          b[r] = tmp;
        }
        int ti = jpvt[j];
        jpvt[j] = jpvt[p];
        jpvt[p] = ti;
      }
    }
    // 4. reflector from x = A[j:m, j]
    cd* x = A + (int64_t)j * lda;
    cd alpha = x[j];
    double xnorm2 = 0.0;
    for (int r = j + 1; r < m; ++r) xnorm2 += abs2(x[r]);
    cd tj = {0.0, 0.0};
    if ((xnorm2 == 0.0 && alpha.im == 0.0) || abs2(alpha) + xnorm2 < DBL_MIN) {
      tj = {0.0, 0.0};  // H_j = I, column left as it is
    } else {
      double nrm = std::sqrt(alpha.re * alpha.re + alpha.im * alpha.im + xnorm2);
      double beta = alpha.re >= 0.0 ? -nrm : nrm;
      tj = {(beta - alpha.re) / beta, -alpha.im / beta};
      cd s = divide({1.0, 0.0}, sub(alpha, {beta, 0.0}));
      for (int r = j + 1; r < m; ++r) x[r] = mul(x[r], s);
      x[j] = {beta, 0.0};
    }
    tau[j] = tj;
    // 5. apply H_j^H = I - conj(tau) v v^H to the columns right of j
    if (tj.re != 0.0 || tj.im != 0.0) {
      cd ct = conj(tj);
#pragma omp parallel for schedule(static)
      for (int t = j + 1; t < n; ++t) {
        cd* a = A + (int64_t)t * lda;
        cd d = a[j];  // v_j = 1
        for (int r = j + 1; r < m; ++r) d = add(d, mul(conj(x[r]), a[r]));
        cd f = mul(ct, d);
        a[j] = sub(a[j], f);
        for (int r = j + 1; r < m; ++r) a[r] = sub(a[r], mul(x[r], f));
      }
    }
  }
  double disc = 0.0;
  for (int t = k; t < n; ++t) disc += col_norm2(A, lda, m, k, t);
  *k_out = k;
  *discarded = disc;
  return 0;
}

}  // namespace

extern "C" {

// Truncated (column-pivoted) Householder QR, in place.
//   A     : m x n column-major, lda >= m; overwritten as described above.
//   tau   : out, k entries.
//   jpvt  : out, n entries; jpvt[t] = original index of the column now at t.
//   k_out : out, number of reflectors k = min(m, n, kmax).
//   discarded : out, ||A[k:m, k:n]||_F^2 after the k steps.
// Returns 0, or -1 on a bad argument.
int oracle_cpqr(int m, int n, int kmax, int pivot, void* A_, int64_t lda, void* tau_, int* jpvt,
                int* k_out, double* discarded) {
  return cpqr_impl(m, n, kmax, pivot, static_cast<cd*>(A_), lda, static_cast<cd*>(tau_), jpvt, k_out, discarded,
                   nullptr, nullptr, nullptr);
}

// The pivoted factorisation of oracle_cpqr with the pivot sequence given:
// order[j] (j < k) is the original index of the column taken at step j.  Writes
// what oracle_cpqr writes, plus chosen2[j] = exact squared residual norm of that
// column at step j and max2[j] = the largest one over all remaining columns, so
// a caller can check that every step took a greedy maximum (within a tolerance
// when several columns tie).  Returns -1 if order[j] is out of range or repeats.
int oracle_cpqr_replay(int m, int n, int kmax, const int* order, void* A_, int64_t lda, void* tau_, int* jpvt,
                       int* k_out, double* discarded, double* chosen2, double* max2) {
  if (!order || !chosen2 || !max2) return -1;
  return cpqr_impl(m, n, kmax, 1, static_cast<cd*>(A_), lda, static_cast<cd*>(tau_), jpvt, k_out, discarded, order,
                   chosen2, max2);
}

// Q[:, :k] = H_0 ... H_{k-1} I[:, :k] from the reflectors left in A by
// oracle_cpqr.  Q is m x k column-major with ldq >= m.
int oracle_form_q(int m, int k, const void* A_, int64_t lda, const void* tau_, void* Q_, int64_t ldq) {
  if (m < 0 || k < 0 || k > m || lda < (m > 1 ? m : 1) || ldq < (m > 1 ? m : 1)) return -1;
  const cd* A = static_cast<const cd*>(A_);
  const cd* tau = static_cast<const cd*>(tau_);
  cd* Q = static_cast<cd*>(Q_);
  for (int t = 0; t < k; ++t) {
    cd* q = Q + (int64_t)t * ldq;
    for (int r = 0; r < m; ++r) q[r] = {0.0, 0.0};
    q[t] = {1.0, 0.0};
  }
  for (int j = k - 1; j >= 0; --j) {
    cd tj = tau[j];
    if (tj.re == 0.0 && tj.im == 0.0) continue;
    const cd* v = A + (int64_t)j * lda;  // v[j] = 1 implicit, v[j+1..] stored
#pragma omp parallel for schedule(static)
    for (int t = j; t < k; ++t) {
      cd* q = Q + (int64_t)t * ldq;
      cd d = q[j];
      for (int r = j + 1; r < m; ++r) d = add(d, mul(conj(v[r]), q[r]));
      cd f = mul(tj, d);
      q[j] = sub(q[j], f);
      for (int r = j + 1; r < m; ++r) q[r] = sub(q[r], mul(v[r], f));
    }
  }
  return 0;
}

// Number of threads the OpenMP runtime will use (1 without OpenMP).
int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"
