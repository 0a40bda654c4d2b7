/* Dense FP64 state-vector oracle in plain C (test infrastructure only).
 *
 * amp(x) = <x| U_L ... U_1 |0^n>  (Sec. I: the amplitude a circuit's tensor network
 * contracts to; Sec. II-A).  The state is 2^n complex128 values, interleaved (re, im).
 * Qubit q is bit (n - 1 - q) of the flat index (qubit 0 most significant).  Gates are
 * applied one at a time, in circuit order, each as a d x d matrix U[out][in] on the
 * amplitudes that differ only in its qubits' bits; a 2-qubit gate on (a, b) has local
 * index 2*bit(a) + bit(b).  Nothing is fused, reordered or blocked beyond splitting the
 * independent amplitude groups of one gate over OpenMP threads.
 *
 * This file is the large-n counterpart of the numpy oracle in statevector.py (same
 * conventions); tests pin the two against each other on small circuits.  It is used
 * to write stored expected values (tests/golden) for circuits too large for numpy.
 */
#include <stdint.h>
#include <string.h>

typedef struct {
  double re, im;
} cplx;

static inline cplx cmul(cplx a, cplx b) {
  cplx r = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
  return r;
}
static inline cplx cadd(cplx a, cplx b) {
  cplx r = {a.re + b.re, a.im + b.im};
  return r;
}

/* insert a zero bit at position p of v */
static inline uint64_t insert_zero(uint64_t v, int p) {
  const uint64_t lo = v & ((1ull << p) - 1);
  return ((v >> p) << (p + 1)) | lo;
}

static void apply_1q(cplx* psi, int n, int q, const double* m) {
  const int p = n - 1 - q;
  const cplx u00 = {m[0], m[1]}, u01 = {m[2], m[3]}, u10 = {m[4], m[5]}, u11 = {m[6], m[7]};
  const int64_t groups = (int64_t)1 << (n - 1);
#pragma omp parallel for schedule(static)
  for (int64_t g = 0; g < groups; ++g) {
    const uint64_t i0 = insert_zero((uint64_t)g, p), i1 = i0 | (1ull << p);
    const cplx a0 = psi[i0], a1 = psi[i1];
    psi[i0] = cadd(cmul(u00, a0), cmul(u01, a1));
    psi[i1] = cadd(cmul(u10, a0), cmul(u11, a1));
  }
}

static void apply_2q(cplx* psi, int n, int qa, int qb, const double* m) {
  const int pa = n - 1 - qa, pb = n - 1 - qb;
  const int lo = pa < pb ? pa : pb, hi = pa < pb ? pb : pa;
  cplx u[4][4];
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) {
      u[r][c].re = m[2 * (4 * r + c)];
      u[r][c].im = m[2 * (4 * r + c) + 1];
    }
  const int64_t groups = (int64_t)1 << (n - 2);
#pragma omp parallel for schedule(static)
  for (int64_t g = 0; g < groups; ++g) {
    const uint64_t base = insert_zero(insert_zero((uint64_t)g, lo), hi);
    uint64_t idx[4];
    for (int l = 0; l < 4; ++l) /* local index l = 2*bit(a) + bit(b) */
      idx[l] = base | ((uint64_t)(l >> 1) << pa) | ((uint64_t)(l & 1) << pb);
    cplx in[4];
    for (int l = 0; l < 4; ++l) in[l] = psi[idx[l]];
    for (int r = 0; r < 4; ++r) {
      cplx acc = {0.0, 0.0};
      for (int c = 0; c < 4; ++c) acc = cadd(acc, cmul(u[r][c], in[c]));
      psi[idx[r]] = acc;
    }
  }
}

/* psi (2^n complex128, caller-owned) <- U_L ... U_1 |0^n>.
 * arity[g] in {1, 2}; qubits[2g], qubits[2g+1]; mats[32g ...] the compact d x d matrix,
 * row-major, interleaved (re, im).  Returns 0, or -1 on a bad argument. */
int sv_final_state(int n, int64_t n_gates, const int32_t* arity, const int32_t* qubits, const double* mats,
                   double* psi_out) {
  if (n < 1 || n > 34 || n_gates < 0) return -1;
  cplx* psi = (cplx*)psi_out;
  const int64_t dim = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < dim; ++i) psi[i].re = psi[i].im = 0.0;
  psi[0].re = 1.0;
  for (int64_t g = 0; g < n_gates; ++g) {
    const int32_t a = qubits[2 * g], b = qubits[2 * g + 1];
    if (arity[g] == 1) {
      if (a < 0 || a >= n) return -1;
      apply_1q(psi, n, a, mats + 32 * g);
    } else if (arity[g] == 2) {
      if (a < 0 || a >= n || b < 0 || b >= n || a == b) return -1;
      apply_2q(psi, n, a, b, mats + 32 * g);
    } else {
      return -1;
    }
  }
  return 0;
}
