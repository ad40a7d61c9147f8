/*
 * Plain CPU oracle of the state-vector gate engine.  TEST INFRASTRUCTURE ONLY:
 * the tests, the package smoke check and the benchmark's CPU-baseline leg are
 * the only code that may load it.  The product path never calls it and shares
 * no code, header, table or helper with it.
 *
 * What it computes (arxiv 2508.13615):
 *   - Sec. 2: every rank holds the same small gate ("logic") matrix, at most
 *     8x8, and applies it to its amplitudes; a gate on target q_T pairs each
 *     amplitude with the one whose index differs in bit q_T (Fig. 1a/1b).
 *   - Sec. 3.1: the "general approach" applies every gate as its full unitary
 *     matrix (2x2 for one qubit, 4x4 for CNOT).  This oracle is that general
 *     approach for every gate, including the diagonal and permutation gates
 *     the GPU path specialises: psi' = U_full psi, one index group at a time.
 *   - Sec. 3.2 / Fig. 5a: QFT from Hadamards and controlled phases; Fig. 6a:
 *     R_k phase rotations.  Listing 1: expectation values of a Hamiltonian
 *     (sum of Pauli words) and gradients for a variational loop.
 *
 * Conventions: qubit q is bit q of the amplitude index (qubit indices grow
 * with the rank distance 2^(q_T-L) in Sec. 2, so the lowest qubit is the
 * least significant bit).  A gate's wires are listed control(s) first, target
 * last; in its 2^m x 2^m matrix the first listed wire is the most significant
 * bit of the local row/column index.  Gate definitions follow the public
 * PennyLane operator definitions, which the paper extends (Sec. 1).
 *
 * Arithmetic is complex128 throughout; sums use Neumaier's compensated
 * summation so the oracle's own rounding stays far below every tolerance.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double _Complex cplx;

/* Gate numbering shared by name with the circuit descriptions. */
enum {
  O_X, O_Y, O_Z, O_H, O_S, O_T, O_RX, O_RY, O_RZ, O_PHASE, O_ROT,
  O_CNOT, O_CZ, O_SWAP, O_CPHASE, O_CRY, O_TOFFOLI, O_U2, O_U4, O_CSWAP, O_DEXC, O_NGATES
};
static const int o_nwires[O_NGATES] = {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 2, 2, 2, 2, 2, 3, 1, 2, 3, 4};
static const int o_nparams[O_NGATES] = {0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 3, 0, 0, 0, 1, 1, 0, 0, 0, 0, 1};

int oracle_gate_wires(int gate) { return (gate >= 0 && gate < O_NGATES) ? o_nwires[gate] : -1; }
int oracle_gate_params(int gate) { return (gate >= 0 && gate < O_NGATES) ? o_nparams[gate] : -1; }

void oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ---- gate matrices, built from their definitions --------------------------- */

static void mat2(cplx* M, cplx a, cplx b, cplx c, cplx d) { M[0] = a; M[1] = b; M[2] = c; M[3] = d; }

/* 2x2 product C = A B (row-major). */
static void matmul2(cplx* C, const cplx* A, const cplx* B) {
  cplx t[4];
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 2; ++c) t[2 * r + c] = A[2 * r] * B[c] + A[2 * r + 1] * B[2 + c];
  memcpy(C, t, sizeof t);
}

/* Single-qubit rotation exp(-i theta sigma / 2) for sigma = X, Y, Z. */
static void rot_x(cplx* M, double th) { double c = cos(th / 2), s = sin(th / 2); mat2(M, c, -I * s, -I * s, c); }
static void rot_y(cplx* M, double th) { double c = cos(th / 2), s = sin(th / 2); mat2(M, c, -s, s, c); }
static void rot_z(cplx* M, double th) { mat2(M, cexp(-I * th / 2), 0, 0, cexp(I * th / 2)); }

/* Embed a 2x2 block U as the controlled block of a dim x dim identity: the
 * block acts on the last two local basis states (all controls = 1). */
static void controlled(cplx* M, int dim, const cplx* U) {
  memset(M, 0, sizeof(cplx) * dim * dim);
  for (int k = 0; k < dim; ++k) M[k * dim + k] = 1;
  int b = dim - 2;
  M[b * dim + b] = U[0];
  M[b * dim + b + 1] = U[1];
  M[(b + 1) * dim + b] = U[2];
  M[(b + 1) * dim + b + 1] = U[3];
}

/*
 * The 2^m x 2^m matrix of `gate` (row-major) into `out` (256 entries suffice),
 * its wire count into *m.  `params` holds the gate's parameters; `user` the
 * caller's row-major matrix for U2/U4 (interleaved re,im).  `inverse` returns
 * the conjugate transpose.  Returns 0, or -1 for an unknown gate.
 */
int oracle_gate_matrix(int gate, const double* params, const double* user, int inverse, double* out_ri, int* m) {
  cplx M[256], A[4], B[4];
  if (gate < 0 || gate >= O_NGATES) return -1;
  int w = o_nwires[gate], dim = 1 << w;
  const double r2 = 1.0 / sqrt(2.0);
  switch (gate) {
    case O_X: mat2(M, 0, 1, 1, 0); break;
    case O_Y: mat2(M, 0, -I, I, 0); break;
    case O_Z: mat2(M, 1, 0, 0, -1); break;
    case O_H: mat2(M, r2, r2, r2, -r2); break;
    case O_S: mat2(M, 1, 0, 0, I); break;
    case O_T: mat2(M, 1, 0, 0, cexp(I * M_PI / 4)); break;
    case O_RX: rot_x(M, params[0]); break;
    case O_RY: rot_y(M, params[0]); break;
    case O_RZ: rot_z(M, params[0]); break;
    case O_PHASE: mat2(M, 1, 0, 0, cexp(I * params[0])); break;
    case O_ROT:  /* Rot(phi, theta, omega) = RZ(omega) RY(theta) RZ(phi) */
      rot_z(A, params[0]);
      rot_y(B, params[1]);
      matmul2(B, B, A);
      rot_z(A, params[2]);
      matmul2(M, A, B);
      break;
    case O_CNOT: mat2(A, 0, 1, 1, 0); controlled(M, 4, A); break;
    case O_CZ: mat2(A, 1, 0, 0, -1); controlled(M, 4, A); break;
    case O_SWAP:
      memset(M, 0, sizeof(cplx) * 16);
      M[0 * 4 + 0] = 1; M[1 * 4 + 2] = 1; M[2 * 4 + 1] = 1; M[3 * 4 + 3] = 1;
      break;
    case O_CPHASE: mat2(A, 1, 0, 0, cexp(I * params[0])); controlled(M, 4, A); break;
    case O_CRY: rot_y(A, params[0]); controlled(M, 4, A); break;
    case O_TOFFOLI: mat2(A, 0, 1, 1, 0); controlled(M, 8, A); break;
    case O_CSWAP:  /* wires (c, a, b): local index 4c + 2a + b; |101> <-> |110> */
      memset(M, 0, sizeof(cplx) * 64);
      for (int k = 0; k < 8; ++k) M[k * 8 + k] = 1;
      M[5 * 8 + 5] = 0; M[6 * 8 + 6] = 0;
      M[5 * 8 + 6] = 1; M[6 * 8 + 5] = 1;
      break;
    case O_DEXC: { /* rotation of the pair |0011> (index 3), |1100> (index 12) */
      const double c = cos(params[0] / 2), s = sin(params[0] / 2);
      memset(M, 0, sizeof(cplx) * 256);
      for (int k = 0; k < 16; ++k) M[k * 16 + k] = 1;
      M[3 * 16 + 3] = c;  M[12 * 16 + 3] = s;
      M[3 * 16 + 12] = -s; M[12 * 16 + 12] = c;
      break;
    }
    case O_U2:
    case O_U4:
      for (int k = 0; k < dim * dim; ++k) M[k] = user[2 * k] + I * user[2 * k + 1];
      break;
  }
  for (int r = 0; r < dim; ++r)
    for (int c = 0; c < dim; ++c) {
      cplx v = inverse ? conj(M[c * dim + r]) : M[r * dim + c];
      out_ri[2 * (r * dim + c)] = creal(v);
      out_ri[2 * (r * dim + c) + 1] = cimag(v);
    }
  *m = w;
  return 0;
}

/* ---- applying a matrix: the general approach -------------------------------- */

/* Global index of local basis state `a` of group `base` (wire k is local bit m-1-k). */
static uint64_t group_index(uint64_t base, const int* wires, int m, int a) {
  uint64_t idx = base;
  for (int k = 0; k < m; ++k)
    if ((a >> (m - 1 - k)) & 1) idx |= (uint64_t)1 << wires[k];
  return idx;
}

/*
 * psi <- U_full psi for the 2^m x 2^m matrix U (interleaved re,im, row-major)
 * acting on `wires`.  Every index whose wire bits are all zero is the base of
 * one group of 2^m amplitudes; the group is gathered, multiplied by U and
 * scattered back.  Wires must be distinct and < n; 1 <= m <= 7 (single gates
 * have at most 4 wires; dense blocks up to 7).
 */
void oracle_apply_matrix(double* psi_ri, int n, const int* wires, int m, const double* U_ri) {
  cplx* psi = (cplx*)psi_ri;
  if (m < 1 || m > 7) return; /* the group buffers hold at most 7 wires (the wrapper rejects more) */
  int dim = 1 << m;
  cplx* U = (cplx*)malloc(sizeof(cplx) * (size_t)dim * (size_t)dim);
  if (!U) return;
  uint64_t N = (uint64_t)1 << n, wmask = 0;
  for (int k = 0; k < dim * dim; ++k) U[k] = U_ri[2 * k] + I * U_ri[2 * k + 1];
  for (int k = 0; k < m; ++k) wmask |= (uint64_t)1 << wires[k];
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < (int64_t)N; ++i) {
    if ((uint64_t)i & wmask) continue;
    cplx v[128], r[128];
    uint64_t idx[128];
    for (int a = 0; a < dim; ++a) {
      idx[a] = group_index((uint64_t)i, wires, m, a);
      v[a] = psi[idx[a]];
    }
    for (int row = 0; row < dim; ++row) {
      cplx s = 0;
      for (int c = 0; c < dim; ++c) s += U[row * dim + c] * v[c];
      r[row] = s;
    }
    for (int a = 0; a < dim; ++a) psi[idx[a]] = r[a];
  }
  free(U);
}

/*
 * Selected amplitudes of U_full psi without forming the whole result: output
 * index k lies in the group whose base is k with its wire bits cleared, at
 * local row = k's wire bits; its value is sum_c U[row][c] psi[group(c)].
 */
void oracle_apply_matrix_at(const double* psi_ri, int n, const int* wires, int m, const double* U_ri,
                            const uint64_t* out_idx, int64_t count, double* out_ri) {
  const cplx* psi = (const cplx*)psi_ri;
  cplx* out = (cplx*)out_ri;
  int dim = 1 << m;
  uint64_t wmask = 0;
  (void)n;
  for (int k = 0; k < m; ++k) wmask |= (uint64_t)1 << wires[k];
  for (int64_t s = 0; s < count; ++s) {
    uint64_t k = out_idx[s], base = k & ~wmask;
    int row = 0;
    for (int q = 0; q < m; ++q) row |= (int)((k >> wires[q]) & 1) << (m - 1 - q);
    cplx acc = 0;
    for (int c = 0; c < dim; ++c) {
      cplx u = U_ri[2 * (row * dim + c)] + I * U_ri[2 * (row * dim + c) + 1];
      acc += u * psi[group_index(base, wires, m, c)];
    }
    out[s] = acc;
  }
}

/* Apply one gate: build its matrix, then the general update. */
int oracle_apply_gate(double* psi_ri, int n, int gate, const int* wires, const double* params,
                      const double* user, int inverse) {
  double U[512];
  int m;
  if (oracle_gate_matrix(gate, params, user, inverse, U, &m)) return -1;
  for (int k = 0; k < m; ++k) {
    if (wires[k] < 0 || wires[k] >= n) return -1;
    for (int j = 0; j < k; ++j)
      if (wires[j] == wires[k]) return -1;
  }
  oracle_apply_matrix(psi_ri, n, wires, m, U);
  return 0;
}

/*
 * Run a circuit in order.  ops is n_ops records of 6 ints:
 * {gate, wire0, wire1, wire2, param_index (-1 none), inverse};
 * `mats` holds 32 doubles (a 4x4 complex matrix) per op for U2/U4.
 */
int oracle_run(double* psi_ri, int n, const int* ops, int n_ops, const double* params, const double* mats) {
  for (int k = 0; k < n_ops; ++k) {
    const int* o = ops + 7 * k; /* gate, 4 wires, parameter index, inverse */
    const double* p = o[5] >= 0 ? params + o[5] : NULL;
    if (oracle_apply_gate(psi_ri, n, o[0], o + 1, p, mats + 32 * k, o[6])) return -1 - k;
  }
  return 0;
}

/* ---- measurement --------------------------------------------------------------- */

/* Neumaier's compensated sum, one term at a time. */
typedef struct { double s, c; } nsum;
static void nadd(nsum* a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
  else a->c += (x - t) + a->s;
  a->s = t;
}

/* <psi|psi>. */
double oracle_norm2(const double* psi_ri, int n) {
  nsum acc = {0, 0};
  uint64_t N = (uint64_t)1 << n;
  for (uint64_t i = 0; i < 2 * N; ++i) nadd(&acc, psi_ri[i] * psi_ri[i]);
  return acc.s + acc.c;
}

/* Matrix element <row|sigma|col> of a single-qubit Pauli sigma = (x, z) bits:
 * I=(0,0), X=(1,0), Z=(0,1), Y=(1,1). */
static cplx pauli_elem(int x, int z, int row, int col) {
  static const cplx Pm[4][4] = {
      {1, 0, 0, 1},    /* I */
      {0, 1, 1, 0},    /* X */
      {1, 0, 0, -1},   /* Z */
      {0, -I, I, 0}};  /* Y */
  return Pm[x + 2 * z][2 * row + col];
}

/*
 * <psi|P|psi> for the Pauli word P = prod_q sigma_q (bit q of x_mask / z_mask
 * selects sigma_q).  Each row k of P has its single nonzero in column k^x_mask,
 * the product of the per-qubit 2x2 entries.
 */
double oracle_pauli_expval(const double* psi_ri, int n, uint64_t x_mask, uint64_t z_mask) {
  const cplx* psi = (const cplx*)psi_ri;
  uint64_t N = (uint64_t)1 << n;
  nsum re = {0, 0};
  for (uint64_t k = 0; k < N; ++k) {
    uint64_t j = k ^ x_mask;
    cplx coef = 1;
    for (int q = 0; q < n; ++q) {
      int x = (int)((x_mask >> q) & 1), z = (int)((z_mask >> q) & 1);
      if (x | z) coef *= pauli_elem(x, z, (int)((k >> q) & 1), (int)((j >> q) & 1));
    }
    nadd(&re, creal(conj(psi[k]) * coef * psi[j]));
  }
  return re.s + re.c;
}

/* sum_w coeff_w <psi|P_w|psi>; per-term values into `per_term` when non-null. */
double oracle_expval(const double* psi_ri, int n, const double* coeff, const uint64_t* x_mask,
                     const uint64_t* z_mask, int n_terms, double* per_term) {
  nsum tot = {0, 0};
  for (int w = 0; w < n_terms; ++w) {
    double v = oracle_pauli_expval(psi_ri, n, x_mask[w], z_mask[w]);
    if (per_term) per_term[w] = v;
    nadd(&tot, coeff[w] * v);
  }
  return tot.s + tot.c;
}
