// Gate validation and lowering to kernel ops (host).
//
// Sec. 2 of arxiv 2508.13615: each process holds the small gate matrix and
// "only takes nonzero elements" of it; the execution pattern depends on the
// gate's character (Pauli-Z only touches amplitudes whose target bit is 1,
// Pauli-X pairs amplitudes, a CNOT's control only selects which amplitudes
// are touched).  Lowering maps every gate of the ABI to one of the kernel
// classes of KKind with exactly those nonzero coefficients.
#include <cmath>
#include <complex>
#include <cstring>

#include "lqs_internal.cuh"

namespace lqs {

using cd = std::complex<double>;

static const int kWires[LQS_NUM_GATES] = {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 2, 2, 2, 2, 2, 3, 1, 2, 3, 4};
static const int kParams[LQS_NUM_GATES] = {0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 3, 0, 0, 0, 1, 1, 0, 0, 0, 0, 1};
static const char* kNames[LQS_NUM_GATES] = {"X",  "Y",    "Z",   "H",    "S",    "T",      "RX",
                                            "RY", "RZ",   "PhaseShift", "Rot", "CNOT", "CZ", "SWAP",
                                            "ControlledPhaseShift", "CRY", "Toffoli", "U2", "U4",
                                            "CSWAP", "DoubleExcitation"};

static void put(KOp& k, int i, cd v) {
  k.m[2 * i] = v.real();
  k.m[2 * i + 1] = v.imag();
}

// Phase factor e^{i a}.
static cd cis(double a) { return cd(std::cos(a), std::sin(a)); }

static KOp phase_op(uint64_t cmask, cd f) {
  KOp k;
  k.kind = K_PHASE;
  k.cmask = cmask;
  put(k, 0, f);
  if (f == cd(-1, 0)) k.special = 1;
  else if (f == cd(0, 1)) k.special = 2;
  else if (f == cd(0, -1)) k.special = 3;
  return k;
}

static KOp diag1_op(int t, uint64_t cmask, cd d0, cd d1) {
  KOp k;
  k.kind = K_DIAG1;
  k.t0 = t;
  k.cmask = cmask;
  put(k, 0, d0);
  put(k, 1, d1);
  return k;
}

static KOp anti1_op(int t, uint64_t cmask, cd f0, cd f1) {
  KOp k;
  k.kind = K_ANTI1;
  k.t0 = t;
  k.cmask = cmask;
  put(k, 0, f0);
  put(k, 1, f1);
  k.special = (f0 == cd(1, 0) && f1 == cd(1, 0)) ? 1 : 0;
  return k;
}

// Dense 2x2 u (row-major); real when every imaginary part is zero.
static KOp dense1_op(int t, uint64_t cmask, const cd* u, bool allow_real) {
  KOp k;
  k.t0 = t;
  k.cmask = cmask;
  bool real = allow_real;
  for (int i = 0; i < 4; ++i) real = real && u[i].imag() == 0.0;
  if (real) {
    k.kind = K_DENSE1R;
    for (int i = 0; i < 4; ++i) k.m[i] = u[i].real();
  } else {
    k.kind = K_DENSE1;
    for (int i = 0; i < 4; ++i) put(k, i, u[i]);
  }
  return k;
}

// Structure-aware lowering of a one-qubit matrix: only nonzero entries used.
static KOp lower_u2(int t, uint64_t cmask, const cd* u, bool general) {
  if (general) return dense1_op(t, cmask, u, false);
  if (u[1] == 0.0 && u[2] == 0.0) {
    if (u[0] == 1.0) return phase_op(cmask | (1ull << t), u[3]);
    return diag1_op(t, cmask, u[0], u[3]);
  }
  if (u[0] == 0.0 && u[3] == 0.0) return anti1_op(t, cmask, u[1], u[2]);
  return dense1_op(t, cmask, u, true);
}

static void adjoint2(cd* u) {  // u <- u^dagger (2x2)
  cd a = std::conj(u[0]), b = std::conj(u[2]), c = std::conj(u[1]), d = std::conj(u[3]);
  u[0] = a; u[1] = b; u[2] = c; u[3] = d;
}

static void rot_z(cd* u, double th) { u[0] = cis(-th / 2); u[1] = 0; u[2] = 0; u[3] = cis(th / 2); }
static void rot_y(cd* u, double th) {
  double c = std::cos(th / 2), s = std::sin(th / 2);
  u[0] = c; u[1] = -s; u[2] = s; u[3] = c;
}
static void rot_x(cd* u, double th) {
  double c = std::cos(th / 2), s = std::sin(th / 2);
  u[0] = c; u[1] = cd(0, -s); u[2] = cd(0, -s); u[3] = c;
}
static void mul2(cd* out, const cd* a, const cd* b) {  // out = a b
  cd r[4];
  r[0] = a[0] * b[0] + a[1] * b[2];
  r[1] = a[0] * b[1] + a[1] * b[3];
  r[2] = a[2] * b[0] + a[3] * b[2];
  r[3] = a[2] * b[1] + a[3] * b[3];
  for (int i = 0; i < 4; ++i) out[i] = r[i];
}

static void with_gen(KOp& k, int slot, int gen, double scale, bool inverse) {
  k.param_slot = slot;
  k.gen = gen;
  k.gen_scale = inverse ? -scale : scale;
}

int lower_gate(int n, int gate, const int* wires, int n_wires, const double* params, int n_params,
               const double* matrix, int inverse, int slot, bool decompose, bool general,
               std::vector<KOp>& out) {
  if (gate < 0 || gate >= LQS_NUM_GATES) return set_error(LQS_ERR_ARG, "unknown gate id " + std::to_string(gate));
  const char* name = kNames[gate];
  if (n_wires != kWires[gate])
    return set_error(LQS_ERR_ARG, std::string(name) + " takes " + std::to_string(kWires[gate]) + " wires, got " +
                                      std::to_string(n_wires));
  if (!wires) return set_error(LQS_ERR_ARG, "wires is NULL");
  for (int i = 0; i < n_wires; ++i) {
    if (wires[i] < 0 || wires[i] >= n)
      return set_error(LQS_ERR_ARG, std::string(name) + ": wire " + std::to_string(wires[i]) + " outside [0, " +
                                        std::to_string(n) + ")");
    for (int j = 0; j < i; ++j)
      if (wires[i] == wires[j]) return set_error(LQS_ERR_ARG, std::string(name) + ": repeated wire");
  }
  if (gate != LQS_U2 && gate != LQS_U4) {
    if (n_params < kParams[gate])
      return set_error(LQS_ERR_ARG, std::string(name) + " takes " + std::to_string(kParams[gate]) + " parameters");
    if (kParams[gate] && !params) return set_error(LQS_ERR_ARG, std::string(name) + ": params is NULL");
    for (int i = 0; i < kParams[gate]; ++i)
      if (!std::isfinite(params[i])) return set_error(LQS_ERR_ARG, std::string(name) + ": non-finite parameter");
  } else if (!matrix) {
    return set_error(LQS_ERR_ARG, std::string(name) + ": matrix is NULL");
  }
  const bool inv = inverse != 0;
  const int t = wires[n_wires - 1];
  const uint64_t tb = 1ull << t;
  cd u[4];
  KOp k;
  switch (gate) {
    case LQS_X: out.push_back(anti1_op(t, 0, 1.0, 1.0)); break;
    case LQS_Y: out.push_back(anti1_op(t, 0, cd(0, -1), cd(0, 1))); break;  // Hermitian: Y^dagger = Y
    case LQS_Z: out.push_back(phase_op(tb, -1.0)); break;
    case LQS_H: {
      const double r = 1.0 / std::sqrt(2.0);
      u[0] = r; u[1] = r; u[2] = r; u[3] = -r;
      out.push_back(dense1_op(t, 0, u, true));
      break;
    }
    case LQS_S: out.push_back(phase_op(tb, inv ? cd(0, -1) : cd(0, 1))); break;
    case LQS_T: out.push_back(phase_op(tb, cis(inv ? -M_PI / 4 : M_PI / 4))); break;
    case LQS_RX:
      rot_x(u, inv ? -params[0] : params[0]);
      k = dense1_op(t, 0, u, !general);
      with_gen(k, slot, G_X, 1.0, inv);
      out.push_back(k);
      break;
    case LQS_RY:
      rot_y(u, inv ? -params[0] : params[0]);
      k = dense1_op(t, 0, u, !general);
      with_gen(k, slot, G_Y, 1.0, inv);
      out.push_back(k);
      break;
    case LQS_RZ:
      rot_z(u, inv ? -params[0] : params[0]);
      k = general ? dense1_op(t, 0, u, false) : diag1_op(t, 0, u[0], u[3]);
      with_gen(k, slot, G_Z, 1.0, inv);
      out.push_back(k);
      break;
    case LQS_PHASE:
      // diag(1, e^{i phi}) = e^{i phi/2} RZ(phi): generator -P1 (scale -2)
      k = phase_op(tb, cis(inv ? -params[0] : params[0]));
      with_gen(k, slot, G_P1, -2.0, inv);
      out.push_back(k);
      break;
    case LQS_ROT: {
      const int s0 = slot < 0 ? -1 : slot, s1 = slot < 0 ? -1 : slot + 1, s2 = slot < 0 ? -1 : slot + 2;
      if (decompose) {
        // RZ(phi) then RY(theta) then RZ(omega); the adjoint reverses the order.
        KOp a, b, c;
        cd v[4];
        rot_z(v, params[0]); a = diag1_op(t, 0, v[0], v[3]); with_gen(a, s0, G_Z, 1.0, false);
        rot_y(v, params[1]); b = dense1_op(t, 0, v, true); with_gen(b, s1, G_Y, 1.0, false);
        rot_z(v, params[2]); c = diag1_op(t, 0, v[0], v[3]); with_gen(c, s2, G_Z, 1.0, false);
        if (!inv) {
          out.push_back(a); out.push_back(b); out.push_back(c);
        } else {
          cd w[4];
          rot_z(w, -params[2]); c = diag1_op(t, 0, w[0], w[3]); with_gen(c, s2, G_Z, 1.0, true);
          rot_y(w, -params[1]); b = dense1_op(t, 0, w, true); with_gen(b, s1, G_Y, 1.0, true);
          rot_z(w, -params[0]); a = diag1_op(t, 0, w[0], w[3]); with_gen(a, s0, G_Z, 1.0, true);
          out.push_back(c); out.push_back(b); out.push_back(a);
        }
      } else {
        cd a[4], b[4], c[4], ab[4];
        rot_z(a, params[0]);
        rot_y(b, params[1]);
        rot_z(c, params[2]);
        mul2(ab, b, a);
        mul2(u, c, ab);
        if (inv) adjoint2(u);
        // always dense: the kernel class of a parametrised gate must not depend on its angles
        out.push_back(dense1_op(t, 0, u, !general));
      }
      break;
    }
    case LQS_CNOT: out.push_back(anti1_op(t, 1ull << wires[0], 1.0, 1.0)); break;
    case LQS_CZ: out.push_back(phase_op((1ull << wires[0]) | tb, -1.0)); break;
    case LQS_SWAP:
      k.kind = K_SWAP;
      k.t0 = wires[0];
      k.t1 = wires[1];
      out.push_back(k);
      break;
    case LQS_CPHASE:
      k = phase_op((1ull << wires[0]) | tb, cis(inv ? -params[0] : params[0]));
      with_gen(k, slot, G_P1, -2.0, inv);
      out.push_back(k);
      break;
    case LQS_CRY:
      rot_y(u, inv ? -params[0] : params[0]);
      k = dense1_op(t, 1ull << wires[0], u, true);
      with_gen(k, slot, G_Y, 1.0, inv);
      out.push_back(k);
      break;
    case LQS_TOFFOLI: out.push_back(anti1_op(t, (1ull << wires[0]) | (1ull << wires[1]), 1.0, 1.0)); break;
    case LQS_CSWAP:  // a SWAP of wires[1], wires[2] under the control wires[0]
      k.kind = K_SWAP;
      k.t0 = wires[1];
      k.t1 = wires[2];
      k.cmask = 1ull << wires[0];
      out.push_back(k);
      break;
    case LQS_DOUBLE_EXCITATION: {
      // CNOTs from w0 to w1, w2, w3 send |0011> to itself and |1100> to
      // |1011>: the pair then differs only in w0, with (w1, w2, w3) = (0, 1, 1)
      // and no other state there.  X on w1 makes that the all-ones control
      // pattern of an RY on w0, which is the rotation; then X and the CNOTs
      // are undone.
      const int w0 = wires[0], w1 = wires[1], w2 = wires[2], w3 = wires[3];
      for (int c : {w1, w2, w3}) out.push_back(anti1_op(c, 1ull << w0, 1.0, 1.0));
      out.push_back(anti1_op(w1, 0, 1.0, 1.0));
      rot_y(u, inv ? -params[0] : params[0]);
      k = dense1_op(w0, (1ull << w1) | (1ull << w2) | (1ull << w3), u, true);
      with_gen(k, slot, G_Y, 1.0, inv);
      out.push_back(k);
      out.push_back(anti1_op(w1, 0, 1.0, 1.0));
      for (int c : {w3, w2, w1}) out.push_back(anti1_op(c, 1ull << w0, 1.0, 1.0));
      break;
    }
    case LQS_U2:
      for (int i = 0; i < 4; ++i) u[i] = cd(matrix[2 * i], matrix[2 * i + 1]);
      for (int i = 0; i < 8; ++i)
        if (!std::isfinite(matrix[i])) return set_error(LQS_ERR_ARG, "U2: non-finite matrix entry");
      if (inv) adjoint2(u);
      out.push_back(lower_u2(t, 0, u, general));
      break;
    case LQS_U4: {
      cd v[16];
      for (int i = 0; i < 32; ++i)
        if (!std::isfinite(matrix[i])) return set_error(LQS_ERR_ARG, "U4: non-finite matrix entry");
      for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
          cd x(matrix[2 * (4 * r + c)], matrix[2 * (4 * r + c) + 1]);
          if (inv) v[4 * c + r] = std::conj(x);
          else v[4 * r + c] = x;
        }
      bool diag = !general;
      for (int r = 0; r < 4 && diag; ++r)
        for (int c = 0; c < 4; ++c)
          if (r != c && v[4 * r + c] != 0.0) { diag = false; break; }
      k.kind = diag ? K_DIAG2 : K_DENSE2;
      k.t0 = wires[0];
      k.t1 = wires[1];
      if (diag) for (int i = 0; i < 4; ++i) put(k, i, v[5 * i]);
      else for (int i = 0; i < 16; ++i) put(k, i, v[i]);
      out.push_back(k);
      break;
    }
  }
  return LQS_OK;
}

int lower_ops(int n, const lqs_op* ops, int n_ops, const double* params, int n_params, bool decompose,
              std::vector<KOp>& out) {
  if (n_ops < 0) return set_error(LQS_ERR_ARG, "n_ops < 0");
  if (n_ops > 0 && !ops) return set_error(LQS_ERR_ARG, "ops is NULL");
  out.reserve(out.size() + (size_t)n_ops);
  for (int i = 0; i < n_ops; ++i) {
    const lqs_op& o = ops[i];
    if (o.gate < 0 || o.gate >= LQS_NUM_GATES)
      return set_error(LQS_ERR_ARG, "op " + std::to_string(i) + ": unknown gate id");
    const int np = kParams[o.gate];
    const double* p = nullptr;
    if (np) {
      if (o.param_idx < 0 || o.param_idx + np > n_params || !params)
        return set_error(LQS_ERR_ARG, "op " + std::to_string(i) + " (" + kNames[o.gate] +
                                          "): param_idx outside the parameter array");
      p = params + o.param_idx;
    }
    const int rc = lower_gate(n, o.gate, o.wires, kWires[o.gate], p, np, o.matrix, o.inverse,
                              np ? o.param_idx : -1, decompose, false, out);
    if (rc != LQS_OK) {
      set_error(rc, "op " + std::to_string(i) + ": " + lqs_last_error());
      return rc;
    }
  }
  return LQS_OK;
}

}  // namespace lqs
