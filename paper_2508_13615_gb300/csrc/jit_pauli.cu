// Compiled Pauli passes: <psi|P_w|psi> for a group of Pauli words, and
// optionally lambda = sum_w c_w P_w psi, as straight-line register-tile
// kernels (the observable of Listing 1's qml.expval(H), and the adjoint
// method's lambda).
//
// A pass covers words whose X/Y qubits fit one tile.  Each thread holds R
// amplitudes of the tile in registers in natural order (thread bits on the
// low tile positions, register bits on the top ones) and a double-float copy
// of the tile sits in shared memory for partners held by other threads.
//   * Diagonal words: <P_w> = sum_j s_w(j) |psi_j|^2 with s_w(j) the parity of
//     j & z_w.  The register part of the sign is applied per thread, once per
//     distinct register Z pattern; one Walsh butterfly over the warp then
//     yields every lane-bit-signed sum at once (lane l holds the sum signed
//     by l's bits), and warp-index and outside-tile bits give uniform signs.
//   * X/Y words: pairs (j, j ^ x) with j's lowest X bit clear, counted once
//     and doubled; the partner comes from registers or the shared copy.
//   * lambda: the diagonal words' coefficients are summed per amplitude
//     first (one real-times-complex product each), the X/Y words add their
//     scaled partners; lambda leaves registers with coalesced direct stores.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "arith.cuh"
#include "jit.h"
#include "lqs_internal.cuh"
#include "measure_common.cuh"
#include "tile.cuh"

namespace lqs {

namespace {

constexpr int kPauliWordsJit = 64;
constexpr int kPauliThreadBits = 8;

std::string hx(uint64_t x) {
  char b[32];
  std::snprintf(b, sizeof b, "0x%llxull", (unsigned long long)x);
  return b;
}

struct JWord {
  uint32_t xl, zl;
  uint64_t ze;
  int ph, lowbit;
};

// Source of one pass.  mode: 1 expectation, 2 lambda (accumulate), 4 lambda
// starts at zero (combined with 2).
std::string pauli_source(const char* aname, int k, int b, const std::vector<JWord>& ws, int mode,
                         std::string& kname) {
  const int tb = kPauliThreadBits, r = k - tb, R = 1 << r;
  const bool exp = mode & 1, lam = mode & 2, fresh = mode & 4;
  const int nw = (int)ws.size();
  std::ostringstream o, pre, post;  // loop body, before the loop, after the loop
  const uint32_t tmask = (1u << tb) - 1u;
  bool need_xa = false;
  for (auto& w : ws)
    if (w.xl & tmask) need_xa = true;
  // element e of thread tid is local index tid + (e << tb)
  auto val = [&](int e) { return "v" + std::to_string(e); };
  o << "    W";
  for (int e = 0; e < R; ++e) o << (e ? ", " : " ") << val(e);
  o << ";\n";
  for (int e = 0; e < R; ++e) o << "    " << val(e) << " = A::load(S0[tid + " << (e << tb) << "u]);\n";
  if (need_xa)
    for (int e = 0; e < R; ++e) o << "    lqs::st_w(&XA[tid + " << (e << tb) << "u], " << val(e) << ");\n";
  // tile-dependent sign parities of the words' Z bits outside the tile
  std::map<uint64_t, std::string> esign;
  for (auto& w : ws)
    if (w.ze && !esign.count(w.ze)) {
      const std::string nm = "es" + std::to_string(esign.size());
      o << "    const bool " << nm << " = (__popcll(base & " << hx(w.ze) << ") & 1) != 0;\n";
      esign.emplace(w.ze, nm);
    }
  if (lam) {
    for (int e = 0; e < R; ++e) {
      o << "    lqs::jit::LAcc<A> l" << e << ";\n";
      if (fresh) o << "    l" << e << ".zero();\n";
      else o << "    l" << e << ".init(A::load(S0L[tid + " << (e << tb) << "u]));\n";
    }
  }
  o << "    __syncthreads();  // the shared copy is complete and the incoming buffers are free\n"
       "    { const uint64_t tn = t + gridDim.x;\n"
       "      if (tn < G.ntiles) {\n"
       "        lqs::jit::seg_copy(G, S0, psi, lqs::tile_base(G, tn), bar, my_roff);\n";
  if (lam && !fresh) o << "        lqs::jit::seg_copy(G, S0L, lam, lqs::tile_base(G, tn), bar, my_roff);\n";
  o << "      } }\n";
  // partner of element e for a word with X mask x: register or shared copy
  auto partner = [&](int e, uint32_t x) {
    const uint32_t xt = x & tmask, xr = x >> tb;
    if (!xt) return val(e ^ (int)xr);
    return "lqs::ld_w(&XA[(tid ^ " + std::to_string(xt) + "u) + " + std::to_string((e ^ (int)xr) << tb) + "u])";
  };
  // per-thread sign parity of a Z mask's thread part (tile independent)
  std::map<uint32_t, std::string> tsign;
  auto thread_sign = [&](uint32_t zt) -> std::string {
    if (!zt) return "false";
    auto it = tsign.find(zt);
    if (it == tsign.end()) {
      const std::string nm = "ts" + std::to_string(tsign.size());
      pre << "  const bool " << nm << " = (__popc(tid & " << zt << "u) & 1) != 0;\n";
      it = tsign.emplace(zt, nm).first;
    }
    return it->second;
  };
  auto tile_sign = [&](uint64_t ze) -> std::string { return ze ? esign.at(ze) : std::string("false"); };
  auto x_ = [](const std::string& a, const std::string& b) {
    if (a == "false") return b;
    if (b == "false") return a;
    return "(" + a + " != " + b + ")";
  };
  int uid = 0;
  if (exp) {
    // diagonal words
    std::map<uint32_t, std::string> walsh;  // register Z pattern -> butterfly result
    std::vector<std::string> pats;          // butterfly results in order
    std::map<uint32_t, int> pat_of;         // register Z pattern -> index in pats
    std::vector<int> dws;                   // the diagonal words
    bool have_p = false;
    for (int w = 0; w < nw; ++w) {
      const JWord& W = ws[w];
      if (W.xl) continue;
      if (!have_p) {
        for (int e = 0; e < R; ++e)
          o << "    const lqs::jit::GAcc<A>::V p" << e << " = lqs::jit::pn2<A>(" << val(e) << ");\n";
        have_p = true;
      }
      const uint32_t zr = W.zl >> tb, zt = W.zl & tmask;
      auto it = walsh.find(zr);
      if (it == walsh.end()) {
        const std::string sn = "d" + std::to_string(uid++);
        o << "    lqs::jit::GAcc<A>::T " << sn << " = lqs::jit::GAcc<A>::zero();\n";
        for (int e = 0; e < R; ++e)
          o << "    lqs::jit::wadd(" << sn << ", p" << e << ", " << ((__builtin_popcount(e & zr) & 1) ? "true" : "false")
            << ");\n";
        const std::string wn = "D" + std::to_string(uid++);
        o << "    const auto " << wn << " = lqs::jit::wht(" << sn << ");\n";
        it = walsh.emplace(zr, wn).first;
        pat_of[zr] = (int)pats.size();
        pats.push_back(wn);
      }
      (void)zt;
      dws.push_back(w);
    }
    // Each diagonal word's value for this tile sits in the butterfly lane of
    // its lane Z bits, signed by its warp and outside-tile Z bits.  Diagonal
    // word k is summed across tiles by lane k mod 32 of every warp (one
    // shuffle per register pattern and one add for all of them) and stored in
    // its slot after the tile loop.
    for (size_t a = 0; 32 * a < dws.size(); ++a) {
      const std::string A_ = std::to_string(a);
      pre << "  uint32_t dsrc" << A_ << " = 0u, dpat" << A_ << " = 0u, dzt" << A_ << " = 0u;\n  uint64_t dze" << A_
          << " = 0ull;\n  int dw" << A_ << " = -1;\n  lqs::jit::LaneAcc<A> dacc" << A_ << ";\n  dacc" << A_
          << ".zero();\n";
      for (size_t kk = 0; kk < 32 && 32 * a + kk < dws.size(); ++kk) {
        const JWord& W = ws[dws[32 * a + kk]];
        const uint32_t zr = W.zl >> tb, zt = W.zl & tmask;
        pre << "  if ((tid & 31u) == " << kk << "u) { dsrc" << A_ << " = " << (zt & 31u) << "u; dpat" << A_ << " = "
            << pat_of[zr] << "u; dzt" << A_ << " = " << (zt & ~31u) << "u; dze" << A_ << " = " << hx(W.ze) << "; dw"
            << A_ << " = " << dws[32 * a + kk] << "; }\n";
      }
      o << "    { auto x = lqs::jit::shfl_idx(" << pats[0] << ", dsrc" << A_ << ");\n";
      for (size_t i = 1; i < pats.size(); ++i)
        o << "      { const auto y = lqs::jit::shfl_idx(" << pats[i] << ", dsrc" << A_ << "); if (dpat" << A_
          << " == " << i << "u) x = y; }\n";
      o << "      dacc" << A_ << ".add(x, ((__popc(tid & dzt" << A_ << ") + __popcll(base & dze" << A_
        << ")) & 1) != 0); }\n";
      post << "  if (dw" << A_ << " >= 0) dacc" << A_ << ".put(wacc + warp * " << nw << " + dw" << A_ << ");\n";
    }
    // X/Y words: pairs with the lowest X bit clear.  Their warp sums go four
    // at a time through one reduce-scatter (gflush4).
    std::vector<std::pair<std::string, int>> pend;
    auto flush = [&](bool all) {
      while (pend.size() >= 4 || (all && !pend.empty())) {
        o << "    lqs::jit::gflush4(";
        for (int i = 0; i < 4; ++i) o << (i < (int)pend.size() ? pend[i].first : "lqs::jit::GAcc<A>::zero()") << ", ";
        for (int i = 0; i < 4; ++i)
          o << (i < (int)pend.size() ? "wacc + warp * " + std::to_string(nw) + " + " + std::to_string(pend[i].second)
                                     : std::string("(double*)0"))
            << (i < 3 ? ", " : ");\n");
        pend.erase(pend.begin(), pend.begin() + std::min<size_t>(4, pend.size()));
      }
    };
    for (int w = 0; w < nw; ++w) {
      const JWord& W = ws[w];
      if (!W.xl) continue;
      const uint32_t zt = W.zl & tmask, zr = W.zl >> tb;
      const std::string acc = "g" + std::to_string(uid++);
      o << "    lqs::jit::GAcc<A>::T " << acc << " = lqs::jit::GAcc<A>::zero();\n    {\n";
      const bool lowreg = W.lowbit >= tb;
      // the pair term of representative j (lowest X bit of j clear):
      // c = psi_{j ^ x}, b = psi_j, sign of j's Z bits
      auto term = [&](const std::string& c, const std::string& b, const std::string& neg) {
        switch (W.ph) {
          case 0: o << "        lqs::jit::gre<A>(" << acc << ", " << c << ", " << b << ", " << neg << ");\n"; break;
          case 1: o << "        lqs::jit::gim<A>(" << acc << ", " << c << ", " << b << ", !(" << neg << "));\n"; break;
          case 2: o << "        lqs::jit::gre<A>(" << acc << ", " << c << ", " << b << ", !(" << neg << "));\n"; break;
          default: o << "        lqs::jit::gim<A>(" << acc << ", " << c << ", " << b << ", " << neg << ");\n"; break;
        }
      };
      const std::string st = x_(thread_sign(zt), tile_sign(W.ze));
      auto neg_at = [&](int e, const std::string& s_) {
        return (__builtin_popcount(e & zr) & 1) ? "!(" + s_ + ")" : s_;
      };
      if (!lowreg && W.lowbit >= 5 && r >= 1) {
        // a warp bit: the two warps of each pair share the pairs (split by
        // the top register bit) instead of one of them idling; the other
        // warp forms the same terms from its side (its own register is the
        // partner value c, the representative's amplitude comes from XA, and
        // the sign is taken at the representative, tid ^ x)
        const int ms = r - 1;
        const uint32_t xt = W.xl & tmask, xr = W.xl >> tb;
        const std::string sx = thread_sign(zt);
        const std::string st1 = x_((__builtin_popcount(xt & zt) & 1) ? "!" + sx : sx, tile_sign(W.ze));
        o << "      if (!((tid >> " << W.lowbit << ") & 1u)) {\n";
        for (int e = 0; e < R; ++e)
          if (!((e >> ms) & 1)) term(partner(e, W.xl), val(e), neg_at(e, st));
        o << "      } else {\n";
        for (int e = 0; e < R; ++e)
          if ((e >> ms) & 1)
            term(val(e ^ (int)xr), "lqs::ld_w(&XA[(tid ^ " + std::to_string(xt) + "u) + " + std::to_string(e << tb) + "u])",
                 neg_at(e, st1));
        o << "      }\n";
      } else if (!lowreg && r >= 1) {
        // a lane bit: both lanes of each pair take half of the pairs (split by
        // the top register bit) in one instruction stream: each lane selects
        // its register operand and the shared-memory position of the other.
        // The lower lane holds the representative, the upper lane its
        // partner; Re(conj(c) b) does not depend on the order of the two,
        // Im(conj(c) b) changes sign, so the upper lanes flip the imaginary
        // forms' sign.
        const int ms = r - 1;
        const uint32_t xt = W.xl & tmask, xr = W.xl >> tb;
        const std::string sx = thread_sign(zt);
        const std::string st1 = x_((__builtin_popcount(xt & zt) & 1) ? "!" + sx : sx, tile_sign(W.ze));
        const std::string hb = "hb" + std::to_string(uid++);
        o << "      const bool " << hb << " = ((tid >> " << W.lowbit << ") & 1u) != 0u;\n";
        for (int i = 0; i < R / 2; ++i) {
          const int e0 = i, e1 = i | (1 << ms);
          const std::string rg = "(" + hb + " ? " + val(e1 ^ (int)xr) + " : " + val(e0) + ")";
          const std::string sm = "lqs::ld_w(&XA[(tid ^ " + std::to_string(xt) + "u) + (" + hb + " ? " +
                                 std::to_string(e1 << tb) + "u : " + std::to_string((e0 ^ (int)xr) << tb) + "u)])";
          const std::string nu = neg_at(e1, st1), nl = neg_at(e0, st);
          const std::string ng = (W.ph & 1) ? "(" + hb + " ? !(" + nu + ") : " + nl + ")"
                                             : "(" + hb + " ? " + nu + " : " + nl + ")";
          term(sm, rg, ng);
        }
      } else {
        if (!lowreg) o << "      if (!((tid >> " << W.lowbit << ") & 1u)) {\n";
        for (int e = 0; e < R; ++e) {
          if (lowreg && ((e >> (W.lowbit - tb)) & 1)) continue;
          term(partner(e, W.xl), val(e), neg_at(e, st));
        }
        if (!lowreg) o << "      }\n";
      }
      o << "    }\n";
      pend.emplace_back(acc, w);
      flush(false);
    }
    flush(true);
  }
  if (lam) {
    // diagonal words: one signed coefficient sum per amplitude
    bool any_diag = false;
    for (auto& W : ws)
      if (!W.xl) any_diag = true;
    if (any_diag) {
      for (int e = 0; e < R; ++e) o << "    lqs::jit::GAcc<A>::T c" << e << " = lqs::jit::GAcc<A>::zero();\n";
      for (int w = 0; w < nw; ++w) {
        const JWord& W = ws[w];
        if (W.xl) continue;
        const uint32_t zt = W.zl & tmask, zr = W.zl >> tb;
        const std::string st = x_(thread_sign(zt), tile_sign(W.ze));
        for (int e = 0; e < R; ++e) {
          const bool cneg = __builtin_popcount(e & zr) & 1;
          o << "    lqs::jit::cadd(c" << e << ", P.c[" << w << "], " << (cneg ? "!(" + st + ")" : st) << ");\n";
        }
      }
      for (int e = 0; e < R; ++e) o << "    l" << e << ".add<0>(" << val(e) << ", lqs::jit::cfin(c" << e << "), false);\n";
    }
    for (int w = 0; w < nw; ++w) {
      const JWord& W = ws[w];
      if (!W.xl) continue;
      // lambda_j += c_w i^ph (-1)^popc((j ^ x) & z) psi_{j ^ x}
      const uint32_t zt = W.zl & tmask, zr = W.zl >> tb, xt = W.xl & tmask, xr = W.xl >> tb;
      const std::string sx = thread_sign(zt);  // parity of (tid ^ xt) & zt = parity(tid & zt) ^ parity(xt & zt)
      const bool xpar = __builtin_popcount(xt & zt) & 1;
      const std::string st = x_(xpar ? "!" + sx : sx, tile_sign(W.ze));
      for (int e = 0; e < R; ++e) {
        const bool cneg = __builtin_popcount((e ^ (int)xr) & zr) & 1;
        o << "    l" << e << ".add<" << W.ph << ">(" << partner(e, W.xl) << ", P.c[" << w << "], "
          << (cneg ? "!(" + st + ")" : st) << ");\n";
      }
    }
    // lambda leaves registers: local index tid + (e << tb) in natural order
    o << "    { S* out = lam + base + st_t;\n";
    for (int e = 0; e < R; ++e) {
      std::string off;
      for (int m = 0; m < r; ++m)
        if ((e >> m) & 1) off += (off.empty() ? "" : " + ") + ("st_" + std::to_string(m));
      o << "      out[" << (off.empty() ? std::string("0") : off) << "] = A::store(l" << e << ".out());\n";
    }
    o << "    }\n";
    pre << "  const uint64_t st_t = (uint64_t)(tid & " << ((1u << b) - 1u) << "u) + lqs::row_offset(G, tid >> " << b
        << ");\n";
    for (int m = 0; m < r; ++m) pre << "  const uint64_t st_" << m << " = 1ull << G.h[" << (tb + m - b) << "];\n";
  }
  const std::string body = o.str(), prel = pre.str(), postl = post.str();
  uint64_t h = 1469598103934665603ull;
  for (unsigned char ch : body + prel + postl + aname) h = (h ^ ch) * 1099511628211ull;
  char nm[40];
  std::snprintf(nm, sizeof nm, "lqs_pauli_%016llx", (unsigned long long)(h ^ ((uint64_t)mode << 56)));
  kname = nm;
  const bool two_in = lam && !fresh;
  std::ostringstream s;
  s << "// compiled Pauli pass: " << nw << " words, mode " << mode << "\n"
    << "typedef unsigned char uint8_t;\ntypedef signed char int8_t;\ntypedef short int16_t;\ntypedef unsigned short uint16_t;\n"
       "typedef unsigned int uint32_t;\ntypedef unsigned long long uint64_t;\n"
    << "#include \"tile.cuh\"\n#include \"jit_dev.cuh\"\n"
    << "typedef " << aname << " A;\n"
    << "struct PArgs {\n  lqs::TileGeom g;\n  lqs::jit::PCoef<A>::T c[" << std::max(nw, 1) << "];\n};\n"
    << "extern \"C\" __global__ void __launch_bounds__(256, 2)\n"
    << kname << "(const A::S* __restrict__ psi, A::S* __restrict__ lam, const __grid_constant__ PArgs P, "
       "double* partial, int pstride, int* status) {\n"
       "  typedef A::S S;\n  typedef A::W W;\n"
       "  extern __shared__ __align__(128) unsigned char smem_raw[];\n"
       "  const lqs::TileGeom& G = P.g;\n"
       "  const uint32_t NT = 1u << G.k;\n"
       "  S* S0 = reinterpret_cast<S*>(smem_raw);\n"
    << "  S* S0L = S0 + NT * " << (two_in ? 1 : 0) << "u;\n"
    << "  W* XA = reinterpret_cast<W*>(S0 + NT * " << (two_in ? 2 : 1) << "u);\n"
    << "  double* wacc = reinterpret_cast<double*>(XA + NT * " << (need_xa ? 1 : 0) << "u);\n"
    << "  uint64_t* bar = reinterpret_cast<uint64_t*>(wacc + " << 8 * std::max(nw, 1) << ");\n"
       "  const uint32_t tid = threadIdx.x, warp = tid >> 5;\n"
       "  (void)S0L; (void)XA; (void)lam; (void)warp;\n"
    << "  for (uint32_t i = tid; i < " << 8 * std::max(nw, 1) << "u; i += blockDim.x) wacc[i] = 0.0;\n"
    << "  uint64_t t = blockIdx.x;\n"
       "  if (tid == 0) {\n    lqs::mbar_init(bar, 1);\n    lqs::fence_mbar_init();\n"
    << "    if (t < G.ntiles) lqs::jit::seg_expect(G, bar, " << (two_in ? 2 : 1) << "u);\n  }\n"
    << "  __syncthreads();\n"
       "  const uint64_t my_roff = tid < (1u << G.r) ? lqs::row_offset(G, tid) : 0ull;\n"
       "  if (t < G.ntiles) {\n    lqs::jit::seg_copy(G, S0, psi, lqs::tile_base(G, t), bar, my_roff);\n";
  if (two_in) s << "    lqs::jit::seg_copy(G, S0L, lam, lqs::tile_base(G, t), bar, my_roff);\n";
  s << "  }\n  uint32_t phase = 0;\n  bool ok = true;\n"
    << prel
    << "  for (; t < G.ntiles; t += gridDim.x) {\n"
       "    const uint64_t base = lqs::tile_base(G, t);\n"
       "    ok = __syncthreads_and(lqs::mbar_wait(bar, phase));\n"
       "    phase ^= 1u;\n    if (!ok) break;\n"
    << "    if (tid == 0 && t + gridDim.x < G.ntiles) lqs::jit::seg_expect(G, bar, " << (two_in ? 2 : 1) << "u);\n"
    << body << "  }\n" << postl
    << "  if (!ok && tid == 0) {\n    lqs::flag_timeout(status, 2);\n    lqs::mbar_wait(bar, phase ^ 1u);\n  }\n"
       "  __syncthreads();\n"
    << "  for (int w = tid; w < " << nw << "; w += blockDim.x) {\n"
       "    double v = 0.0;\n"
       "    for (int q = 0; q < 8; ++q) v += lqs::jit::slot_get<A>(wacc + q * "
    << nw << " + w);\n"
       "    partial[(size_t)w * pstride + blockIdx.x] = v;\n  }\n}\n";
  return s.str();
}

size_t pauli_smem(int k, size_t amp, int nw, int mode, bool need_xa) {
  const bool two_in = (mode & 2) && !(mode & 4);
  return (amp << k) * ((two_in ? 2 : 1) + (need_xa ? 1 : 0)) + sizeof(double) * 8 * std::max(nw, 1) + 16;
}

template <class A> struct PName;
template <> struct PName<ArF32> { static constexpr const char* s = "lqs::ArF32"; };
template <> struct PName<ArF64> { static constexpr const char* s = "lqs::ArF64"; };
template <> struct PName<ArDF> { static constexpr const char* s = "lqs::ArDF"; };

template <class A> typename std::conditional<std::is_same<A, ArF32>::value, float, DF>::type pcoef(double c);
template <> float pcoef<ArF32>(double c) { return (float)c; }
template <> DF pcoef<ArF64>(double c) { return split_const(c); }
template <> DF pcoef<ArDF>(double c) { return split_const(c); }

struct JPass {
  TileGeom g;
  std::vector<JWord> ws;
  std::vector<int> terms;
  int mode = 1;
  bool need_xa = false;
  void* entry = nullptr;
};

}  // namespace

// Plans the passes of a word set and gets (compiling when the mode allows, or
// `force`) their kernels; host only.
template <class A>
static int pauli_prepare_t(int n, int dtype, const lqs_pauli* terms, int n_terms, bool lambda, bool force,
                           std::vector<JPass>& passes, int* compiled) {
  const int k = dtype == LQS_C64 ? 12 : 11, b = dtype == LQS_C64 ? 5 : 4;
  if (n <= k) return set_error(LQS_ERR_UNSUPPORTED, "state fits one tile");
  std::vector<PassPlan> plan;
  std::vector<int> wide;
  LQS_TRY(plan_passes(n, terms, n_terms, k, b, plan, wide, kPauliWordsJit));
  if (!wide.empty()) return set_error(LQS_ERR_UNSUPPORTED, "a word's X/Y qubits do not fit a tile");
  if (plan.empty()) return set_error(LQS_ERR_UNSUPPORTED, "no words");
  const size_t amp = sizeof(typename A::S);
  passes.assign(plan.size(), JPass{});
  std::vector<void*> todo;
  for (size_t pi = 0; pi < plan.size(); ++pi) {
    JPass& P = passes[pi];
    P.g = geom_for(n, plan[pi].Q, k, b, amp);
    P.terms = plan[pi].words;
    P.mode = lambda ? (pi == 0 ? 7 : 3) : 1;
    for (int w : P.terms) {
      const PWord pw = make_pword(P.g, terms[w]);
      P.ws.push_back(JWord{pw.xl, pw.zl, pw.ze, (int)pw.ph, pw.lowbit});
      if (pw.xl & ((1u << kPauliThreadBits) - 1u)) P.need_xa = true;
    }
    std::string key = "pauli";
    key += PName<A>::s;
    const int hdr[4] = {k, b, P.mode, (int)P.ws.size()};
    key.append(reinterpret_cast<const char*>(hdr), sizeof hdr);
    for (const JWord& w : P.ws) key.append(reinterpret_cast<const char*>(&w), sizeof w);
    std::string why;
    const auto gen = [&](std::string& src, std::string& name, std::string&) {
      src = pauli_source(PName<A>::s, k, b, P.ws, P.mode, name);
      return true;
    };
    P.entry = jit_entry_generic(key, gen, true, &why);
    if (!P.entry) return set_error(LQS_ERR_UNSUPPORTED, "Pauli pass not compiled: " + why);
    if (!force && !jit_should_compile(P.entry, n)) return set_error(LQS_ERR_UNSUPPORTED, "Pauli pass not compiled yet");
    if (std::find(todo.begin(), todo.end(), P.entry) == todo.end()) todo.push_back(P.entry);
  }
  int before = 0, good = 0;
  std::string err;
  jit_states(todo, &before, &err);
  LQS_TRY(jit_compile(todo));
  if (jit_states(todo, &good, &err) != LQS_OK) return set_error(LQS_ERR_UNSUPPORTED, "Pauli pass: " + err);
  if (compiled) *compiled = good - before;
  return LQS_OK;
}

template <class A>
static int pauli_compiled_t(SV* sv, const lqs_pauli* terms, int n_terms, void* lam, int arith, double* vals) {
  using CT = typename std::conditional<std::is_same<A, ArF32>::value, float, DF>::type;
  const int n = sv->n;
  const int k = sv->dtype == LQS_C64 ? 12 : 11;
  std::vector<JPass> passes;
  LQS_TRY(pauli_prepare_t<A>(n, sv->dtype, terms, n_terms, lam != nullptr, false, passes, nullptr));
  const size_t amp = sizeof(typename A::S);
  // one grid for every pass (the partial rows share a stride)
  int per_sm = 8;
  for (auto& P : passes) {
    int ps = 0;
    LQS_TRY(jit_occupancy_generic(P.entry, sv->device, pauli_smem(k, amp, (int)P.ws.size(), P.mode, P.need_xa), 256,
                                  &ps));
    per_sm = std::min(per_sm, ps);
  }
  const uint64_t ntiles = 1ull << (n - k);
  const int grid = (int)std::min<uint64_t>(ntiles, (uint64_t)std::max(sv->sms, 1) * std::max(per_sm, 1));
  size_t slots = 0;
  for (auto& P : passes) slots += P.ws.size();
  void* scratch = nullptr;
  LQS_TRY(sv_scratch(sv, 2, sizeof(double) * (slots * grid + slots), &scratch));
  double* partial = static_cast<double*>(scratch);
  double* sums = partial + slots * grid;
  size_t off = 0;
  const std::string pname =
      std::string(lam ? "k_pauli_lambda_jit/" : "k_pauli_jit/") + arith_tag(sv->dtype, arith);
  for (auto& P : passes) {
    const int nw = (int)P.ws.size();
    const size_t coff = (sizeof(TileGeom) + alignof(CT) - 1) / alignof(CT) * alignof(CT);
    std::vector<unsigned char> args((coff + sizeof(CT) * std::max(nw, 1) + 15) / 16 * 16, 0);
    std::memcpy(args.data(), &P.g, sizeof(TileGeom));
    for (int w = 0; w < nw; ++w) {
      const CT c = pcoef<A>(terms[P.terms[w]].coeff);
      std::memcpy(args.data() + coff + sizeof(CT) * w, &c, sizeof(CT));
    }
    const void* psi = sv->d;
    void* lm = lam;
    double* part = partial + off * grid;
    int pstride = grid;
    int* status = sv->d_status;
    void* kp[] = {&psi, &lm, args.data(), &part, &pstride, &status};
    const double S = (double)sv->bytes();
    const double bytes = S * (1.0 + ((P.mode & 2) ? ((P.mode & 4) ? 1.0 : 2.0) : 0.0));
    LQS_TRY(jit_launch_generic(P.entry, sv, (unsigned)grid, 256, pauli_smem(k, amp, nw, P.mode, P.need_xa), kp,
                               pname.c_str(), bytes, 8.0 * nw * (double)sv->N()));
    off += nw;
  }
  k_sum_partials_launch(partial, grid, sums, (int)slots, sv->stream);
  std::vector<double> h(slots);
  LQS_CUDA_TRY(cudaMemcpyAsync(h.data(), sums, sizeof(double) * slots, cudaMemcpyDeviceToHost, sv->stream));
  LQS_CUDA_TRY(cudaStreamSynchronize(sv->stream));
  off = 0;
  for (auto& P : passes)
    for (size_t i = 0; i < P.ws.size(); ++i) {
      const double v = h[off++];
      vals[P.terms[i]] = P.ws[i].xl ? 2.0 * v : v;  // X/Y words counted each pair once
    }
  int status[2] = {0, 0};
  LQS_CUDA_TRY(cudaMemcpy(status, sv->d_status, sizeof status, cudaMemcpyDeviceToHost));
  if (status[0]) {
    cudaMemset(sv->d_status, 0, 64);
    return set_error(LQS_ERR_TIMEOUT, "a tile load did not complete (bounded wait expired)");
  }
  return LQS_OK;
}

int pauli_precompile(int n, int dtype, int arith, const lqs_pauli* terms, int n_terms, bool lambda, int* compiled) {
  std::vector<JPass> passes;
  if (dtype == LQS_C64) return pauli_prepare_t<ArF32>(n, dtype, terms, n_terms, lambda, true, passes, compiled);
  if (arith == LQS_ARITH_F64) return pauli_prepare_t<ArF64>(n, dtype, terms, n_terms, lambda, true, passes, compiled);
  return pauli_prepare_t<ArDF>(n, dtype, terms, n_terms, lambda, true, passes, compiled);
}

int pauli_compiled(SV* sv, const lqs_pauli* terms, int n_terms, void* lam, int arith, double* vals) {
  if (sv->dtype == LQS_C64) return pauli_compiled_t<ArF32>(sv, terms, n_terms, lam, arith, vals);
  if (arith == LQS_ARITH_F64) return pauli_compiled_t<ArF64>(sv, terms, n_terms, lam, arith, vals);
  return pauli_compiled_t<ArDF>(sv, terms, n_terms, lam, arith, vals);
}

}  // namespace lqs
