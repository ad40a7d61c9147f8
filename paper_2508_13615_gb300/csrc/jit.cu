// Segment compiler: a fused segment's register-tile program, compiled into a
// straight-line kernel.  The gates are the paper's pair and quad updates on
// local qubits (Sec. 2, Fig. 1a), here on the qubits of a tile held on chip.
//
// The register-tile interpreter (fused_reg.cu) reads each op of a segment at
// run time: its kind, its register slot, its control pattern and its
// coefficient offsets, and for every amplitude it tests predicates against
// layout tables.  On GB300 that dispatch costs more issue slots than the
// gate arithmetic itself.  Here the same program is written out as CUDA C++
// in which all of that is constant: the register element of every pair, which
// elements a register-held control selects, the thread part of each layout
// (a handful of shifts once per exchange), and the parameter-space offset of
// each coefficient.  Uncontrolled X/CNOT-type swaps become renamings of
// register variables.  The coefficients stay kernel parameters, so circuits
// that differ only in their angles share one compiled kernel.
//
// The source is compiled for sm_103a by NVRTC (loaded with dlopen, so the
// library has no link-time dependency on it) and loaded through the driver
// API (entry points obtained from the runtime), once per structure and
// device; kernels are cached for the life of the process.
#include <dlfcn.h>
#include <cuda.h>
#include <nvrtc.h>

#include <functional>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <sstream>
#include <string>
#include <type_traits>
#include <thread>
#include <unordered_map>
#include <vector>

#include "arith.cuh"
#include "jit.h"
#include "lqs_internal.cuh"
#include "tile.cuh"

#include "jit_headers.inc"  // kJitHeaderNames / kJitHeaderSources (written by the build)

namespace lqs {

// ---------------------------------------------------------------------------
// source generation
// ---------------------------------------------------------------------------
namespace {

std::string replace_all(std::string s, const std::string& a, const std::string& b);

uint32_t host_swz(uint32_t j, int sz) {
  if (sz == 16) return j ^ (((j >> 3) ^ (j >> 6) ^ (j >> 9)) & 7u);
  return j ^ (((j >> 4) ^ (j >> 8)) & 15u);
}

// An exchange's swizzle: swz<sz> with the bank bits of some positions
// changed.  dm[b] lists the positions whose contribution to bank bit b
// flips (jit_dev.cuh pfold); all zero is swz<sz> itself.
//
// The additive form (add) has no swz<sz> base: the bank bits of position j
// are its own low bits changed by the parities in dm, and dm names only
// positions that are thread bits in both layouts of the exchange and changes
// only bank bits that are not register positions.  The swizzled index of a
// thread's amplitude is then its thread part's swizzled index plus its
// register part unchanged (disjoint bits), so each access adds a constant
// offset to one per-thread index instead of XORing it.
struct XSwz {
  uint32_t dm[4] = {0, 0, 0, 0};
  bool add = false;
  bool plain() const { return !(dm[0] | dm[1] | dm[2] | dm[3]); }
};
uint32_t host_xswz(uint32_t j, int sz, const XSwz& x) {
  uint32_t f = 0;
  for (int b = 0; b < 4; ++b) f |= (uint32_t)(__builtin_popcount(j & x.dm[b]) & 1) << b;
  return (x.add ? j : host_swz(j, sz)) ^ f;
}

constexpr int kMaxGradSlotsJit = 128;  // gradient slots per compiled adjoint segment
// Amplitude updates between renormalisations of the double-float registers.
// The updates leave their results unrenormalised (jit_dev.cuh), and the low
// parts grow with each one; a host simulation of 3000 random gates on 12
// qubits kept the error of normalised double-float (2.5e-14) with up to 32
// updates between renormalisations, and 2-5x that at 64-128.
constexpr int kRenormEvery = 16;

// A forward program's unit-row forms leave every amplitude scaled by 1/g, the
// product of their factors.  The scalar commutes with every op, so it is
// folded into the constant of the first merged diagonal run that multiplies
// every amplitude (no controls); without one the store scales by g.  The
// generator and the parameter block both take the run this picks.
int gscale_sink(const TOp* ops, int nops) {
  for (int i = 0; i < nops; ++i)
    if (ops[i].kind == K_DPROD && ops[i].lcmask == 0 && ops[i].ecmask == 0) return i;
  return -1;
}

std::string hex(uint64_t x) {
  char b[32];
  std::snprintf(b, sizeof b, "0x%llxull", (unsigned long long)x);
  return b;
}
std::string hex32(uint32_t x) {
  char b[24];
  std::snprintf(b, sizeof b, "0x%xu", x);
  return b;
}

class SegGen {
 public:
  // adjoint: the kernel carries psi and lambda (same layout and renamings),
  // and ops with a gradient slot (and K_GRAD partials) add Im<lambda|G|psi>.
  SegGen(int k, int b, int r, const char* aname, int amp_bytes, bool adjoint)
      : k_(k), b_(b), r_(r), R_(1 << r), aname_(aname), sz_(amp_bytes), adj_(adjoint),
        xpair_(adjoint && amp_bytes == 16) {}
  void set_folds(const TFold* f) { folds_ = f; }

  // Returns false (with a reason) for a program this generator does not take.
  bool run(const TOp* ops, int nops, int ncoef, int ngrad, std::string& src, std::string& kname, std::string& why);

 private:
  int k_, b_, r_, R_;
  const char* aname_;
  int sz_;
  bool adj_;
  const char* pfx_ = "v";       // variables of the state being emitted ("v" psi, "u" lambda)
  int xb_ = 0;                  // exchange buffer of the next exchange (they alternate)
  // complex128 adjoint: psi and lambda cross each exchange together, through
  // the pair XA/XB or XC/XD (alternating), under one barrier
  bool xpair_ = false;
  int xp_ = 0;
  int next_bar_ = 1;            // next free named barrier id in this tile iteration (0 is the block barrier)
  int slot_[4] = {0, 0, 0, 0};  // register slot m -> local position
  int thr_[16] = {0};           // thread bit m -> local position
  int vm_[16];                  // register element -> variable
  int uid_ = 0;
  std::ostringstream o_;    // tile-loop body
  std::ostringstream pre_;  // before the tile loop (tile-independent per-thread values)
  std::string why_;
  std::vector<std::pair<std::string, int>> pend_;  // gradient partials awaiting a batched warp sum
  int ntab_ = 0;  // entries of the shared table of outside-qubit factor products
  int nut_ = 0;   // entries of the shared tables of tile-independent diagonal runs (UT)
  std::vector<std::string> ofac_;  // per run with outside factors: its per-tile product (OF)
  int lz_ = 0;    // amplitude updates since the registers were last renormalised
  // Exchanges since the last block-wide barrier, for the ordering check of
  // a buffer's next writes (exchange_safe): per exchange its buffer, the warp
  // writing and the warp reading each buffer position, and its barrier's
  // groups (warps agreeing on the tid bits of gmask; 0 = the whole block).
  struct XRec {
    uint32_t bufs;  // buffers written and read by the exchange (bit per buffer)
    bool writes;  // its writes are not yet ordered before everything (no block barrier after them)
    std::vector<uint8_t> wown, rown;
    uint32_t gmask;
  };
  std::vector<XRec> xhist_;
  std::vector<uint8_t> owners(const XSwz& xs) const;
  std::vector<char> reach(int v, size_t from) const;
  bool exchange_safe(int buf, const std::vector<uint8_t>& wown) const;
  int nu_ = 0;    // forward: orthogonal real 2x2 ops applied in unit-row form (their g's scale the store)
  const TFold* folds_ = nullptr;  // permutation runs folded into layout changes (TOp::fold)
  const TFold* wfold_ = nullptr;  // the fold of the exchange being written (owners() maps through it)
  // F x (the linear part of a fold) on local position bits
  static uint32_t fold_lin(const TFold& F, uint32_t x) {
    uint32_t y = 0;
    for (int p = 0; x; ++p, x >>= 1)
      if (x & 1u) y ^= F.col[p];
    return y;
  }

  int nthreads() const { return 1 << (k_ - r_); }
  // Double-float segments take the states' format as a launch-time argument:
  // bit 0, the tiles hold hi/lo float pairs (written by the previous compiled
  // segment of the same call) instead of float64; bit 1, leave hi/lo pairs
  // for the next one.  Both skip the float64 conversions.
  bool split_io() const { return aname_ == std::string("lqs::ArDF"); }
  // Double-float adjoint sweeps un-apply orthogonal real 2x2 ops (RY, H) in
  // the unit-row form too, always pivoting on m00 (one form, no launch-time
  // bit): both states grow by 1/m00 per op, which the host takes out of the
  // gradient partials (seg_scales) and folds into a diagonal run or a final
  // scale; launches whose product of m00's is too small run elsewhere.
  bool unit_adj() const { return adj_ && aname_ == std::string("lqs::ArDF"); }
  // Complex64 forward segments do too little arithmetic per tile to hide a
  // tile load behind it: they keep two incoming buffers (two tiles in flight
  // per CTA) and run every layout exchange through one buffer.
  bool deep() const { return !adj_ && aname_ == std::string("lqs::ArF32"); }
  void flush_pending(bool all);
  // runs f once per state, with V() naming that state's variables
  template <class F>
  void each(F f) {
    pfx_ = "v";
    f();
    if (adj_) {
      pfx_ = "u";
      f();
    }
    pfx_ = "v";
  }
  bool set_layout(uint64_t packed);
  uint32_t je(int e) const {
    uint32_t x = 0;
    for (int m = 0; m < r_; ++m)
      if ((e >> m) & 1) x |= 1u << slot_[m];
    return x;
  }
  int reg_slot(int pos) const {
    for (int m = 0; m < r_; ++m)
      if (slot_[m] == pos) return m;
    return -1;
  }
  uint32_t reg_positions() const {
    uint32_t x = 0;
    for (int m = 0; m < r_; ++m) x |= 1u << slot_[m];
    return x;
  }
  std::string jt_expr() const;
  std::string V(int e) const { return std::string(pfx_) + std::to_string(vm_[e]); }
  std::string Vs(const char* s, int e) const { return std::string(s) + std::to_string(vm_[e]); }
  std::string cref(int i) const { return "P.coef[" + std::to_string(i) + "]"; }
  std::string fresh(const char* p) { return std::string(p) + std::to_string(uid_++); }
  // predicate of the op's thread-held and outside controls ("" when none),
  // and the register-slot mask its register-held controls require
  std::string pred(uint32_t lc, uint64_t ec, uint32_t& regc) const;
  std::string barrier_for(uint64_t to, uint32_t* gmask);
  bool emit_op(const TOp& t);
  XSwz pick_swizzle(const uint32_t* wv, const uint32_t* rv, uint32_t regmask) const;
  // "sj ^ c" or, for an additive swizzle, "sj + c": one access of an exchange
  std::string xacc(const XSwz& xs, uint32_t pos) const {
    return std::string(xs.add ? "sj + " : "sj ^ ") + hex32(host_xswz(pos, sz_, xs));
  }
  std::string swz_expr(const std::string& j, const XSwz& x) const;
  bool emit_grad(const TOp& t);
  bool emit_grad_block(const TOp* ops, int count);
  void emit_layout(const TOp& t);
  int smem_read_degree() const;
  bool store_friendly() const;
  void emit_store();
  bool fail(const std::string& w) {
    why_ = w;
    return false;
  }
};

bool SegGen::set_layout(uint64_t packed) {
  uint32_t seen = 0;
  for (int i = 0; i < k_; ++i) {
    const int p = (int)((packed >> (4 * i)) & 15u);
    if (p >= k_ || ((seen >> p) & 1u)) return false;  // not a permutation of the tile bits
    seen |= 1u << p;
    if (i < r_) slot_[i] = p;
    else thr_[i - r_] = p;
  }
  return true;
}

std::string SegGen::jt_expr() const {
  const int tb = k_ - r_;
  std::string s;
  for (int m = 0; m < tb;) {
    int len = 1;
    while (m + len < tb && thr_[m + len] == thr_[m] + len) ++len;
    const uint32_t mask = (1u << len) - 1u;
    std::string term = m ? "(tid >> " + std::to_string(m) + ")" : std::string("tid");
    if (m + len < 32 && !(m == 0 && len == tb)) term = "(" + term + " & " + hex32(mask) + ")";
    if (thr_[m]) term = "(" + term + " << " + std::to_string(thr_[m]) + ")";
    s += s.empty() ? term : " | " + term;
    m += len;
  }
  return s.empty() ? std::string("0u") : s;
}

std::string SegGen::pred(uint32_t lc, uint64_t ec, uint32_t& regc) const {
  regc = 0;
  uint32_t thc = 0;
  for (int p = 0; p < k_; ++p) {
    if (!((lc >> p) & 1u)) continue;
    const int m = reg_slot(p);
    if (m >= 0) regc |= 1u << m;
    else thc |= 1u << p;
  }
  std::string s;
  if (thc) s = "((jt & " + hex32(thc) + ") == " + hex32(thc) + ")";
  if (ec) s += std::string(s.empty() ? "" : " && ") + "((base & " + hex(ec) + ") == " + hex(ec) + ")";
  return s;
}

// The barrier of one exchange into layout `to`.  Warp-index thread bits that
// keep their position confine the exchange to the warps agreeing on them
// (each group keeps its set of amplitudes), so only those warps synchronise:
// __syncwarp when no warp bit moves, a named barrier per group when some do,
// the block barrier when all do.  Every group barrier of a tile iteration
// gets ids of its own: a warp may reach a later exchange while warps of
// another group are still at an earlier one, and two barrier instances must
// never share an id.  When the ids run out the block barrier is used; block
// barriers (here and at the top of the tile loop) make all ids free again.
std::string SegGen::barrier_for(uint64_t to, uint32_t* gmask) {
  uint32_t fixed = 0, moved = 0;
  for (int m = 5; m < k_ - r_; ++m) {
    const int q = (int)((to >> (4 * (r_ + m))) & 15u);
    if (q == thr_[m]) fixed |= 1u << m;
    else moved |= 1u << m;
  }
  const int groups = 1 << __builtin_popcount(fixed);
  *gmask = fixed;
  if (!moved) return "__syncwarp();";
  if (!fixed || next_bar_ + groups - 1 > 15) {
    next_bar_ = 1;  // every warp passes it after all earlier group barriers completed
    *gmask = 0;
    return "__syncthreads();";
  }
  std::string id;
  int j = 0;
  for (int m = 5; m < k_ - r_; ++m)
    if ((fixed >> m) & 1u) {
      id += " + (((tid >> " + std::to_string(m) + ") & 1u) << " + std::to_string(j) + ")";
      ++j;
    }
  std::string bar = "lqs::jit::bar_group(" + std::to_string(next_bar_) + "u" + id + ", " +
                    std::to_string(32u << __builtin_popcount(moved)) + "u);";
  next_bar_ += groups;
  return bar;
}

// A warp's shared-memory access is served 128 bytes at a time, so the lanes
// of one phase (lane bits 0..nb-1: 8 lanes of 16-byte amplitudes, 16 of
// 8-byte ones) conflict unless their addresses fall in distinct bank groups.
// The bank group of a swizzled position is a linear map F of its bits (the
// low nb bits, plus the folded higher ones).  An exchange is conflict-free on
// both sides when F is one-to-one on the lane positions of the layout that
// writes and on those of the layout that reads.  The default fold of
// positions mod nb fails when two lane positions share a residue, so each
// exchange re-assigns the fold of the higher lane positions when it must
// (a small backtracking search), writes and reads through that swizzle, and
// leaves every other exchange on the default.
XSwz SegGen::pick_swizzle(const uint32_t* wv, const uint32_t* rv, uint32_t regmask) const {
  // wv / rv: the position vectors of the lane bits of the writing and the
  // reading layout (single positions, or their images under a fold);
  // regmask: the register positions of both layouts (0: no additive form)
  const int nb = sz_ == 16 ? 3 : 4;
  XSwz x;
  if (k_ - r_ < nb) return x;
  if (regmask) {
    // the additive form: bank bits are the low position bits, changed only
    // by positions that are thread bits in both layouts, and never on a bank
    // bit that is a register position
    const uint32_t okb = ((1u << nb) - 1u) & ~regmask;
    uint32_t ga[16];
    for (int p = 0; p < 16; ++p) ga[p] = p < nb ? 1u << p : 0u;
    auto bank_a = [&](uint32_t v) {
      uint32_t y = 0;
      for (int p = 0; v; ++p, v >>= 1)
        if (v & 1u) y ^= ga[p];
      return y;
    };
    auto rank_a = [&](const uint32_t* vec) {
      uint32_t span = 1u;
      for (int i = 0; i < nb; ++i) {
        const uint32_t v = bank_a(vec[i]);
        uint32_t next = span;
        for (uint32_t u = 0; u < (1u << nb); ++u)
          if ((span >> u) & 1u) next |= 1u << (u ^ v);
        span = next;
      }
      return span == (nb == 3 ? 0xFFu : 0xFFFFu);
    };
    std::vector<int> fp;  // thread positions above the bank bits met by a lane vector
    for (int i = 0; i < nb; ++i)
      for (uint32_t v : {wv[i], rv[i]})
        for (int p = nb; p < k_; ++p)
          if (((v >> p) & 1u) && !((regmask >> p) & 1u) && std::find(fp.begin(), fp.end(), p) == fp.end())
            fp.push_back(p);
    std::function<bool(size_t)> search_a = [&](size_t i) {
      if (i == fp.size()) return rank_a(wv) && rank_a(rv);
      const int p = fp[i];
      for (uint32_t v = 0; v < (1u << nb); ++v) {
        if (v & ~okb) continue;
        ga[p] = v;
        if (search_a(i + 1)) return true;
      }
      ga[p] = 0;
      return false;
    };
    if (search_a(0)) {
      x.add = true;
      for (int p = nb; p < k_; ++p)
        for (int bb = 0; bb < nb; ++bb)
          if ((ga[p] >> bb) & 1u) x.dm[bb] |= 1u << p;
      return x;
    }
    x = XSwz();
  }
  auto dflt = [&](int p) { return host_swz(1u << p, sz_) & ((1u << nb) - 1u); };  // bank bits of swz<sz>
  uint32_t g[16];
  for (int p = 0; p < 16; ++p) g[p] = dflt(p);
  auto bank = [&](uint32_t v) {
    uint32_t y = 0;
    for (int p = 0; v; ++p, v >>= 1)
      if (v & 1u) y ^= g[p];
    return y;
  };
  auto full_rank = [&](const uint32_t* vec) {
    uint32_t span = 1u;  // bit u set: vector u is in the span
    for (int i = 0; i < nb; ++i) {
      const uint32_t v = bank(vec[i]);
      uint32_t next = span;
      for (uint32_t u = 0; u < (1u << nb); ++u)
        if ((span >> u) & 1u) next |= 1u << (u ^ v);
      span = next;
    }
    return span == (nb == 3 ? 0xFFu : 0xFFFFu);
  };
  if (full_rank(wv) && full_rank(rv)) return x;
  std::vector<int> free_pos;  // positions above the low bits met by a lane vector: their fold can change
  for (int i = 0; i < nb; ++i)
    for (uint32_t v : {wv[i], rv[i]})
      for (int p = nb; p < k_; ++p)
        if (((v >> p) & 1u) && std::find(free_pos.begin(), free_pos.end(), p) == free_pos.end()) free_pos.push_back(p);
  std::function<bool(size_t)> search = [&](size_t i) {
    if (i == free_pos.size()) return full_rank(wv) && full_rank(rv);
    const int p = free_pos[i];
    for (uint32_t v = 1; v < (1u << nb); ++v) {
      g[p] = v;
      if (search(i + 1)) return true;
    }
    g[p] = dflt(p);
    return false;
  };
  if (!search(0)) return x;  // no conflict-free fold found; keep the default
  for (int p = nb; p < k_; ++p) {
    const uint32_t d = g[p] ^ dflt(p);
    for (int bb = 0; bb < nb; ++bb)
      if ((d >> bb) & 1u) x.dm[bb] |= 1u << p;
  }
  return x;
}

std::string SegGen::swz_expr(const std::string& j, const XSwz& x) const {
  std::string e = x.add ? j : "lqs::jit::swz<" + std::to_string(sz_) + ">(" + j + ")";
  if (x.plain()) return e;
  return e + " ^ lqs::jit::pfold(" + j + ", " + hex32(x.dm[0]) + ", " + hex32(x.dm[1]) + ", " + hex32(x.dm[2]) +
         ", " + hex32(x.dm[3]) + ")";
}

// Buffer position -> the warp that holds the amplitude there, in the current
// layout under swizzle xs.
std::vector<uint8_t> SegGen::owners(const XSwz& xs) const {
  std::vector<uint8_t> own((size_t)1 << k_, 0);
  const int nt = nthreads();
  for (int tid = 0; tid < nt; ++tid) {
    uint32_t jt = 0;
    for (int m = 0; m < k_ - r_; ++m)
      if ((tid >> m) & 1) jt |= 1u << thr_[m];
    for (int e = 0; e < R_; ++e) {
      const uint32_t j = jt | je(e);
      own[host_xswz(wfold_ ? (fold_lin(*wfold_, j) ^ wfold_->cst) : j, sz_, xs)] = (uint8_t)(tid >> 5);
    }
  }
  return own;
}

// Warps whose execution after the last recorded barrier is ordered after
// something warp v did before barrier xhist_[from] (every later barrier
// passes the order on to the warps of the group it synchronises).
std::vector<char> SegGen::reach(int v, size_t from) const {
  const int nw = nthreads() / 32;
  std::vector<char> in((size_t)nw, 0);
  in[(size_t)v] = 1;
  for (size_t m = from; m < xhist_.size(); ++m) {
    const uint32_t g = xhist_[m].gmask;
    std::vector<char> nx((size_t)nw, 0);
    for (int u = 0; u < nw; ++u)
      if (in[(size_t)u])
        for (int x = 0; x < nw; ++x)
          if ((((uint32_t)u << 5) & g) == (((uint32_t)x << 5) & g)) nx[(size_t)x] = 1;
    in.swap(nx);
  }
  return in;
}

// Whether the writes of a new exchange into buffer `buf` (position -> writing
// warp) are ordered after every earlier access of the same positions since
// the last block-wide barrier: the earlier writes (before their exchange's
// barrier) and reads (after it).  Group barriers order only the warps of a
// group, so a warp may run an exchange or two ahead of another group.
bool SegGen::exchange_safe(int buf, const std::vector<uint8_t>& wown) const {
  const int nw = nthreads() / 32;
  for (size_t j = 0; j < xhist_.size(); ++j) {
    const XRec& h = xhist_[j];
    if (!((h.bufs >> buf) & 1u)) continue;
    std::vector<std::vector<char>> rw((size_t)nw), rr((size_t)nw);
    for (int v = 0; v < nw; ++v) {
      if (h.writes) rw[(size_t)v] = reach(v, j);
      rr[(size_t)v] = reach(v, j + 1);
    }
    for (size_t p = 0; p < wown.size(); ++p) {
      const int w = wown[p];
      if (h.writes && !rw[h.wown[p]][(size_t)w]) return false;
      if (!rr[h.rown[p]][(size_t)w]) return false;
    }
  }
  return true;
}

void SegGen::emit_layout(const TOp& t) {
  // Each state is written in the current layout and read back in the new one
  // through its own buffer.  The buffers alternate, so one barrier per state
  // suffices: the previous reader of a buffer finished before the
  // intervening exchange's barrier (or the barriers at the top of the tile
  // loop).  A folded permutation run (t.fold) moves every amplitude from its
  // storage position x to F x ^ c on the way: the writes go to the permuted
  // positions, the reads are those of the new layout.
  const TFold* F = t.fold && folds_ ? &folds_[t.fold - 1] : nullptr;
  uint32_t old_je[16];
  for (int e = 0; e < R_; ++e) old_je[e] = je(e);
  const int saved_slot[4] = {slot_[0], slot_[1], slot_[2], slot_[3]};
  int saved_thr[16];
  std::copy(thr_, thr_ + 16, saved_thr);
  // lane position vectors of the writing (through the fold) and the reading layout
  uint32_t wv[4], rv[4];
  for (int i = 0; i < 4; ++i) {
    const int p = i < k_ - r_ ? thr_[i] : 0;
    wv[i] = F ? (uint32_t)F->col[p] : 1u << p;
  }
  for (int i = 0; i < 4; ++i) {
    const int q = r_ + i < k_ ? (int)((t.ecmask >> (4 * (r_ + i))) & 15u) : 0;
    rv[i] = 1u << q;
  }
  uint32_t regmask = 0;  // register positions of the writing and the reading layout (none with a fold)
  if (!F) {
    regmask = reg_positions();
    for (int m = 0; m < r_; ++m) regmask |= 1u << ((t.ecmask >> (4 * m)) & 15u);
  }
  const XSwz xs = pick_swizzle(wv, rv, regmask);
  // the thread's write index: jt itself, or F jt ^ c (c from the tile's outside bits)
  std::string wj = "jt";
  if (F) {
    wj = fresh("fj");
    o_ << "    const uint32_t " << wj << " = jt";
    for (int m = 0; m < k_ - r_; ++m) {
      const int p = thr_[m];
      const uint32_t d = (uint32_t)F->col[p] ^ (1u << p);
      if (d) o_ << " ^ ((0u - ((jt >> " << p << ") & 1u)) & " << hex32(d) << ")";
    }
    if (F->cst) o_ << " ^ " << hex32(F->cst);
    for (int j = 0; j < F->nout; ++j)
      if (F->omask[j]) o_ << " ^ ((0u - lqs::jit::obit(base, " << (int)F->oq[j] << ")) & " << hex32(F->omask[j]) << ")";
    o_ << ";\n";
  }
  std::string jo;
  if (adj_) {
    jo = fresh("jo");
    o_ << "    const uint32_t " << jo << " = " << swz_expr(wj, xs) << ";\n";
  }
  bool first = true;
  // who writes and who reads each buffer position in this exchange (with the
  // fold, for a tile whose outside bits are 0; a folded exchange is fenced by
  // block barriers, which hold for every tile)
  wfold_ = F;
  const std::vector<uint8_t> wown = owners(xs);
  wfold_ = nullptr;
  set_layout(t.ecmask);
  const std::vector<uint8_t> rown = owners(xs);
  std::copy(saved_slot, saved_slot + 4, slot_);
  std::copy(saved_thr, saved_thr + 16, thr_);
  if (xpair_) {
    // both states: writes into the pair, one barrier, reads from the pair.
    // The pair used two exchanges ago was last read before the previous
    // exchange's barrier.
    const int bp = 2 * xp_, bl = 2 * xp_ + 1;
    const char* XP = xp_ ? "XC" : "XA";
    const char* XL = xp_ ? "XD" : "XB";
    xp_ ^= 1;
    bool unsafe = !exchange_safe(bp, wown) || !exchange_safe(bl, wown);
    if (F)
      for (const XRec& h : xhist_) unsafe = unsafe || ((h.bufs >> bp) & 1u) || ((h.bufs >> bl) & 1u);
    if (unsafe) {
      o_ << "    __syncthreads();  // earlier users of these buffers are not ordered before these writes\n";
      next_bar_ = 1;
      xhist_.clear();
    }
    uint32_t gmask = 0;
    std::string bar;
    if (F) {
      bar = "__syncthreads();";
      next_bar_ = 1;
    } else {
      bar = barrier_for(t.ecmask, &gmask);
    }
    if (!gmask) xhist_.clear();
    xhist_.push_back(XRec{(1u << bp) | (1u << bl), gmask != 0, wown, rown, gmask});
    o_ << "    { const uint32_t sj = " << jo << ";\n";
    for (const char* pf : {"v", "u"}) {
      pfx_ = pf;
      for (int e = 0; e < R_; ++e) {
        const uint32_t pos = F ? fold_lin(*F, old_je[e]) : old_je[e];
        o_ << "      lqs::st_w(&" << (pf[0] == 'v' ? XP : XL) << "[" << xacc(xs, pos) << "], " << V(e) << ");\n";
      }
    }
    pfx_ = "v";
    o_ << "    }\n    " << bar << "\n";
    set_layout(t.ecmask);  // validated by the caller
    o_ << "    jt = " << jt_expr() << ";\n";
    o_ << "    { const uint32_t sj = " << swz_expr("jt", xs) << ";\n";
    for (const char* pf : {"v", "u"})
      for (int e = 0; e < R_; ++e)
        o_ << "      " << pf << e << " = lqs::ld_w(&" << (pf[0] == 'v' ? XP : XL) << "[" << xacc(xs, je(e)) << "]);\n";
    o_ << "    }\n";
    for (int e = 0; e < R_; ++e) vm_[e] = e;
    if (t.e0 != t.ecmask) {
      set_layout(t.e0);
      o_ << "    jt = " << jt_expr() << ";\n";
    }
    return;
  }
  each([&]() {
    const int xi = xb_;
    const char* X = xb_ ? "XB" : "XA";
    if (!deep()) xb_ ^= 1;  // deep: XA only (the second incoming buffer took XB's place)
    std::copy(saved_slot, saved_slot + 4, slot_);  // barrier groups compare with the current layout
    std::copy(saved_thr, saved_thr + 16, thr_);
    bool unsafe = !exchange_safe(xi, wown);
    if (F)  // the write positions move with each tile's outside bits: no earlier user of the buffer may be pending
      for (const XRec& h : xhist_) unsafe = unsafe || ((h.bufs >> xi) & 1u);
    if (unsafe) {
      // a warp of another group may still use this buffer's positions from
      // an earlier exchange: wait for the whole block first
      o_ << "    __syncthreads();  // earlier users of this buffer are not ordered before these writes\n";
      next_bar_ = 1;
      xhist_.clear();
    }
    uint32_t gmask = 0;
    std::string bar;
    if (F) {
      bar = "__syncthreads();";
      next_bar_ = 1;
    } else {
      bar = barrier_for(t.ecmask, &gmask);
    }
    if (!gmask) xhist_.clear();
    xhist_.push_back(XRec{1u << xi, gmask != 0, wown, rown, gmask});
    if (adj_) o_ << "    { const uint32_t sj = " << jo << ";\n";
    else o_ << "    { const uint32_t sj = " << swz_expr(wj, xs) << ";\n";
    for (int e = 0; e < R_; ++e) {
      const uint32_t pos = F ? fold_lin(*F, old_je[e]) : old_je[e];
      o_ << "      lqs::st_w(&" << X << "[" << xacc(xs, pos) << "], " << V(e) << ");\n";
    }
    o_ << "    }\n    " << bar << "\n";
    set_layout(t.ecmask);  // validated by the caller
    if (first) o_ << "    jt = " << jt_expr() << ";\n";
    first = false;
    o_ << "    { const uint32_t sj = " << swz_expr("jt", xs) << ";\n";
    for (int e = 0; e < R_; ++e)
      o_ << "      " << pfx_ << e << " = lqs::ld_w(&" << X << "[" << xacc(xs, je(e)) << "]);\n";
    o_ << "    }\n";
  });
  for (int e = 0; e < R_; ++e) vm_[e] = e;
  if (t.e0 != t.ecmask) {  // relabelling SWAPs: from here on amplitudes carry their logical positions
    set_layout(t.e0);
    o_ << "    jt = " << jt_expr() << ";\n";
  }
}

// Worst shared-memory bank conflict of reading the unswizzled incoming tile
// in the current layout: a warp access is served in phases of 128 bytes, and
// lanes of one phase whose amplitudes share a 4-bank group conflict.
int SegGen::smem_read_degree() const {
  const int per_phase = 128 / sz_;
  int worst = 1;
  for (int ph = 0; ph < 32 / per_phase; ++ph) {
    int cnt[32] = {0};
    for (int l = ph * per_phase; l < (ph + 1) * per_phase; ++l) {
      uint32_t j = 0;
      for (int m = 0; m < 5 && m < k_ - r_; ++m)
        if ((l >> m) & 1) j |= 1u << thr_[m];
      worst = std::max(worst, ++cnt[j % per_phase]);
    }
  }
  return worst;
}

// Global stores straight from registers write whole 32-byte sectors when the
// amplitudes of each sector (the lowest tile positions) sit on lane bits.
bool SegGen::store_friendly() const {
  const int need = 32 / sz_;  // amplitudes per sector: positions 0 .. log2(need)-1
  uint32_t lanes = 0;
  for (int m = 0; m < 5 && m < k_ - r_; ++m) lanes |= 1u << thr_[m];
  const uint32_t want = (uint32_t)need - 1u;
  return (lanes & want) == want && b_ >= (need == 4 ? 2 : 1);
}

// The result leaves registers for HBM directly: local index j of the tile is
// amplitude base + (j mod 2^b) + (row j >> b placed on the high tile qubits).
// The thread part of the offset is formed once per thread; the register part
// is a sum of per-slot terms.
void SegGen::emit_store() {
  pre_ << "  uint64_t st_t;\n  { const uint32_t j = " << jt_expr() << ";\n"
       << "    st_t = (uint64_t)(j & " << hex32((1u << b_) - 1u) << ") + lqs::row_offset(G, j >> " << b_ << "); }\n";
  for (int m = 0; m < r_; ++m) {
    const int p = slot_[m];
    if (p < b_) pre_ << "  const uint64_t st_" << m << " = " << (1u << p) << "ull;\n";
    else pre_ << "  const uint64_t st_" << m << " = 1ull << G.h[" << (p - b_) << "];\n";
  }
  each([&]() {
    o_ << "    { S* out = " << (pfx_[0] == 'v' ? "psi" : "lam") << " + base + st_t;\n";
    std::vector<std::string> offs(R_);
    for (int e = 0; e < R_; ++e) {
      for (int m = 0; m < r_; ++m)
        if ((e >> m) & 1) offs[e] += (offs[e].empty() ? "" : " + ") + ("st_" + std::to_string(m));
      if (offs[e].empty()) offs[e] = "0";
    }
    if (split_io()) {  // the next segment of this call reads hi/lo pairs: renormalise, no conversion
      o_ << "      if (fmt & 2u) {\n        W* wo = reinterpret_cast<W*>(out);\n";
      for (int e = 0; e < R_; ++e)
        o_ << "        lqs::jit::renorm<A>(" << V(e) << ");\n        lqs::st_w(&wo[" << offs[e] << "], " << V(e)
           << ");\n";
      o_ << "      } else {\n";
    }
    for (int e = 0; e < R_; ++e)
      o_ << (split_io() ? "  " : "") << "      out[" << offs[e] << "] = A::store(" << V(e) << ");\n";
    if (split_io()) o_ << "      }\n";
    o_ << "    }\n";
  });
}

// Gradient partial of op t (before it is un-applied): Im <lambda|G|psi> over
// the tile's amplitudes that the op's controls select, for generator G on
// its target: X, Y (pairs on the target's register slot), Z (a sign per
// amplitude), or the projector P1 on its control set.  The per-thread sum is
// reduced over the warp into the warp's float64 slot.
// Batched warp sums of pending partials, four at a time (the rest with
// unused slots when `all`).
void SegGen::flush_pending(bool all) {
  while (pend_.size() >= 4 || (all && !pend_.empty())) {
    std::string a[4], sl[4];
    for (int i = 0; i < 4; ++i) {
      if (i < (int)pend_.size()) {
        a[i] = pend_[i].first;
        sl[i] = "wacc + warp * " + std::to_string(kMaxGradSlotsJit) + " + " + std::to_string(pend_[i].second);
      } else {
        a[i] = "lqs::jit::GAcc<A>::zero()";
        sl[i] = "(double*)0";
      }
    }
    o_ << "    lqs::jit::gflush4(" << a[0] << ", " << a[1] << ", " << a[2] << ", " << a[3] << ", " << sl[0] << ", "
       << sl[1] << ", " << sl[2] << ", " << sl[3] << ");\n";
    pend_.erase(pend_.begin(), pend_.begin() + std::min<size_t>(4, pend_.size()));
  }
}

bool SegGen::emit_grad(const TOp& t) {
  if (t.gslot < 0) return true;
  uint32_t regc = 0;
  const std::string p = pred(t.lcmask, t.ecmask, regc);
  auto qual = [&](int e) { return ((uint32_t)e & regc) == regc; };
  const std::string acc = fresh("g");
  // the accumulator lives at tile scope until its batched warp sum
  o_ << "    // gradient slot " << t.gslot << "\n    lqs::jit::GAcc<A>::T " << acc << " = lqs::jit::GAcc<A>::zero();\n    {\n";
  if (!p.empty()) o_ << "      if (" << p << ") {\n";
  if (t.gen == G_P1 || (t.gen == G_Z && !(t.l0 >= 0 && reg_slot(t.l0) >= 0))) {
    // single amplitudes; for Z the sign comes from a thread bit or the tile
    std::string sgn = "false";
    if (t.gen == G_Z) {
      if (t.l0 >= 0) sgn = "((jt >> " + std::to_string(t.l0) + ") & 1u) != 0u";
      else if (t.e0) sgn = "(base & " + hex(t.e0) + ") != 0ull";
      else return fail("Z generator without a target");
    }
    for (int e = 0; e < R_; ++e)
      if (qual(e)) o_ << "        lqs::jit::gim<A>(" << acc << ", " << Vs("u", e) << ", " << Vs("v", e) << ", " << sgn << ");\n";
  } else {
    const int m = t.l0 >= 0 ? reg_slot(t.l0) : -1;
    if (m < 0 || (t.gen != G_X && t.gen != G_Y && t.gen != G_Z)) return fail("generator target not in a register slot");
    for (int e = 0; e < R_; ++e) {
      if ((e >> m) & 1 || !qual(e)) continue;
      const int a = e, b = e | (1 << m);
      if (t.gen == G_X) {  // conj(l0) p1 + conj(l1) p0
        o_ << "        lqs::jit::gim<A>(" << acc << ", " << Vs("u", a) << ", " << Vs("v", b) << ", false);\n";
        o_ << "        lqs::jit::gim<A>(" << acc << ", " << Vs("u", b) << ", " << Vs("v", a) << ", false);\n";
      } else if (t.gen == G_Y) {  // conj(l0)(-i p1) + conj(l1)(i p0)
        o_ << "        lqs::jit::gre<A>(" << acc << ", " << Vs("u", a) << ", " << Vs("v", b) << ", true);\n";
        o_ << "        lqs::jit::gre<A>(" << acc << ", " << Vs("u", b) << ", " << Vs("v", a) << ", false);\n";
      } else {  // Z: conj(l0) p0 - conj(l1) p1
        o_ << "        lqs::jit::gim<A>(" << acc << ", " << Vs("u", a) << ", " << Vs("v", a) << ", false);\n";
        o_ << "        lqs::jit::gim<A>(" << acc << ", " << Vs("u", b) << ", " << Vs("v", b) << ", true);\n";
      }
    }
  }
  if (!p.empty()) o_ << "      }\n";
  o_ << "    }\n";
  pend_.emplace_back(acc, t.gslot);
  flush_pending(false);
  return true;
}

// Gradient partials of the Z / P1 generators of a merged diagonal run (the
// consecutive K_GRAD ops before it): each is a signed sum of the same terms
// w_j = Im(conj(lambda_j) psi_j), so the terms are formed once per amplitude
// and the sums once per pattern (register-held controls, sign slot); the
// thread- or tile-dependent sign and predicate are applied per op.
bool SegGen::emit_grad_block(const TOp* ops, int count) {
  o_ << "    { // gradient partials of a merged diagonal run\n";
  const std::string wn = fresh("w");
  for (int e = 0; e < R_; ++e)
    o_ << "      const lqs::jit::GAcc<A>::V " << wn << "_" << e << " = lqs::jit::wim<A>(" << Vs("u", e) << ", "
       << Vs("v", e) << ");\n";
  std::map<std::pair<uint32_t, int>, std::string> sums, walsh;
  for (int i = 0; i < count; ++i) {
    const TOp& t = ops[i];
    if (t.kind != K_GRAD || (t.gen != G_Z && t.gen != G_P1)) return fail("internal: unexpected op in a gradient block");
    uint32_t regc = 0;
    // register-held controls select elements; thread-held ones make a per-lane
    // predicate; outside ones a per-tile one
    uint32_t thc = 0;
    for (int p = 0; p < k_; ++p)
      if (((t.lcmask >> p) & 1u) && reg_slot(p) < 0) thc |= 1u << p;
    const std::string p = pred(t.lcmask, 0, regc);
    const std::string tp = t.ecmask ? "((base & " + hex(t.ecmask) + ") == " + hex(t.ecmask) + ")" : "true";
    int sm = -1;      // register slot giving the sign, for Z on a register-held target
    int lbit = -1;    // lane bit giving the sign
    std::string rs;   // uniform sign (warp bit or qubit outside the tile)
    if (t.gen == G_Z) {
      if (t.l0 >= 0 && reg_slot(t.l0) >= 0) {
        sm = reg_slot(t.l0);
      } else if (t.l0 >= 0) {
        int m = 0;
        while (m < k_ - r_ && thr_[m] != t.l0) ++m;
        if (m == k_ - r_) return fail("Z target neither in registers nor on a thread bit");
        if (m < 5) lbit = m;
        else rs = "((tid >> " + std::to_string(m) + ") & 1u) != 0u";
      } else if (t.e0) {
        rs = "(base & " + hex(t.e0) + ") != 0ull";
      } else {
        return fail("Z generator without a target");
      }
    }
    const auto key = std::make_pair(regc, sm);
    auto it = sums.find(key);
    if (it == sums.end()) {
      const std::string sn = fresh("s");
      o_ << "      lqs::jit::GAcc<A>::T " << sn << " = lqs::jit::GAcc<A>::zero();\n";
      for (int e = 0; e < R_; ++e)
        if (((uint32_t)e & regc) == regc)
          o_ << "      lqs::jit::wadd(" << sn << ", " << wn << "_" << e << ", " << ((sm >= 0 && ((e >> sm) & 1)) ? "true" : "false")
             << ");\n";
      it = sums.emplace(key, sn).first;
    }
    const std::string slot = "wacc + warp * " + std::to_string(kMaxGradSlotsJit) + " + " + std::to_string(t.gslot);
    if (thc) {  // a per-lane predicate: this partial needs its own warp sum
      std::string val = rs.empty() ? it->second : "lqs::jit::gneg(" + it->second + ", " + rs + ")";
      val = "(" + p + " && " + tp + ") ? " + val + " : lqs::jit::GAcc<A>::zero()";
      if (lbit >= 0) val = "lqs::jit::gneg(" + val + ", ((tid >> " + std::to_string(lbit) + ") & 1u) != 0u)";
      o_ << "      lqs::jit::gflush(" << val << ", " << slot << ");  // gradient slot " << t.gslot << "\n";
      continue;
    }
    // one Walsh butterfly per pattern serves every partial that uses it
    auto wt = walsh.find(key);
    if (wt == walsh.end()) {
      const std::string wv = fresh("W");
      o_ << "      const auto " << wv << " = lqs::jit::wht(" << it->second << ");\n";
      wt = walsh.emplace(key, wv).first;
    }
    const std::string lane = "(tid & 31u) == " + std::to_string(lbit >= 0 ? (1u << lbit) : 0u);
    o_ << "      lqs::jit::gput(" << wt->second << ", " << lane << " && " << tp << ", " << (rs.empty() ? "false" : rs)
       << ", " << slot << ");  // gradient slot " << t.gslot << "\n";
  }
  o_ << "    }\n";
  return true;
}

bool SegGen::emit_op(const TOp& t) {
  uint32_t regc = 0;
  const int c = t.coef;
  auto qual = [&](int e) { return ((uint32_t)e & regc) == regc; };
  if (adj_ && !emit_grad(t)) return false;
  switch (t.kind) {
    case K_LAYOUT:
      return fail("internal: layout reached emit_op");
    case K_GRAD:
      return adj_ ? true : fail("gradient partial outside an adjoint program");
    case K_PHASE: {
      const std::string p = pred(t.lcmask, t.ecmask, regc);
      o_ << "    // phase\n";
      if (!p.empty()) o_ << "    if (" << p << ") {\n";
      each([&]() {
        for (int e = 0; e < R_; ++e) {
          if (!qual(e)) continue;
          const std::string v = V(e);
          switch (t.special) {
            case 1: o_ << "      " << v << " = A::neg(" << v << ");\n"; break;
            case 2: o_ << "      " << v << " = A::mul_i(" << v << ");\n"; break;
            case 3: o_ << "      " << v << " = A::neg(A::mul_i(" << v << "));\n"; break;
            default: o_ << "      " << v << " = lqs::jit::Lz<A>::cmul(" << cref(c) << ", " << v << ");\n"; break;
          }
        }
      });
      if (!p.empty()) o_ << "    }\n";
      return true;
    }
    case K_DIAG1: {
      const std::string p = pred(t.lcmask, t.ecmask, regc);
      o_ << "    // diagonal\n";
      if (!p.empty()) o_ << "    if (" << p << ") {\n";
      const int m = t.l0 >= 0 ? reg_slot(t.l0) : -1;
      if (m >= 0) {
        each([&]() {
          for (int e = 0; e < R_; ++e)
            if (qual(e)) o_ << "      " << V(e) << " = lqs::jit::Lz<A>::cmul(" << cref(c + ((e >> m) & 1)) << ", " << V(e) << ");\n";
        });
      } else {
        const std::string d = fresh("d");
        const std::string bit = t.l0 >= 0 ? "((jt >> " + std::to_string(t.l0) + ") & 1u)"
                                          : "((base & " + hex(t.e0) + ") != 0ull)";
        o_ << "      const C " << d << " = " << bit << " ? " << cref(c + 1) << " : " << cref(c) << ";\n";
        each([&]() {
          for (int e = 0; e < R_; ++e)
            if (qual(e)) o_ << "      " << V(e) << " = lqs::jit::Lz<A>::cmul(" << d << ", " << V(e) << ");\n";
        });
      }
      if (!p.empty()) o_ << "    }\n";
      return true;
    }
    case K_DIAG2: {
      const std::string p = pred(t.lcmask, t.ecmask, regc);
      o_ << "    // two-qubit diagonal\n";
      if (!p.empty()) o_ << "    if (" << p << ") {\n";
      // each target bit: a register slot (known per element) or a runtime bit
      const int m0 = t.l0 >= 0 ? reg_slot(t.l0) : -1, m1 = t.l1 >= 0 ? reg_slot(t.l1) : -1;
      auto rbit = [&](int l, uint64_t em) {
        return l >= 0 ? "((jt >> " + std::to_string(l) + ") & 1u)" : "((base & " + hex(em) + ") != 0ull)";
      };
      const std::string r0 = rbit(t.l0, t.e0), r1 = rbit(t.l1, t.e1);
      std::vector<std::string> fac(R_);
      std::map<int, std::string> sel;  // compile-time pattern -> coefficient expression
      for (int e = 0; e < R_; ++e) {
        if (!qual(e)) continue;
        const int b0 = m0 >= 0 ? (e >> m0) & 1 : -1, b1 = m1 >= 0 ? (e >> m1) & 1 : -1;
        if (b0 >= 0 && b1 >= 0) {
          fac[e] = cref(c + 2 * b0 + b1);
          continue;
        }
        const int key = (b0 + 1) * 3 + (b1 + 1);
        auto it = sel.find(key);
        if (it == sel.end()) {
          std::string ex;
          if (b0 < 0 && b1 >= 0) ex = r0 + " ? " + cref(c + 2 + b1) + " : " + cref(c + b1);
          else if (b0 >= 0 && b1 < 0) ex = r1 + " ? " + cref(c + 2 * b0 + 1) + " : " + cref(c + 2 * b0);
          else
            ex = r0 + " ? (" + r1 + " ? " + cref(c + 3) + " : " + cref(c + 2) + ") : (" + r1 + " ? " + cref(c + 1) +
                 " : " + cref(c) + ")";
          const std::string d = fresh("d");
          o_ << "      const C " << d << " = " << ex << ";\n";
          it = sel.emplace(key, d).first;
        }
        fac[e] = it->second;
      }
      each([&]() {
        for (int e = 0; e < R_; ++e)
          if (qual(e)) o_ << "      " << V(e) << " = lqs::jit::Lz<A>::cmul(" << fac[e] << ", " << V(e) << ");\n";
      });
      if (!p.empty()) o_ << "    }\n";
      return true;
    }
    case K_ANTI1:
    case K_DENSE1:
    case K_DENSE1R: {
      const int m = t.l0 >= 0 ? reg_slot(t.l0) : -1;
      if (m < 0) return fail("single-target op whose target is not in a register slot");
      const std::string p = pred(t.lcmask, t.ecmask, regc);
      if ((regc >> m) & 1u) return fail("control on the target slot");
      const bool plain = t.kind == K_ANTI1 && t.special == 1;
      o_ << "    // " << (t.kind == K_ANTI1 ? "anti-diagonal" : t.kind == K_DENSE1 ? "dense" : "real dense")
         << " on slot " << m << "\n";
      if (plain && p.empty()) {  // a register renaming: no code
        for (int e = 0; e < R_; ++e)
          if (!((e >> m) & 1) && qual(e)) std::swap(vm_[e], vm_[e | (1 << m)]);
        return true;
      }
      if (plain) {
        const std::string q = fresh("p");
        o_ << "    { const bool " << q << " = " << p << ";\n";
        each([&]() {
          for (int e = 0; e < R_; ++e)
            if (!((e >> m) & 1) && qual(e))
              o_ << "      lqs::jit::swap_if(" << q << ", " << V(e) << ", " << V(e | (1 << m)) << ");\n";
        });
        o_ << "    }\n";
        return true;
      }
      if (t.kind == K_ANTI1 && p.empty()) {  // (a, b) <- (f0 b, f1 a): scale in place, then rename
        each([&]() {
          for (int e = 0; e < R_; ++e) {
            if ((e >> m) & 1 || !qual(e)) continue;
            const int a = e, b = e | (1 << m);
            o_ << "    " << V(b) << " = lqs::jit::Lz<A>::cmul(" << cref(c) << ", " << V(b) << ");\n";
            o_ << "    " << V(a) << " = lqs::jit::Lz<A>::cmul(" << cref(c + 1) << ", " << V(a) << ");\n";
          }
        });
        for (int e = 0; e < R_; ++e)
          if (!((e >> m) & 1) && qual(e)) std::swap(vm_[e], vm_[e | (1 << m)]);
        return true;
      }
      if (t.kind == K_DENSE1R && unit_adj() && t.special >= 1 && t.special <= 3) {
        if (!p.empty() || regc) return fail("internal: controlled op marked orthogonal");
        ++nu_;
        const int sg = t.special == 1 ? 1 : -1;
        each([&]() {
          for (int e = 0; e < R_; ++e) {
            if ((e >> m) & 1) continue;
            if (t.special == 3) o_ << "    lqs::jit::u1h<A>(" << V(e) << ", " << V(e | (1 << m)) << ");\n";
            else
              o_ << "    lqs::jit::u1a<A, " << sg << ">(" << V(e) << ", " << V(e | (1 << m)) << ", " << cref(c) << ", "
                 << cref(c + 1) << ");\n";
          }
        });
        return true;
      }
      if (t.kind == K_DENSE1R && !adj_ && t.special == 3) {  // Hadamard pattern: g (a + b, a - b)
        if (!p.empty() || regc) return fail("internal: controlled op marked orthogonal");
        ++nu_;  // its g joins the product; its form bit is unused
        each([&]() {
          for (int e = 0; e < R_; ++e)
            if (!((e >> m) & 1)) o_ << "    lqs::jit::u1h<A>(" << V(e) << ", " << V(e | (1 << m)) << ");\n";
        });
        return true;
      }
      if (t.kind == K_DENSE1R && !adj_ && (t.special == 1 || t.special == 2)) {
        // g times a matrix with a unit entry per row; the form (pivot m00 or
        // m10) is a launch-time bit, so angles do not change the kernel
        if (!p.empty() || regc) return fail("internal: controlled op marked orthogonal");
        const int j = nu_++;
        const int sg = t.special == 1 ? 1 : -1;
        o_ << "    if ((P.usel[" << (j >> 5) << "] >> " << (j & 31) << ") & 1u) {\n";
        for (int form = 1; form >= 0; --form) {
          if (form == 0) o_ << "    } else {\n";
          for (int e = 0; e < R_; ++e) {
            if ((e >> m) & 1) continue;
            o_ << "      lqs::jit::" << (form ? "u1b" : "u1a") << "<A, " << sg << ">(" << V(e) << ", "
               << V(e | (1 << m)) << ", " << cref(c) << ", " << cref(c + 1) << ");\n";
          }
        }
        o_ << "    }\n";
        return true;
      }
      if (!p.empty()) o_ << "    if (" << p << ") {\n";
      each([&]() {
        for (int e = 0; e < R_; ++e) {
          if ((e >> m) & 1 || !qual(e)) continue;
          const std::string a = V(e), b = V(e | (1 << m));
          if (t.kind == K_ANTI1)
            o_ << "      lqs::jit::anti<A>(" << a << ", " << b << ", " << cref(c) << ", " << cref(c + 1) << ");\n";
          else
            o_ << "      lqs::jit::" << (t.kind == K_DENSE1 ? "d1" : "d1r") << "<A>(" << a << ", " << b << ", "
               << cref(c) << ", " << cref(c + 1) << ", " << cref(c + 2) << ", " << cref(c + 3) << ");\n";
        }
      });
      if (!p.empty()) o_ << "    }\n";
      return true;
    }
    case K_SWAP:
    case K_DENSE2: {
      const int ma = t.l0 >= 0 ? reg_slot(t.l0) : -1, mb = t.l1 >= 0 ? reg_slot(t.l1) : -1;
      if (ma < 0 || mb < 0 || ma == mb) return fail("two-target op whose targets are not in register slots");
      const std::string p = pred(t.lcmask, t.ecmask, regc);
      if ((regc >> ma) & 1u || (regc >> mb) & 1u) return fail("control on a target slot");
      const int A_ = 1 << ma, B_ = 1 << mb;
      o_ << "    // " << (t.kind == K_SWAP ? "controlled swap" : "dense 4x4") << " on slots " << ma << ", " << mb
         << "\n";
      if (t.kind == K_SWAP) {
        if (p.empty()) {
          for (int e = 0; e < R_; ++e)
            if (!(e & A_) && !(e & B_) && qual(e)) std::swap(vm_[e | A_], vm_[e | B_]);
          return true;
        }
        const std::string q = fresh("p");
        o_ << "    { const bool " << q << " = " << p << ";\n";
        each([&]() {
          for (int e = 0; e < R_; ++e)
            if (!(e & A_) && !(e & B_) && qual(e))
              o_ << "      lqs::jit::swap_if(" << q << ", " << V(e | A_) << ", " << V(e | B_) << ");\n";
        });
        o_ << "    }\n";
        return true;
      }
      if (!p.empty()) o_ << "    if (" << p << ") {\n";
      each([&]() {
        for (int e = 0; e < R_; ++e) {
          if ((e & A_) || (e & B_) || !qual(e)) continue;
          // amplitude order 2 * bit(t0) + bit(t1)
          o_ << "      lqs::jit::d2<A>(" << V(e) << ", " << V(e | B_) << ", " << V(e | A_) << ", " << V(e | A_ | B_)
             << ", &" << cref(c) << ");\n";
        }
      });
      if (!p.empty()) o_ << "    }\n";
      return true;
    }
    case K_DPROD: {
      // C * prod of f_q over factor qubits q set in the amplitude's index, on
      // amplitudes whose condition bits are all 1.  Pool: C, then the local
      // factors by increasing tile position, then the outside factors by qubit.
      const std::string p = pred(t.lcmask, t.ecmask, regc);
      const uint32_t LF = (uint32_t)t.e1;
      const uint64_t EF = t.e0;
      auto lidx = [&](int q) { return c + 1 + __builtin_popcount(LF & ((1u << q) - 1u)); };
      o_ << "    // merged diagonal run\n";
      if (!p.empty()) o_ << "    if (" << p << ") {\n";
      o_ << "    {\n";
      const uint32_t regpos = reg_positions();
      uint32_t fmask = 0;  // register slots carrying a factor
      for (int m = 0; m < r_; ++m)
        if ((LF >> slot_[m]) & 1u) fmask |= 1u << m;
      std::vector<std::pair<int, int>> outs;  // factors on qubits outside the tile: (qubit, coefficient index)
      for (int q = 0, j = 0; q < 64; ++q)
        if ((EF >> q) & 1ull) outs.emplace_back(q, c + 1 + __builtin_popcount(LF) + j++);
      std::map<uint32_t, std::string> tab;
      std::vector<uint32_t> need;
      for (int e = 0; e < R_; ++e)
        if (qual(e)) need.push_back((uint32_t)e & fmask);
      std::sort(need.begin(), need.end());
      need.erase(std::unique(need.begin(), need.end()), need.end());
      if (!(LF & ~regpos) && outs.empty()) {
        // no factor on a thread bit or outside the tile: the whole table is
        // the same for every thread and tile, formed once per CTA before the
        // tile loop in shared memory (its first barrier orders the fill)
        const int u0 = nut_;
        nut_ += R_;
        pre_ << "  for (uint32_t i = tid; i < " << R_ << "u; i += blockDim.x) {\n    C f = " << cref(c) << ";\n";
        for (int m = 0; m < r_; ++m)
          if ((fmask >> m) & 1u)
            pre_ << "    if ((i >> " << m << ") & 1u) f = A::kmul(" << cref(lidx(slot_[m])) << ", f);\n";
        pre_ << "    UT[" << u0 << "u + i] = f;\n  }\n";
        for (uint32_t key : need) tab[key] = "UT[" + std::to_string(u0 + (int)key) + "u]";
      } else {
        // C times the factors on this thread's bits: the same for every tile,
        // so it is formed once per thread before the tile loop
        std::string h = cref(c);
        if (LF & ~regpos) {
          h = fresh("h");
          pre_ << "  C " << h << " = " << cref(c) << ";\n  { const uint32_t jt = " << jt_expr() << ";\n";
          for (int q = 0; q < k_; ++q)
            if (((LF >> q) & 1u) && !((regpos >> q) & 1u))
              pre_ << "    if ((jt >> " << q << ") & 1u) " << h << " = A::kmul(" << cref(lidx(q)) << ", " << h << ");\n";
          pre_ << "  }\n";
        }
        const std::string a = fresh("a");
        o_ << "      C " << a << " = " << h << ";\n";
        if (!outs.empty()) {
          // The factors on qubits outside the tile depend only on the tile.
          // Groups of up to 4 qubits read a 16-entry table filled once per
          // CTA before the tile loop; a single qubit is a conditional
          // product.  With two groups or more, their product is formed once
          // per tile, one tile ahead, by lane 0 of one warp into a
          // double-buffered shared slot (OF), so each thread pays one
          // product instead of one per group.
          std::vector<std::string> terms;  // one product each, on the tile base `B` into `F`
          for (size_t g0 = 0; g0 < outs.size(); g0 += 4) {
            const size_t m = std::min<size_t>(4, outs.size() - g0);
            if (m == 1) {
              terms.push_back("if ((@B@ >> " + std::to_string(outs[g0].first) + ") & 1ull) @F@ = A::kmul(" +
                              cref(outs[g0].second) + ", @F@);");
              continue;
            }
            const int off = ntab_;
            ntab_ += 1 << m;
            pre_ << "  for (uint32_t i = tid; i < " << (1u << m) << "u; i += blockDim.x) {\n    C f = A::cconst1();\n";
            for (size_t b = 0; b < m; ++b)
              pre_ << "    if (i & " << (1u << b) << "u) f = A::kmul(" << cref(outs[g0 + b].second) << ", f);\n";
            pre_ << "    TBL[" << off << "u + i] = f;\n  }\n";
            std::string ix;
            for (size_t b = 0; b < m; ++b)
              ix += std::string(b ? " | " : "") + "((uint32_t)(@B@ >> " + std::to_string(outs[g0 + b].first) +
                    ") & 1u) << " + std::to_string(b);
            terms.push_back("@F@ = A::kmul(TBL[" + std::to_string(off) + "u + (" + ix + ")], @F@);");
          }
          if (terms.size() == 1) {
            o_ << "      " << replace_all(replace_all(terms[0], "@B@", "base"), "@F@", a) << "\n";
          } else {
            std::string code;
            for (const std::string& tm : terms) code += replace_all(replace_all(tm, "@B@", "ob"), "@F@", "f") + " ";
            o_ << "      " << a << " = lqs::jit::Lz<A>::kmul(OF[@OFCUR@ + " << ofac_.size() << "u], " << a << ");\n";
            ofac_.push_back(code);
          }
        }
        tab[0] = a;
        // products for the needed factor patterns, each from a smaller one
        std::vector<uint32_t> all;
        for (uint32_t key : need)
          for (uint32_t x = key; x; x &= ~(1u << (31 - __builtin_clz(x)))) all.push_back(x);
        std::sort(all.begin(), all.end());
        all.erase(std::unique(all.begin(), all.end()), all.end());
        for (uint32_t key : all) {
          const int m = 31 - __builtin_clz(key);
          const std::string nm = fresh("f");
          o_ << "      const C " << nm << " = lqs::jit::Lz<A>::kmul(" << cref(lidx(slot_[m])) << ", " << tab[key ^ (1u << m)]
             << ");\n";
          tab[key] = nm;
        }
      }
      each([&]() {
        for (int e = 0; e < R_; ++e)
          if (qual(e)) o_ << "      " << V(e) << " = lqs::jit::Lz<A>::cmul(" << tab[(uint32_t)e & fmask] << ", " << V(e) << ");\n";
      });
      o_ << "    }\n";
      if (!p.empty()) o_ << "    }\n";
      return true;
    }
    default:
      return fail("op kind " + std::to_string((int)t.kind) + " has no compiled form");
  }
}

const char* kSkeletonHead = R"(
extern "C" __global__ void __launch_bounds__(@NTH@, @MINB@)
@NAME@(A::S* __restrict__ psi, @LAMP@const __grid_constant__ SegArgs P, @PARTP@int* status@FMTP@) {
  typedef A::S S;
  typedef A::W W;
  typedef A::C C;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const lqs::TileGeom& G = P.g;
  S* S0 = reinterpret_cast<S*>(smem_raw);  // incoming tiles (bulk loads, prefetched one tile ahead)
  S* S0L = S0 + @NT@;                      // incoming lambda tiles (adjoint only)
  W* XA = reinterpret_cast<W*>(S0 + @NT@ * @NIN@);  // layout exchanges alternate between XA and XB
  W* XB = XA + @NT@;
  W* XC = XB + @NT@;  // complex128 adjoint: the second pair of exchange buffers
  W* XD = XC + @NT@;
  double* wacc = reinterpret_cast<double*>(XA + @NT@ * @NX@);  // adjoint: per-warp gradient slots
  uint64_t* bar = reinterpret_cast<uint64_t*>(wacc + @NWACC@);
  const uint32_t tid = threadIdx.x;
  const uint32_t warp = tid >> 5;
  (void)S0L;
  (void)XC;
  (void)XD;
  (void)warp;
  for (uint32_t i = tid; i < @NWACC@; i += blockDim.x) wacc[i] = 0.0;
  uint64_t t = blockIdx.x;
  if (tid == 0) {
    lqs::mbar_init(bar, 1);
    lqs::fence_mbar_init();
    if (t < G.ntiles) lqs::jit::seg_expect(G, bar, @NSTATES@);
  }
  __syncthreads();
  const uint64_t my_roff = tid < (1u << G.r) ? lqs::row_offset(G, tid) : 0ull;
  if (t < G.ntiles) {
    lqs::jit::seg_copy(G, S0, psi, lqs::tile_base(G, t), bar, my_roff);
@LAMCOPY0@  }
  uint32_t phase = 0;
  bool ok = true;
@TBL@@PRE@  for (; t < G.ntiles; t += gridDim.x) {
    const uint64_t base = lqs::tile_base(G, t);
    ok = __syncthreads_and(lqs::mbar_wait(bar, phase));
    phase ^= 1u;
    if (!ok) break;
    // the next phase's byte count goes up before any of its copies is issued
    if (tid == 0 && t + gridDim.x < G.ntiles) lqs::jit::seg_expect(G, bar, @NSTATES@);
)";

// Complex64 forward segments: two incoming buffers and two barriers; tile
// it of this CTA lands in buffer it & 1 (barrier phase (it >> 1) & 1).
const char* kSkeletonHeadDeep = R"(
extern "C" __global__ void __launch_bounds__(@NTH@, @MINB@)
@NAME@(A::S* __restrict__ psi, const __grid_constant__ SegArgs P, int* status, const unsigned fmt) {
  typedef A::S S;
  typedef A::W W;
  typedef A::C C;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const lqs::TileGeom& G = P.g;
  S* S0 = reinterpret_cast<S*>(smem_raw);      // incoming tiles, two buffers (two tiles in flight)
  W* XA = reinterpret_cast<W*>(S0 + @NT@ * 2u);  // every layout exchange
  W* XB = XA;
  uint64_t* bar = reinterpret_cast<uint64_t*>(XA + @NT@);
  const uint32_t tid = threadIdx.x;
  (void)XB;
  (void)fmt;
  uint64_t t = blockIdx.x;
  const uint64_t grid = gridDim.x;
  if (tid == 0) {
    lqs::mbar_init(bar, 1);
    lqs::mbar_init(bar + 1, 1);
    lqs::fence_mbar_init();
    if (t < G.ntiles) lqs::jit::seg_expect(G, bar, 1u);
    if (t + grid < G.ntiles) lqs::jit::seg_expect(G, bar + 1, 1u);
  }
  __syncthreads();
  const uint64_t my_roff = tid < (1u << G.r) ? lqs::row_offset(G, tid) : 0ull;
  if (t < G.ntiles) lqs::jit::seg_copy(G, S0, psi, lqs::tile_base(G, t), bar, my_roff);
  if (t + grid < G.ntiles) lqs::jit::seg_copy(G, S0 + @NT@, psi, lqs::tile_base(G, t + grid), bar + 1, my_roff);
  uint32_t it = 0;
  bool ok = true;
@TBL@@PRE@  for (; t < G.ntiles; t += grid, ++it) {
    const uint64_t base = lqs::tile_base(G, t);
    S* SIN = S0 + @NT@ * (it & 1u);
    uint64_t* BAR = bar + (it & 1u);
    ok = __syncthreads_and(lqs::mbar_wait(BAR, (it >> 1) & 1u));
    if (!ok) break;
    // the byte count of this buffer's next tile goes up before its copies are issued
    if (tid == 0 && t + 2ull * grid < G.ntiles) lqs::jit::seg_expect(G, BAR, 1u);
)";

const char* kSkeletonTailDeep = R"(  }
  if (!ok && tid == 0) {
    lqs::flag_timeout(status, 4);
    lqs::mbar_wait(bar + (it & 1u), (it >> 1) & 1u);  // let the copies in flight land (bounded)
    if (t + grid < G.ntiles) lqs::mbar_wait(bar + ((it + 1u) & 1u), ((it + 1u) >> 1) & 1u);
  }
}
)";

const char* kSkeletonTail = R"(  }
  if (!ok && tid == 0) {
    lqs::flag_timeout(status, 4);
    lqs::mbar_wait(bar, phase ^ 1u);
  }
@GRADOUT@}
)";

const char* kGradOut = R"(  __syncthreads();
  for (int s = tid; s < @NGRAD@; s += blockDim.x) {
    double v = 0.0;
    for (int w = 0; w < @NWARPS@; ++w) v += lqs::jit::slot_get<A>(wacc + w * @SLOTS@ + s);
    partial[(size_t)s * gridDim.x + blockIdx.x] = v;
  }
)";

std::string replace_all(std::string s, const std::string& a, const std::string& b) {
  for (size_t p = s.find(a); p != std::string::npos; p = s.find(a, p + b.size())) s.replace(p, a.size(), b);
  return s;
}

uint64_t fnv1a(const std::string& s) {
  uint64_t h = 1469598103934665603ull;
  for (unsigned char ch : s) {
    h ^= ch;
    h *= 1099511628211ull;
  }
  return h;
}

bool SegGen::run(const TOp* ops, int nops, int ncoef, int ngrad, std::string& src, std::string& kname,
                 std::string& why) {
  if (nops < 1 || ops[0].kind != K_LAYOUT) {
    why = "program does not start with a layout";
    return false;
  }
  if (ngrad > kMaxGradSlotsJit) {
    why = "too many gradient slots";
    return false;
  }
  for (int i = 0; i < nops; ++i)
    if (ops[i].kind == K_LAYOUT) {
      if (!set_layout(ops[i].ecmask) || !set_layout(ops[i].e0)) {
        why = "layout is not a permutation of the tile bits";
        return false;
      }
    }
  // The incoming tile is in natural order.  The program's first layout reads
  // it as is; when the next op is already a layout change whose reads of the
  // unswizzled tile conflict at most 2-way, the tile is read in that layout
  // directly and the exchange is skipped.
  int first = 1;
  uint64_t through = ops[0].ecmask, logical = ops[0].e0;
  if (nops > 1 && ops[1].kind == K_LAYOUT && !ops[1].fold) {
    set_layout(ops[1].ecmask);
    if (smem_read_degree() <= 2) {
      through = ops[1].ecmask;
      logical = ops[1].e0;
      first = 2;
    }
  }
  set_layout(through);
  for (int e = 0; e < R_; ++e) vm_[e] = e;
  o_ << "    uint32_t jt = " << jt_expr() << ";\n";
  each([&]() {
    o_ << "    W";
    for (int e = 0; e < R_; ++e) o_ << (e ? ", " : " ") << pfx_ << e;
    o_ << ";\n";
    const char* sin = pfx_[0] == 'v' ? (deep() ? "SIN" : "S0") : "S0L";
    if (split_io()) {  // the previous segment of this call left hi/lo pairs
      o_ << "    if (fmt & 1u) {\n";
      for (int e = 0; e < R_; ++e)
        o_ << "      " << pfx_ << e << " = lqs::ld_w(reinterpret_cast<const W*>(" << sin << " + (jt + " << hex32(je(e))
           << ")));\n";
      o_ << "    } else {\n";
    }
    for (int e = 0; e < R_; ++e)
      o_ << (split_io() ? "  " : "") << "    " << pfx_ << e << " = A::load(" << sin << "[jt + " << hex32(je(e))
         << "]);\n";
    if (split_io()) o_ << "    }\n";
  });
  if (logical != through) {
    set_layout(logical);
    o_ << "    jt = " << jt_expr() << ";\n";
  }
  if (deep())
    o_ << "    __syncthreads();  // this incoming buffer is free: the tile two ahead goes into it\n"
          "    { const uint64_t tn = t + 2ull * gridDim.x;\n"
          "      if (tn < G.ntiles) {\n"
          "        lqs::jit::seg_copy(G, SIN, psi, lqs::tile_base(G, tn), BAR, my_roff);\n";
  else
    o_ << "    __syncthreads();  // the incoming buffers are free: prefetch the next tile into them\n"
          "    { const uint64_t tn = t + gridDim.x;\n"
          "      if (tn < G.ntiles) {\n"
          "        lqs::jit::seg_copy(G, S0, psi, lqs::tile_base(G, tn), bar, my_roff);\n";
  if (adj_) o_ << "        lqs::jit::seg_copy(G, S0L, lam, lqs::tile_base(G, tn), bar, my_roff);\n";
  o_ << "      } }\n";
  for (int i = first; i < nops; ++i) {
    if (ops[i].kind == K_LAYOUT) {
      if (i == nops - 1 && !ops[i].fold) {
        // The closing layout only restores natural order for the store.  Direct
        // stores need no particular order, so when the current layout, mapped
        // from storage positions to the positions they stand for (relabelled
        // SWAPs), keeps sectors on lane bits, the exchange is skipped.
        int L[16];
        for (int q = 0; q < k_; ++q)
          L[(ops[i].ecmask >> (4 * q)) & 15u] = (int)((ops[i].e0 >> (4 * q)) & 15u);
        const int saved_slot[4] = {slot_[0], slot_[1], slot_[2], slot_[3]};
        int saved_thr[16];
        std::copy(thr_, thr_ + 16, saved_thr);
        for (int m = 0; m < r_; ++m) slot_[m] = L[slot_[m]];
        for (int m = 0; m < k_ - r_; ++m) thr_[m] = L[thr_[m]];
        if (store_friendly()) break;
        std::copy(saved_slot, saved_slot + 4, slot_);
        std::copy(saved_thr, saved_thr + 16, thr_);
      }
      emit_layout(ops[i]);
      continue;
    }
    if (adj_ && ops[i].kind == K_GRAD) {
      int j = i;
      while (j < nops && ops[j].kind == K_GRAD) ++j;
      if (!emit_grad_block(ops + i, j - i)) {
        why = why_;
        return false;
      }
      i = j - 1;
      continue;
    }
    if (!emit_op(ops[i])) {
      why = why_;
      return false;
    }
    const TOp& t = ops[i];
    const bool plain = (t.kind == K_ANTI1 && t.special == 1) || (t.kind == K_PHASE && t.special != 0) ||
                       t.kind == K_SWAP || t.kind == K_GRAD;
    if (!plain && ++lz_ >= kRenormEvery) {
      o_ << "    // renormalise the double-float registers\n";
      each([&]() {
        for (int e = 0; e < R_; ++e) o_ << "    lqs::jit::renorm<A>(" << V(e) << ");\n";
      });
      lz_ = 0;
    }
  }
  flush_pending(true);
  if (nu_ && gscale_sink(ops, nops) < 0) {
    o_ << "    // the product of the unit-row forms' factors\n";
    each([&]() {
      for (int e = 0; e < R_; ++e)
        o_ << "    " << V(e) << " = lqs::jit::Lz<A>::rscale(lqs::jit::Re<A>::get(P.gscale), " << V(e) << ");\n";
    });
  }
  emit_store();  // natural order, or a layout that keeps sectors on lanes
  if (!ofac_.empty()) {
    // per-tile outside-factor products: the next tile's, after this tile's
    // last use of the other buffer; the first tile's before the loop (after
    // a barrier that orders the TBL fill)
    const int nwarps = nthreads() / 32;
    const std::string nof = std::to_string(ofac_.size()) + "u";
    auto fill = [&](std::ostringstream& os, const char* tile, const std::string& slot, const char* ind) {
      os << ind << "if (" << tile << " < G.ntiles && (tid & 31u) == 0u) {\n" << ind << "  const uint64_t ob = lqs::tile_base(G, "
         << tile << ");\n" << ind << "  const uint32_t lw = tid >> 5;\n";
      for (size_t r = 0; r < ofac_.size(); ++r)
        os << ind << "  if (lw == " << (int)r % nwarps << "u) { C f = A::cconst1(); " << ofac_[r] << "OF[" << slot << " + " << r
           << "u] = f; }\n";
      os << ind << "}\n";
    };
    o_ << "    { const uint64_t tno = t + gridDim.x;\n";
    fill(o_, "tno", deep() ? "((it + 1u) & 1u) * " + nof : "phase * " + nof, "      ");
    o_ << "    }\n";
    pre_ << "  __syncthreads();\n";
    fill(pre_, "t", "0u", "  ");
  }
  std::string body = replace_all(o_.str(), "@OFCUR@",
                                 (deep() ? std::string("(it & 1u) * ") : std::string("(phase ^ 1u) * ")) +
                                     std::to_string(ofac_.size()) + "u");
  const uint64_t h = fnv1a(body) ^ (fnv1a(pre_.str()) * 31u) ^ ((uint64_t)ncoef << 48) ^ ((uint64_t)k_ << 40) ^
                     ((uint64_t)b_ << 36) ^ ((uint64_t)ngrad << 24) ^ (adj_ ? 0x5a5aull : 0ull) ^ fnv1a(aname_);
  char nm[40];
  std::snprintf(nm, sizeof nm, adj_ ? "lqs_adj_%016llx" : "lqs_seg_%016llx", (unsigned long long)h);
  kname = nm;
  const int nth = nthreads(), nwarps = nth / 32;
  std::ostringstream s;
  s << "// compiled " << (adj_ ? "adjoint" : "fused") << " segment: " << nops << " ops, " << ncoef
    << " coefficients, " << ngrad << " gradient slots\n"
    << "typedef unsigned char uint8_t;\ntypedef signed char int8_t;\ntypedef short int16_t;\ntypedef unsigned short uint16_t;\n"
       "typedef unsigned int uint32_t;\ntypedef unsigned long long uint64_t;\n"
    << "#include \"tile.cuh\"\n#include \"jit_dev.cuh\"\n"
    << "typedef " << aname_ << " A;\n"
    << "struct SegArgs {\n  lqs::TileGeom g;\n  A::C coef[" << std::max(ncoef, 1) << "];\n";
  if (nu_) s << "  A::C gscale;\n  uint32_t usel[" << (nu_ + 31) / 32 << "];\n";
  s << "};\n";
  std::string head = replace_all(deep() ? kSkeletonHeadDeep : kSkeletonHead, "@NAME@", kname);
  head = replace_all(head, "@NTH@", std::to_string(nth));
  // resident CTAs per SM the register budget aims at: forward 512 threads
  // per SM; adjoint 3 x 128, with 256 threads 2 (4 amplitudes of each state
  // per thread) or 1 (8 or more), with 512 threads 1
  const int minb = !adj_ ? std::max(1, 512 / nth) : nth <= 128 ? 3 : nth >= 512 ? 1 : (R_ * sz_ <= 64 ? 2 : 1);
  head = replace_all(head, "@MINB@", std::to_string(minb));
  head = replace_all(head, "@LAMP@", adj_ ? "A::S* __restrict__ lam, " : "");
  head = replace_all(head, "@PARTP@", adj_ ? "double* partial, " : "");
  head = replace_all(head, "@FMTP@", ", const unsigned fmt");
  head = replace_all(head, "@NT@", std::to_string(1u << k_) + "u");
  head = replace_all(head, "@NIN@", adj_ ? "2u" : "1u");
  head = replace_all(head, "@NX@", xpair_ ? "4u" : "2u");
  head = replace_all(head, "@NSTATES@", adj_ ? "2u" : "1u");
  head = replace_all(head, "@NWACC@", std::to_string(adj_ ? nwarps * kMaxGradSlotsJit : 0) + "u");
  head = replace_all(head, "@LAMCOPY0@",
                     adj_ ? "    lqs::jit::seg_copy(G, S0L, lam, lqs::tile_base(G, t), bar, my_roff);\n" : "");
  head = replace_all(head, "@TBL@",
                     (ntab_ ? "  __shared__ C TBL[" + std::to_string(ntab_) + "];\n" : std::string()) +
                         (nut_ ? "  __shared__ C UT[" + std::to_string(nut_) + "];\n" : std::string()) +
                         (ofac_.empty() ? std::string() : "  __shared__ C OF[" + std::to_string(2 * ofac_.size()) + "];\n"));
  head = replace_all(head, "@PRE@", pre_.str());
  std::string tail = deep() ? kSkeletonTailDeep : kSkeletonTail;
  std::string gout;
  if (adj_) {
    gout = replace_all(kGradOut, "@NGRAD@", std::to_string(ngrad));
    gout = replace_all(gout, "@NWARPS@", std::to_string(nwarps));
    gout = replace_all(gout, "@SLOTS@", std::to_string(kMaxGradSlotsJit));
  }
  tail = replace_all(tail, "@GRADOUT@", gout);
  s << head << body << tail;
  src = s.str();
  return true;
}

}  // namespace

// ---------------------------------------------------------------------------
// NVRTC and driver entry points (resolved at first use)
// ---------------------------------------------------------------------------
namespace {

struct Nvrtc {
  bool tried = false, ok = false;
  std::string err;
  decltype(&nvrtcCreateProgram) create = nullptr;
  decltype(&nvrtcCompileProgram) compile = nullptr;
  decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
  decltype(&nvrtcGetProgramLog) get_log = nullptr;
  decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
  decltype(&nvrtcGetCUBIN) get_cubin = nullptr;
  decltype(&nvrtcDestroyProgram) destroy = nullptr;
  decltype(&nvrtcGetErrorString) errstr = nullptr;
};

struct Driver {
  bool tried = false, ok = false;
  std::string err;
  decltype(&cuModuleLoadData) load = nullptr;
  decltype(&cuModuleGetFunction) get_function = nullptr;
  decltype(&cuFuncSetAttribute) set_attr = nullptr;
  decltype(&cuFuncGetAttribute) get_attr = nullptr;
  decltype(&cuLaunchKernel) launch = nullptr;
  decltype(&cuOccupancyMaxActiveBlocksPerMultiprocessor) occupancy = nullptr;
  decltype(&cuGetErrorString) errstr = nullptr;
};

std::mutex g_load_mu;
Nvrtc g_nvrtc;
Driver g_drv;

bool load_nvrtc() {
  std::lock_guard<std::mutex> lk(g_load_mu);
  Nvrtc& N = g_nvrtc;
  if (N.tried) return N.ok;
  N.tried = true;
  std::vector<std::string> cands;
  if (const char* p = std::getenv("LQS_NVRTC")) cands.push_back(p);
  cands.push_back("libnvrtc.so.13");
  cands.push_back("libnvrtc.so");
  for (const char* env : {"CUDA_HOME", "CUDA_PATH"})
    if (const char* p = std::getenv(env)) cands.push_back(std::string(p) + "/lib64/libnvrtc.so.13");
  cands.push_back("/usr/local/cuda/lib64/libnvrtc.so.13");
  void* h = nullptr;
  for (const auto& c : cands)
    if ((h = dlopen(c.c_str(), RTLD_NOW | RTLD_LOCAL))) break;
  if (!h) {
    N.err = "libnvrtc.so.13 not found (set LQS_NVRTC to its path)";
    return false;
  }
#define LQS_SYM(field, name)                                          \
  N.field = reinterpret_cast<decltype(N.field)>(dlsym(h, name));       \
  if (!N.field) {                                                      \
    N.err = std::string("libnvrtc lacks ") + name;                     \
    return false;                                                      \
  }
  LQS_SYM(create, "nvrtcCreateProgram")
  LQS_SYM(compile, "nvrtcCompileProgram")
  LQS_SYM(log_size, "nvrtcGetProgramLogSize")
  LQS_SYM(get_log, "nvrtcGetProgramLog")
  LQS_SYM(cubin_size, "nvrtcGetCUBINSize")
  LQS_SYM(get_cubin, "nvrtcGetCUBIN")
  LQS_SYM(destroy, "nvrtcDestroyProgram")
  LQS_SYM(errstr, "nvrtcGetErrorString")
#undef LQS_SYM
  N.ok = true;
  return true;
}

bool load_driver() {
  std::lock_guard<std::mutex> lk(g_load_mu);
  Driver& D = g_drv;
  if (D.tried) return D.ok;
  D.tried = true;
  auto get = [&](const char* name, void** fn) {
    cudaDriverEntryPointQueryResult q{};
    const cudaError_t e = cudaGetDriverEntryPointByVersion(name, fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !*fn) {
      D.err = std::string("driver entry point ") + name + " unavailable";
      return false;
    }
    return true;
  };
  D.ok = get("cuModuleLoadData", reinterpret_cast<void**>(&D.load)) &&
         get("cuModuleGetFunction", reinterpret_cast<void**>(&D.get_function)) &&
         get("cuFuncSetAttribute", reinterpret_cast<void**>(&D.set_attr)) &&
         get("cuFuncGetAttribute", reinterpret_cast<void**>(&D.get_attr)) &&
         get("cuLaunchKernel", reinterpret_cast<void**>(&D.launch)) &&
         get("cuOccupancyMaxActiveBlocksPerMultiprocessor", reinterpret_cast<void**>(&D.occupancy)) &&
         get("cuGetErrorString", reinterpret_cast<void**>(&D.errstr));
  return D.ok;
}

int cu_error(CUresult r, const char* what) {
  const char* s = nullptr;
  if (g_drv.errstr) g_drv.errstr(r, &s);
  return set_error(LQS_ERR_CUDA, std::string(what) + ": " + (s ? s : "CUDA driver error") + " (" +
                                     std::to_string((int)r) + ")");
}

}  // namespace

// ---------------------------------------------------------------------------
// cache
// ---------------------------------------------------------------------------
namespace {

constexpr int kJitMaxDevices = 64;
constexpr size_t kJitMaxEntries = 4096;
constexpr int kJitAutoMinQubits = 20;

struct Entry {
  std::string src, name;
  int uses = 0;
  int state = 0;  // 0 not compiled, 1 compiled, 2 failed
  std::vector<char> cubin;
  std::string log;
  CUfunction fn[kJitMaxDevices] = {};
  int per_sm[kJitMaxDevices] = {};
};

std::mutex g_mu;
std::unordered_map<std::string, std::unique_ptr<Entry>> g_cache;
std::atomic<int> g_mode{-1};
std::atomic<int> g_compiled{0}, g_failed{0};
std::atomic<uint64_t> g_launches{0};
std::atomic<uint64_t> g_compile_us{0};
std::string g_last_jit_error;

int mode_now() {
  int m = g_mode.load();
  if (m < 0) {
    m = LQS_JIT_AUTO;
    if (const char* e = std::getenv("LQS_JIT")) {
      const int v = std::atoi(e);
      if (v == LQS_JIT_OFF || v == LQS_JIT_ON || v == LQS_JIT_AUTO) m = v;
    }
    int expect = -1;
    g_mode.compare_exchange_strong(expect, m);
    m = g_mode.load();
  }
  return m;
}

bool wants_compile(const Entry& e, int n) {
  const int m = mode_now();
  if (m == LQS_JIT_ON) return true;
  if (m == LQS_JIT_AUTO) return n >= kJitAutoMinQubits && e.uses >= 2;
  return false;
}

// Compiles one entry (no lock held: NVRTC programs are independent).
void compile_entry(Entry* e) {
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (e->state != 0) return;  // compiled (or rejected) already
  }
  const auto t0 = std::chrono::steady_clock::now();
  const char* dump = std::getenv("LQS_JIT_DUMP");  // keep the generated source and compile log
  if (dump) {
    if (FILE* f = std::fopen((std::string(dump) + "/" + e->name + ".cu").c_str(), "w")) {
      std::fwrite(e->src.data(), 1, e->src.size(), f);
      std::fclose(f);
    }
  }
  Nvrtc& N = g_nvrtc;
  nvrtcProgram prog = nullptr;
  std::string log;
  std::vector<char> cubin;
  bool ok = false;
  if (N.create(&prog, e->src.c_str(), (e->name + ".cu").c_str(), kJitHeaderCount, kJitHeaderSources,
               kJitHeaderNames) == NVRTC_SUCCESS) {
    const char* opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-lineinfo", "-DNDEBUG", "--ptxas-options=-v"};
    const nvrtcResult r = N.compile(prog, dump ? 5 : 4, opts);
    size_t ls = 0;
    if (N.log_size(prog, &ls) == NVRTC_SUCCESS && ls > 1) {
      log.resize(ls);
      N.get_log(prog, &log[0]);
    }
    size_t cs = 0;
    if (r == NVRTC_SUCCESS && N.cubin_size(prog, &cs) == NVRTC_SUCCESS && cs) {
      cubin.resize(cs);
      ok = N.get_cubin(prog, cubin.data()) == NVRTC_SUCCESS;
    } else if (r != NVRTC_SUCCESS && log.empty()) {
      log = N.errstr(r);
    }
    N.destroy(&prog);
  } else {
    log = "nvrtcCreateProgram failed";
  }
  if (dump && !log.empty()) {  // with the dump: ptxas's register, spill and shared-memory report
    if (FILE* f = std::fopen((std::string(dump) + "/" + e->name + ".log").c_str(), "w")) {
      std::fwrite(log.data(), 1, log.size(), f);
      std::fclose(f);
    }
  }
  const auto us = std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now() - t0).count();
  g_compile_us += (uint64_t)us;
  std::lock_guard<std::mutex> lk(g_mu);
  e->cubin = std::move(cubin);
  e->log = std::move(log);
  e->state = ok ? 1 : 2;
  if (ok) ++g_compiled;
  else {
    ++g_failed;
    g_last_jit_error = e->name + ": " + e->log.substr(0, 400);
  }
}

// Compiles entries on up to 8 threads.
void compile_all(const std::vector<Entry*>& todo) {
  if (todo.empty()) return;
  const size_t nt = std::min<size_t>(todo.size(), std::max(1u, std::min(8u, std::thread::hardware_concurrency())));
  std::atomic<size_t> next{0};
  auto work = [&]() {
    for (size_t i; (i = next.fetch_add(1)) < todo.size();) compile_entry(todo[i]);
  };
  std::vector<std::thread> th;
  for (size_t i = 1; i < nt; ++i) th.emplace_back(work);
  work();
  for (auto& t : th) t.join();
}

// Structure key of a program: every field the generated source depends on
// (geometry shape, arithmetic, op fields, coefficient and gradient slot
// indices; not the coefficient values), so the source is generated only the
// first time a structure is met.
std::unordered_map<std::string, Entry*> g_keys;

template <class A>
std::string struct_key(const TileProg<A>& P, int r, bool adjoint, const char* aname) {
  std::string k;
  k.reserve(32 + (size_t)P.nops * 48);
  auto put = [&](const void* p, size_t n) { k.append(static_cast<const char*>(p), n); };
  const int hdr[6] = {P.g.k, P.g.b, r, P.ncoef, adjoint ? P.ngrad : -1, P.nops};
  put(hdr, sizeof hdr);
  k += aname;
  for (int i = 0; i < P.nops; ++i) {
    const TOp& t = P.op[i];
    const uint8_t b8[4] = {t.kind, t.special, t.gen, 0};
    const int8_t s8[4] = {t.l0, t.l1, t.s0, t.s1};
    const int16_t s16[2] = {t.coef, t.gslot};
    put(b8, 4);
    put(s8, 4);
    put(s16, 4);
    put(&t.lcmask, 4);
    put(&t.ecmask, 8);
    put(&t.e0, 8);
    put(&t.e1, 8);
    put(&t.fold, 2);
    if (t.kind == K_LAYOUT && t.fold > 0 && t.fold <= P.nfold) put(&P.fold[t.fold - 1], sizeof(TFold));
  }
  return k;
}

Entry* find_key(const std::string& key, bool count_use) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_keys.find(key);
  if (it == g_keys.end()) return nullptr;
  if (count_use) ++it->second->uses;
  return it->second;
}

Entry* find_or_add(const std::string& src, const std::string& name, bool count_use) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_cache.find(src);
  if (it == g_cache.end()) {
    if (g_cache.size() >= kJitMaxEntries) return nullptr;
    auto e = std::make_unique<Entry>();
    e->src = src;
    e->name = name;
    it = g_cache.emplace(src, std::move(e)).first;
  }
  if (count_use) ++it->second->uses;
  return it->second.get();
}

}  // namespace

template <class A> struct JitTypeName;
template <> struct JitTypeName<ArF32> { static constexpr const char* s = "lqs::ArF32"; };
template <> struct JitTypeName<ArF64> { static constexpr const char* s = "lqs::ArF64"; };
template <> struct JitTypeName<ArDF> { static constexpr const char* s = "lqs::ArDF"; };

template <class A>
int jit_source(const TileProg<A>& P, int r, std::string& src, std::string& name, std::string& why, bool adjoint) {
  SegGen g(P.g.k, P.g.b, r, JitTypeName<A>::s, A::kAmpBytes, adjoint);
  g.set_folds(P.fold);
  return g.run(P.op, P.nops, P.ncoef, adjoint ? P.ngrad : 0, src, name, why) ? LQS_OK : LQS_ERR_UNSUPPORTED;
}

// The cache entry of a program's structure (nullptr when the generator does
// not take it or the cache is full).
template <class A>
static Entry* entry_for(const TileProg<A>& P, int r, bool adjoint, bool count_use, std::string* why) {
  const std::string key = struct_key(P, r, adjoint, JitTypeName<A>::s);
  if (Entry* e = find_key(key, count_use)) return e;
  std::string src, name, w;
  if (jit_source(P, r, src, name, w, adjoint) != LQS_OK) {
    if (why) *why = w;
    return nullptr;
  }
  Entry* e = find_or_add(src, name, count_use);
  if (!e) {
    if (why) *why = "compiled-kernel cache is full";
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  g_keys.emplace(key, e);
  return e;
}

int jit_mode() { return mode_now(); }

bool jit_enabled_for(int n) {
  const int m = mode_now();
  return m == LQS_JIT_ON || (m == LQS_JIT_AUTO && n >= kJitAutoMinQubits);
}

template <class A>
int jit_note(const TileProg<A>& P, int r, int n, bool force, std::vector<void*>& todo) {
  Entry* e = entry_for(P, r, false, true, nullptr);
  if (!e) return LQS_OK;  // the interpreter runs it
  if (e->state == 0 && (force || wants_compile(*e, n)) &&
      std::find(todo.begin(), todo.end(), (void*)e) == todo.end())
    todo.push_back(e);
  return LQS_OK;
}

int jit_compile(const std::vector<void*>& todo) {
  if (todo.empty()) return LQS_OK;
  if (!load_nvrtc()) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_last_jit_error = g_nvrtc.err;
    return set_error(LQS_ERR_UNSUPPORTED, g_nvrtc.err);
  }
  std::vector<Entry*> es;
  for (void* p : todo) es.push_back(static_cast<Entry*>(p));
  compile_all(es);
  return LQS_OK;
}

int jit_states(const std::vector<void*>& todo, int* ok, std::string* err) {
  std::lock_guard<std::mutex> lk(g_mu);
  int good = 0;
  bool bad = false;
  for (void* p : todo) {
    const Entry* e = static_cast<const Entry*>(p);
    if (e->state == 1) {
      ++good;
    } else if (!bad) {
      bad = true;
      if (err) *err = e->name + ": " + e->log.substr(0, 2000);
    }
  }
  if (ok) *ok = good;
  return bad ? LQS_ERR_UNSUPPORTED : LQS_OK;
}

// The kernel of a compiled entry on device `dev` (loaded on first use).
static int entry_function(Entry* e, int dev, size_t smem, int threads, CUfunction* fn, int* per_sm) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!e->fn[dev]) {
    if (!load_driver()) return set_error(LQS_ERR_UNSUPPORTED, g_drv.err);
    LQS_CUDA_TRY(cudaSetDevice(dev));  // makes the device's primary context current on this thread
    CUmodule mod;
    CUresult rr = g_drv.load(&mod, e->cubin.data());
    if (rr != CUDA_SUCCESS) return cu_error(rr, "cuModuleLoadData(compiled segment)");
    CUfunction f;
    rr = g_drv.get_function(&f, mod, e->name.c_str());
    if (rr != CUDA_SUCCESS) return cu_error(rr, "cuModuleGetFunction(compiled segment)");
    rr = g_drv.set_attr(f, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, (int)smem);
    if (rr != CUDA_SUCCESS) return cu_error(rr, "cuFuncSetAttribute(compiled segment)");
    int ps = 0;
    rr = g_drv.occupancy(&ps, f, threads, smem);
    if (rr != CUDA_SUCCESS) return cu_error(rr, "cuOccupancyMaxActiveBlocksPerMultiprocessor");
    e->per_sm[dev] = std::max(ps, 1);
    e->fn[dev] = f;
  }
  *fn = e->fn[dev];
  *per_sm = e->per_sm[dev];
  return LQS_OK;
}

template <class A> struct CoefRe;
template <> struct CoefRe<ArF32> {
  static double get(const float2& c) { return c.x; }
  static double im(const float2& c) { return c.y; }
};
template <> struct CoefRe<ArF64> {
  static double get(const double2& c) { return c.x; }
  static double im(const double2& c) { return c.y; }
};
template <> struct CoefRe<ArDF> {
  static double get(const DFK& c) { return (double)c.re.h + (double)c.re.l; }
  static double im(const DFK& c) { return (double)c.im.h + (double)c.im.l; }
};

static size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Kernel parameter block: the tile geometry, then the used coefficients.  A
// forward program passes its orthogonal real 2x2 ops (special 1, 2) in
// unit-row form (jit_dev.cuh u1a / u1b): k0, k1 in the op's first two
// coefficients, then the product of their factors g and one form bit per op,
// numbered in op order as the generator numbers them.
// Whether a program's orthogonal real 2x2 ops run in unit-row form: every
// forward program, and double-float adjoint programs (one form, pivot m00).
template <class A>
static bool unit_rows(bool forward) {
  return forward || std::is_same<A, ArDF>::value;
}

template <class A>
static std::vector<unsigned char> seg_args(const TileProg<A>& P, bool forward) {
  using C = typename A::C;
  std::vector<C> coef(P.coef, P.coef + P.ncoef);
  std::vector<uint32_t> usel;
  double gprod = 1.0;
  int nu = 0;
  for (int i = 0; unit_rows<A>(forward) && i < P.nops; ++i) {
    const TOp& t = P.op[i];
    if (t.kind != K_DENSE1R || (t.special != 1 && t.special != 2 && t.special != 3)) continue;
    const double m00 = CoefRe<A>::get(coef[t.coef]), m01 = CoefRe<A>::get(coef[t.coef + 1]);
    const double m10 = CoefRe<A>::get(coef[t.coef + 2]), m11 = CoefRe<A>::get(coef[t.coef + 3]);
    const bool form_b = forward && std::fabs(m01) > std::fabs(m00);
    const double g = form_b ? m10 : m00;
    double k0 = 0.0, k1 = 0.0;
    if (g != 0.0) {
      k0 = (form_b ? m00 : m01) / g;
      k1 = (form_b ? m11 : m10) / g;
    }
    coef[t.coef] = A::cconst(k0, 0.0);
    coef[t.coef + 1] = A::cconst(k1, 0.0);
    gprod *= g;
    if ((size_t)(nu >> 5) >= usel.size()) usel.push_back(0u);
    if (form_b) usel[nu >> 5] |= 1u << (nu & 31);
    ++nu;
  }
  const size_t off = round_up(sizeof(TileGeom), alignof(C));
  const size_t nc = (size_t)std::max(P.ncoef, 1);
  const size_t goff = off + nc * sizeof(C);
  const size_t uoff = round_up(goff + sizeof(C), alignof(uint32_t));
  const size_t end = nu ? uoff + usel.size() * sizeof(uint32_t) : goff;
  std::vector<unsigned char> args(round_up(end, 16), 0);
  std::memcpy(args.data(), &P.g, sizeof(TileGeom));
  const int sink = nu ? gscale_sink(P.op, P.nops) : -1;
  if (sink >= 0) {
    C& c0 = coef[P.op[sink].coef];
    c0 = A::cconst(CoefRe<A>::get(c0) * gprod, CoefRe<A>::im(c0) * gprod);
  }
  if (P.ncoef) std::memcpy(args.data() + off, coef.data(), (size_t)P.ncoef * sizeof(C));
  if (nu) {
    const C gc = A::cconst(gprod, 0.0);
    std::memcpy(args.data() + goff, &gc, sizeof(C));
    std::memcpy(args.data() + uoff, usel.data(), usel.size() * sizeof(uint32_t));
  }
  return args;
}

template <class A>
void jit_adjoint_scales(const TileProg<A>& P, std::vector<double>& scale, double* gprod_out) {
  scale.assign((size_t)std::max(P.ngrad, 0), 1.0);
  *gprod_out = 1.0;
  if (!unit_rows<A>(false)) return;
  std::vector<double> g((size_t)P.nops, 0.0);  // the pivot m00 of each unit-row op
  double gprod = 1.0;
  int nu = 0;
  for (int i = 0; i < P.nops; ++i) {
    const TOp& t = P.op[i];
    if (t.kind != K_DENSE1R || (t.special != 1 && t.special != 2 && t.special != 3)) continue;
    g[(size_t)i] = CoefRe<A>::get(P.coef[t.coef]);
    gprod *= g[(size_t)i];
    ++nu;
  }
  const int sink = nu ? gscale_sink(P.op, P.nops) : -1;
  // psi and lambda in registers are S times their values; a partial is
  // taken before its op is un-applied and comes out scaled by S^2
  double S = 1.0;
  for (int i = 0; i < P.nops; ++i) {
    const TOp& t = P.op[i];
    if (t.gslot >= 0 && t.gslot < P.ngrad) scale[(size_t)t.gslot] = 1.0 / (S * S);
    if (g[(size_t)i] != 0.0) S /= g[(size_t)i];
    if (i == sink) S *= gprod;
  }
  *gprod_out = gprod;
}

template <class A>
bool jit_ready(const TileProg<A>& P, int r, const SV* sv) {
  if (!jit_enabled_for(sv->n) || sv->device < 0 || sv->device >= kJitMaxDevices) return false;
  Entry* e = entry_for(P, r, false, false, nullptr);
  return e && e->state == 1;
}

template <class A>
int jit_launch(const TileProg<A>& P, int r, SV* sv, double bytes, double flops, const char* prof_name,
               bool* launched, unsigned fmt) {
  *launched = false;
  if (!jit_ready(P, r, sv)) return LQS_OK;
  Entry* e = entry_for(P, r, false, false, nullptr);
  const int dev = sv->device;
  const int threads = 1 << (P.g.k - r);
  // incoming tile and two exchange buffers, or (complex64) two incoming
  // tiles and one exchange buffer; one or two barriers
  const bool deep = std::is_same<A, ArF32>::value;
  const size_t smem = 3 * ((size_t)sizeof(typename A::S) << P.g.k) + (deep ? 32 : 16);
  CUfunction fn;
  int per_sm;
  LQS_TRY(entry_function(e, dev, smem, threads, &fn, &per_sm));
  std::vector<unsigned char> args = seg_args(P, true);
  void* psi = sv->d;
  int* status = sv->d_status;
  void* kp[] = {&psi, args.data(), &status, &fmt};
  const uint64_t grid = std::min<uint64_t>(P.g.ntiles, (uint64_t)std::max(sv->sms, 1) * per_sm);
  ProfScope ps(sv->stream, prof_name, bytes, flops);
  const CUresult rr = g_drv.launch(fn, (unsigned)grid, 1, 1, threads, 1, 1, (unsigned)smem,
                                   (CUstream)sv->stream, kp, nullptr);
  if (rr != CUDA_SUCCESS) return cu_error(rr, "cuLaunchKernel(compiled segment)");
  count_launch();
  ++g_launches;
  *launched = true;
  return LQS_OK;
}

template <class A>
int jit_adjoint_entry(const TileProg<A>& P, int r, void** entry, std::string* why) {
  Entry* e = entry_for(P, r, true, true, why);
  if (!e) return LQS_ERR_UNSUPPORTED;
  *entry = e;
  return LQS_OK;
}

size_t jit_adjoint_smem(int k, int r, size_t amp_bytes) {
  const int warps = (1 << (k - r)) / 32;
  const size_t tiles = amp_bytes == 16 ? 6 : 4;  // incoming psi and lambda, two (complex128: four) exchange buffers
  return tiles * (amp_bytes << k) + sizeof(double) * warps * kMaxGradSlotsJit + 16;
}

template <class A>
int jit_adjoint_occupancy(void* entry, const TileProg<A>& P, int r, SV* sv, int* per_sm) {
  Entry* e = static_cast<Entry*>(entry);
  if (e->state != 1) return set_error(LQS_ERR_UNSUPPORTED, "compiled adjoint segment is not available");
  const int dev = sv->device;
  if (dev < 0 || dev >= kJitMaxDevices) return set_error(LQS_ERR_UNSUPPORTED, "device index above 63");
  CUfunction fn;
  return entry_function(e, dev, jit_adjoint_smem(P.g.k, r, sizeof(typename A::S)), 1 << (P.g.k - r), &fn, per_sm);
}

template <class A>
int jit_launch_adjoint(void* entry, const TileProg<A>& P, int r, SV* sv, void* lam, double* partial, unsigned grid,
                       double bytes, double flops, const char* prof_name, unsigned fmt) {
  Entry* e = static_cast<Entry*>(entry);
  if (e->state != 1) return set_error(LQS_ERR_UNSUPPORTED, "compiled adjoint segment is not available");
  const int dev = sv->device;
  if (dev < 0 || dev >= kJitMaxDevices) return set_error(LQS_ERR_UNSUPPORTED, "device index above 63");
  const int threads = 1 << (P.g.k - r);
  const size_t smem = jit_adjoint_smem(P.g.k, r, sizeof(typename A::S));
  CUfunction fn;
  int per_sm;
  LQS_TRY(entry_function(e, dev, smem, threads, &fn, &per_sm));
  std::vector<unsigned char> args = seg_args(P, false);
  void* psi = sv->d;
  int* status = sv->d_status;
  void* kp[] = {&psi, &lam, args.data(), &partial, &status, &fmt};
  ProfScope ps(sv->stream, prof_name, bytes, flops);
  const CUresult rr = g_drv.launch(fn, grid, 1, 1, threads, 1, 1, (unsigned)smem, (CUstream)sv->stream, kp, nullptr);
  if (rr != CUDA_SUCCESS) return cu_error(rr, "cuLaunchKernel(compiled adjoint segment)");
  count_launch();
  ++g_launches;
  return LQS_OK;
}

void* jit_entry_generic(const std::string& key,
                        const std::function<bool(std::string& src, std::string& name, std::string& why)>& gen,
                        bool count_use, std::string* why) {
  if (Entry* e = find_key(key, count_use)) return e;
  std::string src, name, w;
  if (!gen(src, name, w)) {
    if (why) *why = w;
    return nullptr;
  }
  Entry* e = find_or_add(src, name, count_use);
  if (!e) {
    if (why) *why = "compiled-kernel cache is full";
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  g_keys.emplace(key, e);
  return e;
}

bool jit_should_compile(void* entry, int n) {
  Entry* e = static_cast<Entry*>(entry);
  std::lock_guard<std::mutex> lk(g_mu);
  return e->state == 1 || (e->state == 0 && wants_compile(*e, n));
}

int jit_occupancy_generic(void* entry, int dev, size_t smem, int threads, int* per_sm) {
  Entry* e = static_cast<Entry*>(entry);
  if (e->state != 1) return set_error(LQS_ERR_UNSUPPORTED, "compiled kernel is not available");
  if (dev < 0 || dev >= kJitMaxDevices) return set_error(LQS_ERR_UNSUPPORTED, "device index above 63");
  CUfunction fn;
  return entry_function(e, dev, smem, threads, &fn, per_sm);
}

int jit_launch_generic(void* entry, SV* sv, unsigned grid, int threads, size_t smem, void** params,
                       const char* prof_name, double bytes, double flops) {
  Entry* e = static_cast<Entry*>(entry);
  if (e->state != 1) return set_error(LQS_ERR_UNSUPPORTED, "compiled kernel is not available");
  const int dev = sv->device;
  if (dev < 0 || dev >= kJitMaxDevices) return set_error(LQS_ERR_UNSUPPORTED, "device index above 63");
  CUfunction fn;
  int per_sm;
  LQS_TRY(entry_function(e, dev, smem, threads, &fn, &per_sm));
  ProfScope ps(sv->stream, prof_name, bytes, flops);
  const CUresult rr = g_drv.launch(fn, grid, 1, 1, threads, 1, 1, (unsigned)smem, (CUstream)sv->stream, params, nullptr);
  if (rr != CUDA_SUCCESS) return cu_error(rr, "cuLaunchKernel(compiled kernel)");
  count_launch();
  ++g_launches;
  return LQS_OK;
}

template int jit_source<ArF32>(const TileProg<ArF32>&, int, std::string&, std::string&, std::string&, bool);
template int jit_source<ArF64>(const TileProg<ArF64>&, int, std::string&, std::string&, std::string&, bool);
template int jit_source<ArDF>(const TileProg<ArDF>&, int, std::string&, std::string&, std::string&, bool);
template int jit_note<ArF32>(const TileProg<ArF32>&, int, int, bool, std::vector<void*>&);
template int jit_note<ArF64>(const TileProg<ArF64>&, int, int, bool, std::vector<void*>&);
template int jit_note<ArDF>(const TileProg<ArDF>&, int, int, bool, std::vector<void*>&);
template int jit_launch<ArF32>(const TileProg<ArF32>&, int, SV*, double, double, const char*, bool*, unsigned);
template bool jit_ready<ArF32>(const TileProg<ArF32>&, int, const SV*);
template void jit_adjoint_scales<ArF32>(const TileProg<ArF32>&, std::vector<double>&, double*);
template int jit_launch<ArF64>(const TileProg<ArF64>&, int, SV*, double, double, const char*, bool*, unsigned);
template bool jit_ready<ArF64>(const TileProg<ArF64>&, int, const SV*);
template void jit_adjoint_scales<ArF64>(const TileProg<ArF64>&, std::vector<double>&, double*);
template int jit_launch<ArDF>(const TileProg<ArDF>&, int, SV*, double, double, const char*, bool*, unsigned);
template bool jit_ready<ArDF>(const TileProg<ArDF>&, int, const SV*);
template void jit_adjoint_scales<ArDF>(const TileProg<ArDF>&, std::vector<double>&, double*);
template int jit_adjoint_entry<ArF32>(const TileProg<ArF32>&, int, void**, std::string*);
template int jit_adjoint_occupancy<ArF32>(void*, const TileProg<ArF32>&, int, SV*, int*);
template int jit_adjoint_occupancy<ArF64>(void*, const TileProg<ArF64>&, int, SV*, int*);
template int jit_adjoint_occupancy<ArDF>(void*, const TileProg<ArDF>&, int, SV*, int*);
template int jit_adjoint_entry<ArF64>(const TileProg<ArF64>&, int, void**, std::string*);
template int jit_adjoint_entry<ArDF>(const TileProg<ArDF>&, int, void**, std::string*);
template int jit_launch_adjoint<ArF32>(void*, const TileProg<ArF32>&, int, SV*, void*, double*, unsigned, double, double,
                                       const char*, unsigned);
template int jit_launch_adjoint<ArF64>(void*, const TileProg<ArF64>&, int, SV*, void*, double*, unsigned, double, double,
                                       const char*, unsigned);
template int jit_launch_adjoint<ArDF>(void*, const TileProg<ArDF>&, int, SV*, void*, double*, unsigned, double, double,
                                      const char*, unsigned);

}  // namespace lqs

using namespace lqs;

extern "C" int lqs_set_jit(int mode) {
  if (mode != LQS_JIT_OFF && mode != LQS_JIT_ON && mode != LQS_JIT_AUTO)
    return set_error(LQS_ERR_ARG, "mode must be LQS_JIT_OFF, LQS_JIT_ON or LQS_JIT_AUTO");
  g_mode.store(mode);
  return LQS_OK;
}

extern "C" int lqs_jit_info(lqs_jit_stats* out) {
  if (!out) return set_error(LQS_ERR_ARG, "out is NULL");
  std::memset(out, 0, sizeof *out);
  out->mode = mode_now();
  out->compiled = g_compiled.load();
  out->failed = g_failed.load();
  out->launches = g_launches.load();
  out->compile_seconds = (double)g_compile_us.load() * 1e-6;
  std::lock_guard<std::mutex> lk(g_mu);
  out->cached = (int)g_cache.size();
  std::snprintf(out->last_error, sizeof out->last_error, "%s", g_last_jit_error.c_str());
  return LQS_OK;
}
