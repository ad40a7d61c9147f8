// Register-resident tile kernel for fused segments.
//
// The paper keeps gates on a process's local qubits free of communication
// (Sec. 2, Fig. 1a); here the qubits of a tile held on chip play that role,
// and a run of gates on them costs one HBM pass.
//
// A tile of 2^k amplitudes (k = r + 9) is spread over 512 threads with
// R = 2^r amplitudes in each thread's registers.  A "layout" assigns r of the
// tile's k local qubits to register index bits and the other 9 to thread
// index bits.  A gate whose non-diagonal targets are register qubits is pure
// register arithmetic: no shared memory, no barrier, no index math beyond
// compile-time register indices.  Controls and diagonal factors on any qubit
// become per-amplitude predicates and selects, since each thread knows the
// local index of every amplitude it holds.  When the next gates need other
// qubits in registers, the host planner inserts a layout change, one
// exchange of the tile through shared memory.
//
// Double buffering: while a tile is being computed in registers, the next
// tile's rows are already streaming into the other shared-memory buffer by
// bulk asynchronous copies; the result is written through the second buffer
// and stored by bulk copies.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <memory>
#include <string>
#include <type_traits>

#include "arith.cuh"
#include "jit.h"
#include "lqs_internal.cuh"
#include "tile.cuh"
#include "tile_ops.cuh"

namespace lqs {

template <class A> int add_tile_op(TileProg<A>& P, const KOp& o, int gslot);
template <class A> void init_prog(TileProg<A>& P, int n, uint64_t Q, int k, int b);

constexpr int kRegThreadBits = 9;
constexpr int kMaxGradSlotsReg = 128;  // gradient slots per compiled adjoint segment
constexpr int kRegThreads = 1 << kRegThreadBits;

template <int R> struct RLog;
template <> struct RLog<8> { static constexpr int r = 3; };
template <> struct RLog<16> { static constexpr int r = 4; };

// Registers per thread per dtype: double-float complex128 keeps 8 amplitudes
// (32 floats), complex64 16 amplitudes (32 floats).
template <class A> struct RegR { static constexpr int R = 8; };
template <> struct RegR<ArF32> { static constexpr int R = 16; };

int reg_tile_qubits(int dtype) { return (dtype == LQS_C64 ? 4 : 3) + kRegThreadBits; }

// Register bits per thread of a compiled forward segment.  The tile keeps its
// reg_tile_qubits; fewer register bits give more threads per tile (2^(k - r)).
// The interpreter keeps RegR's count.
#ifndef LQS_SEG_RBITS_C128
#define LQS_SEG_RBITS_C128 3
#endif
template <class A> struct JitR { static constexpr int r = LQS_SEG_RBITS_C128; };
template <> struct JitR<ArF32> { static constexpr int r = 4; };

// ---------------------------------------------------------------------------
// device side
// ---------------------------------------------------------------------------
template <class A, int R, int M, class F>
__device__ __forceinline__ void for_pairs(F&& f) {
#pragma unroll
  for (int e = 0; e < R; ++e)
    if (!(e & (1 << M))) f(e, e | (1 << M));
}

template <class A, int R, class F>
__device__ __forceinline__ void dispatch_pairs(int slot, F&& f) {
  switch (slot) {
    case 0: for_pairs<A, R, 0>(f); break;
    case 1: for_pairs<A, R, 1>(f); break;
    case 2: for_pairs<A, R, 2>(f); break;
    default: if constexpr (R >= 16) for_pairs<A, R, 3>(f); break;
  }
}

template <class A, int R>
__device__ __forceinline__ void reg_apply(typename A::W (&v)[R], const TOp& o, const typename A::C* coef,
                                          uint64_t base, uint32_t jt, const uint32_t (&je)[R]) {
  using W = typename A::W;
  using C = typename A::C;
  if ((base & o.ecmask) != o.ecmask) return;  // a control outside the tile is 0
  const uint32_t lc = o.lcmask;
  // Controls on local qubits are per-amplitude predicates; gates without them
  // (most of them) take unpredicated code so no selects are spent.
  switch (o.kind) {
    case K_PHASE: {
      const C f = coef[o.coef];
#pragma unroll
      for (int e = 0; e < R; ++e) {
        if (((jt | je[e]) & lc) == lc) v[e] = phase_apply<A>(f, o.special, v[e]);
      }
      break;
    }
    case K_DIAG1: {
      const C d0 = coef[o.coef], d1 = coef[o.coef + 1];
      if (o.s0 >= 0 && lc == 0) {  // target in registers: a fixed pattern over the pairs
        dispatch_pairs<A, R>(o.s0, [&](int e0, int e1) {
          v[e0] = A::cmul(d0, v[e0]);
          v[e1] = A::cmul(d1, v[e1]);
        });
      } else {
        // target on a thread bit or outside the tile: one factor per thread
        const bool hi = o.l0 >= 0 ? ((jt >> o.l0) & 1u) != 0 : (base & o.e0) != 0;
        if (o.s0 >= 0) {
          dispatch_pairs<A, R>(o.s0, [&](int e0, int e1) {
            if (((jt | je[e0]) & lc) != lc) return;
            v[e0] = A::cmul(d0, v[e0]);
            v[e1] = A::cmul(d1, v[e1]);
          });
        } else {
          const C d = hi ? d1 : d0;
#pragma unroll
          for (int e = 0; e < R; ++e)
            if (((jt | je[e]) & lc) == lc) v[e] = A::cmul(d, v[e]);
        }
      }
      break;
    }
    case K_DIAG2: {
#pragma unroll
      for (int e = 0; e < R; ++e) {
        const uint32_t j = jt | je[e];
        if ((j & lc) != lc) continue;
        const int b0 = o.l0 >= 0 ? (int)((j >> o.l0) & 1u) : ((base & o.e0) ? 1 : 0);
        const int b1 = o.l1 >= 0 ? (int)((j >> o.l1) & 1u) : ((base & o.e1) ? 1 : 0);
        v[e] = A::cmul(coef[o.coef + 2 * b0 + b1], v[e]);
      }
      break;
    }
    case K_ANTI1: {
      const C f0 = coef[o.coef], f1 = coef[o.coef + 1];
      const bool plain = o.special == 1;
      if (plain) {
        if (lc == 0) {
          dispatch_pairs<A, R>(o.s0, [&](int e0, int e1) {
            const W a = v[e0];
            v[e0] = v[e1];
            v[e1] = a;
          });
        } else {
          dispatch_pairs<A, R>(o.s0, [&](int e0, int e1) {
            if (((jt | je[e0]) & lc) != lc) return;
            const W a = v[e0];
            v[e0] = v[e1];
            v[e1] = a;
          });
        }
      } else {
        dispatch_pairs<A, R>(o.s0, [&](int e0, int e1) {
          if (((jt | je[e0]) & lc) != lc) return;
          const W a = v[e0], b = v[e1];
          v[e0] = A::cmul(f0, b);
          v[e1] = A::cmul(f1, a);
        });
      }
      break;
    }
    case K_SWAP: {  // targets at slots 1 (t0) and 0 (t1)
#pragma unroll
      for (int e = 0; e < R; e += 4) {
        if (((jt | je[e]) & lc) != lc) continue;
        const W a = v[e + 2];
        v[e + 2] = v[e + 1];
        v[e + 1] = a;
      }
      break;
    }
    case K_DENSE1: {
      const C u00 = coef[o.coef], u01 = coef[o.coef + 1], u10 = coef[o.coef + 2], u11 = coef[o.coef + 3];
      if (lc == 0) {
        dispatch_pairs<A, R>(o.s0, [&](int e0, int e1) {
          const W a = v[e0], b = v[e1];
          v[e0] = A::cmac2(u00, a, u01, b);
          v[e1] = A::cmac2(u10, a, u11, b);
        });
      } else {
        dispatch_pairs<A, R>(o.s0, [&](int e0, int e1) {
          if (((jt | je[e0]) & lc) != lc) return;
          const W a = v[e0], b = v[e1];
          v[e0] = A::cmac2(u00, a, u01, b);
          v[e1] = A::cmac2(u10, a, u11, b);
        });
      }
      break;
    }
    case K_DENSE1R: {
      const typename A::R u00 = CRe<A>::get(coef[o.coef]), u01 = CRe<A>::get(coef[o.coef + 1]),
                          u10 = CRe<A>::get(coef[o.coef + 2]), u11 = CRe<A>::get(coef[o.coef + 3]);
      if (lc == 0) {
        dispatch_pairs<A, R>(o.s0, [&](int e0, int e1) {
          const W a = v[e0], b = v[e1];
          v[e0] = A::rmac2(u00, a, u01, b);
          v[e1] = A::rmac2(u10, a, u11, b);
        });
      } else {
        dispatch_pairs<A, R>(o.s0, [&](int e0, int e1) {
          if (((jt | je[e0]) & lc) != lc) return;
          const W a = v[e0], b = v[e1];
          v[e0] = A::rmac2(u00, a, u01, b);
          v[e1] = A::rmac2(u10, a, u11, b);
        });
      }
      break;
    }
    case K_DENSE2: {  // targets at slots 1 (t0, most significant) and 0 (t1)
#pragma unroll
      for (int e = 0; e < R; e += 4) {
        if (((jt | je[e]) & lc) != lc) continue;
        W x[4] = {v[e], v[e + 1], v[e + 2], v[e + 3]};
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) v[e + rr] = A::cmac4(&coef[o.coef + 4 * rr], x);
      }
      break;
    }
    case K_DPROD: {
      // C * prod over factor qubits q set in the amplitude's index of f_q.
      // e1 = local factor qubits (tile bits), e0 = factor qubits outside the
      // tile; the pool holds C, then local factors, then outside factors, each
      // in increasing qubit order.
      const uint32_t LF = (uint32_t)o.e1;
      C acc = coef[o.coef];
      uint32_t regbits = 0;
#pragma unroll
      for (int m = 0; m < RLog<R>::r; ++m) regbits |= je[1 << m];
      // thread-bit factors (the amplitude's thread part is fixed per thread)
      uint32_t rest = LF & ~regbits & jt;
      while (rest) {
        const int q = __ffs(rest) - 1;
        rest &= rest - 1;
        acc = A::kmul(coef[o.coef + 1 + __popc(LF & ((1u << q) - 1u))], acc);
      }
      uint64_t ef = o.e0;
      int ci = o.coef + 1 + __popc(LF);
      while (ef) {
        const int q = __ffsll((long long)ef) - 1;
        ef &= ef - 1;
        if ((base >> q) & 1ull) acc = A::kmul(coef[ci], acc);
        ++ci;
      }
      // register-bit factors: one per register slot (1 when the slot's qubit
      // carries none), then a doubling table over this thread's amplitudes
      C fm[RLog<R>::r];
#pragma unroll
      for (int m = 0; m < RLog<R>::r; ++m) {
        const uint32_t qb = je[1 << m];
        fm[m] = (LF & qb) ? coef[o.coef + 1 + __popc(LF & (qb - 1u))] : A::cconst1();
      }
      C tab[R];
      tab[0] = acc;
#pragma unroll
      for (int e = 1; e < R; ++e) {
        const int m = 31 - __clz(e);  // highest set bit of e
        tab[e] = A::kmul(fm[m], tab[e ^ (1 << m)]);
      }
      if (lc == 0) {
#pragma unroll
        for (int e = 0; e < R; ++e) v[e] = A::cmul(tab[e], v[e]);
      } else {
#pragma unroll
        for (int e = 0; e < R; ++e)
          if (((jt | je[e]) & lc) == lc) v[e] = A::cmul(tab[e], v[e]);
      }
      break;
    }
    default:
      break;
  }
}

// Exchange-buffer position of local amplitude j: the bits that select a
// 16-byte word within a 128-byte shared-memory wavefront are XORed with a fold
// of the higher bits, so the lanes of a warp hit distinct banks whichever
// qubits the layout puts on them.
template <int SZ>
__device__ __forceinline__ uint32_t swz(uint32_t j) {
  if constexpr (SZ == 16) return j ^ (((j >> 3) ^ (j >> 6) ^ (j >> 9)) & 7u);
  else return j ^ (((j >> 4) ^ (j >> 8)) & 15u);
}

// Register/thread layout: nibble i of `packed` is the local qubit of layout
// slot i; slots 0..r-1 are register bits, slots r..k-1 thread bits.
template <int R>
__device__ __forceinline__ void set_layout(uint64_t packed, uint32_t tid, int k, uint32_t& jt, uint32_t (&je)[R]) {
  constexpr int r = RLog<R>::r;
  jt = 0;
#pragma unroll
  for (int m = 0; m < kRegThreadBits; ++m)
    if (r + m < k) jt |= ((tid >> m) & 1u) << ((packed >> (4 * (r + m))) & 15u);
#pragma unroll
  for (int e = 0; e < R; ++e) {
    uint32_t x = 0;
#pragma unroll
    for (int m = 0; m < r; ++m) x |= (uint32_t)((e >> m) & 1) << ((packed >> (4 * m)) & 15u);
    je[e] = x;
  }
}

template <class A, int R>
__global__ void __launch_bounds__(kRegThreads) k_fused_reg(typename A::S* __restrict__ psi,
                                                           const __grid_constant__ TileProg<A> P, int* status) {
  using S = typename A::S;
  using W = typename A::W;
  static_assert(sizeof(S) == sizeof(W), "in-place working format");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const TileGeom& G = P.g;
  const uint32_t nt = 1u << G.k;
  S* S0 = reinterpret_cast<S*>(smem_raw);  // incoming tiles (bulk loads)
  S* S1 = S0 + nt;                         // layout exchanges and outgoing tiles
  W* X1 = reinterpret_cast<W*>(S1);
  uint64_t* bar = reinterpret_cast<uint64_t*>(S1 + nt);
  const uint32_t tid = threadIdx.x;
  W v[R];
  uint32_t jt, je[R];
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint64_t t = blockIdx.x;
  if (t < G.ntiles && tid < 32) tile_load_issue(G, S0, psi, tile_base(G, t), bar);
  uint32_t phase = 0;
  bool ok = true;
  for (; t < G.ntiles; t += gridDim.x) {
    const uint64_t base = tile_base(G, t);
    ok = __syncthreads_and(mbar_wait(bar, phase));
    phase ^= 1u;
    if (!ok) break;
    // op 0 is the first layout: registers <- incoming tile
    set_layout<R>(P.op[0].ecmask, tid, G.k, jt, je);
#pragma unroll
    for (int e = 0; e < R; ++e) {
      const S s = S0[jt | je[e]];
      v[e] = A::load(s);
    }
    __syncthreads();  // the incoming buffer is free: prefetch the next tile into it
    const uint64_t tn = t + gridDim.x;
    if (tn < G.ntiles && tid < 32) tile_load_issue(G, S0, psi, tile_base(G, tn), bar);
    for (int i = 1; i < P.nops; ++i) {
      const TOp& o = P.op[i];
      if (o.kind == K_LAYOUT) {
        __syncthreads();  // readers of the previous exchange are done
#pragma unroll
        for (int e = 0; e < R; ++e) st_w(&X1[swz<sizeof(S)>(jt | je[e])], v[e]);
        __syncthreads();
        set_layout<R>(o.ecmask, tid, G.k, jt, je);
#pragma unroll
        for (int e = 0; e < R; ++e) v[e] = ld_w(&X1[swz<sizeof(S)>(jt | je[e])]);
        // SWAPs since the previous exchange were relabellings: the read above
        // went through them; from here on amplitudes carry their own labels
        if (o.e0 != o.ecmask) set_layout<R>(o.e0, tid, G.k, jt, je);
      } else {
        reg_apply<A, R>(v, o, P.coef, base, jt, je);
      }
    }
    __syncthreads();  // exchange readers done before the result overwrites the buffer
#pragma unroll
    for (int e = 0; e < R; ++e) S1[jt | je[e]] = A::store(v[e]);
    fence_proxy_async();
    __syncthreads();
    if (tid < 32) tile_store_issue(G, psi, S1, base);
  }
  if (tid < 32) bulk_wait0();
  if (!ok && tid == 0) {
    flag_timeout(status, 4);
    mbar_wait(bar, phase ^ 1u);  // the load that did not complete (bounded)
  }
}

// ---------------------------------------------------------------------------
// host side: layouts
// ---------------------------------------------------------------------------
static bool two_target(const KOp& o) { return o.kind == K_SWAP || o.kind == K_DENSE2; }

// A diagonal run merged into one op: C * prod_q f_q^bit_q on amplitudes whose
// `cond` qubits are all 1.
struct DGroup {
  uint64_t cond = 0, wires = 0;
  std::complex<double> C{1.0, 0.0};
  std::vector<std::pair<int, std::complex<double>>> f;  // (qubit, factor), merged per qubit
  std::vector<int> members;                             // lowered-op indices
  void mul(int q, std::complex<double> fq) {
    for (auto& x : f)
      if (x.first == q) {
        x.second *= fq;
        return;
      }
    f.emplace_back(q, fq);
  }
};

// Express a diagonal op as a group term; false for kinds that do not factor.
// K_DIAG1 (t, d0, d1) = d0 * (d1/d0)^bit_t; K_PHASE (set S, f) = f^bit_q on
// condition S \ {q}, q = the lowest qubit of S.
static bool group_term(const KOp& o, uint64_t& cond, int& q, std::complex<double>& fq, std::complex<double>& C) {
  if (o.kind == K_DIAG1 && o.t0 >= 0) {
    const std::complex<double> d0(o.m[0], o.m[1]), d1(o.m[2], o.m[3]);
    if (std::abs(d0) == 0.0) return false;
    cond = o.cmask;
    q = o.t0;
    fq = d1 / d0;
    C = d0;
    return true;
  }
  if (o.kind == K_PHASE && o.cmask) {
    q = __builtin_ctzll(o.cmask);
    cond = o.cmask & ~(1ull << q);
    fq = std::complex<double>(o.m[0], o.m[1]);
    C = 1.0;
    return true;
  }
  return false;
}

// One entry of the emitted sequence: a lowered op, or a merged group.
struct Ent {
  int op = -1;
  int group = -1;
};

// fold_perm (compiled segments only): runs of CNOT / X gates whose targets are
// tile qubits are not emitted as ops; their affine map is attached to the
// layout change that follows them (TFold), whose exchange then writes every
// amplitude to its permuted position.  The interpreter takes no folds.
template <class A>
static int build_reg_prog(TileProg<A>& P, const std::vector<KOp>& ops, const Segment& seg, int r,
                          std::vector<int>* grad_ops = nullptr, bool fold_perm = false) {
  // grad_ops (compiled adjoint): every parametrised op gets a gradient slot
  // in emission order and grad_ops receives the op of each slot; members of
  // merged diagonal runs are emitted as K_GRAD partials just before their run
  // (diagonal unitaries leave conj(lambda_j) psi_j unchanged, and the run only
  // moved past ops on other wires, which commute with its generators).
  auto has_grad = [&](const KOp& o) { return grad_ops && o.param_slot >= 0 && o.gen != G_NONE; };
  const TileGeom& G = P.g;
  const int k = G.k;
  auto lp = [&](int q) -> int {
    if (q < 0) return -1;
    if (q < G.b) return q;
    for (int m = 0; m < G.r; ++m)
      if (G.h[m] == q) return G.b + m;
    return -1;
  };
  // 1. merge diagonal runs.  Diagonal ops commute with each other and with
  // ops on disjoint wires, so a diagonal op may be delayed until the first
  // later op that touches one of its wires; ops with the same condition set
  // are multiplied into one group.
  std::vector<DGroup> groups;
  std::vector<int> open;  // indices into groups
  std::vector<Ent> seq;
  auto close = [&](size_t oi) {
    const int g = open[oi];
    if (groups[g].members.size() == 1) seq.push_back(Ent{groups[g].members[0], -1});
    else seq.push_back(Ent{-1, g});
    open.erase(open.begin() + oi);
  };
  for (int i : seg.ops) {
    const KOp& o = ops[i];
    uint64_t cond;
    int q;
    std::complex<double> fq, C;
    if (o.diagonal() && group_term(o, cond, q, fq, C)) {
      int g = -1;
      for (int oi : open)
        if (groups[oi].cond == cond) g = oi;
      if (g < 0) {
        groups.emplace_back();
        g = (int)groups.size() - 1;
        groups[g].cond = cond;
        open.push_back(g);
      }
      groups[g].C *= C;
      groups[g].mul(q, fq);
      groups[g].wires |= o.wire_mask();
      groups[g].members.push_back(i);
      continue;
    }
    if (!o.diagonal()) {
      for (size_t oi = open.size(); oi-- > 0;)
        if (groups[open[oi]].wires & o.wire_mask()) close(oi);
    }
    seq.push_back(Ent{i, -1});
  }
  while (!open.empty()) close(open.size() - 1);

  // 2. layouts and emission
  auto nondiag = [&](const Ent& e) { return e.op >= 0 && !ops[e.op].diagonal(); };
  // a gate that only moves amplitudes by an affine map of the tile bits: X or
  // CNOT (at most one control) with its target in the tile
  auto foldable = [&](const KOp& o) {
    return fold_perm && !has_grad(o) && o.kind == K_ANTI1 && o.special == 1 && __builtin_popcountll(o.cmask) <= 1 &&
           lp(o.t0) >= 0;
  };
  auto choose = [&](size_t i, const std::vector<int>& keep) {
    std::vector<int> slot(r, -1);
    auto has = [&](int q) { return std::find(slot.begin(), slot.end(), q) != slot.end(); };
    auto put = [&](int q) {
      if (q < 0 || has(q)) return;
      for (int m = r - 1; m >= 0; --m)
        if (slot[m] < 0) {
          slot[m] = q;
          return;
        }
    };
    size_t j = i;
    while (j < seq.size() && !nondiag(seq[j])) ++j;
    if (j < seq.size() && two_target(ops[seq[j].op])) {
      slot[1] = lp(ops[seq[j].op].t0);
      slot[0] = lp(ops[seq[j].op].t1);
      ++j;
    }
    for (; j < seq.size(); ++j) {
      if (!nondiag(seq[j])) continue;
      const KOp& o = ops[seq[j].op];
      if (foldable(o)) continue;  // folded into a layout change: needs no register slot
      if (two_target(o)) break;  // it will need its own exact placement
      put(lp(o.t0));
      if (std::count(slot.begin(), slot.end(), -1) == 0) break;
    }
    // fill with qubits already in registers (nothing moves for them), then
    // with the highest unused local qubits, leaving low qubits to the thread
    // (lane) bits so shared-memory rows stay contiguous
    for (int q : keep)
      if (std::count(slot.begin(), slot.end(), -1)) put(q);
    for (int q = k - 1; q >= 0 && std::count(slot.begin(), slot.end(), -1); --q) put(q);
    return slot;
  };
  auto pack = [&](const std::vector<int>& slot) {
    uint64_t p = 0;
    for (int m = 0; m < r; ++m) p |= (uint64_t)slot[m] << (4 * m);
    int sl = r;
    for (int q = 0; q < k; ++q)
      if (std::find(slot.begin(), slot.end(), q) == slot.end()) p |= (uint64_t)q << (4 * sl++);
    return p;
  };
  // Uncontrolled SWAPs move no data here: they relabel tile qubits.  pi[l] is
  // the storage position of the amplitude bit that local qubit l denotes;
  // every op is translated through pi, and the next exchange reads the tile
  // through pi and resets it to the identity.
  std::vector<int> pi(k);
  for (int l = 0; l < k; ++l) pi[l] = l;
  auto is_identity = [&]() {
    for (int l = 0; l < k; ++l)
      if (pi[l] != l) return false;
    return true;
  };
  // Thread bits that keep their storage position across a layout change do
  // not move data between the threads they select, so an exchange confined
  // to those groups of threads (often a single warp) needs no block-wide
  // barrier.  A new layout therefore keeps every thread bit whose position
  // stays out of the registers where it was; only the bits vacated by the
  // new register qubits take the qubits that leave the registers.
  uint64_t prev_logical = 0;
  bool have_prev = false;
  auto pack_keep = [&](const std::vector<int>& slot) {
    std::vector<int> pinv(k);
    for (int l = 0; l < k; ++l) pinv[pi[l]] = l;
    std::vector<char> used(k, 0);
    for (int m = 0; m < r; ++m) used[slot[m]] = 1;
    std::vector<int> thr(k - r, -1);
    for (int m = 0; m < k - r; ++m) {
      const int l = pinv[(prev_logical >> (4 * (r + m))) & 15];  // where the bit's data sits now, as a qubit
      if (!used[l]) {
        thr[m] = l;
        used[l] = 1;
      }
    }
    int q = 0;
    for (int m = 0; m < k - r; ++m) {
      if (thr[m] >= 0) continue;
      while (used[q]) ++q;
      thr[m] = q;
      used[q] = 1;
    }
    uint64_t p = 0;
    for (int m = 0; m < r; ++m) p |= (uint64_t)slot[m] << (4 * m);
    for (int m = 0; m < k - r; ++m) p |= (uint64_t)thr[m] << (4 * (r + m));
    return p;
  };
  // The pending folded run, in storage positions: x -> F x ^ c (TFold).
  TFold pend{};
  bool pending = false;
  auto fold_reset = [&]() {
    pend = TFold{};
    for (int p = 0; p < k; ++p) pend.col[p] = (uint16_t)(1u << p);
    pending = false;
  };
  fold_reset();
  auto emit_layout = [&](const std::vector<int>& slot, bool keep) -> int {
    if (P.nops >= kMaxTileOps) return LQS_ERR_UNSUPPORTED;  // the caller splits the segment
    TOp t{};
    t.kind = K_LAYOUT;
    t.gslot = -1;
    if (pending) {
      if (P.nfold >= kMaxTileFolds) return LQS_ERR_UNSUPPORTED;
      P.fold[P.nfold] = pend;
      t.fold = (int16_t)(++P.nfold);
      fold_reset();
    }
    const uint64_t logical = keep && have_prev ? pack_keep(slot) : pack(slot);
    prev_logical = logical;
    have_prev = true;
    uint64_t through = 0;  // the same layout with each position mapped through pi
    for (int i = 0; i < k; ++i) through |= (uint64_t)pi[(logical >> (4 * i)) & 15] << (4 * i);
    t.ecmask = through;
    t.e0 = logical;
    P.op[P.nops++] = t;
    for (int l = 0; l < k; ++l) pi[l] = l;
    return LQS_OK;
  };
  // Tiles arrive and leave in natural order (rows of contiguous amplitudes),
  // so the first and last layouts put the lanes on the lowest qubits
  // (registers on the top r) to read and write shared memory without bank
  // conflicts; layout changes in between go through the swizzled buffer.
  std::vector<int> natural(r);
  for (int m = 0; m < r; ++m) natural[m] = k - r + m;
  std::vector<int> cur = natural;
  LQS_TRY(emit_layout(cur, false));
  // storage position of local qubit q (after relabelling SWAPs), -1 outside the tile
  auto pp = [&](int q) -> int {
    const int l = lp(q);
    return l < 0 ? -1 : pi[l];
  };
  // Composes a foldable gate after the pending map: y -> y ^ y_C e_T for a
  // control on storage position C, y ^ [outside qubit q] e_T, or y ^ e_T.
  // False when the map has no room for another outside control.
  auto fold_in = [&](const KOp& o) -> bool {
    const uint16_t tb = (uint16_t)(1u << pp(o.t0));
    if (!o.cmask) {
      pend.cst ^= tb;
    } else {
      const int q = __builtin_ctzll(o.cmask);
      const int C = pp(q);
      if (C >= 0) {
        for (int p = 0; p < k; ++p)
          if ((pend.col[p] >> C) & 1u) pend.col[p] ^= tb;
        if ((pend.cst >> C) & 1u) pend.cst ^= tb;
        for (int j = 0; j < pend.nout; ++j)
          if ((pend.omask[j] >> C) & 1u) pend.omask[j] ^= tb;
      } else {
        int j = 0;
        while (j < pend.nout && pend.oq[j] != q) ++j;
        if (j == pend.nout) {
          if (pend.nout >= kMaxFoldOut) return false;
          pend.oq[j] = (uint8_t)q;
          pend.omask[j] = 0;
          ++pend.nout;
        }
        pend.omask[j] ^= tb;
      }
    }
    pending = true;
    return true;
  };
  // the layout change that applies a pending fold before entry i
  auto flush_fold = [&](size_t i) -> int {
    if (!pending) return LQS_OK;
    std::vector<int> keep(r);  // the qubits now held in registers
    for (int m = 0; m < r; ++m)
      for (int l = 0; l < k; ++l)
        if (pi[l] == cur[m]) keep[m] = l;
    cur = choose(i, keep);
    return emit_layout(cur, true);
  };
  for (size_t i = 0; i < seq.size(); ++i) {
    if (P.nops >= kMaxTileOps) return LQS_ERR_UNSUPPORTED;
    if (seq[i].op >= 0) {
      const KOp& so = ops[seq[i].op];
      const int la = lp(so.t0), lb = lp(so.t1);
      if (so.kind == K_SWAP && so.cmask == 0 && la >= 0 && lb >= 0) {
        std::swap(pi[la], pi[lb]);
        continue;
      }
      // a permutation whose target is not in registers (or that follows one
      // already folded) joins the pending fold instead of forcing an exchange
      if (foldable(so)) {
        const bool in_reg = std::find(cur.begin(), cur.end(), pp(so.t0)) != cur.end();
        if ((pending || !in_reg) && fold_in(so)) continue;
      }
    }
    LQS_TRY(flush_fold(i));
    if (seq[i].group >= 0) {
      const DGroup& g = groups[seq[i].group];
      for (int mi : g.members) {
        const KOp& mo = ops[mi];
        if (!has_grad(mo)) continue;
        if (P.nops >= kMaxTileOps || (int)grad_ops->size() >= kMaxGradSlotsReg) return LQS_ERR_UNSUPPORTED;
        TOp t{};
        t.kind = K_GRAD;
        t.gen = (uint8_t)mo.gen;
        t.gslot = (int16_t)grad_ops->size();
        t.l0 = t.l1 = -1;
        t.s0 = t.s1 = -1;
        if (mo.t0 >= 0) {
          const int l = pp(mo.t0);
          if (l >= 0) t.l0 = (int8_t)l;
          else t.e0 = 1ull << mo.t0;
        }
        for (int q = 0; q < G.n; ++q) {
          if (!((mo.cmask >> q) & 1)) continue;
          const int l = pp(q);
          if (l >= 0) t.lcmask |= 1u << l;
          else t.ecmask |= 1ull << q;
        }
        P.op[P.nops++] = t;
        grad_ops->push_back(mi);
      }
      auto f = g.f;
      // local factors in increasing storage position, then outside factors by qubit
      std::sort(f.begin(), f.end(), [&](const auto& x, const auto& y) {
        const int a = pp(x.first), b = pp(y.first);
        if ((a < 0) != (b < 0)) return a >= 0;
        return a >= 0 ? a < b : x.first < y.first;
      });
      TOp t{};
      t.kind = K_DPROD;
      t.gslot = -1;
      t.l0 = t.l1 = -1;
      t.s0 = t.s1 = -1;
      for (int q = 0; q < G.n; ++q) {
        if (!((g.cond >> q) & 1)) continue;
        const int l = pp(q);
        if (l >= 0) t.lcmask |= 1u << l;
        else t.ecmask |= 1ull << q;
      }
      const int nc = 1 + (int)f.size();
      if (P.ncoef + nc > kMaxTileCoef) return LQS_ERR_UNSUPPORTED;
      t.coef = (int16_t)P.ncoef;
      P.coef[P.ncoef++] = A::cconst(g.C.real(), g.C.imag());
      uint64_t lf = 0, ef = 0;
      for (auto& x : f) {
        const int l = pp(x.first);
        if (l >= 0) lf |= 1ull << l;
        else ef |= 1ull << x.first;
        P.coef[P.ncoef++] = A::cconst(x.second.real(), x.second.imag());
      }
      t.e1 = lf;
      t.e0 = ef;
      P.op[P.nops++] = t;
      continue;
    }
    const KOp& o = ops[seq[i].op];
    if (!o.diagonal()) {
      const int a = pp(o.t0), b = pp(o.t1);
      const bool fits = two_target(o) ? (cur[1] == a && cur[0] == b)
                                      : std::find(cur.begin(), cur.end(), a) != cur.end();
      if (!fits) {
        std::vector<int> keep(r);  // the qubits now held in registers
        for (int m = 0; m < r; ++m)
          for (int l = 0; l < k; ++l)
            if (pi[l] == cur[m]) keep[m] = l;
        cur = choose(i, keep);
        LQS_TRY(emit_layout(cur, true));  // resets the relabelling
        if (P.nops >= kMaxTileOps) return LQS_ERR_UNSUPPORTED;
      }
    }
    int gslot = -1;
    if (has_grad(o)) {
      if ((int)grad_ops->size() >= kMaxGradSlotsReg) return LQS_ERR_UNSUPPORTED;
      gslot = (int)grad_ops->size();
      grad_ops->push_back(seq[i].op);
    }
    const int rc = add_tile_op(P, o, gslot);
    if (rc != LQS_OK) return LQS_ERR_UNSUPPORTED;
    TOp& t = P.op[P.nops - 1];
    if (!is_identity()) {  // translate the op's local positions to storage positions
      if (t.l0 >= 0) t.l0 = (int8_t)pi[t.l0];
      if (t.l1 >= 0) t.l1 = (int8_t)pi[t.l1];
      uint32_t lc = 0;
      for (int l = 0; l < k; ++l)
        if ((t.lcmask >> l) & 1u) lc |= 1u << pi[l];
      t.lcmask = lc;
    }
    t.s0 = t.s1 = -1;
    if (o.kind == K_DIAG1 && t.l0 >= 0) {  // a diagonal target held in registers
      const auto it = std::find(cur.begin(), cur.end(), (int)t.l0);
      if (it != cur.end()) t.s0 = (int8_t)(it - cur.begin());
    }
    if (!o.diagonal()) {
      t.s0 = (int8_t)(std::find(cur.begin(), cur.end(), pp(o.t0)) - cur.begin());
      t.s1 = o.t1 >= 0 ? (int8_t)(std::find(cur.begin(), cur.end(), pp(o.t1)) - cur.begin()) : (int8_t)-1;
    }
  }
  if (cur != natural || !is_identity() || pending) LQS_TRY(emit_layout(natural, false));
  return LQS_OK;
}

template <class A>
int launch_fused_reg_t(SV* sv, const std::vector<KOp>& ops, const Segment& seg, int k, int b, int arith,
                       unsigned fmt) {
  constexpr int R = RegR<A>::R;
  const int r = RLog<R>::r, rj = JitR<A>::r;
  static thread_local TileProg<A> P;
  init_prog(P, sv->n, seg.qmask, k, b);
  const bool jit = jit_enabled_for(sv->n);  // compiled segments fold permutation runs into exchanges
  LQS_TRY(build_reg_prog(P, ops, seg, jit ? rj : r, nullptr, jit));
  double flops = 0.0;
  for (int i : seg.ops) flops += kop_touched_fraction(ops[i]) * kop_flops_per_amp(ops[i]);
  {
    bool launched = false;
    const std::string jname = std::string("k_fused_reg_jit/") + arith_tag(sv->dtype, arith);
    LQS_TRY(jit_launch(P, jit ? rj : r, sv, 2.0 * (double)sv->bytes(), flops * (double)sv->N(), jname.c_str(),
                       &launched, fmt));
    if (launched) return LQS_OK;
  }
  if (fmt) return set_error(LQS_ERR_CUDA, "internal: a segment planned as compiled code was not launched");
  if (P.nfold || (jit && rj != r)) {  // the interpreter: every gate applied by itself, its own register count
    init_prog(P, sv->n, seg.qmask, k, b);
    LQS_TRY(build_reg_prog(P, ops, seg, r));
  }
  const size_t smem = 2 * ((size_t)sizeof(typename A::S) << k) + 16;
  static bool attr_done = false;
  if (!attr_done) {
    LQS_CUDA_TRY(cudaFuncSetAttribute(k_fused_reg<A, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_done = true;
  }
  int per_sm = 0;
  LQS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused_reg<A, R>, kRegThreads, smem));
  per_sm = std::max(per_sm, 1);
  const uint64_t grid = std::min<uint64_t>(P.g.ntiles, (uint64_t)std::max(sv->sms, 1) * per_sm);
  const std::string pname = std::string("k_fused_reg/") + arith_tag(sv->dtype, arith);
  ProfScope ps(sv->stream, pname.c_str(), 2.0 * (double)sv->bytes(), flops * (double)sv->N());
  k_fused_reg<A, R><<<(unsigned)grid, kRegThreads, smem, sv->stream>>>(static_cast<typename A::S*>(sv->d), P,
                                                                       sv->d_status);
  count_launch();
  LQS_CUDA_TRY(cudaGetLastError());
  return LQS_OK;
}

template <class A>
static int note_reg_prog_t(int n, const std::vector<KOp>& ops, const Segment& seg, int k, int b, bool force,
                           std::vector<void*>& todo) {
  constexpr int R = RegR<A>::R;
  static thread_local TileProg<A> P;
  init_prog(P, n, seg.qmask, k, b);
  LQS_TRY(build_reg_prog(P, ops, seg, JitR<A>::r, nullptr, true));
  return jit_note(P, JitR<A>::r, n, force, todo);
}

int note_reg_prog(int n, int dtype, int arith, const std::vector<KOp>& ops, const Segment& seg, int k, int b,
                  bool force, std::vector<void*>& todo) {
  if (dtype == LQS_C64) return note_reg_prog_t<ArF32>(n, ops, seg, k, b, force, todo);
  if (arith == LQS_ARITH_F64) return note_reg_prog_t<ArF64>(n, ops, seg, k, b, force, todo);
  return note_reg_prog_t<ArDF>(n, ops, seg, k, b, force, todo);
}

// ---------------------------------------------------------------------------
// compiled adjoint (reverse sweep over psi and lambda)
// ---------------------------------------------------------------------------
// The kernel holds two states in registers and four tiles in shared memory
// (incoming psi and lambda, two exchange buffers), so its tiles are smaller
// than the forward kernel's: 2^11 amplitudes for both dtypes.
// Shape of the compiled adjoint: register bits per state and thread bits.
// Measured on GB300 (24-qubit ansatz): complex128 runs fastest with 4
// amplitudes of each state per thread and 512 threads, one CTA per SM (half
// the code per op of 8 amplitudes; 256 threads were 3% slower), complex64
// with 16 per state and 128 threads, three CTAs per SM.
#ifndef LQS_ADJ_THREAD_BITS_C128
#define LQS_ADJ_THREAD_BITS_C128 9
#endif
static void adj_shape(int dtype, int* r, int* tb) {
  *r = dtype == LQS_C64 ? 4 : 2;
  *tb = dtype == LQS_C64 ? 7 : LQS_ADJ_THREAD_BITS_C128;
}
int adjoint_tile_qubits(int dtype) {
  int r, tb;
  adj_shape(dtype, &r, &tb);
  return r + tb;
}

bool reg_adjoint_available(const SV* sv, int) {
  return jit_enabled_for(sv->n) && sv->n > adjoint_tile_qubits(sv->dtype);
}

template <class A>
struct AdjProg {
  TileProg<A> P;
  std::vector<int> gops;  // op (index into rev) of each gradient slot
  std::vector<int> ops;   // the segment's ops (for the profile's flop count)
  void* entry = nullptr;
};

template <class A>
static int adj_build(int n, const std::vector<KOp>& rev, const Segment& seg, int k, int b, int r,
                     std::vector<std::unique_ptr<AdjProg<A>>>& out) {
  auto pr = std::make_unique<AdjProg<A>>();
  init_prog(pr->P, n, seg.qmask, k, b);
  const int rc = build_reg_prog(pr->P, rev, seg, r, &pr->gops, true);
  if (rc == LQS_OK) {
    pr->P.ngrad = (int)pr->gops.size();
    pr->ops = seg.ops;
    out.push_back(std::move(pr));
    return LQS_OK;
  }
  if (rc != LQS_ERR_UNSUPPORTED || seg.ops.size() < 2) return rc;
  Segment lo, hi;  // too many ops, coefficients or gradient slots: split in order
  lo.qmask = hi.qmask = seg.qmask;
  lo.ops.assign(seg.ops.begin(), seg.ops.begin() + seg.ops.size() / 2);
  hi.ops.assign(seg.ops.begin() + seg.ops.size() / 2, seg.ops.end());
  LQS_TRY(adj_build(n, rev, lo, k, b, r, out));
  return adj_build(n, rev, hi, k, b, r, out);
}

// Plans the reverse sweep, builds its programs and compiles the missing
// kernels (host only).  *compiled (optional) gets the number of kernels this
// call compiled.
template <class A>
static int adj_prepare_t(int n, int dtype, const std::vector<KOp>& rev, std::vector<std::unique_ptr<AdjProg<A>>>& progs,
                         int* compiled, bool force) {
  int r, tb;
  adj_shape(dtype, &r, &tb);
  const int k = r + tb, b = dtype == LQS_C64 ? 5 : 4;
  if (n <= k) return set_error(LQS_ERR_UNSUPPORTED, "state fits one adjoint tile");
  PlanCfg pc;
  pc.k = k;
  pc.b = b;
  pc.max_ops = kMaxTileOps;
  std::vector<Segment> segs;
  LQS_TRY(plan_segments(n, rev, pc, segs));
  for (const Segment& sg : segs) LQS_TRY(adj_build(n, rev, sg, k, b, r, progs));
  std::vector<void*> todo;
  for (auto& pr : progs) {
    std::string why;
    if (jit_adjoint_entry(pr->P, r, &pr->entry, &why) != LQS_OK)
      return set_error(LQS_ERR_UNSUPPORTED, "adjoint segment not compiled: " + why);
    if (!force && !jit_should_compile(pr->entry, n))
      return set_error(LQS_ERR_UNSUPPORTED, "adjoint segment not compiled yet");
    if (std::find(todo.begin(), todo.end(), pr->entry) == todo.end()) todo.push_back(pr->entry);
  }
  int before = 0;
  std::string err;
  jit_states(todo, &before, &err);
  LQS_TRY(jit_compile(todo));
  int good = 0;
  if (jit_states(todo, &good, &err) != LQS_OK) return set_error(LQS_ERR_UNSUPPORTED, "adjoint segment: " + err);
  if (compiled) *compiled = good - before;
  return LQS_OK;
}

template <class A>
static int run_adjoint_compiled_t(SV* sv, const std::vector<KOp>& rev, void* lam, int arith,
                                  std::vector<int>& slot_op, std::vector<double>& slot_scale, double** partial_out,
                                  int* grid_out) {
  int r, tb;
  adj_shape(sv->dtype, &r, &tb);
  const int n = sv->n, k = r + tb;
  std::vector<std::unique_ptr<AdjProg<A>>> progs;
  LQS_TRY(adj_prepare_t<A>(n, sv->dtype, rev, progs, nullptr, false));
  size_t nslots = 0;
  for (auto& pr : progs) nslots += pr->gops.size();
  // unit-row un-applies scale psi and lambda by up to 1 / (product of the
  // segment's pivots); a product below 2^-40 (angles within about 1e-12**(1/m)
  // of pi) would take them out of float32 range, so the interpreter runs it
  std::vector<std::vector<double>> scales(progs.size());
  for (size_t j = 0; j < progs.size(); ++j) {
    double gprod = 1.0;
    jit_adjoint_scales(progs[j]->P, scales[j], &gprod);
    if (!(std::fabs(gprod) >= 0x1p-40))
      return set_error(LQS_ERR_UNSUPPORTED, "compiled adjoint: a segment's rotations are too close to pi");
  }
  // one grid for all segments (the partial sums share a layout): as many
  // CTAs as the least occupant kernel keeps resident
  int per_sm = 8;
  for (auto& pr : progs) {
    int ps = 0;
    LQS_TRY(jit_adjoint_occupancy(pr->entry, pr->P, r, sv, &ps));
    per_sm = std::min(per_sm, ps);
  }
  const uint64_t ntiles = 1ull << (n - k);
  const unsigned grid = (unsigned)std::min<uint64_t>(ntiles, (uint64_t)std::max(sv->sms, 1) * std::max(per_sm, 1));
  void* scratch = nullptr;
  LQS_TRY(sv_scratch(sv, 1, sizeof(double) * (std::max<size_t>(nslots, 1) * (grid + 1)), &scratch));
  double* partial = static_cast<double*>(scratch);
  const std::string pname = std::string("k_adjoint_jit/") + arith_tag(sv->dtype, arith);
  size_t off = 0;
  for (size_t j = 0; j < progs.size(); ++j) {
    auto& pr = progs[j];
    // both states un-apply every op; each gradient slot is about 8 flops per amplitude
    double fl = 8.0 * (double)pr->gops.size();
    for (int i : pr->ops) fl += 2.0 * kop_touched_fraction(rev[i]) * kop_flops_per_amp(rev[i]);
    // consecutive double-float segments pass psi and lambda as hi/lo float
    // pairs; the sweep reads and leaves float64 states
    const unsigned fmt = (j > 0 ? 1u : 0u) | (j + 1 < progs.size() ? 2u : 0u);
    LQS_TRY(jit_launch_adjoint(pr->entry, pr->P, r, sv, lam, partial + off * grid, grid, 4.0 * (double)sv->bytes(),
                               fl * (double)sv->N(), pname.c_str(), fmt));
    off += pr->gops.size();
    slot_op.insert(slot_op.end(), pr->gops.begin(), pr->gops.end());
    for (size_t q = 0; q < pr->gops.size(); ++q) slot_scale.push_back(q < scales[j].size() ? scales[j][q] : 1.0);
  }
  *partial_out = partial;
  *grid_out = (int)grid;
  return LQS_OK;
}

int adjoint_precompile(int n, int dtype, int arith, const std::vector<KOp>& rev, int* compiled) {
  if (dtype == LQS_C64) {
    std::vector<std::unique_ptr<AdjProg<ArF32>>> p;
    return adj_prepare_t<ArF32>(n, dtype, rev, p, compiled, true);
  }
  if (arith == LQS_ARITH_F64) {
    std::vector<std::unique_ptr<AdjProg<ArF64>>> p;
    return adj_prepare_t<ArF64>(n, dtype, rev, p, compiled, true);
  }
  std::vector<std::unique_ptr<AdjProg<ArDF>>> p;
  return adj_prepare_t<ArDF>(n, dtype, rev, p, compiled, true);
}

int run_adjoint_compiled(SV* sv, const std::vector<KOp>& rev, void* lam, int arith, std::vector<int>& slot_op,
                         std::vector<double>& slot_scale, double** partial, int* grid) {
  slot_op.clear();
  slot_scale.clear();
  if (sv->dtype == LQS_C64)
    return run_adjoint_compiled_t<ArF32>(sv, rev, lam, arith, slot_op, slot_scale, partial, grid);
  if (arith == LQS_ARITH_F64)
    return run_adjoint_compiled_t<ArF64>(sv, rev, lam, arith, slot_op, slot_scale, partial, grid);
  return run_adjoint_compiled_t<ArDF>(sv, rev, lam, arith, slot_op, slot_scale, partial, grid);
}

int launch_fused_reg(SV* sv, const std::vector<KOp>& ops, const Segment& seg, int k, int b, int arith,
                     unsigned fmt) {
  if (sv->dtype == LQS_C64) return launch_fused_reg_t<ArF32>(sv, ops, seg, k, b, arith, fmt);
  if (arith == LQS_ARITH_F64) return launch_fused_reg_t<ArF64>(sv, ops, seg, k, b, arith, fmt);
  return launch_fused_reg_t<ArDF>(sv, ops, seg, k, b, arith, fmt);
}

// True when a double-float forward segment runs as exactly one compiled
// kernel right now: launch_segment's routing (more than one op, the
// register tile's shape), a program that fits one kernel, and its kernel
// compiled.  Only such launches can hand hi/lo pairs to one another.
bool seg_split_capable(const SV* sv, const std::vector<KOp>& ops, const Segment& seg, int k, int b, int arith) {
  if (sv->dtype != LQS_C128 || arith == LQS_ARITH_F64 || seg.ops.size() < 2) return false;
  if (k != reg_tile_qubits(sv->dtype) || !jit_enabled_for(sv->n)) return false;
  static thread_local TileProg<ArDF> P;
  init_prog(P, sv->n, seg.qmask, k, b);
  if (build_reg_prog(P, ops, seg, JitR<ArDF>::r, nullptr, true) != LQS_OK) return false;  // launched split in two
  return jit_ready(P, JitR<ArDF>::r, sv);
}

}  // namespace lqs
