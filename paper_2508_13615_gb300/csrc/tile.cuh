// Shared-memory tiles of the state vector and the bulk-copy engine plumbing.
//
// A tile is the set of 2^k amplitudes that agree on every qubit outside a
// qubit set Q = {0 .. b-1} U {h_0 < .. < h_{r-1}} (k = b + r).  In the tile,
// local bit i < b is qubit i and local bit b + m is qubit h_m; a tile's
// amplitudes are 2^r rows of 2^b contiguous amplitudes, so one bulk
// asynchronous copy (cp.async.bulk, the TMA engine's untiled form) moves one
// row.  The paper keeps gates on "local" qubits inside one process's memory
// (Sec. 2, Fig. 1a); on one GPU the analogue of a process's local vector is a
// tile held in shared memory.
#pragma once
#ifndef __CUDACC_RTC__  // runtime-compiled segment kernels bring their own integer types
#include <cuda_runtime.h>
#include <stdint.h>
#endif

#include "arith.cuh"

namespace lqs {

constexpr int kMaxTileOps = 128;
constexpr int kMaxTileCoef = 448;
constexpr int kMaxTileBits = 14;
constexpr int kTileThreads = 256;
constexpr int kTileWarps = kTileThreads / 32;
constexpr uint32_t kSpinLimit = 1u << 22;  // bounded mbarrier waits: at most this many polls ...
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // ... and at most 2 s of the global timer, then error flag

struct TileGeom {
  int n, k, b, r;
  int h[kMaxTileBits];     // high tile qubits, ascending
  uint64_t ntiles;
  uint32_t row_bytes;      // 2^b * amplitude bytes
};

// Kernel op inside a tile.  Local bit positions are tile bits; masks named e*
// are global qubit masks for qubits outside the tile.
struct TOp {
  uint8_t kind, special, nfix, gen;
  int8_t l0, l1;           // local target bits (-1: none / outside the tile)
  int16_t coef;            // index of the first coefficient in the pool
  uint32_t lcmask;         // local control bits
  uint8_t fix[4];          // local fixed bits (targets + local controls), ascending
  uint64_t ecmask;         // controls outside the tile: the op applies on tiles where all are 1
  uint64_t e0, e1;         // diagonal ops: target bits outside the tile
  int16_t gslot;           // adjoint: gradient slot (-1 none)
  int8_t s0, s1;           // register-tile kernel: register slots of the targets
  int16_t fold;            // layout changes: 1 + index of the permutation folded into it (0: none)
  int16_t pad;
};

// A run of CNOT / X gates whose targets are tile qubits, folded into the layout
// exchange that follows it.  Such gates only move amplitudes: each maps local
// index bits x to x ^ x_c e_t (or x ^ e_t, or x ^ [outside bit q] e_t), so a
// run of them is an affine map x -> F x ^ c over GF(2).  The exchange writes the
// amplitude at storage position x to F x ^ c instead of x, which applies the
// whole run for the cost of the exchange it shares.  col[p] = F e_p; c = cst
// ^ the omask[j] of every outside qubit oq[j] that is 1 on this tile.
constexpr int kMaxFoldOut = 6;
constexpr int kMaxTileFolds = 24;
struct TFold {
  uint16_t col[kMaxTileBits];
  uint16_t cst;
  uint8_t nout, pad;
  uint8_t oq[kMaxFoldOut];
  uint16_t omask[kMaxFoldOut];
};

template <class A>
struct TileProg {
  TileGeom g;
  int nops;
  int ncoef;               // coefficients used in the pool
  int ngrad;               // adjoint: number of gradient slots
  int nfold;               // permutation runs folded into layout changes (compiled segments only)
  TOp op[kMaxTileOps];
  typename A::C coef[kMaxTileCoef];
  TFold fold[kMaxTileFolds];
};

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t ins0(uint32_t g, const uint8_t* fix, int nfix) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if (i < nfix) {
      const int p = fix[i];
      g = ((g >> p) << (p + 1)) | (g & ((1u << p) - 1u));
    }
  return g;
}

// Base index of tile t: t's bits placed on the qubits outside the tile.
__device__ __forceinline__ uint64_t tile_base(const TileGeom& G, uint64_t t) {
  uint64_t x = t << G.b;
  for (int m = 0; m < G.r; ++m) {
    const int p = G.h[m];
    x = ((x >> p) << (p + 1)) | (x & ((1ull << p) - 1));
  }
  return x;
}

// Global offset (in amplitudes) of tile row `row` relative to the tile base.
__device__ __forceinline__ uint64_t row_offset(const TileGeom& G, uint32_t row) {
  uint64_t off = 0;
  for (int m = 0; m < G.r; ++m) off |= (uint64_t)((row >> m) & 1u) << G.h[m];
  return off;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait: false when it gave up (the caller flags an error).  A poll
// may suspend the thread for a hardware-chosen time, so besides the poll count
// the global timer bounds the wait: it is read every 64 polls, and the wait
// gives up once kWaitLimitNs have passed since the first reading.  A wait that
// completes within 63 polls never reads it.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  uint64_t t0 = 0;
  for (uint32_t it = 0; it < kSpinLimit; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 63u) == 63u) {
      const uint64_t now = globaltimer_ns();
      if (it == 63u) t0 = now;
      else if (now - t0 > kWaitLimitNs) return false;
    }
  }
  return false;
}
__device__ __forceinline__ void bulk_g2s(void* dst_smem, const void* src_gmem, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void bulk_s2g(void* dst_gmem, const void* src_smem, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst_gmem),
               "r"(smem_u32(src_smem)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Warp 0 issues the row copies of one tile into `buf`; they complete on `bar`,
// whose expected byte count the caller has already raised (tile_expect).
template <class S>
__device__ __forceinline__ void tile_load_rows(const TileGeom& G, S* buf, const S* src, uint64_t base,
                                               uint64_t* bar) {
  const int lane = threadIdx.x & 31;
  const uint32_t nrows = 1u << G.r;
  const uint32_t per_row = 1u << G.b;
  for (uint32_t row = lane; row < nrows; row += 32)
    bulk_g2s(buf + (size_t)row * per_row, src + base + row_offset(G, row), G.row_bytes, bar);
}

// Lane 0 of warp 0 arrives on `bar` expecting `ntiles` tiles of bytes; the
// barrier is initialised with one arrival, so this is the phase's only arrive.
__device__ __forceinline__ void tile_expect(const TileGeom& G, uint64_t* bar, uint32_t ntiles) {
  if ((threadIdx.x & 31) == 0) mbar_expect_tx(bar, ntiles * (1u << G.r) * G.row_bytes);
  __syncwarp();
}

// Warp 0 loads one tile into `buf`.
template <class S>
__device__ __forceinline__ void tile_load_issue(const TileGeom& G, S* buf, const S* psi, uint64_t base,
                                                uint64_t* bar) {
  tile_expect(G, bar, 1);
  tile_load_rows(G, buf, psi, base, bar);
}

// Warp 0 issues the row stores of one tile and waits until shared memory has
// been read (so the buffer can be refilled).
template <class S>
__device__ __forceinline__ void tile_store_issue(const TileGeom& G, S* psi, const S* buf, uint64_t base) {
  const int lane = threadIdx.x & 31;
  const uint32_t nrows = 1u << G.r;
  const uint32_t per_row = 1u << G.b;
  for (uint32_t row = lane; row < nrows; row += 32)
    bulk_s2g(psi + base + row_offset(G, row), buf + (size_t)row * per_row, G.row_bytes);
  bulk_commit();
  bulk_wait_read0();
  __syncwarp();
}

// Error flag for bounded waits (status[0] = code, status[1] = block).
__device__ __forceinline__ void flag_timeout(int* status, int code) {
  if (status) {
    atomicCAS(status, 0, code);
    status[1] = blockIdx.x;
  }
}

}  // namespace lqs
