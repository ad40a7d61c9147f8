// Dense blocks on the tensor cores (complex64 states).
//
// A run of gates confined to the m lowest qubits is one 2^m x 2^m complex
// matrix U: the general approach of Sec. 3.1 (multiply by the gate's dense
// matrix) applied to a set of qubits instead of one gate, so that a long run
// costs one pass over the state.  Row r of the state, psi[r 2^m + k] for
// k < 2^m, becomes U times itself.  With each row stored as 2^(m+1) floats
// (re, im interleaved), every row update is the real product y = x W with
//   W[2k][2j] = Re U[j][k],  W[2k+1][2j] = -Im U[j][k],
//   W[2k][2j+1] = Im U[j][k], W[2k+1][2j+1] = Re U[j][k],
// and a tile of 128 rows is one matrix product D = X W on the fifth-generation
// tensor cores: tcgen05.mma, kind::tf32, M = 128, N = K = 64 (m = 5), the
// accumulator D in tensor memory (TMEM).
//
// Precision: TF32 keeps 10 mantissa bits.  Both operands are split into a
// TF32 leading part and a float32 residual (x = x_l + x_r exactly), and three
// products x_l W_l + x_l W_r + x_r W_l are accumulated in float32 (the
// 3xTF32 method); the dropped x_r W_r and the truncation of the residuals are
// below 2^-20 relative, about float32 accuracy.
//
// Data path per CTA (persistent, 128 threads, two CTAs per SM): W's leading
// parts and residuals are loaded once by TMA; each tile of 128 rows (32 KB)
// arrives by TMA with the 128-byte swizzle the tensor cores read (two slabs
// of 32 floats per row), is split in shared memory by all threads, multiplied
// by 24 MMAs issued from one thread, and leaves TMEM through tcgen05.ld into
// the (then free) residual buffer, from where a TMA store writes it back.  The
// next tile's load is issued as soon as the products are complete and the
// store runs while the next tile is split, so both overlap the CTA's work.
// Every wait is bounded: on a timeout the kernel flags the state's status
// word, waits (bounded) for its own work in flight, frees TMEM and returns.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "lqs_internal.cuh"
#include "tile.cuh"

namespace lqs {
namespace {

constexpr int kTM = 128;                 // rows per tile (MMA M)
constexpr int kTK = 64;                  // floats per row = MMA K = MMA N (m = 5)
constexpr int kSlab = 32;                // floats per 128-byte swizzled row of a slab
constexpr int kNSlab = kTK / kSlab;      // slabs along K
constexpr int kBlockThreads = 128;       // one warpgroup: warp w reads TMEM lanes 32w..32w+31
constexpr uint32_t kTmemCols = 64;       // the float32 accumulator, N columns
constexpr uint32_t kTileBytes = kTM * kTK * 4;
constexpr uint32_t kBBytes = kTK * kTK * 4;

struct BlockSmem {
  float x[kTM * kTK];    // incoming tile (slab s at s * kTM * kSlab), then its TF32 leading parts
  float xr[kTM * kTK];   // residuals, same layout
  float bl[kTK * kTK];   // W^T (N rows x K, K-major) leading parts, slab s at s * kTK * kSlab
  float br[kTK * kTK];   // W^T residuals
  uint64_t bar_x, bar_b, bar_mma;
  uint32_t tmem;
};
constexpr size_t kBlockSmemBytes = sizeof(BlockSmem) + 1024;  // + alignment slack

// Instruction descriptor of tcgen05.mma kind::tf32: float32 accumulator
// (bits 4-5 = 1), TF32 A and B (bits 7-9, 10-12 = 2), both K-major (bits 15,
// 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTK >> 3) << 17) |
                            ((uint32_t)(kTM >> 4) << 24);

// Shared-memory operand descriptor, K-major with the 128-byte swizzle: start
// address >> 4 (bits 0-13), leading offset (unused for this layout, 1),
// stride between 8-row groups 1024 bytes >> 4 (bits 32-45), descriptor
// version 1 (bits 46-47), layout SWIZZLE_128B = 2 (bits 61-63).  Slabs are
// 1024-byte aligned; K steps inside a slab advance the start address.
__device__ __forceinline__ uint64_t desc_sw128(const void* p) {
  const uint32_t a = smem_u32(p);
  return (uint64_t)((a & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, const void* src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(map), "r"(x),
               "r"(y), "r"(smem_u32(src))
               : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(kIdesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// 32 consecutive float32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// x rounded to TF32 (10 mantissa bits, low 13 bits zero)
__device__ __forceinline__ float tf32_lead(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__global__ void __launch_bounds__(kBlockThreads) k_block_tc(const __grid_constant__ CUtensorMap tm_x,
                                                          const __grid_constant__ CUtensorMap tm_b,
                                                          float* __restrict__ psi, uint64_t ntiles, int* status) {
  extern __shared__ unsigned char smem_raw[];
  BlockSmem& S = *reinterpret_cast<BlockSmem*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const uint32_t tid = threadIdx.x, warp = tid >> 5;
  uint64_t t = blockIdx.x;
  if (tid == 0) {
    mbar_init(&S.bar_x, 1);
    mbar_init(&S.bar_b, 1);
    mbar_init(&S.bar_mma, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(&S.tmem, kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem;
  bool x_pending = false;  // a tile load is in flight (thread 0's view)
  if (tid == 0) {
    mbar_expect_tx(&S.bar_b, 2 * kBBytes);
    for (int s = 0; s < kNSlab; ++s) {
      tma_load_2d(S.bl + s * kTK * kSlab, &tm_b, s * kSlab, 0, &S.bar_b);
      tma_load_2d(S.br + s * kTK * kSlab, &tm_b, s * kSlab, kTK, &S.bar_b);
    }
    if (t < ntiles) {
      mbar_expect_tx(&S.bar_x, kTileBytes);
      for (int s = 0; s < kNSlab; ++s)
        tma_load_2d(S.x + s * kTM * kSlab, &tm_x, s * kSlab, (int)(t * kTM), &S.bar_x);
      x_pending = true;
    }
  }
  // every wait's outcome is agreed on by the whole CTA, so all threads leave together
  bool ok = __syncthreads_and(mbar_wait(&S.bar_b, 0));
  bool mma_pending = false;
  uint32_t px = 0, pm = 0;
  for (; ok && t < ntiles; t += gridDim.x) {
    // the residual buffer also stages the previous tile's results for its
    // TMA store: the store must have read it before the split rewrites it
    if (tid == 0) bulk_wait_read0();
    ok = __syncthreads_and(mbar_wait(&S.bar_x, px));
    if (!ok) break;
    px ^= 1u;
    x_pending = false;
    // split the tile into TF32 leading parts (in place) and residuals; the
    // layout is the same for both, so every thread takes any 16 bytes
    float4* x4 = reinterpret_cast<float4*>(S.x);
    float4* r4 = reinterpret_cast<float4*>(S.xr);
#pragma unroll 4
    for (int i = (int)tid; i < kTM * kTK / 4; i += kBlockThreads) {
      const float4 v = x4[i];
      const float4 l = make_float4(tf32_lead(v.x), tf32_lead(v.y), tf32_lead(v.z), tf32_lead(v.w));
      x4[i] = l;
      r4[i] = make_float4(v.x - l.x, v.y - l.y, v.z - l.z, v.w - l.w);
    }
    fence_proxy_async();  // the tensor cores read shared memory through the async proxy
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      // x_l W_l + x_l W_r + x_r W_l, K = 8 TF32 (32 bytes) per MMA
#pragma unroll
      for (int term = 0; term < 3; ++term)
#pragma unroll
        for (int s = 0; s < kNSlab; ++s)
#pragma unroll
          for (int kk = 0; kk < kSlab / 8; ++kk) {
            const float* a = (term == 2 ? S.xr : S.x) + s * kTM * kSlab + kk * 8;
            const float* b = (term == 1 ? S.br : S.bl) + s * kTK * kSlab + kk * 8;
            mma_tf32(tmem, desc_sw128(a), desc_sw128(b), (term | s | kk) ? 1u : 0u);
          }
      mma_commit(&S.bar_mma);
    }
    mma_pending = true;
    ok = __syncthreads_and(mbar_wait(&S.bar_mma, pm));
    if (!ok) break;
    pm ^= 1u;
    mma_pending = false;
    tc_fence_after();
    // the tile buffers are free again: fetch the next tile while this one leaves TMEM
    const uint64_t tn = t + gridDim.x;
    if (tid == 0 && tn < ntiles) {
      mbar_expect_tx(&S.bar_x, kTileBytes);
      for (int s = 0; s < kNSlab; ++s)
        tma_load_2d(S.x + s * kTM * kSlab, &tm_x, s * kSlab, (int)(tn * kTM), &S.bar_x);
      x_pending = true;
    }
    // row r = 32w + lane of the tile is TMEM lane r: its 64 output floats go
    // to the residual buffer in the tensor map's layout (slab h, 16-byte
    // chunk c of the row at chunk position c ^ (r mod 8)), then one TMA store
    // per slab writes the tile back
    const uint32_t r = warp * 32u + (tid & 31u);
#pragma unroll
    for (int h = 0; h < kTK / 32; ++h) {
      uint32_t v[32];
      tmem_ld32(tmem + ((warp * 32u) << 16) + (uint32_t)(h * 32), v);
      tmem_wait_ld();
      float* slab_row = S.xr + h * kTM * kSlab + r * kSlab;
#pragma unroll
      for (int c = 0; c < 8; ++c)
        *reinterpret_cast<float4*>(slab_row + 4 * (c ^ (int)(r & 7u))) =
            make_float4(__uint_as_float(v[4 * c]), __uint_as_float(v[4 * c + 1]), __uint_as_float(v[4 * c + 2]),
                        __uint_as_float(v[4 * c + 3]));
    }
    fence_proxy_async();  // the TMA store reads shared memory through the async proxy
    tc_fence_before();
    __syncthreads();  // results staged; TMEM is rewritten by the next tile's products
    tc_fence_after();
    if (tid == 0) {
      for (int s = 0; s < kNSlab; ++s) tma_store_2d(&tm_x, s * kSlab, (int)(t * kTM), S.xr + s * kTM * kSlab);
      bulk_commit();
    }
  }
  if (!ok) {
    if (tid == 0) flag_timeout(status, 8);
    // bounded waits for the work this CTA may still have in flight
    if (mma_pending) mbar_wait(&S.bar_mma, pm);
    if (tid == 0 && x_pending) mbar_wait(&S.bar_x, px);
  }
  if (tid == 0) bulk_wait0();  // the last stores have left shared memory and completed
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
  static std::once_flag once;
  static EncodeTiled fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  });
  return fn;
}

// rows x 64 floats, row-major, loaded in boxes of 32 floats x box_rows with the 128-byte swizzle
int make_map(CUtensorMap* map, void* base, uint64_t rows, uint32_t box_rows) {
  EncodeTiled enc = encode_fn();
  if (!enc) return set_error(LQS_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled is not available");
  const cuuint64_t dims[2] = {(cuuint64_t)kTK, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)kTK * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)kSlab, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(LQS_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return LQS_OK;
}

// TF32 leading part of x (round to nearest, ties to even, at 10 mantissa bits)
float tf32_round_host(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  if ((u & 0x7F800000u) != 0x7F800000u) {
    u += 0xFFFu + ((u >> 13) & 1u);
    u &= 0xFFFFE000u;
  }
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

}  // namespace

// One lowered op applied to a register of kBlockQubits qubits (host, complex
// double): the semantics of each kernel op kind (lqs_internal.cuh) on the 32
// amplitudes, controls included.
static void kop_apply_small(const KOp& o, std::complex<double>* v) {
  using Z = std::complex<double>;
  const int N = 1 << kBlockQubits;
  const uint64_t cm = o.cmask;
  auto coef = [&](int i) { return Z(o.m[2 * i], o.m[2 * i + 1]); };
  auto on = [&](int i) { return ((uint64_t)i & cm) == cm; };
  const int T0 = o.t0 >= 0 ? 1 << o.t0 : 0, T1 = o.t1 >= 0 ? 1 << o.t1 : 0;
  switch (o.kind) {
    case K_PHASE: {
      const Z f = o.special == 1 ? Z(-1, 0) : o.special == 2 ? Z(0, 1) : o.special == 3 ? Z(0, -1) : coef(0);
      for (int i = 0; i < N; ++i)
        if (on(i)) v[i] *= f;
      break;
    }
    case K_DIAG1:
      for (int i = 0; i < N; ++i)
        if (on(i)) v[i] *= coef((i & T0) ? 1 : 0);
      break;
    case K_DIAG2:
      for (int i = 0; i < N; ++i)
        if (on(i)) v[i] *= coef(2 * ((i & T0) ? 1 : 0) + ((i & T1) ? 1 : 0));
      break;
    case K_ANTI1:
      for (int i = 0; i < N; ++i) {
        if ((i & T0) || !on(i)) continue;
        const Z a = v[i], b = v[i | T0];
        if (o.special == 1) {
          v[i] = b;
          v[i | T0] = a;
        } else {
          v[i] = coef(0) * b;
          v[i | T0] = coef(1) * a;
        }
      }
      break;
    case K_SWAP:
      for (int i = 0; i < N; ++i) {
        if (!(i & T0) || (i & T1) || !on(i)) continue;
        std::swap(v[i], v[i ^ T0 ^ T1]);
      }
      break;
    case K_DENSE1:
    case K_DENSE1R:
      for (int i = 0; i < N; ++i) {
        if ((i & T0) || !on(i)) continue;
        const Z a = v[i], b = v[i | T0];
        Z u[4];
        for (int k = 0; k < 4; ++k) u[k] = o.kind == K_DENSE1 ? coef(k) : Z(o.m[k], 0.0);
        v[i] = u[0] * a + u[1] * b;
        v[i | T0] = u[2] * a + u[3] * b;
      }
      break;
    case K_DENSE2:
      for (int i = 0; i < N; ++i) {
        if ((i & T0) || (i & T1) || !on(i)) continue;
        const int id[4] = {i, i | T1, i | T0, i | T0 | T1};  // local index 2 bit(t0) + bit(t1)
        Z x[4], y[4];
        for (int r = 0; r < 4; ++r) x[r] = v[id[r]];
        for (int r = 0; r < 4; ++r) {
          y[r] = 0;
          for (int c = 0; c < 4; ++c) y[r] += coef(4 * r + c) * x[c];
        }
        for (int r = 0; r < 4; ++r) v[id[r]] = y[r];
      }
      break;
    default:
      break;
  }
}

void block_matrix(const std::vector<KOp>& ops, const std::vector<int>& idx, double* U) {
  const int N = 1 << kBlockQubits;
  std::complex<double> col[1 << kBlockQubits];
  for (int k = 0; k < N; ++k) {
    for (int j = 0; j < N; ++j) col[j] = j == k ? 1.0 : 0.0;
    for (int i : idx) kop_apply_small(ops[i], col);
    for (int j = 0; j < N; ++j) {
      U[2 * (j * N + k)] = col[j].real();
      U[2 * (j * N + k) + 1] = col[j].imag();
    }
  }
}

double block_weight(const KOp& op) {
  switch (op.kind) {
    case K_DENSE2: return 4.0;
    case K_DENSE1:
    case K_DENSE1R: return 1.0;
    default: return 0.25;
  }
}

int apply_block(SV* sv, const double* matrix) {
  const int m = kBlockQubits, dim = 1 << m;
  // W^T in N-major rows (row n = output float, K contiguous), leading parts in
  // rows 0..63 and residuals in rows 64..127
  std::vector<float> B((size_t)2 * kTK * kTK);
  for (int j = 0; j < dim; ++j)
    for (int k = 0; k < dim; ++k) {
      const double re = matrix[2 * (j * dim + k)], im = matrix[2 * (j * dim + k) + 1];
      // W[2k + c][2j + c'] -> Bt[2j + c'][2k + c]
      const double w[2][2] = {{re, im}, {-im, re}};  // w[c][c']
      for (int c = 0; c < 2; ++c)
        for (int cp = 0; cp < 2; ++cp) {
          const double v = w[c][cp];
          const float lead = tf32_round_host((float)v);
          const size_t at = (size_t)(2 * j + cp) * kTK + (size_t)(2 * k + c);
          B[at] = lead;
          B[(size_t)kTK * kTK + at] = (float)(v - (double)lead);
        }
    }
  void* dB = nullptr;
  LQS_TRY(sv_scratch(sv, 2, B.size() * sizeof(float), &dB));
  LQS_CUDA_TRY(cudaMemcpyAsync(dB, B.data(), B.size() * sizeof(float), cudaMemcpyHostToDevice, sv->stream));
  const uint64_t rows = sv->N() >> m;
  CUtensorMap tm_x, tm_b;
  LQS_TRY(make_map(&tm_x, sv->d, rows, kTM));
  LQS_TRY(make_map(&tm_b, dB, 2 * kTK, kTK));
  static std::once_flag attr;
  cudaError_t ae = cudaSuccess;
  std::call_once(attr, [&] {
    ae = cudaFuncSetAttribute(k_block_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBlockSmemBytes);
  });
  LQS_CUDA_TRY(ae);
  const uint64_t ntiles = rows / kTM;
  const unsigned grid = (unsigned)std::min<uint64_t>(ntiles, (uint64_t)std::max(sv->sms, 1) * 2);
  ProfScope ps(sv->stream, "k_block_tc/tf32x3", 2.0 * (double)sv->bytes(), 8.0 * dim * (double)sv->N());
  k_block_tc<<<grid, kBlockThreads, kBlockSmemBytes, sv->stream>>>(tm_x, tm_b, static_cast<float*>(sv->d), ntiles,
                                                                  sv->d_status);
  count_launch();
  LQS_CUDA_TRY(cudaGetLastError());
  return LQS_OK;
}

}  // namespace lqs

using namespace lqs;

extern "C" int lqs_block_matrix(const lqs_op* ops, int n_ops, const double* params, int n_params, double* matrix) {
  if (!matrix) return set_error(LQS_ERR_ARG, "matrix is NULL");
  if (n_ops < 0 || (n_ops > 0 && !ops)) return set_error(LQS_ERR_ARG, "bad ops");
  std::vector<KOp> kops;
  LQS_TRY(lower_ops(kBlockQubits, ops, n_ops, params, n_params, false, kops));  // wires must be < 5
  std::vector<int> idx(kops.size());
  for (size_t i = 0; i < idx.size(); ++i) idx[i] = (int)i;
  block_matrix(kops, idx, matrix);
  return LQS_OK;
}

extern "C" int lqs_apply_block(lqs_sv* h, int m, const double* matrix) {
  void* dptr = nullptr;
  int n = 0, dtype = 0;
  LQS_TRY(lqs_sv_info(h, &dptr, &n, &dtype));  // validates the handle
  if (!matrix) return set_error(LQS_ERR_ARG, "matrix is NULL");
  SV* sv = reinterpret_cast<SV*>(h);
  if (sv->dtype != LQS_C64) return set_error(LQS_ERR_UNSUPPORTED, "tensor-core blocks take complex64 states");
  if (m != kBlockQubits) return set_error(LQS_ERR_UNSUPPORTED, "tensor-core blocks have m = 5 qubits");
  if (sv->n < m + 7) return set_error(LQS_ERR_UNSUPPORTED, "tensor-core blocks need at least m + 7 qubits");
  const int dim = 1 << m;
  for (int i = 0; i < 2 * dim * dim; ++i)
    if (!std::isfinite(matrix[i])) return set_error(LQS_ERR_ARG, "matrix has a non-finite entry");
  return apply_block(sv, matrix);
}
