// Allocation-free expectation value (lqs_expval_static): the expectation of
// a Hamiltonian given as a sum of Pauli words (Listing 1), without any device
// allocation.
//
// Some callers cannot allocate device memory at the point where they need a
// measurement: hosts whose memory pool owns all device memory and forbids
// driver allocations, and latency-critical loops that cannot afford the
// device-wide synchronisation cudaFree implies.  lqs_expval_static serves
// them: it needs no handle and uses a fixed scratch array compiled into the
// library instead of cudaMalloc.  It is synchronous: it ends by copying the
// results to host memory and waiting for its stream, so it cannot be called
// on a stream that is being captured into a CUDA graph: on such a stream it
// returns LQS_ERR_ARG before enqueuing anything, leaving the capture intact.
//
// The scratch array is a file-scope __device__ variable, so every GPU that
// loads the library holds it until the process exits.  In host code its name
// is only a host-side stand-in, so its device address is looked up once per
// device with cudaGetSymbolAddress (on the first call made on that device,
// with the device current) and passed to the kernels.  The stream must belong
// to the current device.  All calls share the array: calls whose work
// overlaps on the GPU (other streams, other host threads) race on it and must
// be serialised by the caller.
//
// Accuracy: complex128 amplitudes are split into double-float pairs (about
// 47 significant bits) and their products accumulate in double-float chains
// of 64 terms, then in float64, so each <P_w> carries a relative error of
// about 1e-14 rather than float64's 1e-16; complex64 products are formed in
// float32 and accumulated the same way.
#include <mutex>

#include "arith.cuh"
#include "lqs_internal.cuh"

namespace lqs {

// Layout of the static scratch (doubles): per-term partial sums, one row of
// kStaticGrid blocks per term, then the per-term sums, then the total.
constexpr int kStaticMaxTerms = 64;
constexpr int kStaticGrid = 1024;
constexpr size_t kStaticScratchDoubles = (size_t)kStaticMaxTerms * kStaticGrid + kStaticMaxTerms + 1;

static __device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];

struct StaticTerm {
  uint64_t x, z;
  int lowbit;  // lowest X/Y qubit, -1 for a diagonal word
  int ph;      // number of Y factors mod 4
};

static LQS_HD DFC widen(const float2& w) { return DFC{DF{w.x, 0.f}, DF{w.y, 0.f}}; }
static LQS_HD DFC widen(const double2& w) { return DFC{d2df(w.x), d2df(w.y)}; }

// acc += sign * Re(conj(a) b)   or   acc += sign * Im(conj(a) b)
__device__ __forceinline__ void add_re(DAcc& A, const DFC& a, const DFC& b, bool neg) {
  df_mac(A, neg ? df_neg(a.re) : a.re, b.re);
  df_mac(A, neg ? df_neg(a.im) : a.im, b.im);
}
__device__ __forceinline__ void add_im(DAcc& A, const DFC& a, const DFC& b, bool neg) {
  df_mac(A, neg ? df_neg(a.re) : a.re, b.im);
  df_mac(A, neg ? a.im : df_neg(a.im), b.re);
}

// <P> for one word: pairs (j, j^x) with j's lowest X bit clear (counted
// twice: the two orders are complex conjugates), or all j for a diagonal
// word.  One float64 partial per block into row `row` of the scratch.
template <class S>
__global__ void __launch_bounds__(256) k_static_word(const S* __restrict__ psi, uint64_t N, StaticTerm t,
                                                     double* scratch, int row) {
  __shared__ double red[256];
  DAcc acc{0.f, 0.f};
  double dacc = 0.0;
  int cnt = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t count = t.lowbit < 0 ? N : N / 2;
  for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < count; g += stride) {
    uint64_t j = g;
    if (t.lowbit >= 0) j = ((g >> t.lowbit) << (t.lowbit + 1)) | (g & ((1ull << t.lowbit) - 1));
    const DFC b = widen(psi[j]);
    const DFC a = t.lowbit < 0 ? b : widen(psi[j ^ t.x]);
    const bool neg = __popcll(j & t.z) & 1;
    switch (t.ph) {
      case 0: add_re(acc, a, b, neg); break;
      case 1: add_im(acc, a, b, !neg); break;
      case 2: add_re(acc, a, b, !neg); break;
      default: add_im(acc, a, b, neg); break;
    }
    if (++cnt == 64) {  // short double-float chains, then float64
      dacc += df2d(df_norm(acc));
      acc = DAcc{0.f, 0.f};
      cnt = 0;
    }
  }
  dacc += df2d(df_norm(acc));
  red[threadIdx.x] = (t.lowbit < 0 ? 1.0 : 2.0) * dacc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) scratch[(size_t)row * kStaticGrid + blockIdx.x] = red[0];
}

// Per-term sums over the used blocks (fixed order), then the total
// sum_w c_w <P_w>; written after the partial rows.
struct StaticCoeffs {
  double c[kStaticMaxTerms];
};
__global__ void k_static_reduce(double* scratch, int n_terms, int grid, StaticCoeffs C) {
  __shared__ double red[256];
  double* sums = scratch + (size_t)kStaticMaxTerms * kStaticGrid;
  for (int w = 0; w < n_terms; ++w) {
    double s = 0.0;
    for (int b = threadIdx.x; b < grid; b += blockDim.x) s += scratch[(size_t)w * kStaticGrid + b];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
      if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
      __syncthreads();
    }
    if (threadIdx.x == 0) sums[w] = red[0];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double e = 0.0;
    for (int w = 0; w < n_terms; ++w) e += C.c[w] * sums[w];
    sums[kStaticMaxTerms] = e;
  }
}

// Device address of the scratch array, looked up once per device.
static std::mutex g_static_mu;
static double* g_static_ptr[64] = {nullptr};

static int static_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(LQS_ERR_UNSUPPORTED, std::string("no CUDA device: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= 64) return set_error(LQS_ERR_UNSUPPORTED, "device index above 63");
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(static scratch)");
    g_static_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_static_ptr[dev];
  return LQS_OK;
}

}  // namespace lqs

using namespace lqs;

extern "C" int lqs_expval_static(const void* psi_device, int n_qubits, int dtype, void* cuda_stream,
                                 const lqs_pauli* terms, int n_terms, double* out_host, double* per_term_host) {
  if (!psi_device) return set_error(LQS_ERR_ARG, "psi_device is NULL");
  if (n_qubits < 1 || n_qubits > 36) return set_error(LQS_ERR_ARG, "n_qubits must be in [1, 36]");
  if (dtype != LQS_C64 && dtype != LQS_C128) return set_error(LQS_ERR_ARG, "dtype must be LQS_C64 or LQS_C128");
  if (!out_host) return set_error(LQS_ERR_ARG, "out_host is NULL");
  if (n_terms < 0 || (n_terms > 0 && !terms)) return set_error(LQS_ERR_ARG, "bad terms");
  if (n_terms > kStaticMaxTerms)
    return set_error(LQS_ERR_ARG, "lqs_expval_static takes at most " + std::to_string(kStaticMaxTerms) +
                                      " Pauli terms (its fixed scratch holds " + std::to_string(kStaticMaxTerms) +
                                      " x " + std::to_string(kStaticGrid) + " partial sums); use lqs_expval");
  const uint64_t N = 1ull << n_qubits;
  for (int i = 0; i < n_terms; ++i)
    if ((terms[i].x_mask | terms[i].z_mask) & ~(N - 1))
      return set_error(LQS_ERR_ARG, "term " + std::to_string(i) + " acts on a qubit >= n");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int sms = 0, dev = 0, sdev = 0;
  LQS_CUDA_TRY(cudaGetDevice(&dev));
  // The call ends with a copy to pageable host memory and a stream
  // synchronisation, neither of which a graph capture admits: refuse before
  // anything is enqueued, so the caller's capture stays valid.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  LQS_CUDA_TRY(cudaStreamIsCapturing(st, &cap));
  if (cap != cudaStreamCaptureStatusNone)
    return set_error(LQS_ERR_ARG, "lqs_expval_static is synchronous and cannot run on a stream that is being "
                                  "captured into a CUDA graph; call it outside the capture");
  LQS_CUDA_TRY(cudaStreamGetDevice(st, &sdev));
  if (sdev != dev)
    return set_error(LQS_ERR_ARG, "cuda_stream belongs to device " + std::to_string(sdev) +
                                      " but the current device is " + std::to_string(dev) +
                                      ": make the stream's device current first");
  double* scratch = nullptr;
  LQS_TRY(static_scratch(&scratch));
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t want = (N + 255) / 256;
  const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(want, std::min<uint64_t>(kStaticGrid, (uint64_t)std::max(sms, 1) * 8)));
  StaticCoeffs C{};
  for (int w = 0; w < n_terms; ++w) {
    const lqs_pauli& p = terms[w];
    StaticTerm t;
    t.x = p.x_mask;
    t.z = p.z_mask;
    t.lowbit = p.x_mask ? __builtin_ctzll(p.x_mask) : -1;
    t.ph = __builtin_popcountll(p.x_mask & p.z_mask) & 3;
    C.c[w] = p.coeff;
    if (dtype == LQS_C64)
      k_static_word<float2><<<grid, 256, 0, st>>>(static_cast<const float2*>(psi_device), N, t, scratch, w);
    else
      k_static_word<double2><<<grid, 256, 0, st>>>(static_cast<const double2*>(psi_device), N, t, scratch, w);
    count_launch();
    LQS_CUDA_TRY(cudaGetLastError());
  }
  k_static_reduce<<<1, 256, 0, st>>>(scratch, n_terms, grid, C);
  count_launch();
  LQS_CUDA_TRY(cudaGetLastError());
  const double* sums = scratch + (size_t)kStaticMaxTerms * kStaticGrid;
  LQS_CUDA_TRY(cudaMemcpyAsync(out_host, sums + kStaticMaxTerms, sizeof(double), cudaMemcpyDeviceToHost, st));
  if (per_term_host && n_terms > 0)
    LQS_CUDA_TRY(cudaMemcpyAsync(per_term_host, sums, sizeof(double) * n_terms, cudaMemcpyDeviceToHost, st));
  LQS_CUDA_TRY(cudaStreamSynchronize(st));
  return LQS_OK;
}
