// C ABI entry points (include/lqs.h): validation, handles, dispatch.
//
// The calls follow the paper's circuit model: gates from its gate set applied
// to qubits of one state (Sec. 2, Sec. 3.2), expectation values of a
// Hamiltonian given as a sum of Pauli words and gradients with respect to the
// gate parameters (Listing 1).  Each gate is routed by class and by the
// qubits it touches (Sec. 2, Fig. 1).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <memory>
#include <vector>

#include "arith.cuh"
#include "jit.h"
#include "measure_common.cuh"
#include "lqs_internal.cuh"

namespace lqs {

static thread_local std::string g_err;
static std::atomic<uint64_t> g_launches{0};
static std::atomic<int> g_arith{LQS_ARITH_DF};

int set_error(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cuda_error(cudaError_t e, const char* what) {
  const int code = (e == cudaErrorMemoryAllocation) ? LQS_ERR_OOM : LQS_ERR_CUDA;
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return code;
}

void count_launch(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// ---- launch profiling --------------------------------------------------------
struct ProfRec {
  std::string name;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaStream_t st = nullptr;
  double bytes = 0, flops = 0;
};
static std::mutex g_prof_mu;
static bool g_prof_on = false;
static std::vector<ProfRec> g_prof;
static std::vector<cudaEvent_t> g_event_pool;

static cudaEvent_t pool_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

ProfScope::ProfScope(cudaStream_t s, const char* name, double bytes, double flops) : st(s) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (!g_prof_on) return;
  ProfRec r;
  r.name = name;
  r.st = s;
  r.bytes = bytes;
  r.flops = flops;
  r.e0 = pool_event();
  r.e1 = pool_event();
  cudaEventRecord(r.e0, s);
  idx = (int)g_prof.size();
  g_prof.push_back(r);
}
ProfScope::~ProfScope() {
  if (idx < 0) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (idx < (int)g_prof.size()) cudaEventRecord(g_prof[idx].e1, g_prof[idx].st);
}

const char* arith_tag(int dtype, int arith) {
  if (dtype == LQS_C64) return "f32";
  return arith == LQS_ARITH_F64 ? "f64" : "df";
}

double kop_touched_fraction(const KOp& o) {
  const double c = std::ldexp(1.0, -__builtin_popcountll(o.cmask));
  return o.kind == K_SWAP ? 0.5 * c : c;
}
double kop_flops_per_amp(const KOp& o) {
  switch (o.kind) {
    case K_PHASE: return o.special ? 0.0 : 6.0;
    case K_DIAG1: return 6.0;
    case K_DIAG2: return 6.0;
    case K_ANTI1: return o.special == 1 ? 0.0 : 6.0;
    case K_SWAP: return 0.0;
    case K_DENSE1: return 14.0;
    case K_DENSE1R: return 6.0;
    case K_DENSE2: return 30.0;
  }
  return 0.0;
}

int current_arith(int requested) {
  if (requested == LQS_ARITH_F64 || requested == LQS_ARITH_DF) return requested;
  return g_arith.load();
}

int sv_scratch(SV* sv, int slot, size_t bytes, void** out) {
  if (slot < 0 || slot > 2) return set_error(LQS_ERR_ARG, "internal: scratch slot");
  if (sv->scratch_bytes[slot] < bytes) {
    if (sv->scratch[slot]) {
      LQS_CUDA_TRY(cudaStreamSynchronize(sv->stream));
      cudaFree(sv->scratch[slot]);
      sv->scratch[slot] = nullptr;
      sv->scratch_bytes[slot] = 0;
    }
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) return cuda_error(e, "cudaMalloc(scratch)");
    sv->scratch[slot] = p;
    sv->scratch_bytes[slot] = bytes;
  }
  *out = sv->scratch[slot];
  return LQS_OK;
}

static int check_sv(const lqs_sv* h) {
  if (!h) return set_error(LQS_ERR_ARG, "state handle is NULL");
  return LQS_OK;
}

static SV* S_(lqs_sv* h) { return reinterpret_cast<SV*>(h); }
static const SV* S_(const lqs_sv* h) { return reinterpret_cast<const SV*>(h); }

__global__ void k_set_basis_f(float2* psi, uint64_t N, uint64_t x) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride)
    psi[i] = make_float2(i == x ? 1.f : 0.f, 0.f);
}
__global__ void k_set_basis_d(double2* psi, uint64_t N, uint64_t x) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride)
    psi[i] = make_double2(i == x ? 1.0 : 0.0, 0.0);
}

// sum |a - b|^2 and sum |b|^2 for states of possibly different dtypes:
// double-float per thread (chains of at most 64 terms), float64 per block.
template <class SA, class SB>
__global__ void k_distance(const SA* __restrict__ a, const SB* __restrict__ b, uint64_t N, double* part) {
  __shared__ double r0[256], r1[256];
  auto wd = [](const auto& v) -> DFC {
    if constexpr (sizeof(v) == 8) return DFC{DF{v.x, 0.f}, DF{v.y, 0.f}};
    else return DFC{d2df(v.x), d2df(v.y)};
  };
  double d0 = 0.0, d1 = 0.0;
  DAcc x{0.f, 0.f}, y{0.f, 0.f};
  int cnt = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
    const DFC va = wd(a[i]), vb = wd(b[i]);
    const DF dr = df_sub(va.re, vb.re), di = df_sub(va.im, vb.im);
    df_mac(x, dr, dr);
    df_mac(x, di, di);
    df_mac(y, vb.re, vb.re);
    df_mac(y, vb.im, vb.im);
    if (++cnt == 64) {
      d0 += df2d(df_norm(x));
      d1 += df2d(df_norm(y));
      x = DAcc{0.f, 0.f};
      y = DAcc{0.f, 0.f};
      cnt = 0;
    }
  }
  d0 += df2d(df_norm(x));
  d1 += df2d(df_norm(y));
  r0[threadIdx.x] = d0;
  r1[threadIdx.x] = d1;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      r0[threadIdx.x] += r0[threadIdx.x + w];
      r1[threadIdx.x] += r1[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = r0[0];
    part[2 * blockIdx.x + 1] = r1[0];
  }
}

// Dense-block extraction for the tensor cores.  A scan in circuit order keeps
// open runs, each a set of gates whose wires stay within one set W of at
// most kBlockQubits qubits (any qubits; W grows with the run), the runs' sets
// pairwise disjoint.  A gate joins the runs it touches, merged into one, when
// their qubits and its own number at most kBlockQubits; otherwise it closes
// every run it touches and opens a new one.  A closed run whose dense weight reaches the threshold
// becomes one block.  The other gates keep their circuit order, and each
// block takes the place of its run's last gate: the gates of the run that it
// moves past act on other qubits (a gate on W would have joined or closed the
// run), so they commute with it.  The tensor-core kernel works on qubits
// 0..kBlockQubits-1: W's qubits above that range are swapped with free
// qubits of the range before the block (uncontrolled SWAPs, which the fused
// segments around it apply as relabellings of their tile qubits) and back
// after it, and the block matrix is composed from the run's gates relabelled
// the same way.  A window that needs SWAPs must reach twice the threshold,
// for the passes its SWAPs may add.  emit(ops, U): U is a block matrix, or
// null for gates of the fused stream.
template <class Emit>
static void split_blocks(const std::vector<KOp>& kops, double threshold, Emit&& emit) {
  const uint64_t low = (1ull << kBlockQubits) - 1;
  struct Run {
    uint64_t W = 0;
    std::vector<int> ops;
    double weight = 0.0;
  };
  std::vector<Run> open, blocks;
  auto close = [&](size_t r) {
    const bool swaps = (open[r].W & ~low) != 0;
    if (open[r].weight >= (swaps ? 2.0 : 1.0) * threshold) blocks.push_back(open[r]);
    open.erase(open.begin() + (long)r);
  };
  for (int i = 0; i < (int)kops.size(); ++i) {
    const uint64_t w = kops[i].wire_mask();
    std::vector<size_t> hit;
    for (size_t r = 0; r < open.size(); ++r)
      if (open[r].W & w) hit.push_back(r);
    uint64_t uni = w;
    for (size_t r : hit) uni |= open[r].W;
    if (!hit.empty() && __builtin_popcountll(uni) <= kBlockQubits) {
      // the gate joins the runs it touches, merged into one (their gates in circuit order)
      Run& R = open[hit[0]];
      for (size_t h = hit.size(); h-- > 1;) {
        Run& Q = open[hit[h]];
        R.ops.insert(R.ops.end(), Q.ops.begin(), Q.ops.end());
        R.weight += Q.weight;
        open.erase(open.begin() + (long)hit[h]);
      }
      std::sort(R.ops.begin(), R.ops.end());
      R.W = uni;
      R.ops.push_back(i);
      R.weight += block_weight(kops[i]);
      continue;
    }
    for (size_t h = hit.size(); h-- > 0;) close(hit[h]);
    if (__builtin_popcountll(w) <= kBlockQubits) {
      Run R;
      R.W = w;
      R.ops.push_back(i);
      R.weight = block_weight(kops[i]);
      open.push_back(std::move(R));
    }
  }
  while (!open.empty()) close(open.size() - 1);
  // the output: gates in circuit order, each block in place of its run's last gate
  std::vector<int> block_of(kops.size(), -1), last_of(kops.size(), -1);
  for (size_t bI = 0; bI < blocks.size(); ++bI) {
    for (int i : blocks[bI].ops) block_of[(size_t)i] = (int)bI;
    last_of[(size_t)blocks[bI].ops.back()] = (int)bI;
  }
  std::vector<KOp> pending;
  auto flush_pending = [&]() {
    if (!pending.empty()) emit(std::move(pending), nullptr);
    pending.clear();
  };
  for (int i = 0; i < (int)kops.size(); ++i) {
    if (block_of[(size_t)i] < 0) {
      pending.push_back(kops[i]);
      continue;
    }
    if (last_of[(size_t)i] < 0) continue;
    const Run& R = blocks[(size_t)last_of[(size_t)i]];
    // map: each qubit of W above the range takes a free qubit of the range
    int to[64];
    for (int q = 0; q < 64; ++q) to[q] = q;
    std::vector<KOp> sw;
    uint64_t freel = low & ~R.W;
    for (uint64_t hi = R.W & ~low; hi; hi &= hi - 1) {
      const int q = __builtin_ctzll(hi);
      const int sl = __builtin_ctzll(freel);
      freel &= freel - 1;
      to[q] = sl;
      to[sl] = q;
      KOp k;
      k.kind = K_SWAP;
      k.t0 = sl;
      k.t1 = q;
      sw.push_back(k);
    }
    std::vector<KOp> rel;
    for (int j : R.ops) {
      KOp k = kops[(size_t)j];
      if (k.t0 >= 0) k.t0 = to[k.t0];
      if (k.t1 >= 0) k.t1 = to[k.t1];
      uint64_t cm = 0;
      for (uint64_t c = k.cmask; c; c &= c - 1) cm |= 1ull << to[__builtin_ctzll(c)];
      k.cmask = cm;
      rel.push_back(k);
    }
    std::vector<int> all(rel.size());
    for (size_t j = 0; j < all.size(); ++j) all[j] = (int)j;
    double U[2 << (2 * kBlockQubits)];
    block_matrix(rel, all, U);
    pending.insert(pending.end(), sw.begin(), sw.end());
    flush_pending();
    emit(std::vector<KOp>(), U);
    pending.insert(pending.end(), sw.begin(), sw.end());
  }
  flush_pending();
}

}  // namespace lqs

using namespace lqs;

extern "C" {

int lqs_sv_distance(lqs_sv* ha, lqs_sv* hb, double* diff2_host, double* norm2_b_host) {
  LQS_TRY(check_sv(ha));
  LQS_TRY(check_sv(hb));
  if (!diff2_host || !norm2_b_host) return set_error(LQS_ERR_ARG, "output pointer is NULL");
  SV* A = S_(ha);
  SV* B = S_(hb);
  if (A->n != B->n) return set_error(LQS_ERR_ARG, "states have different qubit counts");
  LQS_CUDA_TRY(cudaStreamSynchronize(A->stream));
  LQS_CUDA_TRY(cudaStreamSynchronize(B->stream));
  const int grid = std::max(1, std::min<int>((int)std::min<uint64_t>((A->N() + 255) / 256, 1u << 20), A->sms * 4));
  void* scratch = nullptr;
  LQS_TRY(sv_scratch(B, 2, sizeof(double) * 2 * grid, &scratch));
  double* part = static_cast<double*>(scratch);
  cudaStream_t st = B->stream;
  {
    ProfScope ps(st, "k_distance", (double)(A->bytes() + B->bytes()), 0.0);
    if (A->dtype == LQS_C64 && B->dtype == LQS_C64)
      k_distance<float2, float2><<<grid, 256, 0, st>>>((const float2*)A->d, (const float2*)B->d, A->N(), part);
    else if (A->dtype == LQS_C64)
      k_distance<float2, double2><<<grid, 256, 0, st>>>((const float2*)A->d, (const double2*)B->d, A->N(), part);
    else if (B->dtype == LQS_C64)
      k_distance<double2, float2><<<grid, 256, 0, st>>>((const double2*)A->d, (const float2*)B->d, A->N(), part);
    else
      k_distance<double2, double2><<<grid, 256, 0, st>>>((const double2*)A->d, (const double2*)B->d, A->N(), part);
    count_launch();
  }
  LQS_CUDA_TRY(cudaGetLastError());
  std::vector<double> h(2 * grid);
  LQS_CUDA_TRY(cudaMemcpyAsync(h.data(), part, sizeof(double) * 2 * grid, cudaMemcpyDeviceToHost, st));
  LQS_CUDA_TRY(cudaStreamSynchronize(st));
  double d0 = 0.0, d1 = 0.0;
  for (int i = 0; i < grid; ++i) {
    d0 += h[2 * i];
    d1 += h[2 * i + 1];
  }
  *diff2_host = d0;
  *norm2_b_host = d1;
  return LQS_OK;
}


const char* lqs_last_error(void) { return g_err.c_str(); }

int lqs_profile_start(void) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (auto& r : g_prof) {
    g_event_pool.push_back(r.e0);
    g_event_pool.push_back(r.e1);
  }
  g_prof.clear();
  g_prof_on = true;
  return LQS_OK;
}

int lqs_profile_stop(lqs_launch_record* out, int cap, int* count) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_on = false;
  for (auto& r : g_prof) cudaEventSynchronize(r.e1);
  if (count) *count = (int)g_prof.size();
  for (int i = 0; out && i < cap && i < (int)g_prof.size(); ++i) {
    const ProfRec& r = g_prof[i];
    std::memset(out[i].kernel, 0, sizeof out[i].kernel);
    std::strncpy(out[i].kernel, r.name.c_str(), sizeof out[i].kernel - 1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.e0, r.e1);
    out[i].ms = ms;
    out[i].bytes = r.bytes;
    out[i].flops = r.flops;
  }
  return LQS_OK;
}

int lqs_version(void) { return 100; }

uint64_t lqs_kernel_launches(void) { return g_launches.load(); }

int lqs_set_arith(int arith) {
  if (arith != LQS_ARITH_AUTO && arith != LQS_ARITH_F64 && arith != LQS_ARITH_DF)
    return set_error(LQS_ERR_ARG, "arith must be LQS_ARITH_AUTO, LQS_ARITH_F64 or LQS_ARITH_DF");
  g_arith.store(arith == LQS_ARITH_AUTO ? LQS_ARITH_DF : arith);
  return LQS_OK;
}

int lqs_sv_alloc(int n_qubits, int dtype, void* device_ptr, void* cuda_stream, lqs_sv** out) {
  if (!out) return set_error(LQS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n_qubits < 1 || n_qubits > 36) return set_error(LQS_ERR_ARG, "n_qubits must be in [1, 36]");
  if (dtype != LQS_C64 && dtype != LQS_C128) return set_error(LQS_ERR_ARG, "dtype must be LQS_C64 or LQS_C128");
  if (device_ptr && (reinterpret_cast<uintptr_t>(device_ptr) & 255u))
    return set_error(LQS_ERR_ARG, "device_ptr must be 256-byte aligned");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(LQS_ERR_UNSUPPORTED, std::string("no CUDA device: ") + cudaGetErrorString(e));
  SV* sv = new SV();
  sv->n = n_qubits;
  sv->dtype = dtype;
  sv->stream = static_cast<cudaStream_t>(cuda_stream);
  sv->device = dev;
  cudaDeviceGetAttribute(&sv->sms, cudaDevAttrMultiProcessorCount, dev);
  if (device_ptr) {
    sv->d = device_ptr;
    sv->owns = false;
  } else {
    e = cudaMalloc(&sv->d, sv->bytes());
    if (e != cudaSuccess) {
      delete sv;
      return cuda_error(e, "cudaMalloc(state)");
    }
    sv->owns = true;
  }
  e = cudaMalloc(&sv->d_status, 64);
  if (e == cudaSuccess) e = cudaMemsetAsync(sv->d_status, 0, 64, sv->stream);
  if (e != cudaSuccess) {
    if (sv->owns) cudaFree(sv->d);
    delete sv;
    return cuda_error(e, "cudaMalloc(status)");
  }
  *out = reinterpret_cast<lqs_sv*>(sv);
  return LQS_OK;
}

int lqs_sv_free(lqs_sv* h) {
  if (!h) return LQS_OK;
  SV* sv = S_(h);
  cudaStreamSynchronize(sv->stream);
  for (int i = 0; i < 3; ++i)
    if (sv->scratch[i]) cudaFree(sv->scratch[i]);
  if (sv->d_status) cudaFree(sv->d_status);
  if (sv->owns && sv->d) cudaFree(sv->d);
  delete sv;
  return LQS_OK;
}

int lqs_sv_info(const lqs_sv* h, void** device_ptr, int* n_qubits, int* dtype) {
  LQS_TRY(check_sv(h));
  const SV* sv = S_(h);
  if (device_ptr) *device_ptr = sv->d;
  if (n_qubits) *n_qubits = sv->n;
  if (dtype) *dtype = sv->dtype;
  return LQS_OK;
}

int lqs_sv_set_basis(lqs_sv* h, uint64_t x) {
  LQS_TRY(check_sv(h));
  SV* sv = S_(h);
  if (x >= sv->N()) return set_error(LQS_ERR_ARG, "basis index >= 2^n");
  const unsigned grid = (unsigned)std::min<uint64_t>((sv->N() + 255) / 256, (uint64_t)sv->sms * 8);
  ProfScope ps(sv->stream, "k_set_basis", (double)sv->bytes(), 0.0);
  if (sv->dtype == LQS_C64) k_set_basis_f<<<grid, 256, 0, sv->stream>>>((float2*)sv->d, sv->N(), x);
  else k_set_basis_d<<<grid, 256, 0, sv->stream>>>((double2*)sv->d, sv->N(), x);
  count_launch();
  LQS_CUDA_TRY(cudaGetLastError());
  return LQS_OK;
}

int lqs_sv_copy_from_host(lqs_sv* h, const void* host) {
  LQS_TRY(check_sv(h));
  if (!host) return set_error(LQS_ERR_ARG, "host is NULL");
  SV* sv = S_(h);
  LQS_CUDA_TRY(cudaMemcpyAsync(sv->d, host, sv->bytes(), cudaMemcpyHostToDevice, sv->stream));
  return LQS_OK;
}

int lqs_sv_copy_to_host(const lqs_sv* h, void* host) {
  LQS_TRY(check_sv(h));
  if (!host) return set_error(LQS_ERR_ARG, "host is NULL");
  const SV* sv = S_(h);
  LQS_CUDA_TRY(cudaMemcpyAsync(host, sv->d, sv->bytes(), cudaMemcpyDeviceToHost, sv->stream));
  LQS_CUDA_TRY(cudaStreamSynchronize(sv->stream));
  return LQS_OK;
}

int lqs_sv_copy_to_host_async(const lqs_sv* h, void* host) {
  LQS_TRY(check_sv(h));
  if (!host) return set_error(LQS_ERR_ARG, "host is NULL");
  const SV* sv = S_(h);
  LQS_CUDA_TRY(cudaMemcpyAsync(host, sv->d, sv->bytes(), cudaMemcpyDeviceToHost, sv->stream));
  return LQS_OK;
}

int lqs_sv_sync(lqs_sv* h) {
  LQS_TRY(check_sv(h));
  SV* sv = S_(h);
  LQS_CUDA_TRY(cudaStreamSynchronize(sv->stream));
  int status[4] = {0, 0, 0, 0};
  LQS_CUDA_TRY(cudaMemcpy(status, sv->d_status, sizeof status, cudaMemcpyDeviceToHost));
  if (status[0]) {
    cudaMemsetAsync(sv->d_status, 0, 64, sv->stream);
    return set_error(LQS_ERR_TIMEOUT, "a device-side wait gave up (code " + std::to_string(status[0]) + ")");
  }
  return LQS_OK;
}

int lqs_apply_gate(lqs_sv* h, int gate, const int* wires, int n_wires, const double* params, int n_params,
                   int inverse) {
  LQS_TRY(check_sv(h));
  SV* sv = S_(h);
  std::vector<KOp> ops;
  const double* matrix = nullptr;
  if (gate == LQS_U2 || gate == LQS_U4) {
    const int need = gate == LQS_U2 ? 8 : 32;
    if (!params || n_params != need)
      return set_error(LQS_ERR_ARG, std::string(gate == LQS_U2 ? "U2" : "U4") + " needs its matrix as " +
                                        std::to_string(need) + " doubles in params");
    matrix = params;
  }
  LQS_TRY(lower_gate(sv->n, gate, wires, n_wires, params, n_params, matrix, inverse, -1, false, false, ops));
  const int arith = current_arith(LQS_ARITH_AUTO);
  for (const KOp& k : ops) LQS_TRY(launch_gate(sv, k, arith));
  return LQS_OK;
}

int lqs_apply_matrix(lqs_sv* h, const int* wires, int n_wires, const double* matrix) {
  LQS_TRY(check_sv(h));
  SV* sv = S_(h);
  if (n_wires != 1 && n_wires != 2) return set_error(LQS_ERR_ARG, "lqs_apply_matrix takes 1 or 2 wires");
  std::vector<KOp> ops;
  LQS_TRY(lower_gate(sv->n, n_wires == 1 ? LQS_U2 : LQS_U4, wires, n_wires, nullptr, 0, matrix, 0, -1, false, true,
                     ops));
  const int arith = current_arith(LQS_ARITH_AUTO);
  for (const KOp& k : ops) LQS_TRY(launch_gate(sv, k, arith));
  return LQS_OK;
}

int lqs_apply_fused(lqs_sv* h, const lqs_op* ops, int n_ops, const double* params, int n_params,
                    const lqs_fuse_cfg* cfg) {
  LQS_TRY(check_sv(h));
  SV* sv = S_(h);
  std::vector<KOp> kops;
  LQS_TRY(lower_ops(sv->n, ops, n_ops, params, n_params, false, kops));
  lqs_fuse_cfg tuned;
  if (!cfg && tuned_cfg(sv->n, sv->dtype, ops, n_ops, &tuned)) cfg = &tuned;  // lqs_autotune_fused's choice
  PlanCfg pc;
  int arith = LQS_ARITH_AUTO;
  LQS_TRY(resolve_cfg(sv->n, sv->dtype, cfg, pc, &arith));
  // Pieces in execution order: fused runs of lowered ops, and dense blocks
  // on qubits 0..4 for the tensor cores (complex64).
  struct Piece {
    std::vector<KOp> ops;
    std::vector<Segment> segs;
    bool block = false;
    double U[2 << (2 * kBlockQubits)];
  };
  std::vector<std::unique_ptr<Piece>> pieces;
  const double tc_weight = !cfg || cfg->tc_blocks == 0 ? 16.0 : (double)cfg->tc_blocks;
  if (sv->dtype == LQS_C64 && sv->n >= kBlockQubits + 7 && tc_weight > 0) {
    split_blocks(kops, tc_weight, [&](std::vector<KOp>&& run, const double* U) {
      if (U) {
        pieces.emplace_back(new Piece());
        pieces.back()->block = true;
        std::memcpy(pieces.back()->U, U, sizeof(pieces.back()->U));
      } else {
        if (pieces.empty() || pieces.back()->block) pieces.emplace_back(new Piece());
        for (KOp& k : run) pieces.back()->ops.push_back(k);
      }
    });
  } else {
    pieces.emplace_back(new Piece());
    pieces.back()->ops = std::move(kops);
  }
  for (auto& p : pieces)
    if (!p->block) LQS_TRY(plan_segments(sv->n, p->ops, pc, p->segs));
  if (jit_enabled_for(sv->n)) {  // compile the structures this call needs, in parallel, before launching
    std::vector<void*> todo;
    for (auto& p : pieces)
      for (const Segment& s : p->segs) LQS_TRY(jit_collect(sv->n, sv->dtype, arith, p->ops, s, pc, false, todo));
    const int rc = jit_compile(todo);
    if (rc != LQS_OK && jit_mode() == LQS_JIT_ON) return rc;
  }
  // Consecutive compiled double-float segments hand the state to one another
  // as hi/lo float pairs (no float64 conversions in between); the first
  // reads float64 and the last writes it, so the call leaves a complex128
  // state as always.
  std::vector<std::pair<const Piece*, const Segment*>> order;
  for (auto& p : pieces) {
    if (p->block) order.emplace_back(p.get(), nullptr);
    for (const Segment& s : p->segs) order.emplace_back(p.get(), &s);
  }
  const int kk = std::min(pc.k, sv->n), bb = std::min(pc.b, kk);
  std::vector<char> split(order.size(), 0);
  for (size_t i = 0; i < order.size(); ++i)
    split[i] = order[i].second && seg_split_capable(sv, order[i].first->ops, *order[i].second, kk, bb, arith);
  for (size_t i = 0; i < order.size(); ++i) {
    const Piece* p = order[i].first;
    if (!order[i].second) {
      LQS_TRY(apply_block(sv, p->U));
      continue;
    }
    const unsigned fmt = split[i] ? (i > 0 && split[i - 1] ? 1u : 0u) | (i + 1 < order.size() && split[i + 1] ? 2u : 0u)
                                  : 0u;
    LQS_TRY(launch_segment(sv, p->ops, *order[i].second, pc, arith, fmt));
  }
  return LQS_OK;
}

int lqs_jit_precompile_expval(int n_qubits, int dtype, int arith, const lqs_pauli* terms, int n_terms, int lambda,
                              int* n_compiled) {
  if (n_compiled) *n_compiled = 0;
  if (n_qubits < 1 || n_qubits > 36) return set_error(LQS_ERR_ARG, "n_qubits must be in [1, 36]");
  if (dtype != LQS_C64 && dtype != LQS_C128) return set_error(LQS_ERR_ARG, "bad dtype");
  if (arith != LQS_ARITH_AUTO && arith != LQS_ARITH_F64 && arith != LQS_ARITH_DF)
    return set_error(LQS_ERR_ARG, "arith must be LQS_ARITH_AUTO, LQS_ARITH_F64 or LQS_ARITH_DF");
  if (n_terms < 0 || (n_terms > 0 && !terms)) return set_error(LQS_ERR_ARG, "bad terms");
  const uint64_t all = n_qubits >= 64 ? ~0ull : ((1ull << n_qubits) - 1);
  for (int i = 0; i < n_terms; ++i)
    if ((terms[i].x_mask | terms[i].z_mask) & ~all) return set_error(LQS_ERR_ARG, "a term acts on a qubit >= n");
  if (n_terms == 0 || n_qubits <= (dtype == LQS_C64 ? 12 : 11)) return LQS_OK;  // nothing compiled for these
  const int rc = pauli_precompile(n_qubits, dtype, current_arith(arith), terms, n_terms, lambda != 0, n_compiled);
  if (rc == LQS_ERR_UNSUPPORTED && std::string(lqs_last_error()).find("do not fit") != std::string::npos)
    return LQS_OK;  // words wider than a tile run on the interpreter passes
  return rc;
}

int lqs_jit_precompile_adjoint(int n_qubits, int dtype, int arith, const lqs_op* ops, int n_ops,
                               const double* params, int n_params, int* n_compiled) {
  if (n_compiled) *n_compiled = 0;
  if (n_qubits < 1 || n_qubits > 36) return set_error(LQS_ERR_ARG, "n_qubits must be in [1, 36]");
  if (dtype != LQS_C64 && dtype != LQS_C128) return set_error(LQS_ERR_ARG, "bad dtype");
  if (arith != LQS_ARITH_AUTO && arith != LQS_ARITH_F64 && arith != LQS_ARITH_DF)
    return set_error(LQS_ERR_ARG, "arith must be LQS_ARITH_AUTO, LQS_ARITH_F64 or LQS_ARITH_DF");
  std::vector<KOp> kops;
  LQS_TRY(lower_ops(n_qubits, ops, n_ops, params, n_params, true, kops));
  std::vector<KOp> rev;
  rev.reserve(kops.size());
  for (size_t i = kops.size(); i-- > 0;) rev.push_back(inverse_op(kops[i]));
  const int ar = current_arith(arith);
  if (n_qubits <= adjoint_tile_qubits(dtype)) return LQS_OK;  // one tile: the interpreter sweep runs it
  return adjoint_precompile(n_qubits, dtype, ar, rev, n_compiled);
}

int lqs_jit_precompile(int n_qubits, int dtype, int arith, const lqs_op* ops, int n_ops, const double* params,
                       int n_params, const lqs_fuse_cfg* cfg, int* n_compiled) {
  if (n_compiled) *n_compiled = 0;
  if (n_qubits < 1 || n_qubits > 36) return set_error(LQS_ERR_ARG, "n_qubits must be in [1, 36]");
  if (dtype != LQS_C64 && dtype != LQS_C128) return set_error(LQS_ERR_ARG, "bad dtype");
  if (arith != LQS_ARITH_AUTO && arith != LQS_ARITH_F64 && arith != LQS_ARITH_DF)
    return set_error(LQS_ERR_ARG, "arith must be LQS_ARITH_AUTO, LQS_ARITH_F64 or LQS_ARITH_DF");
  std::vector<KOp> kops;
  LQS_TRY(lower_ops(n_qubits, ops, n_ops, params, n_params, false, kops));
  PlanCfg pc;
  int ar = LQS_ARITH_AUTO;
  LQS_TRY(resolve_cfg(n_qubits, dtype, cfg, pc, &ar));
  if (arith != LQS_ARITH_AUTO) ar = arith;
  std::vector<Segment> segs;
  LQS_TRY(plan_segments(n_qubits, kops, pc, segs));
  std::vector<void*> todo;
  for (const Segment& s : segs) LQS_TRY(jit_collect(n_qubits, dtype, ar, kops, s, pc, true, todo));
  LQS_TRY(jit_compile(todo));
  int ok = 0;
  std::string err;
  const int st = jit_states(todo, &ok, &err);
  if (n_compiled) *n_compiled = ok;
  if (st != LQS_OK) return set_error(LQS_ERR_UNSUPPORTED, "segment compilation failed: " + err);
  return LQS_OK;
}

int lqs_plan_fused(int n_qubits, int dtype, const lqs_op* ops, int n_ops, const lqs_fuse_cfg* cfg,
                   int* n_segments, uint64_t* seg_qubit_mask, int cap, int* op_segment) {
  if (n_qubits < 1 || n_qubits > 36) return set_error(LQS_ERR_ARG, "n_qubits must be in [1, 36]");
  if (dtype != LQS_C64 && dtype != LQS_C128) return set_error(LQS_ERR_ARG, "bad dtype");
  if (!n_segments) return set_error(LQS_ERR_ARG, "n_segments is NULL");
  if (n_ops < 0 || (n_ops > 0 && !ops)) return set_error(LQS_ERR_ARG, "bad ops");
  // The plan depends only on gate classes and wires: lower with zero angles.
  int np_needed = 0;
  for (int i = 0; i < n_ops; ++i) np_needed = std::max(np_needed, ops[i].param_idx + 3);
  std::vector<double> zeros((size_t)std::max(np_needed, 1), 0.0);
  // Map lowered ops back to the caller's ops: lower one op at a time.
  std::vector<KOp> kops;
  std::vector<int> owner;
  for (int i = 0; i < n_ops; ++i) {
    const size_t before = kops.size();
    LQS_TRY(lower_ops(n_qubits, ops + i, 1, zeros.data(), (int)zeros.size(), false, kops));
    owner.insert(owner.end(), kops.size() - before, i);
  }
  PlanCfg pc;
  int arith = LQS_ARITH_AUTO;
  LQS_TRY(resolve_cfg(n_qubits, dtype, cfg, pc, &arith));
  std::vector<Segment> segs;
  LQS_TRY(plan_segments(n_qubits, kops, pc, segs));
  *n_segments = (int)segs.size();
  if (seg_qubit_mask)
    for (int s = 0; s < (int)segs.size() && s < cap; ++s) seg_qubit_mask[s] = segs[s].qmask;
  if (op_segment) {
    for (int i = 0; i < n_ops; ++i) op_segment[i] = -1;
    for (int s = 0; s < (int)segs.size(); ++s)
      for (int k : segs[s].ops) op_segment[owner[k]] = s;
  }
  return LQS_OK;
}

int lqs_norm2(lqs_sv* h, double* out_host) {
  LQS_TRY(check_sv(h));
  if (!out_host) return set_error(LQS_ERR_ARG, "out_host is NULL");
  return run_norm2(S_(h), current_arith(LQS_ARITH_AUTO), out_host);
}

int lqs_expval(lqs_sv* h, const lqs_pauli* terms, int n_terms, double* out_host, double* per_term_host) {
  LQS_TRY(check_sv(h));
  SV* sv = S_(h);
  if (!out_host) return set_error(LQS_ERR_ARG, "out_host is NULL");
  if (n_terms < 0 || (n_terms > 0 && !terms)) return set_error(LQS_ERR_ARG, "bad terms");
  const uint64_t lim = sv->N() - 1;
  for (int i = 0; i < n_terms; ++i)
    if ((terms[i].x_mask | terms[i].z_mask) & ~lim)
      return set_error(LQS_ERR_ARG, "term " + std::to_string(i) + " acts on a qubit >= n");
  PlanCfg pc;
  int arith = LQS_ARITH_AUTO;
  LQS_TRY(resolve_cfg(sv->n, sv->dtype, nullptr, pc, &arith));
  return run_expval(sv, terms, n_terms, pc, arith, out_host, per_term_host, nullptr);
}

int lqs_adjoint_grad(lqs_sv* h, const lqs_op* ops, int n_ops, const double* params, int n_params,
                     const lqs_pauli* terms, int n_terms, double* grads_host, double* energy_host) {
  LQS_TRY(check_sv(h));
  SV* sv = S_(h);
  if (n_params < 0 || (n_params > 0 && !grads_host)) return set_error(LQS_ERR_ARG, "grads_host is NULL");
  if (n_terms < 0 || (n_terms > 0 && !terms)) return set_error(LQS_ERR_ARG, "bad terms");
  const uint64_t lim = sv->N() - 1;
  for (int i = 0; i < n_terms; ++i)
    if ((terms[i].x_mask | terms[i].z_mask) & ~lim)
      return set_error(LQS_ERR_ARG, "term " + std::to_string(i) + " acts on a qubit >= n");
  std::vector<KOp> kops;
  LQS_TRY(lower_ops(sv->n, ops, n_ops, params, n_params, true, kops));
  PlanCfg pc;
  int arith = LQS_ARITH_AUTO;
  LQS_TRY(resolve_cfg(sv->n, sv->dtype, nullptr, pc, &arith));
  return run_adjoint(sv, kops, n_params, terms, n_terms, pc, arith, grads_host, energy_host);
}

// Host-side check of the double-float conversions (no device needed): for
// each input x, out[2i] = hi + lo widened exactly, out[2i+1] = the double the
// store path produces.  Exposed for CPU tests of the bit manipulation.
int lqs_debug_df_roundtrip(const double* in, double* out, int64_t count) {
  if (!in || !out || count < 0) return set_error(LQS_ERR_ARG, "bad arguments");
  for (int64_t i = 0; i < count; ++i) {
    const DF v = d2df(in[i]);
    out[2 * i] = (double)v.h + (double)v.l;
    out[2 * i + 1] = df2d(v);
  }
  return LQS_OK;
}

}  // extern "C"
