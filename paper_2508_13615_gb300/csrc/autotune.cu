// Autotuner for the fused path: picks the tile shape and segment length of
// lqs_apply_fused for a circuit structure by timing candidates on the GPU.
// The paper has no tuner; its kernels are fixed per gate class (Sec. 2).
//
// The register-tile kernels fix the tile width k (the registers and thread
// bits of a thread block); what varies is the number b of low contiguous
// qubits every tile keeps (longer bulk-copy rows and coalesced stores against
// fewer free tile qubits for the planner) and a cap on gates per segment
// (shorter straight-line kernels against more passes).  Each candidate is
// applied twice untimed (compiled kernels are built then) and timed over
// `repeats` applications with CUDA events on the state's stream; the fastest
// is remembered per (qubits, dtype, circuit structure) and used by
// lqs_apply_fused when it is called without a configuration.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "lqs_internal.cuh"

namespace lqs {

static std::mutex g_tune_mu;
static std::map<std::string, lqs_fuse_cfg> g_tuned;

// Circuit structure: gate kinds and wires (angles and matrices only change
// coefficients, not the plan).
static std::string tune_key(int n, int dtype, const lqs_op* ops, int n_ops) {
  std::string k;
  k.reserve(16 + (size_t)n_ops * 20);
  const int hdr[3] = {n, dtype, n_ops};
  k.append(reinterpret_cast<const char*>(hdr), sizeof hdr);
  for (int i = 0; i < n_ops; ++i) {
    const int32_t rec[5] = {ops[i].gate, ops[i].wires[0], ops[i].wires[1], ops[i].wires[2], ops[i].wires[3]};
    k.append(reinterpret_cast<const char*>(rec), sizeof rec);
  }
  return k;
}

bool tuned_cfg(int n, int dtype, const lqs_op* ops, int n_ops, lqs_fuse_cfg* out) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tuned.find(tune_key(n, dtype, ops, n_ops));
  if (it == g_tuned.end()) return false;
  *out = it->second;
  return true;
}

}  // namespace lqs

using namespace lqs;

extern "C" int lqs_autotune_fused(lqs_sv* h, const lqs_op* ops, int n_ops, const double* params, int n_params,
                                  int repeats, lqs_fuse_cfg* best) {
  if (!h) return set_error(LQS_ERR_ARG, "sv is NULL");
  if (!best) return set_error(LQS_ERR_ARG, "best is NULL");
  if (n_ops < 0 || (n_ops > 0 && !ops)) return set_error(LQS_ERR_ARG, "bad ops");
  if (repeats < 1 || repeats > 100) return set_error(LQS_ERR_ARG, "repeats must be in [1, 100]");
  void* dptr = nullptr;
  int n = 0, dtype = 0;
  LQS_TRY(lqs_sv_info(h, &dptr, &n, &dtype));
  SV* sv = reinterpret_cast<SV*>(h);
  *best = lqs_fuse_cfg{0, 0, 0, 0};
  const int k = reg_tile_qubits(dtype);
  if (n <= k || n_ops == 0) return LQS_OK;  // one tile (or nothing): no choice to make
  std::vector<lqs_fuse_cfg> cand;
  const int b0 = dtype == LQS_C64 ? 5 : 4;
  for (int b : {b0 - 1, b0, b0 + 1})
    for (int mo : {0, 48}) cand.push_back(lqs_fuse_cfg{0, b, 0, mo});
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  LQS_CUDA_TRY(cudaEventCreate(&e0));
  LQS_CUDA_TRY(cudaEventCreate(&e1));
  float best_ms = 0.f;
  int rc = LQS_OK;
  for (const lqs_fuse_cfg& c : cand) {
    for (int w = 0; w < 2 && rc == LQS_OK; ++w) rc = lqs_apply_fused(h, ops, n_ops, params, n_params, &c);
    if (rc != LQS_OK) break;
    cudaEventRecord(e0, sv->stream);
    for (int i = 0; i < repeats && rc == LQS_OK; ++i) rc = lqs_apply_fused(h, ops, n_ops, params, n_params, &c);
    cudaEventRecord(e1, sv->stream);
    if (rc != LQS_OK) break;
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      rc = cuda_error(cudaGetLastError(), "autotune timing");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (best_ms == 0.f || ms < best_ms) {
      best_ms = ms;
      *best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != LQS_OK) return rc;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned[tune_key(n, dtype, ops, n_ops)] = *best;
  return LQS_OK;
}
