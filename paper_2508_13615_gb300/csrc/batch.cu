// Batches of small independent circuits.
//
// lqs_batch_run takes many small circuits (each with its own qubit count,
// gates, parameters and observable), runs forward + expectation + adjoint
// gradient for each, and returns energies and gradients.
#include <algorithm>
#include <vector>

#include "lqs_internal.cuh"

using namespace lqs;

extern "C" int lqs_batch_run(const lqs_batch_item* items, int n_items, int dtype, void* cuda_stream) {
  if (n_items < 0 || (n_items > 0 && !items)) return set_error(LQS_ERR_ARG, "bad batch");
  if (dtype != LQS_C64 && dtype != LQS_C128) return set_error(LQS_ERR_ARG, "bad dtype");
  for (int i = 0; i < n_items; ++i) {
    const lqs_batch_item& it = items[i];
    if (it.n_qubits < 1 || it.n_qubits > 30) return set_error(LQS_ERR_ARG, "batch item qubit count outside [1, 30]");
    if (!it.energy) return set_error(LQS_ERR_ARG, "batch item energy pointer is NULL");
  }
  for (int i = 0; i < n_items; ++i) {
    const lqs_batch_item& it = items[i];
    lqs_sv* sv = nullptr;
    LQS_TRY(lqs_sv_alloc(it.n_qubits, dtype, nullptr, cuda_stream, &sv));
    int rc = lqs_sv_set_basis(sv, 0);
    if (rc == LQS_OK) rc = lqs_apply_fused(sv, it.ops, it.n_ops, it.params, it.n_params, nullptr);
    if (rc == LQS_OK) {
      if (it.grads) {
        rc = lqs_adjoint_grad(sv, it.ops, it.n_ops, it.params, it.n_params, it.terms, it.n_terms, it.grads,
                              it.energy);
      } else {
        rc = lqs_expval(sv, it.terms, it.n_terms, it.energy, nullptr);
      }
    }
    lqs_sv_free(sv);
    if (rc != LQS_OK) return rc;
  }
  return LQS_OK;
}
