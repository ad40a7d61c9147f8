// Segment compiler interface (internal): see jit.cu.
#pragma once
#include <string>
#include <vector>

#include "lqs_internal.cuh"
#include "tile.cuh"

namespace lqs {

int jit_mode();
// Whether compiled segments may run for an n-qubit state under the current mode.
bool jit_enabled_for(int n);
// CUDA C++ source of a register-tile program (LQS_ERR_UNSUPPORTED for a
// program the generator does not take; the interpreter runs those).
template <class A>
int jit_source(const TileProg<A>& P, int r, std::string& src, std::string& name, std::string& why,
               bool adjoint = false);
// Counts one use of the program's structure and queues it for compilation
// when the mode asks for it (or `force`).
template <class A>
int jit_note(const TileProg<A>& P, int r, int n, bool force, std::vector<void*>& todo);
// Compiles queued structures in parallel.
int jit_compile(const std::vector<void*>& todo);
// After jit_compile: *ok = structures in `todo` that compiled; LQS_ERR_UNSUPPORTED
// (with the first failure's log in *err) when any did not.
int jit_states(const std::vector<void*>& todo, int* ok, std::string* err);
// Launches the compiled kernel of the program if there is one (*launched
// tells); otherwise does nothing and the caller runs the interpreter.
template <class A>
int jit_launch(const TileProg<A>& P, int r, SV* sv, double bytes, double flops, const char* prof_name,
               bool* launched);

// Compiled adjoint: the cache entry of a reverse-sweep program (queued for
// compilation by the caller through jit_compile), its shared-memory size,
// and its launch over psi and lambda writing per-block partial sums
// partial[slot * grid + block].
template <class A>
int jit_adjoint_entry(const TileProg<A>& P, int r, void** entry, std::string* why);
size_t jit_adjoint_smem(int k, int r, size_t amp_bytes);
template <class A>
int jit_adjoint_occupancy(void* entry, const TileProg<A>& P, int r, SV* sv, int* per_sm);
template <class A>
int jit_launch_adjoint(void* entry, const TileProg<A>& P, int r, SV* sv, void* lam, double* partial, unsigned grid,
                       double bytes, double flops, const char* prof_name);

}  // namespace lqs
