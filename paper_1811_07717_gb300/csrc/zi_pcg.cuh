// Solver entry points shared between the libzi translation units.
#pragma once

#include "zi_internal.cuh"

namespace zi {

int check_opts(const zi_solver_opts* o);
int transfer_impl(zi_system* S, const zi_solver_opts* o, double* Tout, int32_t* iters, double* relres,
                  cudaStream_t user);
void choose_layout(int ncol, int* ld, int* cptv64, int* cptv32);
void solver_scratch_free(zi_system* S);
void solver_invalidate(zi_system* S);  // the system's values changed

}  // namespace zi
