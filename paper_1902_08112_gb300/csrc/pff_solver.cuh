// Solver-level entry points shared by pff_solver.cu and pff_api.cu.
#pragma once

#include <string>

#include "pff_internal.cuh"

namespace pff {

template <typename T>
// preset = false: the caller already wrote y = x on eliminated rows and 0 elsewhere
cudaError_t apply_level(pff_hierarchy* h, int l, int op, const T* x, T* y, int phi_bits, bool preset = true);
template <typename T>
cudaError_t diagonal_level(pff_hierarchy* h, int l, T* d);
cudaError_t residual_fine(pff_hierarchy* h, double* R);
cudaError_t propagate_state(pff_hierarchy* h, bool values = true);   // values=false: masks only
// propagate_state once if the fine state changed since the last propagation
cudaError_t refresh_state(pff_hierarchy* h);
cudaError_t setup(pff_hierarchy* h);
void drop_graph(pff_hierarchy* h);
template <typename T>
cudaError_t smooth(pff_hierarchy* h, int l, const T* b, T* x, int zero_guess);
cudaError_t coarse_solve(pff_hierarchy* h, const double* b, double* x);
cudaError_t vcycle(pff_hierarchy* h, const double* r, double* z);
pff_status fgmres(pff_hierarchy* h, const double* b, double* x, double rtol, int m, int maxit,
                  pff_solve_info* info, std::string& err);

}  // namespace pff
