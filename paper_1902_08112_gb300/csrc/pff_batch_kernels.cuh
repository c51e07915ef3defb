// Launchers of the batched kernels (pff_batch_kernels.cu).  'blocks' is the grid width per instance.
#pragma once

#include "pff_batch.cuh"

namespace pff {

constexpr int kBPartials = 64;   // partial sums per instance in batched reductions

template <typename T>
cudaError_t bl_init_masked(const BLevel* L, int n, int blocks, int sx, int sy, int phi_bits, T v, cudaStream_t s);
template <typename T>
cudaError_t bl_cheb(const BLevel* L, int n, int blocks, int sr, int st, int sd, int sx, const double* coef, int first,
                    cudaStream_t s, int stn = -1);
template <typename T>
cudaError_t bl_sub(const BLevel* L, int n, int blocks, int sa, int sb, int sc, cudaStream_t s);
template <typename T>
cudaError_t bl_copy(const BLevel* L, int n, int blocks, int ss, int sd, int block, cudaStream_t s);
template <typename Ti, typename To>
cudaError_t bl_convert(const BLevel* L, int n, int blocks, int ss, int sd, int mode, cudaStream_t s);
cudaError_t bl_axpby64(const BLevel* L, int n, int blocks, const double* a, int sx, double b, int sy, int invert_a,
                       cudaStream_t s);
template <typename T>
cudaError_t bl_restrict(const BLevel* Lc, const BLevel* Lf, int n, int blocks, int sf, int sc, cudaStream_t s);
template <typename T>
cudaError_t bl_prolongate_add(const BLevel* Lc, const BLevel* Lf, int n, int blocks, int sc, int sf, cudaStream_t s);
template <typename T>
cudaError_t bl_dots2(const BLevel* L, int n, int sa, int sb, double* part, double* out, cudaStream_t s);
// k < 0: the number of basis vectors is (*kcol) + 1 (device column counter)
cudaError_t bl_multidot(const BLevel* L, int n, int k, int sw, double* part, int kmax, double* h, int ldh,
                        cudaStream_t s, const int* kcol = nullptr);
cudaError_t bl_multi_axpy(const BLevel* L, int n, int blocks, int k, const double* h, int ldh, int sw, cudaStream_t s,
                          const int* kcol = nullptr);
cudaError_t bl_norm(const BLevel* L, int n, int sw, double* part, double* out, cudaStream_t s);
// kk (nullable): per-instance number of columns
cudaError_t bl_gemv_add(const BLevel* L, int n, int blocks, int k, const double* y, int ldy, int sx, cudaStream_t s,
                        const int* kk = nullptr);
template <typename T>
cudaError_t bl_cg_r(const BLevel* L, int n, int blocks, int sr, int sq, int sz, const double* alpha2, cudaStream_t s);
template <typename T>
cudaError_t bl_cg_p(const BLevel* L, int n, int blocks, int sp, int sz, const double* beta2, cudaStream_t s);
template <typename T>
cudaError_t bl_start_vector(const BLevel* L, int n, int blocks, int sv, const uint64_t* seeds, int level,
                            cudaStream_t s);

}  // namespace pff
