// Descriptors of batched launches: many independent instances (hierarchies) processed by one
// launch per level and operation.  A BLevel describes one instance at one level; batched kernels
// find their instance from the launch index and their vectors through selectors.
#pragma once

#include "pff_internal.cuh"
#include "pff_q1.cuh"

namespace pff {

// vector selectors: (id | column << 8); the column picks a Krylov vector V_j / Z_j
enum : int {
    BV_W32 = 0,    // + k, k = 0..5: level FP32 work vectors
    BV_W64 = 6,    // + k, k = 0..5: level FP64 work vectors
    BV_T64 = 12,   // + k, k = 0..3: FP64 temporaries of the finest level
    BV_KV = 16,    // FGMRES basis V (finest level)
    BV_KZ = 17,    // FGMRES preconditioned basis Z (finest level)
    BV_R = 18,     // residual -A(U) (finest level)
    BV_U = 19,     // state U (FP64, this level)
    BV_PHIOLD = 20,
    BV_N = 21
};

struct BLevel {
    Geom g;
    int valid;                  // the instance has this level
    const int* on;              // device flag of the instance, 0 = skipped by every batched kernel (the
                                // batched FGMRES retires converged instances through it); nullptr = on
    const int* col;             // device Krylov column counter of the batch (selector columns kColJ, kColJ1)
    const uint8_t* mask;
    const float* qpd32;
    const float2* qpd64;
    float* dinv32;
    double* dinv64;
    void* vec[BV_N];
    Q1Consts k;                 // apply constants of this instance and level
};

__host__ __device__ inline int bsel(int id, int col = 0) { return id | (col << 8); }

// selector columns read from the batch's device counter: column *col and *col + 1, so that one
// captured Arnoldi step serves every column j
constexpr int kColJ = 0xFE, kColJ1 = 0xFF;

__device__ __forceinline__ bool bon(const BLevel& d) { return d.valid && (!d.on || *d.on != 0); }

template <typename T>
__device__ __forceinline__ T* bvec(const BLevel& L, int sel) {
    char* p = reinterpret_cast<char*>(L.vec[sel & 0xFF]);
    int col = sel >> 8;
    if (col >= kColJ) col = *L.col + (col - kColJ);
    if (col) p += (size_t)col * (size_t)n_dofs(L.g) * sizeof(T);
    return reinterpret_cast<T*>(p);
}

// batched Q1 applies: y(sy) = G~ x(sx) on every valid instance of a level (eliminated rows of y must
// be preset); tile_start: prefix sums of the instances' tile counts for this kernel style
// cell = true (3D): the per-cell kernel with shared-memory derivatives (tiles of the FP32 per-cell
// style, q1_cell_tiles_match_f32())
// Persistent launches: at most max_ctas CTAs (0: one per tile) loop over the flattened tiles of all
// instances; tile_start[n] holds the total in device memory.
cudaError_t launch_q1_apply_batched(int dim, bool fp64, bool blockdiag, bool lanes, const BLevel* L, int n,
                                    const int* tile_start, int total_tiles, int sx, int sy, int phi_bits,
                                    cudaStream_t s, bool cell = false, int max_ctas = 0);
bool q1_cell_tiles_match_f32();
// set the kernels' shared-memory attributes (once per device, before any stream capture)
cudaError_t q1_batched_prepare();
// resident CTAs per SM of a batched apply kernel (the largest useful persistent grid is SMs times this)
int q1_batched_ctas_per_sm(int dim, bool fp64, bool cell);
// tile count of one instance for a kernel style (host)
int q1_tiles(const Geom& g, bool fp64, bool lanes);

}  // namespace pff
