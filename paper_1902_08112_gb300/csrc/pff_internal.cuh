// Internal declarations of the pff CUDA library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/pff.h"

namespace pff {

constexpr int MASK_U_ALL = PFF_MASK_UX | PFF_MASK_UY | PFF_MASK_UZ;
constexpr int PHI_BITS_ALL = PFF_MASK_ACTIVE | PFF_MASK_PHI_DIR;

// Material/physics constants in the form the kernels use.
struct Phys {
    double mu, lam;      // Lame coefficients
    double Gc, kappa, eps, p;
    double f;            // factor on the phi-equation elastic term
    int split;           // 0: no split; 1: Miehe split of E_s (Sec. 2.1)
};

// 1D Lagrange shape functions on [0,1] at the (deg+1)-point Gauss rule: value N1[a][q],
// derivative D1[a][q] (reference), weights w1[q].
struct Tables {
    double N1[3][3];
    double D1[3][3];
    double w1[3];
};

// Geometry of one uniform level.
struct Geom {
    int dim, deg;
    int nc[3];           // cells per axis (1 beyond dim)
    int nn[3];           // nodes per axis (1 beyond dim)
    int64_t n_nodes, n_cells;
    double h[3];         // cell edge lengths (1 beyond dim)
    const double* es;    // per-cell factor on E (n_cells, device), nullptr = uniform modulus
    const uint8_t* cm;   // per-cell domain mask (n_cells, device, nonzero = in), nullptr = box
};

__host__ __device__ inline bool cell_in(const Geom& g, int64_t cell) { return !g.cm || g.cm[cell] != 0; }

__host__ __device__ inline int64_t n_dofs(const Geom& g) { return (int64_t)(g.dim + 1) * g.n_nodes; }

// component of a DoF index in a component-blocked vector of up to 4 blocks of nn entries
// (comparisons instead of a 64-bit division)
__device__ __forceinline__ int dof_comp(int64_t i, int64_t nn) {
    return (int)(i >= nn) + (int)(i >= 2 * nn) + (int)(i >= 3 * nn);
}

// Device arrays of one level.
struct Level {
    Geom g;
    uint8_t* mask = nullptr;     // node masks (Dirichlet u bits, active bit)
    double* U64 = nullptr;       // restricted state (n_dofs)
    double* pt64 = nullptr;      // restricted extrapolation (n_nodes)
    float* U32 = nullptr;
    float* pt32 = nullptr;
    double* dinv64 = nullptr;    // inverse operator diagonal (1 on eliminated rows)
    float* dinv32 = nullptr;
    void* w[2][6] = {{nullptr}}; // V-cycle work vectors, [0]=FP32, [1]=FP64
    float* qpd32 = nullptr;      // Q1: Gauss-point linearisation coefficients, FP32
    float2* qpd64 = nullptr;     // Q1: the same as df64 pairs (hi, lo)
    double* es_buf = nullptr;    // storage of g.es once a varying modulus is set
    uint8_t* cm_buf = nullptr;   // storage of g.cm (domains cut from the box)
    float* qps32 = nullptr;      // Q1 with the Miehe split: Gauss-point tangent data, FP32
    float2* qps64 = nullptr;     // the same as df64 pairs
    double lam_min[2] = {1, 1};  // eigenvalue estimates of D^-1 G_bb, blocks u / phi
    double lam_max[2] = {1, 1};
};

// Operator selector for the cell kernel.
enum CellOp : int { OP_APPLY = 0, OP_APPLY_BLOCKDIAG = 1, OP_RESIDUAL = 2, OP_DIAGONAL = 3 };

template <typename T>
struct CellArgs {
    Geom g;
    Phys ph;
    Tables tb;
    const T* x;          // input vector (apply) or nullptr
    T* y;                // output
    const T* U;          // state [u | phi]
    const T* pt;         // extrapolation phi~
    const uint8_t* mask;
    int phi_bits;        // mask bits that eliminate phi DoFs (apply); 0 disables elimination
    int u_bits;          // mask bits that eliminate u DoFs
};

// ---------------------------------------------------------------- launchers (pff_ops.cu)
template <typename T>
cudaError_t launch_cell_op(int op, const CellArgs<T>& a, cudaStream_t s);

// y_i = eliminated(i) ? x_i : 0     (x may be null: constrained entries get 'diag_one')
template <typename T>
cudaError_t launch_init_masked(const Geom& g, const uint8_t* mask, int u_bits, int phi_bits,
                               const T* x, T* y, T eliminated_value, cudaStream_t s);
// the same on the nodes [node0, node1) only (all components), FP64
cudaError_t launch_init_masked_nodes(const Geom& g, const uint8_t* mask, int u_bits, int phi_bits, const double* x,
                                     double* y, int64_t node0, int64_t node1, cudaStream_t s);

// ---------------------------------------------------------------- vector kernels (pff_vec.cu)
cudaError_t launch_restrict_state(const Geom& gc, const Geom& gf, const double* Uf, const double* ptf,
                                  const uint8_t* maskf, double* Uc, double* ptc, uint8_t* maskc,
                                  bool phi_max_q1, cudaStream_t s);
cudaError_t launch_cast_f64_f32(const double* a, float* b, int64_t n, cudaStream_t s);
cudaError_t launch_cast_f32_f64(const float* a, double* b, int64_t n, cudaStream_t s);
cudaError_t launch_face_mask(const Geom& g, unsigned faces, const uint8_t* extra, uint8_t* mask,
                             cudaStream_t s);
cudaError_t launch_set_active(const Geom& g, const uint8_t* active, uint8_t* mask, cudaStream_t s);
cudaError_t launch_get_active(const Geom& g, const uint8_t* mask, uint8_t* active, cudaStream_t s);
template <typename T>
cudaError_t launch_restrict(const Geom& gc, const Geom& gf, const T* rf, T* rc, const uint8_t* maskc,
                            cudaStream_t s);
template <typename T>
cudaError_t launch_prolongate_add(const Geom& gc, const Geom& gf, const T* ec, T* xf,
                                  const uint8_t* maskf, cudaStream_t s);
template <typename T>
cudaError_t launch_invert_diag(T* d, int64_t n, cudaStream_t s);

// Chebyshev smoother update: r -= t; d = c1[b] d + c2[b] dinv r; x += d  (b = block of i)
template <typename T>
cudaError_t launch_cheb_update(const Geom& g, T* r, const T* t, T* d, const T* dinv, T* x,
                               double c1u, double c1p, double c2u, double c2p, int first,
                               cudaStream_t s, const uint8_t* mask = nullptr, T* tn = nullptr);
// elementwise helpers
template <typename T>
cudaError_t launch_axpby(int64_t n, double a, const T* x, double b, T* y, cudaStream_t s);  // y = a x + b y
template <typename T>
cudaError_t launch_sub(int64_t n, const T* a, const T* b, T* c, cudaStream_t s);            // c = a - b
template <typename T>
cudaError_t launch_copy_block(const Geom& g, int block, const T* src, T* dst, cudaStream_t s); // dst = src on block, 0 elsewhere
template <typename T>
cudaError_t launch_mask_copy(const Geom& g, const uint8_t* mask, const T* src, T* dst, int free_only,
                             cudaStream_t s);

// Deterministic blocked dot products: out[k] = sum over block k (k=0 u, 1 phi) of a_i b_i w_i
// (w may be null).  Results in double on the device (out[0..1]).  'scratch' holds the
// per-CTA partial sums (2 * dot_partials() doubles).
int dot_partials();
template <typename T>
cudaError_t launch_block_dots(const Geom& g, const T* a, const T* b, const T* w, double* scratch,
                              double* out, cudaStream_t s);

// start vector of the CG eigenvalue estimate: SplitMix64 counter-based values in [-1,1) on
// free DoFs, 0 on eliminated ones.
template <typename T>
cudaError_t launch_start_vector(const Geom& g, const uint8_t* mask, uint64_t seed, int level, T* v,
                                cudaStream_t s);

// Jacobi-PCG step pieces for the blocked eigenvalue estimate (device scalars)
template <typename T>
cudaError_t launch_cg_update_r(const Geom& g, T* r, const T* q, const T* dinv, T* z,
                               const double* alpha2, cudaStream_t s);
template <typename T>
cudaError_t launch_cg_update_p(const Geom& g, T* p, const T* z, const double* beta2,
                               cudaStream_t s);

// lumped Gauss-Lobatto mass and active set (Algorithm 1 step 3)
cudaError_t launch_lumped_mass(const Geom& g, double* M, cudaStream_t s);
cudaError_t launch_active_set(const Geom& g, const double* R, const double* M, const double* U,
                              const double* phi_old, double c, double threshold, int tie_scale, uint8_t* mask,
                              int* counts, cudaStream_t s);
cudaError_t launch_newton_rhs(const Geom& g, const double* R, const double* t, const double* U,
                              const double* phi_old, const uint8_t* mask, double* Rt, cudaStream_t s);
cudaError_t launch_coarsen_cells(const Geom& gc, const Geom& gf, const double* sf, double* sc, cudaStream_t s);
cudaError_t launch_count_nonpositive(int64_t n, const double* v, int* bad, cudaStream_t s);
cudaError_t launch_coarsen_cell_mask(const Geom& gc, const Geom& gf, const uint8_t* mf, uint8_t* mc, cudaStream_t s);
cudaError_t launch_outside_nodes(const Geom& g, uint8_t* mask, cudaStream_t s);
cudaError_t launch_face_sum(const Geom& g, int axis, int side, int comp, const double* R, double* out,
                            cudaStream_t s);
cudaError_t launch_extrapolate(int64_t n, const double* phi_nm1, const double* phi_nm2, double* out,
                               cudaStream_t s);
// U = u_dirichlet on the Dirichlet displacement DoFs of mask (prescribed boundary values)
cudaError_t launch_lift_dirichlet(const Geom& g, const uint8_t* mask, const double* ud, double* U, cudaStream_t s);
cudaError_t launch_active_delta(const Geom& g, const double* U, const double* phi_old,
                                const uint8_t* mask, double* delta, cudaStream_t s);

// FGMRES kernels
cudaError_t launch_multidot(int64_t n, const double* V, int64_t ld, int k, const double* w,
                            double* scratch, double* h, cudaStream_t s);
cudaError_t launch_multi_axpy(int64_t n, const double* V, int64_t ld, int k, const double* h,
                              double* w, cudaStream_t s);  // w -= V h
cudaError_t launch_norm2(int64_t n, const double* w, double* scratch, double* out, cudaStream_t s);
cudaError_t launch_scale_copy(int64_t n, const double* w, const double* nrm, double* v,
                              cudaStream_t s);  // v = w / *nrm
cudaError_t launch_gemv_add(int64_t n, const double* Z, int64_t ld, int k, const double* y,
                            double* x, cudaStream_t s);   // x += Z y

}  // namespace pff

// The opaque hierarchy of the C ABI.
constexpr int kLevelScal = 256, kLevelScratch = 1024;

// Smallest 3D level that the per-cell applies with shared-memory derivatives serve by default: below
// about two waves of their CTAs the lane and per-cell-gather kernels finish sooner.
constexpr int64_t kCellMinCells = 100000;

struct pff_hierarchy {
    pff_mesh mesh;
    pff_params prm;
    cudaStream_t stream = nullptr;
    int L = 0;
    pff::Phys ph;
    pff::Tables tb;
    std::vector<pff::Level> lv;
    // fine-level data
    uint8_t* dir_mask = nullptr;     // Dirichlet-only mask of the finest level
    double* phi_old = nullptr;
    double* lumped = nullptr;
    double* R = nullptr;             // residual (n_dofs)
    double* tmp64[4] = {nullptr, nullptr, nullptr, nullptr};  // fine FP64 temporaries
    uint8_t* prev_active = nullptr;
    double* udir = nullptr;          // prescribed displacement values on Dirichlet DoFs (dim * n_nodes), or none
    bool has_udir = false;
    int* d_counts = nullptr;         // device counters
    double* d_scal = nullptr;        // device scalars (dots, CG coefficients)
    // setup runs the levels concurrently: one stream per level, a private region of CG scalars
    // (kLevelScal doubles) and of dot partials (kLevelScratch doubles) per level
    double* d_scal_lv = nullptr;
    double* d_scratch_lv = nullptr;
    cudaStream_t lv_stream[16] = {};
    cudaEvent_t lv_event[17] = {};
    double* d_scratch = nullptr;     // per-CTA partial sums
    // Krylov workspace
    int kr_m = 0;
    double* kr_V = nullptr;
    double* kr_Z = nullptr;
    double* kr_h = nullptr;          // device column of H (2 * (m + 1))
    bool has_state = false;
    bool fast_q1 = true;             // Q1 levels use the linearisation-data kernels of pff_q1.cu
    int q1_style = 52;               // bit 0/1: lanes for FP64/FP32; bit 2/3: lanes with global atomics for FP64/FP32;
                                     // bit 4/6 (FP64), 5/7 (FP32): per cell with shared-memory derivatives and
                                     // global atomics on 3D levels of at least kCellMinCells cells / on every
                                     // 3D level
    bool use_graphs = true;          // replay the V-cycle body from a captured CUDA graph
    cudaGraphExec_t vgraph = nullptr;   // captured V-cycle body (valid until the next setup)
    long long vgraph_nodes = 0;
    bool active_known = false;       // an active set has been computed or set
    bool derived_dirty = false;      // fine U changed; coarse levels, FP32 copies, Gauss-point data not yet
    bool stale = true;               // preconditioner data out of date
    std::vector<void*> allocs;       // every device allocation, freed on destroy
    // kernel timing: event pairs per class, recorded while prof_on
    bool prof_on = false;
    std::vector<cudaEvent_t> ev_pool;
    // host-buffer apply: device copies of x and y, copy streams, one event per slab and stage
    double* hx = nullptr;
    double* hy = nullptr;
    cudaStream_t cs_in = nullptr, cs_out = nullptr;
    std::vector<cudaEvent_t> slab_ev;
    size_t ev_used = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof[PFF_PROF_NCLASS];
    std::string err;
};

namespace pff {
// Process-wide count of kernel launches issued by this library (tracing; read through
// pff_launch_count).  Each launcher passes its cudaGetLastError() result through here.
cudaError_t count_launch(cudaError_t e);
long long launch_count();
void add_launches(long long n);   // graph replays add their node count; a capture takes its own back
}  // namespace pff
