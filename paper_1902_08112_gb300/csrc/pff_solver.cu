// Host orchestration of the solver stack (all arithmetic runs in the kernels of pff_ops.cu
// and pff_vec.cu; the host only sequences launches and keeps O(restart^2) Krylov scalars).
//
//  setup      level diagonals (Sec. 4.1 remark) and eigenvalue bounds of D^-1 G_bb from
//             10 Jacobi-preconditioned CG steps per block (Sec. 3.2.1)
//  smooth     block-diagonal Chebyshev-Jacobi S_full (Sec. 3.2.1, 3.3)
//  coarse     Chebyshev as solver on [0.9 lmin, 1.2 lmax] (Sec. 3.2.2), block forward
//             substitution
//  vcycle     P_full^-1 = MG(G~) (Sec. 3.3)
//  fgmres     right-preconditioned flexible GMRES, CGS2 Arnoldi, Givens (outer solver, Sec. 5)
//  newton     one primal-dual active-set step (Algorithm 1)
#include <math.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "pff_q1.cuh"
#include "pff_solver.cuh"

namespace pff {

template <typename T> static T* stU(Level& L);
template <> double* stU<double>(Level& L) { return L.U64; }
template <> float* stU<float>(Level& L) { return L.U32; }
template <typename T> static T* stPt(Level& L);
template <> double* stPt<double>(Level& L) { return L.pt64; }
template <> float* stPt<float>(Level& L) { return L.pt32; }
template <typename T> static T* dinv(Level& L);
template <> double* dinv<double>(Level& L) { return L.dinv64; }
template <> float* dinv<float>(Level& L) { return L.dinv32; }
template <typename T> static constexpr int prec_index() { return sizeof(T) == 8 ? 1 : 0; }
template <typename T> static T* work(Level& L, int k) { return reinterpret_cast<T*>(L.w[prec_index<T>()][k]); }

#define CK(expr)                                  \
    do {                                          \
        cudaError_t e_ = (expr);                  \
        if (e_ != cudaSuccess) return e_;         \
    } while (0)

static cudaEvent_t next_event(pff_hierarchy* h) {
    if (h->ev_used == h->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        h->ev_pool.push_back(e);
    }
    return h->ev_pool[h->ev_used++];
}

template <typename T>
cudaError_t apply_level(pff_hierarchy* h, int l, int op, const T* x, T* y, int phi_bits, bool preset) {
    CK(refresh_state(h));
    Level& L = h->lv[l];
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (h->prof_on) {
        e0 = next_event(h);
        e1 = next_event(h);
        if (e0 && e1) CK(cudaEventRecord(e0, h->stream));
    }
    if (preset) CK(launch_init_masked<T>(L.g, L.mask, MASK_U_ALL, phi_bits, x, y, T(0), h->stream));
    if (h->fast_q1 && L.g.deg == 1 && h->ph.split && L.qps64 && (op == OP_APPLY || op == OP_APPLY_BLOCKDIAG)) {
        const bool bd = op == OP_APPLY_BLOCKDIAG;
        if constexpr (sizeof(T) == 8)
            CK(launch_q1_apply_split64(L.g, h->ph, L.qps64, (const double*)x, (double*)y, L.mask, phi_bits, bd,
                                       h->stream));
        else
            CK(launch_q1_apply_split32(L.g, h->ph, L.qps32, (const float*)x, (float*)y, L.mask, phi_bits, bd,
                                       h->stream));
    } else if (h->fast_q1 && L.g.deg == 1 && !h->ph.split && (op == OP_APPLY || op == OP_APPLY_BLOCKDIAG)) {
        const bool bd = op == OP_APPLY_BLOCKDIAG;
        if constexpr (sizeof(T) == 8)
            CK(launch_q1_apply64(L.g, h->ph, L.qpd64, (const double*)x, (double*)y, L.mask, phi_bits, bd,
                                 (h->q1_style & 1) != 0, h->stream, (h->q1_style & 4) != 0,
                                 (h->q1_style & 64) != 0 ||
                                     ((h->q1_style & 16) != 0 && L.g.n_cells >= kCellMinCells)));
        else
            CK(launch_q1_apply32(L.g, h->ph, L.qpd32, (const float*)x, (float*)y, L.mask, phi_bits, bd,
                                 (h->q1_style & 2) != 0, h->stream, (h->q1_style & 8) != 0,
                                 (h->q1_style & 128) != 0 ||
                                     ((h->q1_style & 32) != 0 && L.g.n_cells >= kCellMinCells)));
    } else if (h->fast_q1 && L.g.deg == 2 && L.g.dim == 3 && !h->ph.split && L.qpd64 &&
               (op == OP_APPLY || op == OP_APPLY_BLOCKDIAG)) {
        const bool bd = op == OP_APPLY_BLOCKDIAG;
        if constexpr (sizeof(T) == 8)
            CK(launch_q2_apply64(L.g, h->ph, L.qpd64, (const double*)x, (double*)y, L.mask, phi_bits, bd, h->stream));
        else
            CK(launch_q2_apply32(L.g, h->ph, L.qpd32, (const float*)x, (float*)y, L.mask, phi_bits, bd, h->stream));
    } else {
        CellArgs<T> a;
        a.g = L.g;
        a.ph = h->ph;
        a.tb = h->tb;
        a.x = x;
        a.y = y;
        a.U = stU<T>(L);
        a.pt = stPt<T>(L);
        a.mask = L.mask;
        a.phi_bits = phi_bits;
        a.u_bits = MASK_U_ALL;
        CK(launch_cell_op<T>(op, a, h->stream));
    }
    if (e0 && e1) {
        CK(cudaEventRecord(e1, h->stream));
        const int cls = sizeof(T) == 4 ? PFF_PROF_APPLY32 : (l == h->L - 1 ? PFF_PROF_APPLY64_FINE : PFF_PROF_APPLY64_COARSE);
        h->prof[cls].push_back({e0, e1});
    }
    return cudaSuccess;
}
template cudaError_t apply_level<double>(pff_hierarchy*, int, int, const double*, double*, int, bool);
template cudaError_t apply_level<float>(pff_hierarchy*, int, int, const float*, float*, int, bool);

template <typename T>
cudaError_t diagonal_level(pff_hierarchy* h, int l, T* d) {
    CK(refresh_state(h));
    Level& L = h->lv[l];
    CK(launch_init_masked<T>(L.g, L.mask, MASK_U_ALL, PHI_BITS_ALL, (const T*)nullptr, d, T(1), h->stream));
    if constexpr (sizeof(T) == 8) {
        if (h->fast_q1 && L.g.deg == 1 && !h->ph.split)
            return launch_q1_diagonal(L.g, h->ph, L.qpd64, L.mask, (double*)d, h->stream);
    }
    CellArgs<T> a;
    a.g = L.g;
    a.ph = h->ph;
    a.tb = h->tb;
    a.x = nullptr;
    a.y = d;
    a.U = stU<T>(L);
    a.pt = stPt<T>(L);
    a.mask = L.mask;
    a.phi_bits = PHI_BITS_ALL;
    a.u_bits = MASK_U_ALL;
    return launch_cell_op<T>(OP_DIAGONAL, a, h->stream);
}
template cudaError_t diagonal_level<double>(pff_hierarchy*, int, double*);
template cudaError_t diagonal_level<float>(pff_hierarchy*, int, float*);

cudaError_t residual_fine(pff_hierarchy* h, double* R) {
    Level& L = h->lv[h->L - 1];
    CK(cudaMemsetAsync(R, 0, sizeof(double) * n_dofs(L.g), h->stream));
    if (h->fast_q1 && L.g.deg == 1 && !h->ph.split) return launch_q1_residual(L.g, h->ph, L.U64, L.pt64, R, h->stream);
    CellArgs<double> a;
    a.g = L.g;
    a.ph = h->ph;
    a.tb = h->tb;
    a.x = nullptr;
    a.y = R;
    a.U = L.U64;
    a.pt = L.pt64;
    a.mask = L.mask;
    a.phi_bits = 0;
    a.u_bits = 0;
    return launch_cell_op<double>(OP_RESIDUAL, a, h->stream);
}

// Fine state -> all coarser levels (coincident nodes) and FP32 copies.
cudaError_t refresh_state(pff_hierarchy* h) {
    return h->derived_dirty ? propagate_state(h, true) : cudaSuccess;
}

cudaError_t propagate_state(pff_hierarchy* h, bool values) {
    if (values) h->derived_dirty = false;
    for (int l = h->L - 2; l >= 0; --l) {
        Level& C = h->lv[l];
        Level& F = h->lv[l + 1];
        CK(launch_restrict_state(C.g, F.g, F.U64, F.pt64, F.mask, C.U64, C.pt64, C.mask, h->prm.coarse_phi_max != 0,
                                 h->stream));
    }
    for (auto& L : h->lv) {
        if (!values) break;     // only the masks changed: FP32 copies and Gauss-point data stay valid
        CK(launch_cast_f64_f32(L.U64, L.U32, n_dofs(L.g), h->stream));
        CK(launch_cast_f64_f32(L.pt64, L.pt32, L.g.n_nodes, h->stream));
        if (L.qpd64 && !h->ph.split) {
            if (L.g.deg == 1) CK(launch_q1_linearize(L.g, h->ph, L.U64, L.pt64, L.qpd32, L.qpd64, h->stream));
            else CK(launch_q2_linearize(L.g, h->ph, L.U64, L.pt64, L.qpd32, L.qpd64, h->stream));
        }
        if (L.qps64 && h->ph.split)
            CK(launch_q1_linearize_split(L.g, h->ph, L.U64, L.pt64, L.qps32, L.qps64, h->stream));
    }
    h->stale = true;
    return cudaSuccess;
}

// ---------------------------------------------------------------- eigenvalue estimate
// Device scalar layout in h->d_scal (doubles):
//   [0..1] rz, [2..3] pq, [4..5] alpha, [6..7] beta, [8..9] rz_new, [10..11] stopped flag,
//   [16 .. 16 + 2*2*maxsteps) alpha/beta history per block, [256..] misc (FGMRES)
static constexpr int S_RZ = 0, S_PQ = 2, S_AL = 4, S_BE = 6, S_RZN = 8, S_STOP = 10, S_HIST = 16;
static constexpr int MAX_CG = 50;

__global__ void k_cg_alpha(double* s) {
    const int b = threadIdx.x;
    if (b >= 2) return;
    const double rz = s[S_RZ + b], pq = s[S_PQ + b];
    if (s[S_STOP + b] != 0.0 || !(rz > 0.0) || !(pq > 0.0)) {
        s[S_STOP + b] = 1.0;
        s[S_AL + b] = 0.0;
    } else {
        s[S_AL + b] = rz / pq;
    }
}

__global__ void k_cg_beta(double* s, int it) {
    const int b = threadIdx.x;
    if (b >= 2) return;
    double* hist = s + S_HIST;   // [it][b][alpha, beta]
    if (s[S_STOP + b] != 0.0) {
        s[S_BE + b] = 0.0;
        hist[(it * 2 + b) * 2 + 0] = 0.0;
        hist[(it * 2 + b) * 2 + 1] = -1.0;   // marks a step not taken
        return;
    }
    const double beta = s[S_RZN + b] / s[S_RZ + b];
    s[S_BE + b] = beta;
    hist[(it * 2 + b) * 2 + 0] = s[S_AL + b];
    hist[(it * 2 + b) * 2 + 1] = beta;
    s[S_RZ + b] = s[S_RZN + b];
}

// Sturm count of eigenvalues of the symmetric tridiagonal (a, e) below x.
__device__ int sturm_count(const double* a, const double* e, int k, double x) {
    int cnt = 0;
    double q = 1.0;
    for (int j = 0; j < k; ++j) {
        const double off = j > 0 ? e[j - 1] * e[j - 1] : 0.0;
        q = (a[j] - x) - (j > 0 ? off / q : 0.0);
        if (q == 0.0) q = -1e-300;
        if (q < 0.0) ++cnt;
    }
    return cnt;
}

// Lanczos tridiagonal from CG coefficients (T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1},
// T_j,j+1 = sqrt(beta_j)/alpha_j) and its extreme eigenvalues by multisection: one warp per
// (block, extreme); each round the 32 lanes evaluate Sturm counts at 32 interior points of the
// bracket and the bracket shrinks to the sub-interval where the count crosses the target
// (count >= 1 for the smallest eigenvalue, count >= k for the largest).
__global__ void k_cg_eigs(const double* s, int steps, double* out /* lmin_u, lmax_u, lmin_p, lmax_p */) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w >= 4) return;
    const int b = w >> 1, want_max = w & 1;
    const double* hist = s + S_HIST;
    double a[MAX_CG], e[MAX_CG];
    int k = 0;
    for (int it = 0; it < steps; ++it) {
        const double al = hist[(it * 2 + b) * 2 + 0], be = hist[(it * 2 + b) * 2 + 1];
        if (be < 0.0 && al == 0.0) break;
        k = it + 1;
    }
    if (k == 0) {
        if (lane == 0) out[2 * b + want_max] = 1.0;
        return;
    }
    for (int j = 0; j < k; ++j) {
        const double al = hist[(j * 2 + b) * 2 + 0], be = hist[(j * 2 + b) * 2 + 1];
        a[j] = 1.0 / al;
        if (j > 0) {
            const double alp = hist[((j - 1) * 2 + b) * 2 + 0], bep = hist[((j - 1) * 2 + b) * 2 + 1];
            a[j] += bep / alp;
        }
        e[j] = sqrt(be) / al;
    }
    double lo = 1e300, hi = -1e300;   // Gershgorin bracket
    for (int j = 0; j < k; ++j) {
        const double r = (j > 0 ? fabs(e[j - 1]) : 0.0) + (j + 1 < k ? fabs(e[j]) : 0.0);
        lo = fmin(lo, a[j] - r);
        hi = fmax(hi, a[j] + r);
    }
    const int target = want_max ? k : 1;
    for (int round = 0; round < 16; ++round) {
        const double x = lo + (hi - lo) * (double)(lane + 1) / 33.0;
        const unsigned hit = __ballot_sync(0xffffffffu, sturm_count(a, e, k, x) >= target);
        const int first = hit ? __ffs(hit) - 1 : 32;   // first lane whose point reaches the target
        const double nlo = first == 0 ? lo : lo + (hi - lo) * (double)first / 33.0;
        const double nhi = first == 32 ? hi : lo + (hi - lo) * (double)(first + 1) / 33.0;
        if (!(nhi - nlo < hi - lo)) break;
        lo = nlo;
        hi = nhi;
    }
    if (lane == 0) out[2 * b + want_max] = 0.5 * (lo + hi);
}

template <typename T>
static cudaError_t eigen_estimate(pff_hierarchy* h, int l, double* d_out) {
    Level& L = h->lv[l];
    cudaStream_t s = h->stream;
    T* r = work<T>(L, 2);
    T* z = work<T>(L, 3);
    T* q = work<T>(L, 4);
    T* p = work<T>(L, 5);
    double* sc = h->d_scal_lv + (size_t)kLevelScal * l;         // per level: setup runs levels concurrently
    double* scratch = h->d_scratch_lv + (size_t)kLevelScratch * l;
    static_assert(S_HIST + 4 * MAX_CG <= kLevelScal, "CG scalars exceed the per-level region");
    const int steps = std::min(h->prm.cg_steps, MAX_CG);
    CK(cudaMemsetAsync(sc, 0, sizeof(double) * (S_HIST + 4 * MAX_CG), s));
    CK(launch_start_vector<T>(L.g, L.mask, h->prm.seed, l, r, s));
    // z = dinv r (an update with the zeroed alpha), p = z
    CK(launch_cg_update_r<T>(L.g, r, r, dinv<T>(L), z, sc + S_AL, s));
    CK(cudaMemcpyAsync(p, z, sizeof(T) * n_dofs(L.g), cudaMemcpyDeviceToDevice, s));
    CK(launch_block_dots<T>(L.g, r, z, (const T*)nullptr, scratch, sc + S_RZ, s));
    for (int it = 0; it < steps; ++it) {
        CK(apply_level<T>(h, l, OP_APPLY_BLOCKDIAG, p, q, PHI_BITS_ALL));
        CK(launch_block_dots<T>(L.g, p, q, (const T*)nullptr, scratch, sc + S_PQ, s));
        k_cg_alpha<<<1, 32, 0, s>>>(sc);
        CK(count_launch(cudaGetLastError()));
        CK(launch_cg_update_r<T>(L.g, r, q, dinv<T>(L), z, sc + S_AL, s));
        CK(launch_block_dots<T>(L.g, r, z, (const T*)nullptr, scratch, sc + S_RZN, s));
        k_cg_beta<<<1, 32, 0, s>>>(sc, it);
        CK(count_launch(cudaGetLastError()));
        CK(launch_cg_update_p<T>(L.g, p, z, sc + S_BE, s));
    }
    k_cg_eigs<<<1, 128, 0, s>>>(sc, steps, d_out);
    return count_launch(cudaGetLastError());
}

void drop_graph(pff_hierarchy* h) {
    if (h->vgraph) cudaGraphExecDestroy(h->vgraph);
    h->vgraph = nullptr;
    h->vgraph_nodes = 0;
}

cudaError_t setup(pff_hierarchy* h) {
    CK(refresh_state(h));
    cudaStream_t s = h->stream;
    drop_graph(h);
    const bool f32 = h->prm.mg_precision == 32;
    double* d_eigs = h->d_scal + 512;   // 4 per level
    // The levels' diagonals and eigenvalue estimates are independent (each level has its own
    // vectors, diagonal, CG scalars and partial sums): fork one stream per level from the library
    // stream and join them before the bounds are read.  The small levels' launch latencies then
    // overlap the fine level's work.
    CK(cudaEventRecord(h->lv_event[h->L], s));
    for (int l = 0; l < h->L; ++l) {
        Level& L = h->lv[l];
        cudaStream_t ls = h->lv_stream[l];
        CK(cudaStreamWaitEvent(ls, h->lv_event[h->L], 0));
        h->stream = ls;   // every launch of this level's setup goes to its stream
        cudaError_t e = diagonal_level<double>(h, l, L.dinv64);
        if (e == cudaSuccess) e = launch_invert_diag<double>(L.dinv64, n_dofs(L.g), ls);
        if (e == cudaSuccess) e = launch_cast_f64_f32(L.dinv64, L.dinv32, n_dofs(L.g), ls);
        // the coarsest level's bounds feed the FP64 coarse solver; the others the smoother
        if (e == cudaSuccess) e = (f32 && l > 0) ? eigen_estimate<float>(h, l, d_eigs + 4 * l)
                                                 : eigen_estimate<double>(h, l, d_eigs + 4 * l);
        if (e == cudaSuccess) e = cudaEventRecord(h->lv_event[l], ls);
        h->stream = s;
        if (e != cudaSuccess) return e;
        CK(cudaStreamWaitEvent(s, h->lv_event[l], 0));
    }
    std::vector<double> eig(4 * h->L);
    CK(cudaMemcpyAsync(eig.data(), d_eigs, sizeof(double) * 4 * h->L, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int l = 0; l < h->L; ++l) {
        for (int b = 0; b < 2; ++b) {
            h->lv[l].lam_min[b] = eig[4 * l + 2 * b];
            h->lv[l].lam_max[b] = eig[4 * l + 2 * b + 1];
        }
    }
    h->stale = false;
    return cudaSuccess;
}

// ---------------------------------------------------------------- Chebyshev
// Coefficients of a k-step Chebyshev recurrence on [alpha, beta] (Saad Alg. 12.1):
// step 0: d = (1/theta) z ; step s>0: d = rho_s rho_{s-1} d + (2 rho_s / delta) z.
struct ChebCoef {
    std::vector<double> c1, c2;
};
static ChebCoef cheb_coefs(double alpha, double beta, int k) {
    ChebCoef c;
    const double theta = 0.5 * (beta + alpha), delta = 0.5 * (beta - alpha);
    const double sigma1 = theta / delta;
    double rho = 1.0 / sigma1;
    c.c1.push_back(0.0);
    c.c2.push_back(1.0 / theta);
    for (int s = 1; s < k; ++s) {
        const double rn = 1.0 / (2.0 * sigma1 - rho);
        c.c1.push_back(rn * rho);
        c.c2.push_back(2.0 * rn / delta);
        rho = rn;
    }
    return c;
}

static int coarse_steps(double alpha, double beta, double rtol, int maxit) {
    const double sigma1 = (beta + alpha) / (beta - alpha);
    const double k = ceil(acosh(1.0 / rtol) / acosh(sigma1));
    int ki = (int)std::min<double>(k, (double)maxit);
    return std::max(1, ki);
}

// Operator of the V-cycle residuals: G~ (P_full) or its block diagonal (P_diag, Sec. 3.3).
static int mg_op(const pff_hierarchy* h) { return h->prm.preconditioner == 1 ? OP_APPLY_BLOCKDIAG : OP_APPLY; }

// Run the recurrence on the residual r (modified in place) with the block-diagonal operator;
// mode 1: x = correction, mode 2: x += correction.  ku/kp: steps per block (the longer block
// keeps iterating; the other block's coefficients become zero-updates once finished).
template <typename T>
static cudaError_t cheb_run(pff_hierarchy* h, int l, T* r, T* x, const ChebCoef& cu, const ChebCoef& cp,
                            int mode) {
    Level& L = h->lv[l];
    T* d = work<T>(L, 3);
    T* t = work<T>(L, 4);
    const int k = (int)std::max(cu.c2.size(), cp.c2.size());
    // first step; every update except the last also presets t for the next apply
    CK(launch_cheb_update<T>(L.g, r, (const T*)nullptr, d, dinv<T>(L), x, 0.0, 0.0, cu.c2[0], cp.c2[0], mode,
                             h->stream, L.mask, k > 1 ? t : (T*)nullptr));
    for (int st = 1; st < k; ++st) {
        CK(apply_level<T>(h, l, OP_APPLY_BLOCKDIAG, d, t, PHI_BITS_ALL, false));
        const bool uon = st < (int)cu.c2.size(), pon = st < (int)cp.c2.size();
        CK(launch_cheb_update<T>(L.g, r, t, d, dinv<T>(L), x, uon ? cu.c1[st] : 0.0, pon ? cp.c1[st] : 0.0,
                                 uon ? cu.c2[st] : 0.0, pon ? cp.c2[st] : 0.0, 0, h->stream, L.mask,
                                 st + 1 < k ? t : (T*)nullptr));
    }
    return cudaSuccess;
}

template <typename T>
cudaError_t smooth(pff_hierarchy* h, int l, const T* b, T* x, int zero_guess) {
    Level& L = h->lv[l];
    T* r = work<T>(L, 2);
    const int64_t nd = n_dofs(L.g);
    if (zero_guess) {
        CK(cudaMemcpyAsync(r, b, sizeof(T) * nd, cudaMemcpyDeviceToDevice, h->stream));
    } else {
        T* t = work<T>(L, 4);
        CK(apply_level<T>(h, l, mg_op(h), x, t, PHI_BITS_ALL));
        CK(launch_sub<T>(nd, b, t, r, h->stream));
    }
    const double sf = h->prm.cheb_safety, ra = h->prm.cheb_ratio;
    ChebCoef cu = cheb_coefs(ra * sf * L.lam_max[0], sf * L.lam_max[0], h->prm.cheb_degree);
    ChebCoef cp = cheb_coefs(ra * sf * L.lam_max[1], sf * L.lam_max[1], h->prm.cheb_degree);
    return cheb_run<T>(h, l, r, x, cu, cp, zero_guess ? 1 : 2);
}
template cudaError_t smooth<double>(pff_hierarchy*, int, const double*, double*, int);
template cudaError_t smooth<float>(pff_hierarchy*, int, const float*, float*, int);

// FP64 coarse solve on level 0: u block first, then phi block with the coupling G_phiu x_u
// moved to the right-hand side (P_full); both blocks at once without the coupling (P_diag).
cudaError_t coarse_solve(pff_hierarchy* h, const double* b, double* x) {
    Level& L = h->lv[0];
    const int64_t nd = n_dofs(L.g);
    double* r = work<double>(L, 2);
    double* t = work<double>(L, 4);
    double* xp = work<double>(L, 5);
    const double au = 0.9 * L.lam_min[0], bu = 1.2 * L.lam_max[0];
    const double ap = 0.9 * L.lam_min[1], bp = 1.2 * L.lam_max[1];
    const int ku = coarse_steps(au, bu, h->prm.coarse_rtol, h->prm.coarse_maxit);
    const int kp = coarse_steps(ap, bp, h->prm.coarse_rtol, h->prm.coarse_maxit);
    ChebCoef cu = cheb_coefs(au, bu, ku), cp = cheb_coefs(ap, bp, kp);
    ChebCoef none;
    none.c1.assign(1, 0.0);
    none.c2.assign(1, 0.0);
    if (h->prm.preconditioner == 1) {
        CK(cudaMemcpyAsync(r, b, sizeof(double) * nd, cudaMemcpyDeviceToDevice, h->stream));
        return cheb_run<double>(h, 0, r, x, cu, cp, 1);
    }
    // u block
    CK(launch_copy_block<double>(L.g, 0, b, r, h->stream));
    CK(cheb_run<double>(h, 0, r, x, cu, none, 1));
    // phi block: r = (b - G x_u) restricted to phi
    CK(apply_level<double>(h, 0, OP_APPLY, x, t, PHI_BITS_ALL));
    CK(launch_sub<double>(nd, b, t, r, h->stream));
    CK(launch_copy_block<double>(L.g, 1, r, r, h->stream));
    CK(cheb_run<double>(h, 0, r, xp, none, cp, 1));
    return launch_axpby<double>(nd, 1.0, xp, 1.0, x, h->stream);
}

// V-cycle on level l: b -> x (level work vectors 0 = b, 1 = x of each level).
template <typename T>
static cudaError_t vcycle_rec(pff_hierarchy* h, int l) {
    Level& L = h->lv[l];
    T* b = work<T>(L, 0);
    T* x = work<T>(L, 1);
    if (l == 0) {
        if (sizeof(T) == 8) return coarse_solve(h, (const double*)b, (double*)x);
        double* b64 = work<double>(L, 0);
        double* x64 = work<double>(L, 1);
        CK(launch_cast_f32_f64((const float*)b, b64, n_dofs(L.g), h->stream));
        CK(coarse_solve(h, b64, x64));
        return launch_cast_f64_f32(x64, (float*)x, n_dofs(L.g), h->stream);
    }
    Level& C = h->lv[l - 1];
    const int64_t nd = n_dofs(L.g);
    T* r = work<T>(L, 2);
    T* t = work<T>(L, 4);
    CK(smooth<T>(h, l, b, x, 1));
    CK(apply_level<T>(h, l, mg_op(h), x, t, PHI_BITS_ALL));
    CK(launch_sub<T>(nd, b, t, r, h->stream));
    CK(launch_restrict<T>(C.g, L.g, r, work<T>(C, 0), C.mask, h->stream));
    CK(vcycle_rec<T>(h, l - 1));
    CK(launch_prolongate_add<T>(C.g, L.g, work<T>(C, 1), x, L.mask, h->stream));
    return smooth<T>(h, l, b, x, 0);
}

// The V-cycle between the fixed level buffers (input work 0, output work 1 of the finest level).
// On a non-default stream it is captured once per setup into a CUDA graph and replayed: every
// kernel argument (Chebyshev coefficients included) is fixed between setups.
template <typename T>
static cudaError_t vcycle_body(pff_hierarchy* h) {
    if (!h->use_graphs || h->stream == nullptr) return vcycle_rec<T>(h, h->L - 1);
    if (!h->vgraph) {
        cudaGraph_t g = nullptr;
        const bool prof = h->prof_on;
        h->prof_on = false;                   // no timing events inside the captured body
        CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        const long long c0 = launch_count();
        cudaError_t e = vcycle_rec<T>(h, h->L - 1);
        cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
        h->prof_on = prof;
        if (e != cudaSuccess || e2 != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            h->use_graphs = false;            // fall back to direct launches from now on
            return vcycle_rec<T>(h, h->L - 1);
        }
        e = cudaGraphInstantiate(&h->vgraph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            cudaGetLastError();
            h->vgraph = nullptr;
            h->use_graphs = false;
            return vcycle_rec<T>(h, h->L - 1);
        }
        h->vgraph_nodes = launch_count() - c0;
        add_launches(-h->vgraph_nodes);       // captured kernels run only when replayed
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (h->prof_on) {
        e0 = next_event(h);
        e1 = next_event(h);
        if (e0 && e1) CK(cudaEventRecord(e0, h->stream));
    }
    CK(cudaGraphLaunch(h->vgraph, h->stream));
    if (e0 && e1) {
        CK(cudaEventRecord(e1, h->stream));
        h->prof[PFF_PROF_VCYCLE].push_back({e0, e1});
    }
    add_launches(h->vgraph_nodes);
    return cudaSuccess;
}

cudaError_t vcycle(pff_hierarchy* h, const double* r, double* z) {
    CK(refresh_state(h));
    Level& F = h->lv[h->L - 1];
    const int64_t nd = n_dofs(F.g);
    if (h->prm.mg_precision == 32) {
        float* b = work<float>(F, 0);
        // b = free ? (float) r : 0
        CK(launch_mask_copy<double>(F.g, F.mask, r, h->tmp64[3], 1, h->stream));
        CK(launch_cast_f64_f32(h->tmp64[3], b, nd, h->stream));
        CK(vcycle_body<float>(h));
        CK(launch_cast_f32_f64(work<float>(F, 1), z, nd, h->stream));
    } else {
        CK(launch_mask_copy<double>(F.g, F.mask, r, work<double>(F, 0), 1, h->stream));
        CK(vcycle_body<double>(h));
        CK(cudaMemcpyAsync(z, work<double>(F, 1), sizeof(double) * nd, cudaMemcpyDeviceToDevice, h->stream));
    }
    return launch_mask_copy<double>(F.g, F.mask, r, z, 0, h->stream);
}

// ---------------------------------------------------------------- FGMRES
pff_status fgmres(pff_hierarchy* h, const double* b, double* x, double rtol, int m, int maxit,
                  pff_solve_info* info, std::string& err) {
    cudaStream_t s = h->stream;
    const int fine = h->L - 1;
    Level& F = h->lv[fine];
    const int64_t n = n_dofs(F.g);
    double* V = h->kr_V;
    double* Z = h->kr_Z;
    double* w = h->tmp64[0];
    double* dsc = h->d_scal + 256;   // [0] norm, [1..] h1, h2 buffers in kr_h
    double* h1 = h->kr_h;
    double* h2 = h->kr_h + (m + 1);
    std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m, 0.0), sn(m, 0.0), g(m + 1, 0.0), hv(2 * (m + 1) + 1);
    auto fail = [&](const char* what, cudaError_t e) {
        err = std::string(what) + ": " + cudaGetErrorString(e);
        return PFF_ECUDA;
    };
#define KC(expr, what)                              \
    do {                                            \
        cudaError_t e_ = (expr);                    \
        if (e_ != cudaSuccess) return fail(what, e_); \
    } while (0)
    auto true_res = [&](double* out) -> cudaError_t {
        CK(apply_level<double>(h, fine, OP_APPLY, x, w, PHI_BITS_ALL));
        CK(launch_sub<double>(n, b, w, w, s));
        CK(launch_norm2(n, w, h->d_scratch, dsc, s));
        CK(cudaMemcpyAsync(out, dsc, sizeof(double), cudaMemcpyDeviceToHost, s));
        return cudaStreamSynchronize(s);
    };
    double beta0 = 0.0;
    KC(true_res(&beta0), "fgmres residual");
    if (!std::isfinite(beta0)) {
        err = "non-finite initial residual";
        return PFF_ENONFINITE;
    }
    const double target = rtol * beta0;
    int its = 0;
    double beta = beta0;
    bool first = true;
    while (true) {
        if (!first) KC(true_res(&beta), "fgmres residual");
        first = false;
        if (!std::isfinite(beta)) {
            err = "non-finite residual";
            return PFF_ENONFINITE;
        }
        if (beta <= target || its >= maxit || beta == 0.0) break;
        // V_0 = w / beta   (w holds b - G x)
        KC(launch_scale_copy(n, w, dsc, V, s), "fgmres scale");
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int k = 0;
        for (int j = 0; j < m; ++j) {
            double* Vj = V + (int64_t)j * n;
            double* Zj = Z + (int64_t)j * n;
            double* Vn = V + (int64_t)(j + 1) * n;
            KC(vcycle(h, Vj, Zj), "vcycle");
            KC(apply_level<double>(h, fine, OP_APPLY, Zj, Vn, PHI_BITS_ALL), "apply");
            // classical Gram-Schmidt, twice
            KC(launch_multidot(n, V, n, j + 1, Vn, h->d_scratch, h1, s), "multidot");
            KC(launch_multi_axpy(n, V, n, j + 1, h1, Vn, s), "axpy");
            KC(launch_multidot(n, V, n, j + 1, Vn, h->d_scratch, h2, s), "multidot");
            KC(launch_multi_axpy(n, V, n, j + 1, h2, Vn, s), "axpy");
            KC(launch_norm2(n, Vn, h->d_scratch, dsc, s), "norm");
            KC(launch_scale_copy(n, Vn, dsc, Vn, s), "scale");
            KC(cudaMemcpyAsync(hv.data(), h->kr_h, sizeof(double) * 2 * (m + 1), cudaMemcpyDeviceToHost, s), "copy");
            KC(cudaMemcpyAsync(hv.data() + 2 * (m + 1), dsc, sizeof(double), cudaMemcpyDeviceToHost, s), "copy");
            KC(cudaStreamSynchronize(s), "sync");
            for (int i = 0; i <= j; ++i) H[i * m + j] = hv[i] + hv[(m + 1) + i];
            const double hn = hv[2 * (m + 1)];
            if (!std::isfinite(hn)) {
                err = "non-finite Arnoldi norm";
                return PFF_ENONFINITE;
            }
            H[(j + 1) * m + j] = hn;
            for (int i = 0; i < j; ++i) {
                const double t = cs[i] * H[i * m + j] + sn[i] * H[(i + 1) * m + j];
                H[(i + 1) * m + j] = -sn[i] * H[i * m + j] + cs[i] * H[(i + 1) * m + j];
                H[i * m + j] = t;
            }
            const double den = hypot(H[j * m + j], H[(j + 1) * m + j]);
            cs[j] = H[j * m + j] / den;
            sn[j] = H[(j + 1) * m + j] / den;
            H[j * m + j] = den;
            H[(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            ++its;
            k = j + 1;
            if (fabs(g[j + 1]) <= target || its >= maxit) break;
        }
        std::vector<double> y(k, 0.0);
        for (int i = k - 1; i >= 0; --i) {
            double acc = g[i];
            for (int c = i + 1; c < k; ++c) acc -= H[i * m + c] * y[c];
            y[i] = acc / H[i * m + i];
        }
        KC(cudaMemcpyAsync(h1, y.data(), sizeof(double) * k, cudaMemcpyHostToDevice, s), "copy y");
        KC(launch_gemv_add(n, Z, n, k, h1, x, s), "update");
    }
    double res = 0.0;
    KC(true_res(&res), "fgmres residual");
#undef KC
    if (info) {
        info->iterations = its;
        info->res0 = beta0;
        info->res_final = res;
        info->converged = res <= target * (1.0 + 1e-12) || beta0 == 0.0;
    }
    if (!std::isfinite(res)) {
        err = "non-finite final residual";
        return PFF_ENONFINITE;
    }
    if (!(res <= target * (1.0 + 1e-12) || beta0 == 0.0)) {
        err = "FGMRES reached maxit";
        return PFF_ENOCONV;
    }
    return PFF_OK;
}

}  // namespace pff
