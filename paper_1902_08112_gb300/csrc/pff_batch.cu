// Batches: many independent instances (hierarchies) advanced together, one launch per level and
// operation.  A pff_batch is a view over existing hierarchies (all on one stream, same dimension,
// Q1, FP32 V-cycle): per (instance, level) descriptors live in device memory, the applies map a
// flattened CTA index to (instance, tile), and every other kernel runs one grid row per instance.
//
// The V-cycle runs in lockstep over level indices (0 = every instance's coarsest level):
// instance i takes part in level l when it has more than l levels, and enters the cycle at its own
// finest level.  FGMRES keeps its Hessenberg matrices and Givens rotations per instance on the host
// and drops converged instances from the descriptor tables.  Per-instance results are the same as
// the single-instance path up to rounding.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "pff_batch.cuh"
#include "pff_batch_kernels.cuh"
#include "pff_q1.cuh"
#include "pff_solver.cuh"

using namespace pff;

struct pff_batch {
    int n = 0, dim = 3, Lmax = 0, m = 0;
    std::vector<pff_hierarchy*> hs;
    cudaStream_t stream = nullptr;
    std::vector<char> valid;                 // instance currently processed
    std::vector<std::vector<BLevel>> h_lv;   // [l][i]
    std::vector<BLevel> h_fine;              // [i]: the instance's finest level
    BLevel* d_lv = nullptr;                  // Lmax * n
    BLevel* d_fine = nullptr;                // n
    int* d_tiles = nullptr;                  // [(l * 2 + style) * (n + 1)], l = Lmax is the fine table
    std::vector<int> tot;                    // totals per (l, style)
    std::vector<int> blocks;                 // grid width per level (elementwise); blocks[Lmax] = fine
    std::vector<int64_t> cells;              // cells per level over the valid instances
    double* d_part = nullptr;                // partial sums
    double* d_vals = nullptr;                // per-instance scalars
    double* d_coef = nullptr;                // Chebyshev tables (smoother and coarse)
    size_t coef_cap = 0;                     // allocated doubles of d_coef
    uint64_t* d_seeds = nullptr;
    int cheb_k = 4, coarse_k = 1;
    // batched FGMRES state on the device (per instance): flags read by every batched kernel, the
    // Hessenberg matrices, Givens rotations and right-hand sides, iteration counts and targets
    int* d_on = nullptr;                     // n: instance active in the current Arnoldi step
    int* d_cyc = nullptr;                    // n: instance takes part in the current restart cycle
    int* d_col = nullptr;                    // 1: Krylov column j of the next Arnoldi step
    int* d_its = nullptr;                    // n
    int* d_k = nullptr;                      // n: Krylov dimension of the cycle
    int* d_flags = nullptr;                  // n: bit 0 non-finite residual, bit 1 non-finite Arnoldi norm
    int* d_count = nullptr;                  // [0] instances on after the last step, [1] maxit, [2] instances on with
                                             // the FP64 V-cycle, [3] iterations before an FP32-MG instance switches
    int* d_prec = nullptr;                   // n: V-cycle precision of the instance in the current solve (32 / 64)
    int* d_save = nullptr;                   // n: the FGMRES flags while a V-cycle runs on a precision's subset
    int switch_its = 10;                     // FP32 V-cycle batches: FP64 V-cycle after this many iterations (0: never)
    double* d_fg = nullptr;                  // per instance: beta, target, g (m + 1), cs, sn, y (m each), H
    int* h_status = nullptr;                 // pinned host mirror: [0] count, [1 ..] flags / its
    cudaEvent_t ev_step[2] = {nullptr, nullptr};
    cudaGraphExec_t step_graph = nullptr;    // one captured Arnoldi step (every column j)
    cudaGraphExec_t step_graph_mixed = nullptr;   // the same with the V-cycle split by instance precision
    int graph_key = -1;                      // coarse_k the graph was captured with
    bool use_graphs = true;
    long long graph_nodes = 0, graph_nodes_mixed = 0;
    // autotuned level operators: per lockstep level (Lmax = the fine table) and precision (0 FP32,
    // 1 FP64) the kernel family (1 small-level kernels, 2 per-cell kernels) and the persistent grid
    // (CTAs per SM; 0 = one CTA per tile), with the measured time of one apply
    struct Tune { int style = 0, cps = 0; double ms = 0.0; };
    std::vector<Tune> tune;                  // (Lmax + 1) * 2
    bool tuned = false;
    int sms = 0;
    bool mg64 = false;                       // FP64 V-cycle (mg_precision 64 in every instance)
    int style = 0;                           // level-operator kernels: 0 by level size, 1 small-level, 2 per-cell
    bool stale = true;
    bool dirty = false;                      // instances changed: device state rebuilt before the next call
    std::vector<pff_newton_info> last;       // per instance: the last batched Newton step (pff_batch_poll)
    std::vector<void*> allocs;
    std::string err;
};

namespace {

constexpr int kStyleF32 = 0, kStyleF64 = 1;   // FP32 per-cell kernel, df64 lane kernel
constexpr int kMaxCG = 50;

#define BCK(...)                                  \
    do {                                          \
        cudaError_t e_ = (__VA_ARGS__);           \
        if (e_ != cudaSuccess) return e_;         \
    } while (0)

template <typename T>
cudaError_t balloc(pff_batch* b, T** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T) + 16);
    if (e != cudaSuccess) return e;
    b->allocs.push_back(q);
    *p = reinterpret_cast<T*>(q);
    return cudaMemsetAsync(q, 0, count * sizeof(T) + 16, b->stream);
}

BLevel make_desc(pff_hierarchy* h, int l, bool valid, const int* on, const int* col) {
    BLevel d;
    memset(&d, 0, sizeof(d));
    Level& L = h->lv[l];
    d.g = L.g;
    d.valid = valid ? 1 : 0;
    d.on = on;
    d.col = col;
    d.mask = L.mask;
    d.qpd32 = L.qpd32;
    d.qpd64 = L.qpd64;
    d.dinv32 = L.dinv32;
    d.dinv64 = L.dinv64;
    for (int k = 0; k < 6; ++k) {
        d.vec[BV_W32 + k] = L.w[0][k];
        d.vec[BV_W64 + k] = L.w[1][k];
    }
    d.vec[BV_U] = L.U64;
    if (l == h->L - 1) {
        for (int k = 0; k < 4; ++k) d.vec[BV_T64 + k] = h->tmp64[k];
        d.vec[BV_KV] = h->kr_V;
        d.vec[BV_KZ] = h->kr_Z;
        d.vec[BV_R] = h->R;
        d.vec[BV_PHIOLD] = h->phi_old;
    }
    d.k = make_q1_consts(L.g, h->ph);
    return d;
}

int grid_w(int64_t n) {
    int64_t b = (n + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 1024));
}

__global__ void kb_set_flags(int n, int v, int* __restrict__ on) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) on[i] = v;
}

// every instance on (the state between batched FGMRES solves)
cudaError_t set_all_on(pff_batch* b) {
    kb_set_flags<<<std::max(1, std::min(64, (b->n + 255) / 256)), 256, 0, b->stream>>>(b->n, 1, b->d_on);
    return count_launch(cudaGetLastError());
}

// rebuild and upload descriptor tables and tile prefixes for the instances flagged in b->valid
cudaError_t upload(pff_batch* b) {
    const int n = b->n;
    std::vector<int> tiles((size_t)(b->Lmax + 1) * 2 * (n + 1), 0);
    b->tot.assign((size_t)(b->Lmax + 1) * 2, 0);
    b->blocks.assign(b->Lmax + 1, 1);
    b->cells.assign(b->Lmax + 1, 0);
    for (int l = 0; l <= b->Lmax; ++l) {
        for (int i = 0; i < n; ++i) {
            pff_hierarchy* h = b->hs[i];
            const bool fine = l == b->Lmax;
            const int li = fine ? h->L - 1 : l;
            const bool has = li < h->L;
            BLevel d = make_desc(h, has ? li : 0, has && b->valid[i], b->d_on ? b->d_on + i : nullptr, b->d_col);
            if (fine) b->h_fine[i] = d; else b->h_lv[l][i] = d;
            for (int st = 0; st < 2; ++st) {
                int* pre = &tiles[((size_t)l * 2 + st) * (n + 1)];
                const int t = d.valid ? q1_tiles(d.g, st == kStyleF64, st == kStyleF64) : 0;
                pre[i + 1] = pre[i] + t;
            }
            if (d.valid) {
                b->blocks[l] = std::max(b->blocks[l], grid_w(n_dofs(d.g)));
                b->cells[l] += d.g.n_cells;
            }
        }
        for (int st = 0; st < 2; ++st) b->tot[(size_t)l * 2 + st] = tiles[((size_t)l * 2 + st) * (n + 1) + n];
    }
    for (int l = 0; l < b->Lmax; ++l)
        BCK(cudaMemcpyAsync(b->d_lv + (size_t)l * n, b->h_lv[l].data(), sizeof(BLevel) * n, cudaMemcpyHostToDevice,
                            b->stream));
    BCK(cudaMemcpyAsync(b->d_fine, b->h_fine.data(), sizeof(BLevel) * n, cudaMemcpyHostToDevice, b->stream));
    BCK(cudaMemcpyAsync(b->d_tiles, tiles.data(), sizeof(int) * tiles.size(), cudaMemcpyHostToDevice, b->stream));
    if (b->d_on) BCK(set_all_on(b));
    // the host vectors are reused at the next upload: make the copies complete first
    return cudaStreamSynchronize(b->stream);
}

const BLevel* tab(pff_batch* b, int l) { return l == b->Lmax ? b->d_fine : b->d_lv + (size_t)l * b->n; }

// y(sy) = G~ x(sx) on level l (l == Lmax: each instance's finest level), precision by fp64.  The
// kernel family and persistent grid come from the autotuner (style 0), else from the fixed rule
// (3D levels of at least kCellMinCells cells over the batch run the per-cell kernel with
// shared-memory derivatives) or the forced style.
cudaError_t b_apply(pff_batch* b, int l, bool fp64, bool blockdiag, int sx, int sy, int phi_bits, bool preset = true,
                    int force_style = 0, int force_cps = -1) {
    const BLevel* L = tab(b, l);
    int style = force_style ? force_style : b->style;
    int cps = force_cps >= 0 ? force_cps : 0;
    if (!force_style && style == 0 && b->tuned) {
        const pff_batch::Tune& t = b->tune[(size_t)l * 2 + (fp64 ? 1 : 0)];
        style = t.style;
        if (force_cps < 0) cps = t.cps;
    }
    const bool cell = b->dim == 3 && q1_cell_tiles_match_f32() &&
                      (style == 2 || (style == 0 && b->cells[l] >= kCellMinCells));
    const int st = (fp64 && !cell) ? kStyleF64 : kStyleF32;
    if (preset) {
        if (fp64) BCK(bl_init_masked<double>(L, b->n, b->blocks[l], sx, sy, phi_bits, 0.0, b->stream));
        else BCK(bl_init_masked<float>(L, b->n, b->blocks[l], sx, sy, phi_bits, 0.f, b->stream));
    }
    return launch_q1_apply_batched(b->dim, fp64, blockdiag, fp64 && !cell, L, b->n,
                                   b->d_tiles + ((size_t)l * 2 + st) * (b->n + 1), b->tot[(size_t)l * 2 + st], sx, sy,
                                   phi_bits, b->stream, cell, cps > 0 ? cps * b->sms : 0);
}

double* smooth_coef(pff_batch* b, int l, int step) { return b->d_coef + ((size_t)l * b->cheb_k + step) * b->n * 4; }
double* coarse_coef(pff_batch* b, int phase, int step) {
    return b->d_coef + (size_t)b->Lmax * b->cheb_k * b->n * 4 + ((size_t)phase * b->coarse_k + step) * b->n * 4;
}

// Chebyshev recurrence on level l in precision T from r (W2) into x (W1); mode 1: x = corr, 2: x += corr
template <typename T>
cudaError_t b_cheb_run(pff_batch* b, int l, int K, bool coarse, int phase, int sx, int mode) {
    const BLevel* L = tab(b, l);
    const int W = sizeof(T) == 8 ? BV_W64 : BV_W32;
    const int r = bsel(W + 2), d = bsel(W + 3), t = bsel(W + 4);
    // every update except the last also presets t for the next apply
    BCK(bl_cheb<T>(L, b->n, b->blocks[l], r, -1, d, sx, coarse ? coarse_coef(b, phase, 0) : smooth_coef(b, l, 0), mode,
                   b->stream, K > 1 ? t : -1));
    for (int s = 1; s < K; ++s) {
        BCK(b_apply(b, l, sizeof(T) == 8, true, d, t, PHI_BITS_ALL, false));
        BCK(bl_cheb<T>(L, b->n, b->blocks[l], r, t, d, sx, coarse ? coarse_coef(b, phase, s) : smooth_coef(b, l, s), 0,
                       b->stream, s + 1 < K ? t : -1));
    }
    return cudaSuccess;
}

// Smoother on level l in precision T: zero guess (x = S b) or x += S (b - G x)
template <typename T>
cudaError_t b_smooth(pff_batch* b, int l, bool zero_guess) {
    const BLevel* L = tab(b, l);
    const int W = sizeof(T) == 8 ? BV_W64 : BV_W32;
    const int bb = bsel(W + 0), x = bsel(W + 1), r = bsel(W + 2), t = bsel(W + 4);
    if (zero_guess) {
        BCK(bl_copy<T>(L, b->n, b->blocks[l], bb, r, -1, b->stream));
    } else {
        BCK(b_apply(b, l, sizeof(T) == 8, false, x, t, PHI_BITS_ALL));
        BCK(bl_sub<T>(L, b->n, b->blocks[l], bb, t, r, b->stream));
    }
    return b_cheb_run<T>(b, l, b->cheb_k, false, 0, x, zero_guess ? 1 : 2);
}

// FP64 coarse solve on level 0: b (W64_0) -> x (W64_1), u block then phi block
cudaError_t b_coarse(pff_batch* b) {
    const BLevel* L = tab(b, 0);
    const int w = b->blocks[0];
    const int bb = bsel(BV_W64 + 0), x = bsel(BV_W64 + 1), r = bsel(BV_W64 + 2), t = bsel(BV_W64 + 4),
              xp = bsel(BV_W64 + 5);
    BCK(bl_copy<double>(L, b->n, w, bb, r, 0, b->stream));
    BCK(b_cheb_run<double>(b, 0, b->coarse_k, true, 0, x, 1));
    BCK(b_apply(b, 0, true, false, x, t, PHI_BITS_ALL));
    BCK(bl_sub<double>(L, b->n, w, bb, t, r, b->stream));
    BCK(bl_copy<double>(L, b->n, w, r, r, 1, b->stream));
    BCK(b_cheb_run<double>(b, 0, b->coarse_k, true, 1, xp, 1));
    return bl_axpby64(L, b->n, w, nullptr, xp, 1.0, x, 0, b->stream);
}

// z (fine selector) = V-cycle(v (fine selector)); levels in precision T, FP64 coarse solve
template <typename T>
cudaError_t b_vcycle_t(pff_batch* b, int sv, int sz) {
    const int F = b->Lmax;
    const int W = sizeof(T) == 8 ? BV_W64 : BV_W32;
    const bool f64 = sizeof(T) == 8;
    BCK(bl_convert<double, T>(tab(b, F), b->n, b->blocks[F], sv, bsel(W + 0), 1, b->stream));
    for (int l = b->Lmax - 1; l >= 1; --l) {
        BCK(b_smooth<T>(b, l, true));
        BCK(b_apply(b, l, f64, false, bsel(W + 1), bsel(W + 4), PHI_BITS_ALL));
        BCK(bl_sub<T>(tab(b, l), b->n, b->blocks[l], bsel(W + 0), bsel(W + 4), bsel(W + 2), b->stream));
        BCK(bl_restrict<T>(tab(b, l - 1), tab(b, l), b->n, b->blocks[l - 1], bsel(W + 2), bsel(W + 0), b->stream));
    }
    if (!f64) BCK(bl_convert<float, double>(tab(b, 0), b->n, b->blocks[0], bsel(BV_W32 + 0), bsel(BV_W64 + 0), 0, b->stream));
    BCK(b_coarse(b));
    if (!f64) BCK(bl_convert<double, float>(tab(b, 0), b->n, b->blocks[0], bsel(BV_W64 + 1), bsel(BV_W32 + 1), 0, b->stream));
    for (int l = 1; l < b->Lmax; ++l) {
        BCK(bl_prolongate_add<T>(tab(b, l - 1), tab(b, l), b->n, b->blocks[l], bsel(W + 1), bsel(W + 1), b->stream));
        BCK(b_smooth<T>(b, l, false));
    }
    BCK(bl_convert<T, double>(tab(b, F), b->n, b->blocks[F], bsel(W + 1), sz, 0, b->stream));
    return bl_convert<double, double>(tab(b, F), b->n, b->blocks[F], sv, sz, 2, b->stream);
}

cudaError_t b_vcycle(pff_batch* b, int sv, int sz) {
    return b->mg64 ? b_vcycle_t<double>(b, sv, sz) : b_vcycle_t<float>(b, sv, sz);
}

// ---------------------------------------------------------------- batched eigenvalue estimates
// scalar layout per level run: [0,2n) rz, [2n,4n) pq, [4n,6n) alpha, [6n,8n) beta, [8n,10n) rz_new,
// [10n,12n) stopped, then history [it][inst][block][alpha, beta]
__global__ void kb_cg_alpha(double* s, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * n) return;
    const double rz = s[i], pq = s[2 * n + i];
    if (s[10 * n + i] != 0.0 || !(rz > 0.0) || !(pq > 0.0)) {
        s[10 * n + i] = 1.0;
        s[4 * n + i] = 0.0;
    } else {
        s[4 * n + i] = rz / pq;
    }
}
__global__ void kb_cg_beta(double* s, int n, int it) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * n) return;
    double* hist = s + 12 * n + (size_t)it * 4 * n;
    if (s[10 * n + i] != 0.0) {
        s[6 * n + i] = 0.0;
        hist[2 * i] = 0.0;
        hist[2 * i + 1] = -1.0;
        return;
    }
    const double beta = s[8 * n + i] / s[i];
    s[6 * n + i] = beta;
    hist[2 * i] = s[4 * n + i];
    hist[2 * i + 1] = beta;
    s[i] = s[8 * n + i];
}
__device__ int b_sturm(const double* a, const double* e, int k, double x) {
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
// one CTA per instance, one warp per (block, extreme): Lanczos tridiagonal and multisection
__global__ void kb_cg_eigs(const double* s, int n, int steps, double* out /* [inst][4] */) {
    const int inst = blockIdx.x;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w >= 4) return;
    const int blk = w >> 1, want_max = w & 1;
    const int i = 2 * inst + blk;
    const double* hist = s + 12 * n;
    double a[kMaxCG], e[kMaxCG];
    int k = 0;
    for (int it = 0; it < steps; ++it) {
        const double al = hist[(size_t)it * 4 * n + 2 * i], be = hist[(size_t)it * 4 * n + 2 * i + 1];
        if (be < 0.0 && al == 0.0) break;
        k = it + 1;
    }
    if (k == 0) {
        if (lane == 0) out[4 * inst + 2 * blk + want_max] = 1.0;
        return;
    }
    for (int j = 0; j < k; ++j) {
        const double al = hist[(size_t)j * 4 * n + 2 * i], be = hist[(size_t)j * 4 * n + 2 * i + 1];
        a[j] = 1.0 / al;
        if (j > 0) {
            const double alp = hist[(size_t)(j - 1) * 4 * n + 2 * i], bep = hist[(size_t)(j - 1) * 4 * n + 2 * i + 1];
            a[j] += bep / alp;
        }
        e[j] = sqrt(be) / al;
    }
    double lo = 1e300, hi = -1e300;
    for (int j = 0; j < k; ++j) {
        const double r = (j > 0 ? fabs(e[j - 1]) : 0.0) + (j + 1 < k ? fabs(e[j]) : 0.0);
        lo = fmin(lo, a[j] - r);
        hi = fmax(hi, a[j] + r);
    }
    const int target = want_max ? k : 1;
    for (int round = 0; round < 16; ++round) {
        const double x = lo + (hi - lo) * (double)(lane + 1) / 33.0;
        const unsigned hit = __ballot_sync(0xffffffffu, b_sturm(a, e, k, x) >= target);
        const int first = hit ? __ffs(hit) - 1 : 32;
        const double nlo = first == 0 ? lo : lo + (hi - lo) * (double)first / 33.0;
        const double nhi = first == 32 ? hi : lo + (hi - lo) * (double)(first + 1) / 33.0;
        if (!(nhi - nlo < hi - lo)) break;
        lo = nlo;
        hi = nhi;
    }
    if (lane == 0) out[4 * inst + 2 * blk + want_max] = 0.5 * (lo + hi);
}

template <typename T>
cudaError_t b_eigen_level(pff_batch* b, int l, int steps, uint64_t* seeds, double* d_out) {
    const BLevel* L = tab(b, l);
    const int n = b->n, w = b->blocks[l];
    const int W = sizeof(T) == 8 ? BV_W64 : BV_W32;
    const int r = bsel(W + 2), z = bsel(W + 3), q = bsel(W + 4), p = bsel(W + 5);
    double* s = b->d_vals;
    BCK(cudaMemsetAsync(s, 0, sizeof(double) * (12 * (size_t)n + (size_t)steps * 4 * n), b->stream));
    BCK(bl_start_vector<T>(L, n, w, r, seeds, l, b->stream));
    BCK(bl_cg_r<T>(L, n, w, r, r, z, s + 4 * n, b->stream));   // alpha = 0: z = dinv r
    BCK(bl_copy<T>(L, n, w, z, p, -1, b->stream));
    BCK(bl_dots2<T>(L, n, r, z, b->d_part, s, b->stream));
    const int tb = (2 * n + 127) / 128;
    for (int it = 0; it < steps; ++it) {
        BCK(b_apply(b, l, sizeof(T) == 8, true, p, q, PHI_BITS_ALL));
        BCK(bl_dots2<T>(L, n, p, q, b->d_part, s + 2 * n, b->stream));
        kb_cg_alpha<<<tb, 128, 0, b->stream>>>(s, n);
        BCK(count_launch(cudaGetLastError()));
        BCK(bl_cg_r<T>(L, n, w, r, q, z, s + 4 * n, b->stream));
        BCK(bl_dots2<T>(L, n, r, z, b->d_part, s + 8 * n, b->stream));
        kb_cg_beta<<<tb, 128, 0, b->stream>>>(s, n, it);
        BCK(count_launch(cudaGetLastError()));
        BCK(bl_cg_p<T>(L, n, w, p, z, s + 6 * n, b->stream));
    }
    kb_cg_eigs<<<n, 128, 0, b->stream>>>(s, n, steps, d_out);
    return count_launch(cudaGetLastError());
}

struct HostCheb {
    std::vector<double> c1, c2;
};
HostCheb host_cheb(double alpha, double beta, int k) {
    HostCheb c;
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
int host_coarse_steps(double alpha, double beta, double rtol, int maxit) {
    const double sigma1 = (beta + alpha) / (beta - alpha);
    const double k = ceil(acosh(1.0 / rtol) / acosh(sigma1));
    return std::max(1, (int)std::min<double>(k, (double)maxit));
}

void drop_step_graph(pff_batch* b);

// ---------------------------------------------------------------- autotuner
// Choices are cached for the process by (dimension, precision, log2 of the level's cells over the
// batch, log2 of its instances), so batches of a similar make-up (e.g. successive compositions of a
// serving loop) reuse them.
struct TuneKey {
    int dim, prec, lc, ln;
    bool operator<(const TuneKey& o) const {
        return std::tie(dim, prec, lc, ln) < std::tie(o.dim, o.prec, o.lc, o.ln);
    }
};
std::mutex g_tune_mutex;
std::map<TuneKey, pff_batch::Tune> g_tune_cache;

int ilog2(int64_t v) {
    int r = 0;
    while (v > 1) { v >>= 1; ++r; }
    return r;
}

// Time every candidate (kernel family x persistent grid) of the level operator on each level and
// precision the batch uses, with CUDA events over a few launches on the level's scratch vectors
// (work vectors 3 -> 4, free at setup time), and keep the fastest.
cudaError_t b_autotune(pff_batch* b) {
    const int n = b->n;
    b->tune.assign((size_t)(b->Lmax + 1) * 2, pff_batch::Tune());
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    BCK(cudaEventCreate(&e0));
    cudaError_t err = cudaEventCreate(&e1);
    if (err != cudaSuccess) {
        cudaEventDestroy(e0);
        return err;
    }
    for (int l = 0; l <= b->Lmax && err == cudaSuccess; ++l) {
        if (b->cells[l] == 0) continue;
        for (int prec = 0; prec < 2 && err == cudaSuccess; ++prec) {
            // FP64 operators run on the fine table and the coarse level (FGMRES, coarse solve) or, with
            // the FP64 V-cycle, everywhere; FP32 operators on the V-cycle levels of an FP32 V-cycle
            const bool used = prec == 1 ? (l == b->Lmax || l == 0 || b->mg64) : (!b->mg64 && l > 0 && l < b->Lmax);
            if (!used) continue;
            const TuneKey key{b->dim, prec, ilog2(b->cells[l]), ilog2(n)};
            {
                std::lock_guard<std::mutex> lock(g_tune_mutex);
                auto it = g_tune_cache.find(key);
                if (it != g_tune_cache.end()) {
                    b->tune[(size_t)l * 2 + prec] = it->second;
                    continue;
                }
            }
            const int W = prec ? BV_W64 : BV_W32;
            pff_batch::Tune best;
            best.ms = -1.0;
            const int nstyles = b->dim == 3 ? 2 : 1;
            for (int style = 1; style <= nstyles && err == cudaSuccess; ++style) {
                const bool cell = style == 2;
                const int res = q1_batched_ctas_per_sm(b->dim, prec == 1, cell);
                const int tiles = b->tot[(size_t)l * 2 + ((prec == 1 && !cell) ? kStyleF64 : kStyleF32)];
                std::vector<int> cands{0};
                for (int c : {std::max(1, res / 2), res})
                    if ((int64_t)c * b->sms < tiles && std::find(cands.begin(), cands.end(), c) == cands.end())
                        cands.push_back(c);
                for (int c : cands) {
                    err = b_apply(b, l, prec == 1, false, bsel(W + 3), bsel(W + 4), PHI_BITS_ALL, true, style, c);
                    if (err == cudaSuccess) err = cudaEventRecord(e0, b->stream);
                    for (int r = 0; r < 3 && err == cudaSuccess; ++r)
                        err = b_apply(b, l, prec == 1, false, bsel(W + 3), bsel(W + 4), PHI_BITS_ALL, true, style, c);
                    if (err == cudaSuccess) err = cudaEventRecord(e1, b->stream);
                    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
                    float ms = 0.f;
                    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
                    if (err != cudaSuccess) break;
                    if (best.ms < 0.0 || ms / 3.0 < best.ms) {
                        best.style = style;
                        best.cps = c;
                        best.ms = ms / 3.0;
                    }
                }
            }
            if (err == cudaSuccess) {
                b->tune[(size_t)l * 2 + prec] = best;
                std::lock_guard<std::mutex> lock(g_tune_mutex);
                g_tune_cache[key] = best;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err == cudaSuccess) b->tuned = true;
    return err;
}

// diagonals per instance, batched eigenvalue estimates, coefficient tables
cudaError_t b_setup(pff_batch* b) {
    const int n = b->n;
    for (int i = 0; i < n; ++i) {
        pff_hierarchy* h = b->hs[i];
        for (int l = 0; l < h->L; ++l) {
            Level& L = h->lv[l];
            BCK(diagonal_level<double>(h, l, L.dinv64));
            BCK(launch_invert_diag<double>(L.dinv64, n_dofs(L.g), b->stream));
            BCK(launch_cast_f64_f32(L.dinv64, L.dinv32, n_dofs(L.g), b->stream));
        }
    }
    if (!b->tuned && b->style == 0) BCK(b_autotune(b));
    const int steps = std::min(b->hs[0]->prm.cg_steps, kMaxCG);
    double* d_eig = b->d_vals + 12 * (size_t)n + (size_t)kMaxCG * 4 * n;   // [l][inst][4]
    for (int l = 0; l < b->Lmax; ++l) {
        if (l == 0 || b->mg64) BCK(b_eigen_level<double>(b, l, steps, b->d_seeds, d_eig + (size_t)l * 4 * n));
        else BCK(b_eigen_level<float>(b, l, steps, b->d_seeds, d_eig + (size_t)l * 4 * n));
    }
    std::vector<double> eig((size_t)b->Lmax * 4 * n);
    BCK(cudaMemcpyAsync(eig.data(), d_eig, sizeof(double) * eig.size(), cudaMemcpyDeviceToHost, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    // smoother coefficients [l][step][inst][4], coarse [phase][step][inst][4]
    const pff_params& prm = b->hs[0]->prm;
    std::vector<int> ku(n), kp(n);
    int kmax = 1;
    for (int i = 0; i < n; ++i) {
        const double* e0 = &eig[4 * (size_t)i];
        ku[i] = host_coarse_steps(0.9 * e0[0], 1.2 * e0[1], prm.coarse_rtol, prm.coarse_maxit);
        kp[i] = host_coarse_steps(0.9 * e0[2], 1.2 * e0[3], prm.coarse_rtol, prm.coarse_maxit);
        kmax = std::max(kmax, std::max(ku[i], kp[i]));
    }
    b->coarse_k = kmax;
    std::vector<double> coef(((size_t)b->Lmax * b->cheb_k + 2 * (size_t)kmax) * n * 4, 0.0);
    for (int l = 0; l < b->Lmax; ++l)
        for (int i = 0; i < n; ++i) {
            if (l >= b->hs[i]->L) continue;
            for (int blk = 0; blk < 2; ++blk) {
                const double lm = eig[((size_t)l * n + i) * 4 + 2 * blk + 1];
                HostCheb c = host_cheb(prm.cheb_ratio * prm.cheb_safety * lm, prm.cheb_safety * lm, b->cheb_k);
                for (int s = 0; s < b->cheb_k; ++s) {
                    double* dst = &coef[(((size_t)l * b->cheb_k + s) * n + i) * 4];
                    dst[0 + blk] = c.c1[s];
                    dst[2 + blk] = c.c2[s];
                }
            }
        }
    const size_t cbase = (size_t)b->Lmax * b->cheb_k * n * 4;
    for (int i = 0; i < n; ++i) {
        const double* e0 = &eig[4 * (size_t)i];
        HostCheb cu = host_cheb(0.9 * e0[0], 1.2 * e0[1], ku[i]);
        HostCheb cp = host_cheb(0.9 * e0[2], 1.2 * e0[3], kp[i]);
        for (int s = 0; s < ku[i]; ++s) {
            double* dst = &coef[cbase + (((size_t)0 * kmax + s) * n + i) * 4];
            dst[0] = cu.c1[s];
            dst[2] = cu.c2[s];
        }
        for (int s = 0; s < kp[i]; ++s) {
            double* dst = &coef[cbase + (((size_t)1 * kmax + s) * n + i) * 4];
            dst[1] = cp.c1[s];
            dst[3] = cp.c2[s];
        }
        for (int l = 0; l < b->hs[i]->L; ++l)
            for (int blk = 0; blk < 2; ++blk) {
                b->hs[i]->lv[l].lam_min[blk] = eig[((size_t)l * n + i) * 4 + 2 * blk];
                b->hs[i]->lv[l].lam_max[blk] = eig[((size_t)l * n + i) * 4 + 2 * blk + 1];
            }
    }
    // the table keeps its address across setups (the captured Arnoldi step reads it); it is only
    // reallocated, and the graph dropped, when it has to grow
    if (coef.size() > b->coef_cap) {
        drop_step_graph(b);
        BCK(cudaStreamSynchronize(b->stream));
        if (b->d_coef) {
            for (auto it = b->allocs.begin(); it != b->allocs.end(); ++it)
                if (*it == b->d_coef) { cudaFree(*it); b->allocs.erase(it); break; }
            b->d_coef = nullptr;
        }
        const size_t cap = coef.size() + coef.size() / 2;
        BCK(balloc(b, &b->d_coef, cap));
        b->coef_cap = cap;
    }
    BCK(cudaMemcpyAsync(b->d_coef, coef.data(), sizeof(double) * coef.size(), cudaMemcpyHostToDevice, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    for (auto* h : b->hs) h->stale = false;
    b->stale = false;
    return cudaSuccess;
}

// ---------------------------------------------------------------- batched FGMRES
// Per-instance FGMRES scalars live on the device (layout of d_fg per instance, stride fg_stride):
// [0] beta (current true residual), [1] target, [2] beta_0, [3, m + 4) g, then cs (m), sn (m),
// y (m), H ((m + 1) x m, row-major).
__host__ __device__ inline int fg_stride(int m) { return 3 + (m + 1) + 3 * m + (m + 1) * m; }
constexpr int kFgG = 3;

// Start of a restart cycle: instance i iterates while its true residual beta_i is finite and above
// target_i and its iteration budget lasts; g = beta e_1, column counter 0, count of active instances.
__global__ void kb_fg_begin(int n, int m, int maxit, double rtol, int first, int base_prec, int switch_its,
                            double* __restrict__ fg, int* __restrict__ its, int* __restrict__ cyc,
                            int* __restrict__ on, int* __restrict__ k, int* __restrict__ flags,
                            int* __restrict__ prec, int* __restrict__ col, int* __restrict__ count) {
    __shared__ int cnt, c64;
    if (threadIdx.x == 0) cnt = c64 = 0;
    __syncthreads();
    const int st = fg_stride(m);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double* f = fg + (size_t)i * st;
        const double beta = f[0];
        if (first) {
            f[1] = rtol * beta;
            f[2] = beta;
            its[i] = 0;
            flags[i] = 0;
            prec[i] = base_prec;
        }
        const bool finite = isfinite(beta);
        if (!finite) flags[i] |= 1;
        const int need = finite && !(beta <= f[1] || its[i] >= maxit || beta == 0.0);
        cyc[i] = need;
        on[i] = need;
        k[i] = 0;
        double* g = f + kFgG;
        g[0] = beta;
        for (int r = 1; r <= m; ++r) g[r] = 0.0;
        if (need) atomicAdd(&cnt, 1);
        if (need && prec[i] == 64) atomicAdd(&c64, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        *col = 0;
        count[0] = cnt;
        count[1] = maxit;        // read by the captured Arnoldi steps
        count[2] = c64;
        count[3] = switch_its;
    }
}

// One Arnoldi step's scalar work for every active instance (column j = *col): the new Hessenberg
// column from the two Gram-Schmidt passes and the norm, the previous Givens rotations, a new one,
// the updated residual estimate |g_{j+1}|; an instance that reaches its target or its iteration cap
// is switched off.  Then the column counter advances.
// A still-active FP32-MG instance that has taken count[3] iterations switches to the FP64 V-cycle
// (flexible GMRES admits a different preconditioner in every iteration).
__global__ void kb_fg_arnoldi(int n, int m, const double* __restrict__ h, const double* __restrict__ nrm,
                              double* __restrict__ fg, int* __restrict__ its, int* __restrict__ on,
                              int* __restrict__ k, int* __restrict__ flags, int* __restrict__ prec,
                              int* __restrict__ col, int* __restrict__ count) {
    __shared__ int cnt, c64;
    const int j = *col, maxit = count[1], sw = count[3];
    if (threadIdx.x == 0) cnt = c64 = 0;
    __syncthreads();
    const int st = fg_stride(m);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        if (!on[i] || j >= m) {
            if (j >= m) on[i] = 0;
            continue;
        }
        double* f = fg + (size_t)i * st;
        double* g = f + kFgG;
        double* cs = g + (m + 1);
        double* sn = cs + m;
        double* H = sn + 2 * m;
        const double* hi = h + (size_t)i * 2 * (m + 1);
        for (int r = 0; r <= j; ++r) H[(size_t)r * m + j] = hi[r] + hi[(m + 1) + r];
        const double hn = nrm[i];
        if (!isfinite(hn)) {
            flags[i] |= 2;
            on[i] = 0;
            continue;
        }
        H[(size_t)(j + 1) * m + j] = hn;
        for (int r = 0; r < j; ++r) {
            const double a = H[(size_t)r * m + j], bb = H[(size_t)(r + 1) * m + j];
            H[(size_t)r * m + j] = cs[r] * a + sn[r] * bb;
            H[(size_t)(r + 1) * m + j] = -sn[r] * a + cs[r] * bb;
        }
        const double den = hypot(H[(size_t)j * m + j], H[(size_t)(j + 1) * m + j]);
        cs[j] = H[(size_t)j * m + j] / den;
        sn[j] = H[(size_t)(j + 1) * m + j] / den;
        H[(size_t)j * m + j] = den;
        H[(size_t)(j + 1) * m + j] = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        its[i] += 1;
        k[i] = j + 1;
        if (fabs(g[j + 1]) <= f[1] || its[i] >= maxit || j + 1 >= m) {
            on[i] = 0;
        } else {
            atomicAdd(&cnt, 1);
            if (prec[i] == 32 && sw > 0 && its[i] >= sw) prec[i] = 64;
            if (prec[i] == 64) atomicAdd(&c64, 1);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        *col = j + 1;
        count[0] = cnt;
        count[2] = c64;
    }
}

// V-cycle of one precision's subset: mode 0 keeps the FGMRES flags and leaves the FP32-MG instances
// on, mode 1 the FP64-MG ones, mode 2 restores the flags
__global__ void kb_prec_subset(int n, int mode, int* __restrict__ on, int* __restrict__ save,
                               const int* __restrict__ prec) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (mode == 0) save[i] = on[i];
        const int o = save[i];
        on[i] = mode == 2 ? o : (o && prec[i] == (mode == 0 ? 32 : 64));
    }
}

// y = H_k^-1 g_k (back substitution) for every instance of the cycle; then the cycle's instances
// are switched on again for the update x += Z y
__global__ void kb_fg_solve(int n, int m, double* __restrict__ fg, const int* __restrict__ k,
                            const int* __restrict__ cyc, int* __restrict__ on) {
    const int st = fg_stride(m);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double* f = fg + (size_t)i * st;
        const double* g = f + kFgG;
        double* y = f + kFgG + (m + 1) + 2 * m;
        const double* H = y + m;
        const int ki = cyc[i] ? k[i] : 0;
        for (int r = m - 1; r >= ki; --r) y[r] = 0.0;
        for (int r = ki - 1; r >= 0; --r) {
            double acc = g[r];
            for (int c = r + 1; c < ki; ++c) acc -= H[(size_t)r * m + c] * y[c];
            y[r] = acc / H[(size_t)r * m + r];
        }
        on[i] = cyc[i];
    }
}

// beta_i (the fg slot 0) from the norms of a batched reduction
__global__ void kb_fg_take_beta(int n, int m, const double* __restrict__ nrm, double* __restrict__ fg) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        fg[(size_t)i * fg_stride(m)] = nrm[i];
}

cudaError_t fg_launch_checked(cudaError_t e) { return count_launch(e == cudaSuccess ? cudaGetLastError() : e); }

// One Arnoldi step of every active instance at column j = *col (all selectors through the device
// counter, so the same launches serve every j): z_j = MG(v_j), w = G~ z_j, classical Gram-Schmidt
// twice, v_{j+1} = w / |w|, then the scalar step on the device.
cudaError_t b_arnoldi_step(pff_batch* b, bool mixed) {
    const int n = b->n, m = b->m, F = b->Lmax;
    cudaStream_t s = b->stream;
    double* d_nrm = b->d_vals;
    double* d_h = b->d_vals + n;
    const int vj = bsel(BV_KV, kColJ), zj = bsel(BV_KZ, kColJ), vn = bsel(BV_KV, kColJ1);
    if (mixed) {
        const int tb = std::max(1, std::min(64, (n + 255) / 256));
        kb_prec_subset<<<tb, 256, 0, s>>>(n, 0, b->d_on, b->d_save, b->d_prec);
        BCK(fg_launch_checked(cudaSuccess));
        BCK(b_vcycle_t<float>(b, vj, zj));
        kb_prec_subset<<<tb, 256, 0, s>>>(n, 1, b->d_on, b->d_save, b->d_prec);
        BCK(fg_launch_checked(cudaSuccess));
        BCK(b_vcycle_t<double>(b, vj, zj));
        kb_prec_subset<<<tb, 256, 0, s>>>(n, 2, b->d_on, b->d_save, b->d_prec);
        BCK(fg_launch_checked(cudaSuccess));
    } else {
        BCK(b_vcycle(b, vj, zj));
    }
    BCK(b_apply(b, F, true, false, zj, vn, PHI_BITS_ALL));
    BCK(bl_multidot(tab(b, F), n, -1, vn, b->d_part, m + 1, d_h, 2 * (m + 1), s, b->d_col));
    BCK(bl_multi_axpy(tab(b, F), n, b->blocks[F], -1, d_h, 2 * (m + 1), vn, s, b->d_col));
    BCK(bl_multidot(tab(b, F), n, -1, vn, b->d_part, m + 1, d_h + (m + 1), 2 * (m + 1), s, b->d_col));
    BCK(bl_multi_axpy(tab(b, F), n, b->blocks[F], -1, d_h + (m + 1), 2 * (m + 1), vn, s, b->d_col));
    BCK(bl_norm(tab(b, F), n, vn, b->d_part, d_nrm, s));
    BCK(bl_axpby64(tab(b, F), n, b->blocks[F], d_nrm, vn, 0.0, vn, 1, s));
    kb_fg_arnoldi<<<1, 256, 0, s>>>(n, m, d_h, d_nrm, b->d_fg, b->d_its, b->d_on, b->d_k, b->d_flags, b->d_prec,
                                    b->d_col, b->d_count);
    return fg_launch_checked(cudaSuccess);
}

void drop_step_graph(pff_batch* b) {
    if (b->step_graph) cudaGraphExecDestroy(b->step_graph);
    if (b->step_graph_mixed) cudaGraphExecDestroy(b->step_graph_mixed);
    b->step_graph = b->step_graph_mixed = nullptr;
    b->graph_key = -1;
    b->graph_nodes = 0;
}

cudaError_t capture_step(pff_batch* b, bool mixed, cudaGraphExec_t* out, long long* nodes) {
    cudaGraph_t g = nullptr;
    BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    const long long c0 = launch_count();
    cudaError_t e = b_arnoldi_step(b, mixed);
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess && !g) e = cudaErrorUnknown;
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    if (g) cudaGraphDestroy(g);
    *nodes = launch_count() - c0;
    add_launches(-*nodes);        // captured kernels run only when replayed
    return e;
}

// The Arnoldi step, captured once into a CUDA graph (and once more with the V-cycle split by instance
// precision) and replayed for every column, restart cycle and later solve of the batch: every
// argument of its launches is fixed (descriptor tables, vector selectors, coefficient tables) or read
// from device memory (column, flags, precisions).  Re-captured when the coarse solver's step count
// changes (the shape of the V-cycle).  Direct launches on the legacy default stream, which cannot be
// captured.
cudaError_t b_run_step(pff_batch* b, bool mixed) {
    if (!b->use_graphs || b->stream == nullptr) return b_arnoldi_step(b, mixed);
    if ((b->step_graph || b->step_graph_mixed) && b->graph_key != b->coarse_k) drop_step_graph(b);
    cudaGraphExec_t* ge = mixed ? &b->step_graph_mixed : &b->step_graph;
    long long* nodes = mixed ? &b->graph_nodes_mixed : &b->graph_nodes;
    if (!*ge) {
        cudaError_t e = capture_step(b, mixed, ge, nodes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            *ge = nullptr;
            b->use_graphs = false;        // direct launches from now on
            return b_arnoldi_step(b, mixed);
        }
        b->graph_key = b->coarse_k;
    }
    BCK(cudaGraphLaunch(*ge, b->stream));
    add_launches(*nodes);
    return cudaSuccess;
}

// solve G~ x = b per instance: b in T64[1], x in T64[2] (fine selectors).  The host launches the
// steps and reads one counter per step (one step behind, so the GPU never waits for the host); every
// scalar of the method stays on the device.
pff_status b_fgmres(pff_batch* b, double rtol, int maxit, pff_solve_info* info) {
    const int n = b->n, m = b->m, F = b->Lmax;
    cudaStream_t s = b->stream;
    const int sb = bsel(BV_T64 + 1), sx = bsel(BV_T64 + 2), sw = bsel(BV_T64 + 0);
    double* d_nrm = b->d_vals;
    // host mirror: [0] active after a cycle start, [1 + 2 (j & 1)] active and [2 + 2 (j & 1)] active with the
    // FP64 V-cycle after step j (alternating slots), [5 ..) flags
    int* hs = b->h_status;
    const int base_prec = b->mg64 ? 64 : 32;
    bool mixed = false;
    for (int q = 1; q < 5; ++q) hs[q] = 0;
    auto fail = [&](cudaError_t e) {
        b->err = std::string("batched FGMRES: ") + cudaGetErrorString(e);
        return PFF_ECUDA;
    };
#define BKC(...)                            \
    do {                                    \
        cudaError_t e_ = (__VA_ARGS__);     \
        if (e_ != cudaSuccess) return fail(e_); \
    } while (0)
    const int tb = std::max(1, std::min(64, (n + 255) / 256));
    // true residual of every instance -> beta (fg slot 0)
    auto true_res = [&]() -> cudaError_t {
        kb_set_flags<<<tb, 256, 0, s>>>(n, 1, b->d_on);
        BCK(fg_launch_checked(cudaSuccess));
        BCK(b_apply(b, F, true, false, sx, sw, PHI_BITS_ALL));
        BCK(bl_sub<double>(tab(b, F), n, b->blocks[F], sb, sw, sw, s));
        BCK(bl_norm(tab(b, F), n, sw, b->d_part, d_nrm, s));
        kb_fg_take_beta<<<tb, 256, 0, s>>>(n, m, d_nrm, b->d_fg);
        return fg_launch_checked(cudaSuccess);
    };
    auto begin = [&](int first) -> cudaError_t {
        kb_fg_begin<<<1, 256, 0, s>>>(n, m, maxit, rtol, first, base_prec, b->mg64 ? 0 : b->switch_its, b->d_fg,
                                      b->d_its, b->d_cyc, b->d_on, b->d_k, b->d_flags, b->d_prec, b->d_col,
                                      b->d_count);
        BCK(fg_launch_checked(cudaSuccess));
        BCK(cudaMemcpyAsync(hs, b->d_count, sizeof(int), cudaMemcpyDeviceToHost, s));
        BCK(cudaMemcpyAsync(hs + 5, b->d_flags, sizeof(int) * n, cudaMemcpyDeviceToHost, s));
        return cudaStreamSynchronize(s);
    };
    auto check_flags = [&](const char* what) -> bool {
        for (int i = 0; i < n; ++i)
            if (hs[5 + i]) {
                b->err = std::string("non-finite ") + what + " in instance " + std::to_string(i);
                set_all_on(b);
                return true;
            }
        return false;
    };
    b->valid.assign(n, 1);
    BKC(upload(b));
    BKC(true_res());
    BKC(begin(1));
    if (check_flags("initial residual")) return PFF_ENONFINITE;
    while (hs[0] > 0) {
        // V_0 = w / beta on the active instances (w = b - G x from the true residual)
        BKC(bl_axpby64(tab(b, F), n, b->blocks[F], d_nrm, sw, 0.0, bsel(BV_KV, 0), 1, s));
        for (int j = 0; j < m; ++j) {
            BKC(b_run_step(b, mixed && !b->mg64));
            BKC(cudaMemcpyAsync(hs + 1 + 2 * (j & 1), b->d_count, sizeof(int), cudaMemcpyDeviceToHost, s));
            BKC(cudaMemcpyAsync(hs + 2 + 2 * (j & 1), b->d_count + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
            BKC(cudaEventRecord(b->ev_step[j & 1], s));
            if (j >= 1) {
                BKC(cudaEventSynchronize(b->ev_step[(j - 1) & 1]));
                if (hs[1 + 2 * ((j - 1) & 1)] == 0) break;   // every instance stopped at step j - 1
                if (hs[2 + 2 * ((j - 1) & 1)] > 0) mixed = true;   // an instance switched to the FP64 V-cycle
            }
        }
        if (hs[0] > 0 && !mixed) {
            BKC(cudaStreamSynchronize(s));
            // a switch decided in the last step of the cycle
            for (int q = 0; q < 2; ++q)
                if (hs[2 + 2 * q] > 0) mixed = true;
        }
        kb_fg_solve<<<tb, 256, 0, s>>>(n, m, b->d_fg, b->d_k, b->d_cyc, b->d_on);
        BKC(fg_launch_checked(cudaSuccess));
        const int ldy = fg_stride(m);
        BKC(bl_gemv_add(tab(b, F), n, b->blocks[F], m, b->d_fg + kFgG + (m + 1) + 2 * m, ldy, sx, s, b->d_k));
        BKC(true_res());
        BKC(begin(0));
        if (check_flags("residual or Arnoldi norm")) return PFF_ENONFINITE;
    }
    BKC(set_all_on(b));
#undef BKC
    // final true residuals (fg slot 0), targets and iteration counts
    std::vector<double> fgh((size_t)n * fg_stride(m));
    std::vector<int> its(n);
    if (cudaMemcpyAsync(fgh.data(), b->d_fg, sizeof(double) * fgh.size(), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(its.data(), b->d_its, sizeof(int) * n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(cudaGetLastError());
    pff_status st = PFF_OK;
    for (int i = 0; i < n; ++i) {
        const double* f = &fgh[(size_t)i * fg_stride(m)];
        const double res = f[0], target = f[1], res0 = f[2];
        const bool conv = res <= target * (1.0 + 1e-12) || res0 == 0.0;
        if (info) {
            info[i].iterations = its[i];
            info[i].res0 = res0;
            info[i].res_final = res;
            info[i].converged = conv ? 1 : 0;
        }
        if (!std::isfinite(res)) {
            b->err = "non-finite final residual in instance " + std::to_string(i);
            st = PFF_ENONFINITE;
        } else if (!conv && st == PFF_OK) {
            b->err = "batched FGMRES reached maxit";
            st = PFF_ENOCONV;
        }
    }
    return st;
}

// The device-side state of a batch (descriptor tables, reduction scratch, FGMRES state, captured
// graphs, tuning): released and rebuilt from the current instance list when it changes.
void release_state(pff_batch* b) {
    drop_step_graph(b);
    for (cudaEvent_t& e : b->ev_step) {
        if (e) cudaEventDestroy(e);
        e = nullptr;
    }
    if (b->h_status) cudaFreeHost(b->h_status);
    b->h_status = nullptr;
    for (void* p : b->allocs) cudaFree(p);
    b->allocs.clear();
    b->d_lv = b->d_fine = nullptr;
    b->d_tiles = nullptr;
    b->d_part = b->d_vals = b->d_coef = b->d_fg = nullptr;
    b->coef_cap = 0;
    b->d_seeds = nullptr;
    b->d_on = b->d_cyc = b->d_col = b->d_its = b->d_k = b->d_flags = b->d_count = b->d_prec = b->d_save = nullptr;
    b->tuned = false;
    b->stale = true;
    b->use_graphs = true;
}

void free_batch(pff_batch* b) {
    release_state(b);
    delete b;
}

cudaError_t build_state(pff_batch* b) {
    const int n = b->n, restart = b->m;
    b->Lmax = 0;
    for (auto* h : b->hs) b->Lmax = std::max(b->Lmax, h->L);
    b->valid.assign(n, 1);
    b->h_lv.assign(b->Lmax, std::vector<BLevel>(n));
    b->h_fine.assign(n, BLevel());
    cudaError_t e = balloc(b, &b->d_lv, (size_t)b->Lmax * n);
    if (e == cudaSuccess) e = balloc(b, &b->d_fine, (size_t)n);
    if (e == cudaSuccess) e = balloc(b, &b->d_tiles, (size_t)(b->Lmax + 1) * 2 * (n + 1));
    if (e == cudaSuccess) e = balloc(b, &b->d_part, (size_t)n * (restart + 2) * kBPartials * 2);
    if (e == cudaSuccess) e = balloc(b, &b->d_vals, (size_t)n * (12 + 4 * kMaxCG + 4 * b->Lmax + 4 * (restart + 2)));
    if (e == cudaSuccess) e = balloc(b, &b->d_seeds, (size_t)n);
    if (e == cudaSuccess) e = balloc(b, &b->d_on, (size_t)n);
    if (e == cudaSuccess) e = balloc(b, &b->d_cyc, (size_t)n);
    if (e == cudaSuccess) e = balloc(b, &b->d_col, (size_t)4);
    if (e == cudaSuccess) e = balloc(b, &b->d_its, (size_t)n);
    if (e == cudaSuccess) e = balloc(b, &b->d_k, (size_t)n);
    if (e == cudaSuccess) e = balloc(b, &b->d_flags, (size_t)n);
    if (e == cudaSuccess) e = balloc(b, &b->d_count, (size_t)4);
    if (e == cudaSuccess) e = balloc(b, &b->d_fg, (size_t)n * fg_stride(restart));
    if (e == cudaSuccess) e = balloc(b, &b->d_prec, (size_t)n);
    if (e == cudaSuccess) e = balloc(b, &b->d_save, (size_t)n);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_status, sizeof(int) * (size_t)(n + 5));
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&b->ev_step[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = q1_batched_prepare();
    if (e == cudaSuccess) {
        int dev = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    }
    if (e == cudaSuccess) {
        std::vector<uint64_t> seeds(n);
        for (int i = 0; i < n; ++i) seeds[i] = b->hs[i]->prm.seed;
        e = cudaMemcpyAsync(b->d_seeds, seeds.data(), sizeof(uint64_t) * n, cudaMemcpyHostToDevice, b->stream);
    }
    if (e == cudaSuccess) e = upload(b);   // synchronises: the seeds' host vector may go
    if (e == cudaSuccess) b->dirty = false;
    return e;
}

// an instance a batch can hold: Q1, same dimension, stream, V-cycle precision and Chebyshev degree as
// the batch's first instance, P_full, no split, the Q1 fast path
bool batch_compatible(const pff_hierarchy* h, const pff_hierarchy* ref) {
    return h && h->mesh.degree == 1 && h->mesh.dim == ref->mesh.dim && h->stream == ref->stream &&
           h->prm.mg_precision == ref->prm.mg_precision && h->prm.preconditioner == 0 && h->prm.split == 0 &&
           h->prm.cheb_degree == ref->prm.cheb_degree && h->fast_q1;
}

pff_status b_fail(pff_batch* b, pff_status st, const std::string& msg) {
    if (b) b->err = msg;
    return st;
}

}  // namespace

#define BCUDA_OR_FAIL(b, ...)                                                                         \
    do {                                                                                              \
        cudaError_t e_ = (__VA_ARGS__);                                                               \
        if (e_ != cudaSuccess) return b_fail(b, PFF_ECUDA, std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// ensure every instance has a Krylov workspace of restart m (pff_api.cu)
extern pff_status pff_internal_ensure_krylov(pff_hierarchy* h, int m);

extern "C" pff_status pff_batch_create(int n, pff_hierarchy* const* hs, int restart, pff_batch** out) {
    if (!out) return PFF_EINVAL;
    *out = nullptr;
    if (n < 0 || (n > 0 && !hs) || restart < 1 || restart > 200) return PFF_EINVAL;
    for (int i = 0; i < n; ++i)
        if (!batch_compatible(hs[i], hs[0])) return PFF_EINVAL;
    pff_batch* b = new (std::nothrow) pff_batch();
    if (!b) return PFF_ENOMEM;
    b->m = restart;
    b->hs.assign(hs, hs + n);
    b->n = n;
    b->last.assign(n, pff_newton_info());
    b->dirty = true;
    if (n > 0) {
        b->dim = hs[0]->mesh.dim;
        b->mg64 = hs[0]->prm.mg_precision == 64;
        b->stream = hs[0]->stream;
        b->cheb_k = hs[0]->prm.cheb_degree;
        pff_status st = PFF_OK;
        for (auto* h : b->hs) {
            st = pff_internal_ensure_krylov(h, restart);
            if (st != PFF_OK) break;
        }
        if (st == PFF_OK) {
            cudaError_t e = build_state(b);
            if (e != cudaSuccess) st = e == cudaErrorMemoryAllocation ? PFF_ENOMEM : PFF_ECUDA;
        }
        if (st != PFF_OK) {
            cudaGetLastError();
            free_batch(b);
            return st;
        }
    }
    *out = b;
    return PFF_OK;
}

// rebuild the device state after submit/retire; an empty batch has nothing to run
static pff_status ensure_built(pff_batch* b) {
    if (b->n == 0) return b_fail(b, PFF_ESTATE, "the batch holds no instance");
    if (!b->dirty) return PFF_OK;
    BCUDA_OR_FAIL(b, cudaStreamSynchronize(b->stream));
    release_state(b);
    cudaError_t e = build_state(b);
    if (e != cudaSuccess) {
        cudaGetLastError();
        release_state(b);
        b->dirty = true;
        return b_fail(b, e == cudaErrorMemoryAllocation ? PFF_ENOMEM : PFF_ECUDA,
                      std::string("batch rebuild: ") + cudaGetErrorString(e));
    }
    return PFF_OK;
}

extern "C" pff_status pff_batch_submit(pff_batch* b, pff_hierarchy* h, int* index) {
    if (!b || !h) return PFF_EINVAL;
    if (b->n > 0 && !batch_compatible(h, b->hs[0]))
        return b_fail(b, PFF_EINVAL, "instance incompatible with the batch (dimension, stream, precision, options)");
    if (b->n == 0 && !batch_compatible(h, h)) return b_fail(b, PFF_EINVAL, "instance cannot be batched (Q1, P_full, no split)");
    for (auto* g : b->hs)
        if (g == h) return b_fail(b, PFF_EINVAL, "instance already in the batch");
    pff_status st = pff_internal_ensure_krylov(h, b->m);
    if (st != PFF_OK) return b_fail(b, st, "Krylov workspace of the submitted instance");
    if (b->n == 0) {
        b->dim = h->mesh.dim;
        b->mg64 = h->prm.mg_precision == 64;
        b->stream = h->stream;
        b->cheb_k = h->prm.cheb_degree;
    }
    b->hs.push_back(h);
    b->last.push_back(pff_newton_info());
    b->n = (int)b->hs.size();
    b->dirty = true;
    if (index) *index = b->n - 1;
    return PFF_OK;
}

extern "C" pff_status pff_batch_retire(pff_batch* b, int index) {
    if (!b) return PFF_EINVAL;
    if (index < 0 || index >= b->n) return b_fail(b, PFF_EINVAL, "index out of range");
    if (b->stream) BCUDA_OR_FAIL(b, cudaStreamSynchronize(b->stream));
    b->hs.erase(b->hs.begin() + index);
    b->last.erase(b->last.begin() + index);
    b->n = (int)b->hs.size();
    b->dirty = true;
    return PFF_OK;
}

extern "C" int pff_batch_size(const pff_batch* b) { return b ? b->n : -1; }

extern "C" pff_status pff_batch_poll(const pff_batch* b, int index, pff_newton_info* info) {
    if (!b || !info || index < 0 || index >= b->n) return PFF_EINVAL;
    *info = b->last[index];
    return PFF_OK;
}

extern "C" pff_status pff_batch_destroy(pff_batch* b) {
    if (!b) return PFF_OK;
    cudaStreamSynchronize(b->stream);
    free_batch(b);
    return PFF_OK;
}

extern "C" pff_status pff_batch_setup(pff_batch* b) {
    if (!b) return PFF_EINVAL;
    {
        const pff_status sb = ensure_built(b);
        if (sb != PFF_OK) return sb;
    }
    for (auto* h : b->hs)
        if (!h->has_state) return b_fail(b, PFF_ESTATE, "batch setup before pff_set_state of every instance");
    for (auto* h : b->hs) BCUDA_OR_FAIL(b, refresh_state(h));
    b->valid.assign(b->n, 1);
    BCUDA_OR_FAIL(b, upload(b));
    BCUDA_OR_FAIL(b, b_setup(b));
    return PFF_OK;
}

static pff_status ensure_batch_setup(pff_batch* b) {
    bool stale = b->stale;
    for (auto* h : b->hs) stale = stale || h->stale;
    if (stale) return pff_batch_setup(b);
    return PFF_OK;
}

extern "C" pff_status pff_batch_vcycle(pff_batch* b, const double* const* r, double* const* z) {
    if (!b || !r || !z) return PFF_EINVAL;
    {
        const pff_status sb = ensure_built(b);
        if (sb != PFF_OK) return sb;
    }
    pff_status st = ensure_batch_setup(b);
    if (st != PFF_OK) return st;
    for (int i = 0; i < b->n; ++i) {
        pff_hierarchy* h = b->hs[i];
        const size_t nd = (size_t)n_dofs(h->lv[h->L - 1].g);
        BCUDA_OR_FAIL(b, cudaMemcpyAsync(h->tmp64[1], r[i], nd * sizeof(double), cudaMemcpyDeviceToDevice, b->stream));
    }
    b->valid.assign(b->n, 1);
    BCUDA_OR_FAIL(b, upload(b));
    BCUDA_OR_FAIL(b, b_vcycle(b, bsel(BV_T64 + 1), bsel(BV_T64 + 2)));
    for (int i = 0; i < b->n; ++i) {
        pff_hierarchy* h = b->hs[i];
        const size_t nd = (size_t)n_dofs(h->lv[h->L - 1].g);
        BCUDA_OR_FAIL(b, cudaMemcpyAsync(z[i], h->tmp64[2], nd * sizeof(double), cudaMemcpyDeviceToDevice, b->stream));
    }
    return PFF_OK;
}

extern "C" pff_status pff_batch_gmres_solve(pff_batch* b, const double* const* rhs, double* const* x, double rtol,
                                            int maxit, pff_solve_info* info) {
    if (!b || !rhs || !x) return PFF_EINVAL;
    {
        const pff_status sb = ensure_built(b);
        if (sb != PFF_OK) return sb;
    }
    if (!(rtol > 0 && rtol < 1) || maxit < 1) return b_fail(b, PFF_EINVAL, "need 0 < rtol < 1 and maxit >= 1");
    pff_status st = ensure_batch_setup(b);
    if (st != PFF_OK) return st;
    for (int i = 0; i < b->n; ++i) {
        pff_hierarchy* h = b->hs[i];
        const size_t nd = (size_t)n_dofs(h->lv[h->L - 1].g);
        BCUDA_OR_FAIL(b, cudaMemcpyAsync(h->tmp64[1], rhs[i], nd * sizeof(double), cudaMemcpyDeviceToDevice, b->stream));
        BCUDA_OR_FAIL(b, cudaMemcpyAsync(h->tmp64[2], x[i], nd * sizeof(double), cudaMemcpyDeviceToDevice, b->stream));
    }
    st = b_fgmres(b, rtol, maxit, info);
    if (st != PFF_OK && st != PFF_ENOCONV) return st;
    for (int i = 0; i < b->n; ++i) {
        pff_hierarchy* h = b->hs[i];
        const size_t nd = (size_t)n_dofs(h->lv[h->L - 1].g);
        BCUDA_OR_FAIL(b, cudaMemcpyAsync(x[i], h->tmp64[2], nd * sizeof(double), cudaMemcpyDeviceToDevice, b->stream));
    }
    BCUDA_OR_FAIL(b, cudaStreamSynchronize(b->stream));
    return st;
}

// Newton step of every instance (Algorithm 1), the linear solves batched.
extern pff_status pff_internal_newton_prepare(pff_hierarchy* h, double* U, int* n_act, int* n_chg, double* res);
extern pff_status pff_internal_newton_finish(pff_hierarchy* h, double* U);

extern "C" pff_status pff_batch_newton_step(pff_batch* b, double* const* U, pff_newton_info* infos) {
    if (!b || !U) return PFF_EINVAL;
    {
        const pff_status sb = ensure_built(b);
        if (sb != PFF_OK) return sb;
    }
    const int n = b->n;
    std::vector<int> na(n), nc(n);
    std::vector<double> res(n);
    for (int i = 0; i < n; ++i) {
        pff_status st = pff_internal_newton_prepare(b->hs[i], U[i], &na[i], &nc[i], &res[i]);
        if (st != PFF_OK) return b_fail(b, st, "instance " + std::to_string(i) + ": " + b->hs[i]->err);
    }
    b->stale = true;
    pff_status st = ensure_batch_setup(b);
    if (st != PFF_OK) return st;
    // rhs R~ is in tmp64[1] of each instance; dU in tmp64[2] starts at 0
    for (int i = 0; i < n; ++i) {
        pff_hierarchy* h = b->hs[i];
        const size_t nd = (size_t)n_dofs(h->lv[h->L - 1].g);
        BCUDA_OR_FAIL(b, cudaMemsetAsync(h->tmp64[2], 0, nd * sizeof(double), b->stream));
    }
    std::vector<pff_solve_info> si(n);
    st = b_fgmres(b, b->hs[0]->prm.newton_rtol, 200, si.data());
    if (st != PFF_OK && st != PFF_ENOCONV) return st;
    for (int i = 0; i < n; ++i) {
        pff_status s2 = pff_internal_newton_finish(b->hs[i], U[i]);
        if (s2 != PFF_OK) return b_fail(b, s2, "instance " + std::to_string(i) + ": " + b->hs[i]->err);
        pff_newton_info& li = b->last[i];
        li.n_active = na[i];
        li.n_changed = nc[i];
        li.res_norm = res[i];
        li.solve = si[i];
        li.converged = (nc[i] == 0 && res[i] <= b->hs[i]->prm.tol_as) ? 1 : 0;
        if (infos) infos[i] = li;
    }
    BCUDA_OR_FAIL(b, cudaStreamSynchronize(b->stream));
    return st;
}

extern "C" pff_status pff_batch_set_kernel_style(pff_batch* b, int style) {
    if (!b) return PFF_EINVAL;
    if (style < 0 || style > 2) return b_fail(b, PFF_EINVAL, "kernel style must be 0, 1 or 2");
    b->style = style;
    return PFF_OK;
}

extern "C" pff_status pff_batch_set_precision_switch(pff_batch* b, int iterations) {
    if (!b) return PFF_EINVAL;
    if (iterations < 0) return b_fail(b, PFF_EINVAL, "iterations must be >= 0");
    b->switch_its = iterations;
    return PFF_OK;
}

extern "C" pff_status pff_batch_mg_precisions(pff_batch* b, int* precisions) {
    if (!b || !precisions) return PFF_EINVAL;
    {
        const pff_status sb = ensure_built(b);
        if (sb != PFF_OK) return sb;
    }
    BCUDA_OR_FAIL(b, cudaMemcpyAsync(precisions, b->d_prec, sizeof(int) * b->n, cudaMemcpyDeviceToHost, b->stream));
    BCUDA_OR_FAIL(b, cudaStreamSynchronize(b->stream));
    for (int i = 0; i < b->n; ++i)
        if (precisions[i] != 32 && precisions[i] != 64) precisions[i] = b->mg64 ? 64 : 32;   // before any solve
    return PFF_OK;
}

extern "C" pff_status pff_batch_tuning(pff_batch* b, int level, int precision, int* style, int* ctas_per_sm,
                                       double* ms) {
    if (!b) return PFF_EINVAL;
    if (precision != 32 && precision != 64) return b_fail(b, PFF_EINVAL, "precision must be 32 or 64");
    if (level < -1 || level >= b->Lmax) return b_fail(b, PFF_EINVAL, "level out of range");
    if (!b->tuned || b->dirty) return b_fail(b, PFF_ESTATE, "the batch has not been tuned (pff_batch_setup with style 0)");
    const pff_batch::Tune& t = b->tune[(size_t)(level < 0 ? b->Lmax : level) * 2 + (precision == 64 ? 1 : 0)];
    if (style) *style = t.style;
    if (ctas_per_sm) *ctas_per_sm = t.cps;
    if (ms) *ms = t.ms;
    return PFF_OK;
}

extern "C" pff_status pff_batch_apply_jacobian(pff_batch* b, int level, int precision, const void* const* x,
                                               void* const* y) {
    if (!b || !x || !y) return PFF_EINVAL;
    {
        const pff_status sb = ensure_built(b);
        if (sb != PFF_OK) return sb;
    }
    if (precision != 32 && precision != 64) return b_fail(b, PFF_EINVAL, "precision must be 32 or 64");
    if (level < -1 || level >= b->Lmax) return b_fail(b, PFF_EINVAL, "level out of range");
    for (auto* h : b->hs)
        if (!h->has_state) return b_fail(b, PFF_ESTATE, "batch apply before pff_set_state of every instance");
    for (auto* h : b->hs) BCUDA_OR_FAIL(b, refresh_state(h));
    const int l = level < 0 ? b->Lmax : level;
    const size_t es = precision == 64 ? sizeof(double) : sizeof(float);
    const int W = precision == 64 ? BV_W64 : BV_W32;
    b->valid.assign(b->n, 1);
    BCUDA_OR_FAIL(b, upload(b));
    auto vec_of = [&](int i, int k) -> std::pair<void*, size_t> {
        pff_hierarchy* h = b->hs[i];
        const int li = level < 0 ? h->L - 1 : level;
        if (li >= h->L) return {nullptr, 0};
        Level& L = h->lv[li];
        return {L.w[precision == 64 ? 1 : 0][k], (size_t)n_dofs(L.g) * es};
    };
    for (int i = 0; i < b->n; ++i) {
        auto v = vec_of(i, 3);
        if (v.first) BCUDA_OR_FAIL(b, cudaMemcpyAsync(v.first, x[i], v.second, cudaMemcpyDeviceToDevice, b->stream));
    }
    BCUDA_OR_FAIL(b, b_apply(b, l, precision == 64, false, bsel(W + 3), bsel(W + 4), PHI_BITS_ALL));
    for (int i = 0; i < b->n; ++i) {
        auto v = vec_of(i, 4);
        if (v.first) BCUDA_OR_FAIL(b, cudaMemcpyAsync(y[i], v.first, v.second, cudaMemcpyDeviceToDevice, b->stream));
    }
    return PFF_OK;
}

extern "C" const char* pff_batch_last_error(const pff_batch* b) { return b ? b->err.c_str() : "null batch"; }
