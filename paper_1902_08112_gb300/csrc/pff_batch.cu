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
#include <new>
#include <string>
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
    uint64_t* d_seeds = nullptr;
    int cheb_k = 4, coarse_k = 1;
    bool mg64 = false;                       // FP64 V-cycle (mg_precision 64 in every instance)
    int style = 0;                           // level-operator kernels: 0 by level size, 1 small-level, 2 per-cell
    bool stale = true;
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

BLevel make_desc(pff_hierarchy* h, int l, bool valid) {
    BLevel d;
    memset(&d, 0, sizeof(d));
    Level& L = h->lv[l];
    d.g = L.g;
    d.valid = valid ? 1 : 0;
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
            BLevel d = make_desc(h, has ? li : 0, has && b->valid[i]);
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
    // the host vectors are reused at the next upload: make the copies complete first
    return cudaStreamSynchronize(b->stream);
}

const BLevel* tab(pff_batch* b, int l) { return l == b->Lmax ? b->d_fine : b->d_lv + (size_t)l * b->n; }

// y(sy) = G~ x(sx) on level l (l == Lmax: each instance's finest level), precision by fp64
cudaError_t b_apply(pff_batch* b, int l, bool fp64, bool blockdiag, int sx, int sy, int phi_bits, bool preset = true) {
    const BLevel* L = tab(b, l);
    // 3D levels of at least kCellMinCells cells over the batch: the per-cell kernel with
    // shared-memory derivatives, on the tiles of the FP32 per-cell style
    const bool cell = b->dim == 3 && q1_cell_tiles_match_f32() &&
                      (b->style == 2 || (b->style == 0 && b->cells[l] >= kCellMinCells));
    const int st = (fp64 && !cell) ? kStyleF64 : kStyleF32;
    if (preset) {
        if (fp64) BCK(bl_init_masked<double>(L, b->n, b->blocks[l], sx, sy, phi_bits, 0.0, b->stream));
        else BCK(bl_init_masked<float>(L, b->n, b->blocks[l], sx, sy, phi_bits, 0.f, b->stream));
    }
    return launch_q1_apply_batched(b->dim, fp64, blockdiag, fp64, L, b->n,
                                   b->d_tiles + ((size_t)l * 2 + st) * (b->n + 1), b->tot[(size_t)l * 2 + st], sx, sy,
                                   phi_bits, b->stream, cell);
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
    if (b->d_coef) {
        for (auto it = b->allocs.begin(); it != b->allocs.end(); ++it)
            if (*it == b->d_coef) { cudaFree(*it); b->allocs.erase(it); break; }
        b->d_coef = nullptr;
    }
    BCK(balloc(b, &b->d_coef, coef.size()));
    BCK(cudaMemcpyAsync(b->d_coef, coef.data(), sizeof(double) * coef.size(), cudaMemcpyHostToDevice, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    for (auto* h : b->hs) h->stale = false;
    b->stale = false;
    return cudaSuccess;
}

// ---------------------------------------------------------------- batched FGMRES
// solve G~ x = b per instance: b in T64[1], x in T64[2] (fine selectors)
pff_status b_fgmres(pff_batch* b, double rtol, int maxit, pff_solve_info* info) {
    const int n = b->n, m = b->m, F = b->Lmax;
    cudaStream_t s = b->stream;
    const int sb = bsel(BV_T64 + 1), sx = bsel(BV_T64 + 2), sw = bsel(BV_T64 + 0);
    double* d_nrm = b->d_vals;                              // n
    double* d_h = b->d_vals + n;                            // n * 2(m+1)  (h1 | h2)
    double* d_y = d_h + (size_t)n * 2 * (m + 1);            // n * m
    std::vector<double> beta0(n), beta(n), target(n), hv((size_t)n * 2 * (m + 1)), nrm(n);
    std::vector<int> its(n, 0);
    std::vector<char> all(n, 1);
    auto fail = [&](cudaError_t e) {
        b->err = std::string("batched FGMRES: ") + cudaGetErrorString(e);
        return PFF_ECUDA;
    };
#define BKC(...)                            \
    do {                                    \
        cudaError_t e_ = (__VA_ARGS__);     \
        if (e_ != cudaSuccess) return fail(e_); \
    } while (0)
    auto true_res = [&](std::vector<double>& out) -> cudaError_t {
        BCK(b_apply(b, F, true, false, sx, sw, PHI_BITS_ALL));
        BCK(bl_sub<double>(tab(b, F), n, b->blocks[F], sb, sw, sw, s));
        BCK(bl_norm(tab(b, F), n, sw, b->d_part, d_nrm, s));
        BCK(cudaMemcpyAsync(out.data(), d_nrm, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
        return cudaStreamSynchronize(s);
    };
    b->valid = all;
    BKC(upload(b));
    BKC(true_res(beta0));
    for (int i = 0; i < n; ++i) {
        if (!std::isfinite(beta0[i])) {
            b->err = "non-finite initial residual in instance " + std::to_string(i);
            return PFF_ENONFINITE;
        }
        target[i] = rtol * beta0[i];
    }
    beta = beta0;
    std::vector<std::vector<double>> H(n), g(n), cs(n), sn(n);
    bool first = true;
    while (true) {
        if (!first) {
            b->valid = all;
            BKC(upload(b));
            BKC(true_res(beta));
        }
        first = false;
        std::vector<char> act(n, 0);
        int nact = 0;
        for (int i = 0; i < n; ++i) {
            if (!std::isfinite(beta[i])) {
                b->err = "non-finite residual in instance " + std::to_string(i);
                return PFF_ENONFINITE;
            }
            act[i] = !(beta[i] <= target[i] || its[i] >= maxit || beta[i] == 0.0);
            nact += act[i];
        }
        if (!nact) break;
        b->valid = act;
        BKC(upload(b));
        BKC(bl_axpby64(tab(b, F), n, b->blocks[F], d_nrm, sw, 0.0, bsel(BV_KV, 0), 1, s));   // V0 = w / beta
        std::vector<int> k(n, 0);
        for (int i = 0; i < n; ++i) {
            H[i].assign((size_t)(m + 1) * m, 0.0);
            g[i].assign(m + 1, 0.0);
            cs[i].assign(m, 0.0);
            sn[i].assign(m, 0.0);
            g[i][0] = beta[i];
        }
        std::vector<char> inner = act;
        for (int j = 0; j < m; ++j) {
            BKC(b_vcycle(b, bsel(BV_KV, j), bsel(BV_KZ, j)));
            BKC(b_apply(b, F, true, false, bsel(BV_KZ, j), bsel(BV_KV, j + 1), PHI_BITS_ALL));
            const int vn = bsel(BV_KV, j + 1);
            BKC(bl_multidot(tab(b, F), n, j + 1, vn, b->d_part, m + 1, d_h, 2 * (m + 1), s));
            BKC(bl_multi_axpy(tab(b, F), n, b->blocks[F], j + 1, d_h, 2 * (m + 1), vn, s));
            BKC(bl_multidot(tab(b, F), n, j + 1, vn, b->d_part, m + 1, d_h + (m + 1), 2 * (m + 1), s));
            BKC(bl_multi_axpy(tab(b, F), n, b->blocks[F], j + 1, d_h + (m + 1), 2 * (m + 1), vn, s));
            BKC(bl_norm(tab(b, F), n, vn, b->d_part, d_nrm, s));
            BKC(bl_axpby64(tab(b, F), n, b->blocks[F], d_nrm, vn, 0.0, vn, 1, s));
            BKC(cudaMemcpyAsync(hv.data(), d_h, sizeof(double) * hv.size(), cudaMemcpyDeviceToHost, s));
            BKC(cudaMemcpyAsync(nrm.data(), d_nrm, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
            BKC(cudaStreamSynchronize(s));
            bool changed = false;
            int left = 0;
            for (int i = 0; i < n; ++i) {
                if (!inner[i]) continue;
                const double* hi = &hv[(size_t)i * 2 * (m + 1)];
                std::vector<double>& Hi = H[i];
                for (int r = 0; r <= j; ++r) Hi[(size_t)r * m + j] = hi[r] + hi[(m + 1) + r];
                if (!std::isfinite(nrm[i])) {
                    b->err = "non-finite Arnoldi norm in instance " + std::to_string(i);
                    return PFF_ENONFINITE;
                }
                Hi[(size_t)(j + 1) * m + j] = nrm[i];
                for (int r = 0; r < j; ++r) {
                    const double t = cs[i][r] * Hi[(size_t)r * m + j] + sn[i][r] * Hi[(size_t)(r + 1) * m + j];
                    Hi[(size_t)(r + 1) * m + j] = -sn[i][r] * Hi[(size_t)r * m + j] + cs[i][r] * Hi[(size_t)(r + 1) * m + j];
                    Hi[(size_t)r * m + j] = t;
                }
                const double den = hypot(Hi[(size_t)j * m + j], Hi[(size_t)(j + 1) * m + j]);
                cs[i][j] = Hi[(size_t)j * m + j] / den;
                sn[i][j] = Hi[(size_t)(j + 1) * m + j] / den;
                Hi[(size_t)j * m + j] = den;
                Hi[(size_t)(j + 1) * m + j] = 0.0;
                g[i][j + 1] = -sn[i][j] * g[i][j];
                g[i][j] = cs[i][j] * g[i][j];
                ++its[i];
                k[i] = j + 1;
                if (fabs(g[i][j + 1]) <= target[i] || its[i] >= maxit) {
                    inner[i] = 0;
                    changed = true;
                } else {
                    ++left;
                }
            }
            if (!left) break;
            if (changed) {
                b->valid = inner;
                BKC(upload(b));
            }
        }
        // x += Z y for the instances of this cycle
        std::vector<double> y((size_t)n * m, 0.0);
        for (int i = 0; i < n; ++i) {
            if (!act[i]) continue;
            for (int r = k[i] - 1; r >= 0; --r) {
                double acc = g[i][r];
                for (int c = r + 1; c < k[i]; ++c) acc -= H[i][(size_t)r * m + c] * y[(size_t)i * m + c];
                y[(size_t)i * m + r] = acc / H[i][(size_t)r * m + r];
            }
        }
        b->valid = act;
        BKC(upload(b));
        BKC(cudaMemcpyAsync(d_y, y.data(), sizeof(double) * y.size(), cudaMemcpyHostToDevice, s));
        int kmax = 0;
        for (int i = 0; i < n; ++i) kmax = std::max(kmax, act[i] ? k[i] : 0);
        BKC(bl_gemv_add(tab(b, F), n, b->blocks[F], kmax, d_y, m, sx, s));
        BKC(cudaStreamSynchronize(s));
    }
    std::vector<double> res(n);
    b->valid = all;
    BKC(upload(b));
    BKC(true_res(res));
#undef BKC
    pff_status st = PFF_OK;
    for (int i = 0; i < n; ++i) {
        const bool conv = res[i] <= target[i] * (1.0 + 1e-12) || beta0[i] == 0.0;
        if (info) {
            info[i].iterations = its[i];
            info[i].res0 = beta0[i];
            info[i].res_final = res[i];
            info[i].converged = conv ? 1 : 0;
        }
        if (!std::isfinite(res[i])) {
            b->err = "non-finite final residual";
            st = PFF_ENONFINITE;
        } else if (!conv && st == PFF_OK) {
            b->err = "batched FGMRES reached maxit";
            st = PFF_ENOCONV;
        }
    }
    return st;
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
    if (n < 1 || !hs || restart < 1 || restart > 200) return PFF_EINVAL;
    for (int i = 0; i < n; ++i) {
        if (!hs[i]) return PFF_EINVAL;
        if (hs[i]->mesh.degree != 1 || hs[i]->mesh.dim != hs[0]->mesh.dim) return PFF_EINVAL;
        if (hs[i]->stream != hs[0]->stream) return PFF_EINVAL;
        if (hs[i]->prm.mg_precision != hs[0]->prm.mg_precision || hs[i]->prm.preconditioner != 0 || hs[i]->prm.split != 0 || hs[i]->prm.cheb_degree != hs[0]->prm.cheb_degree) return PFF_EINVAL;
        if (!hs[i]->fast_q1) return PFF_EINVAL;
    }
    pff_batch* b = new (std::nothrow) pff_batch();
    if (!b) return PFF_ENOMEM;
    b->n = n;
    b->dim = hs[0]->mesh.dim;
    b->m = restart;
    b->mg64 = hs[0]->prm.mg_precision == 64;
    b->hs.assign(hs, hs + n);
    b->stream = hs[0]->stream;
    b->cheb_k = hs[0]->prm.cheb_degree;
    for (auto* h : b->hs) b->Lmax = std::max(b->Lmax, h->L);
    b->valid.assign(n, 1);
    b->h_lv.assign(b->Lmax, std::vector<BLevel>(n));
    b->h_fine.resize(n);
    pff_status st = PFF_OK;
    for (auto* h : b->hs) {
        st = pff_internal_ensure_krylov(h, restart);
        if (st != PFF_OK) break;
    }
    cudaError_t e = cudaSuccess;
    if (st == PFF_OK) {
        e = balloc(b, &b->d_lv, (size_t)b->Lmax * n);
        if (e == cudaSuccess) e = balloc(b, &b->d_fine, (size_t)n);
        if (e == cudaSuccess) e = balloc(b, &b->d_tiles, (size_t)(b->Lmax + 1) * 2 * (n + 1));
        if (e == cudaSuccess) e = balloc(b, &b->d_part, (size_t)n * (restart + 2) * kBPartials * 2);
        if (e == cudaSuccess) e = balloc(b, &b->d_vals, (size_t)n * (12 + 4 * kMaxCG + 4 * b->Lmax + 4 * (restart + 2)));
        if (e == cudaSuccess) e = balloc(b, &b->d_seeds, (size_t)n);
        if (e == cudaSuccess) {
            std::vector<uint64_t> seeds(n);
            for (int i = 0; i < n; ++i) seeds[i] = b->hs[i]->prm.seed;
            e = cudaMemcpyAsync(b->d_seeds, seeds.data(), sizeof(uint64_t) * n, cudaMemcpyHostToDevice, b->stream);
        }
        if (e == cudaSuccess) e = upload(b);
        if (e != cudaSuccess) st = e == cudaErrorMemoryAllocation ? PFF_ENOMEM : PFF_ECUDA;
    }
    if (st != PFF_OK) {
        cudaGetLastError();
        for (void* p : b->allocs) cudaFree(p);
        delete b;
        return st;
    }
    *out = b;
    return PFF_OK;
}

extern "C" pff_status pff_batch_destroy(pff_batch* b) {
    if (!b) return PFF_OK;
    cudaStreamSynchronize(b->stream);
    for (void* p : b->allocs) cudaFree(p);
    delete b;
    return PFF_OK;
}

extern "C" pff_status pff_batch_setup(pff_batch* b) {
    if (!b) return PFF_EINVAL;
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
    st = b_fgmres(b, 1e-8, 200, si.data());
    if (st != PFF_OK && st != PFF_ENOCONV) return st;
    for (int i = 0; i < n; ++i) {
        pff_status s2 = pff_internal_newton_finish(b->hs[i], U[i]);
        if (s2 != PFF_OK) return b_fail(b, s2, "instance " + std::to_string(i) + ": " + b->hs[i]->err);
        if (infos) {
            infos[i].n_active = na[i];
            infos[i].n_changed = nc[i];
            infos[i].res_norm = res[i];
            infos[i].solve = si[i];
            infos[i].converged = (nc[i] == 0 && res[i] <= b->hs[i]->prm.tol_as) ? 1 : 0;
        }
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

extern "C" pff_status pff_batch_apply_jacobian(pff_batch* b, int level, int precision, const void* const* x,
                                               void* const* y) {
    if (!b || !x || !y) return PFF_EINVAL;
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
