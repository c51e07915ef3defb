// Batched element-wise, transfer and reduction kernels: grid.y = instance, grid.x strides over
// that instance's vector at one level.  Instances without the level (BLevel::valid == 0) exit.
// Reductions are two-stage with a fixed number of partials per instance, so results do not
// depend on which other instances share the launch.
#include "pff_batch.cuh"
#include "pff_batch_kernels.cuh"

namespace pff {

static constexpr int kT = 256;

#define BSTRIDE(i, n) \
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

__device__ __forceinline__ bool belim(uint8_t m, int c, int dim, int phi_bits) {
    return c < dim ? ((m >> c) & 1) != 0 : (m & phi_bits) != 0;
}

template <typename T>
__global__ void kb_init_masked(const BLevel* __restrict__ L, int sx, int sy, int phi_bits, T elim_val) {
    const BLevel& d = L[blockIdx.y];
    if (!bon(d)) return;
    const int64_t nn = d.g.n_nodes, nd = n_dofs(d.g);
    const T* x = sx >= 0 ? bvec<T>(d, sx) : nullptr;
    T* y = bvec<T>(d, sy);
    BSTRIDE(i, nd) {
        const int c = dof_comp(i, nn);
        const bool e = belim(d.mask[i - c * nn], c, d.g.dim, phi_bits);
        y[i] = e ? (x ? x[i] : elim_val) : T(0);
    }
}

// Chebyshev step with per-instance coefficients coef[inst * 4 + (c1u, c1p, c2u, c2p)]; with
// stn >= 0 it also writes the preset of the next apply into stn (d on eliminated rows, else 0)
template <typename T>
__global__ void kb_cheb(const BLevel* __restrict__ L, int sr, int st, int sd, int sx, const double* __restrict__ coef,
                        int first, int stn) {
    const BLevel& d = L[blockIdx.y];
    if (!bon(d)) return;
    const int64_t nd = n_dofs(d.g), nu = d.g.n_nodes * d.g.dim;
    const double* cf = coef + 4 * blockIdx.y;
    const T c1u = (T)cf[0], c1p = (T)cf[1], c2u = (T)cf[2], c2p = (T)cf[3];
    T* r = bvec<T>(d, sr);
    const T* t = st >= 0 ? bvec<T>(d, st) : nullptr;
    T* dd = bvec<T>(d, sd);
    T* x = bvec<T>(d, sx);
    T* tn = stn >= 0 ? bvec<T>(d, stn) : nullptr;
    const int64_t nn = d.g.n_nodes;
    const T* dinv = sizeof(T) == 8 ? (const T*)d.dinv64 : (const T*)d.dinv32;
    BSTRIDE(i, nd) {
        const bool u = i < nu;
        const T c1 = u ? c1u : c1p, c2 = u ? c2u : c2p;
        T di;
        if (first) {
            di = c2 * dinv[i] * r[i];
            x[i] = first == 1 ? di : x[i] + di;
        } else {
            const T ri = r[i] - t[i];
            r[i] = ri;
            di = c1 * dd[i] + c2 * dinv[i] * ri;
            x[i] += di;
        }
        dd[i] = di;
        if (tn) {
            const int c = dof_comp(i, nn);
            tn[i] = belim(d.mask[i - c * nn], c, d.g.dim, PHI_BITS_ALL) ? di : T(0);
        }
    }
}

template <typename T>
__global__ void kb_sub(const BLevel* __restrict__ L, int sa, int sb, int sc) {
    const BLevel& d = L[blockIdx.y];
    if (!bon(d)) return;
    const int64_t nd = n_dofs(d.g);
    const T* a = bvec<T>(d, sa);
    const T* b = bvec<T>(d, sb);
    T* c = bvec<T>(d, sc);
    BSTRIDE(i, nd) c[i] = a[i] - b[i];
}

template <typename T>
__global__ void kb_copy(const BLevel* __restrict__ L, int ss, int sd, int block) {
    const BLevel& d = L[blockIdx.y];
    if (!bon(d)) return;
    const int64_t nd = n_dofs(d.g), nu = d.g.n_nodes * d.g.dim;
    const T* s = bvec<T>(d, ss);
    T* t = bvec<T>(d, sd);
    BSTRIDE(i, nd) {
        const bool keep = block < 0 || (block == 0 ? i < nu : i >= nu);
        t[i] = keep ? s[i] : T(0);
    }
}

// dst (To) = free ? (To) src : (free_only ? 0 : dst-unchanged...) ; mode 0: dst = (To) src on all
// entries, mode 1: dst = free ? src : 0, mode 2: dst = eliminated ? src : dst
template <typename Ti, typename To>
__global__ void kb_convert(const BLevel* __restrict__ L, int ss, int sd, int mode) {
    const BLevel& d = L[blockIdx.y];
    if (!bon(d)) return;
    const int64_t nn = d.g.n_nodes, nd = n_dofs(d.g);
    const Ti* s = bvec<Ti>(d, ss);
    To* t = bvec<To>(d, sd);
    BSTRIDE(i, nd) {
        if (mode == 0) { t[i] = (To)s[i]; continue; }
        const int c = dof_comp(i, nn);
        const bool e = belim(d.mask[i - c * nn], c, d.g.dim, PHI_BITS_ALL);
        if (mode == 1) t[i] = e ? To(0) : (To)s[i];
        else if (e) t[i] = (To)s[i];
    }
}

// y = a x + b y with per-instance scalars a_i = sa[inst], b_i = sb (host constant) or per instance
__global__ void kb_axpby64(const BLevel* __restrict__ L, const double* __restrict__ a, int sx, double b, int sy,
                           int invert_a) {
    const BLevel& d = L[blockIdx.y];
    if (!bon(d)) return;
    const int64_t nd = n_dofs(d.g);
    double ai = a ? a[blockIdx.y] : 1.0;
    if (invert_a) ai = ai > 0.0 ? 1.0 / ai : 0.0;
    const double* x = bvec<double>(d, sx);
    double* y = bvec<double>(d, sy);
    BSTRIDE(i, nd) y[i] = b == 0.0 ? ai * x[i] : ai * x[i] + b * y[i];
}

// ---------------------------------------------------------------- transfers
template <typename T>
__device__ __forceinline__ T bp1w(int i, int I, int nc) {   // Q1 only
    int m = i / 2;
    if (m > nc - 1) m = nc - 1;
    const int a = I - m;
    if (a < 0 || a > 1) return T(0);
    const T t = T(i - 2 * m) / T(2);
    return a == 0 ? T(1) - t : t;
}

template <typename T>
__global__ void kb_restrict(const BLevel* __restrict__ Lc, const BLevel* __restrict__ Lf, int sf, int sc) {
    const BLevel& F = Lf[blockIdx.y];
    const BLevel& C = Lc[blockIdx.y];
    if (!bon(F) || !bon(C)) return;
    const Geom& gc = C.g;
    const Geom& gf = F.g;
    const T* rf = bvec<T>(F, sf);
    T* rc = bvec<T>(C, sc);
    BSTRIDE(n, gc.n_nodes) {
        const int I = (int)(n % gc.nn[0]);
        const int64_t r = n / gc.nn[0];
        const int J = (int)(r % gc.nn[1]), K = (int)(r / gc.nn[1]);
        T acc[4] = {T(0), T(0), T(0), T(0)};
        const int k0 = gc.dim == 3 ? max(0, 2 * K - 1) : 0, k1 = gc.dim == 3 ? min(gf.nn[2] - 1, 2 * K + 1) : 0;
        for (int k = k0; k <= k1; ++k) {
            const T wk = gc.dim == 3 ? bp1w<T>(k, K, gc.nc[2]) : T(1);
            if (wk == T(0)) continue;
            for (int j = max(0, 2 * J - 1); j <= min(gf.nn[1] - 1, 2 * J + 1); ++j) {
                const T wj = bp1w<T>(j, J, gc.nc[1]);
                if (wj == T(0)) continue;
                for (int i = max(0, 2 * I - 1); i <= min(gf.nn[0] - 1, 2 * I + 1); ++i) {
                    const T wi = bp1w<T>(i, I, gc.nc[0]);
                    if (wi == T(0)) continue;
                    const T w = wi * wj * wk;
                    const int64_t f = (int64_t)i + (int64_t)gf.nn[0] * ((int64_t)j + (int64_t)gf.nn[1] * k);
                    for (int c = 0; c <= gc.dim; ++c) acc[c] += w * rf[c * gf.n_nodes + f];
                }
            }
        }
        const uint8_t m = C.mask[n];
        for (int c = 0; c <= gc.dim; ++c) rc[c * gc.n_nodes + n] = belim(m, c, gc.dim, PHI_BITS_ALL) ? T(0) : acc[c];
    }
}

template <typename T>
__global__ void kb_prolongate_add(const BLevel* __restrict__ Lc, const BLevel* __restrict__ Lf, int sc, int sf) {
    const BLevel& F = Lf[blockIdx.y];
    const BLevel& C = Lc[blockIdx.y];
    if (!bon(F) || !bon(C)) return;
    const Geom& gc = C.g;
    const Geom& gf = F.g;
    const T* ec = bvec<T>(C, sc);
    T* xf = bvec<T>(F, sf);
    BSTRIDE(n, gf.n_nodes) {
        int idx[3];
        idx[0] = (int)(n % gf.nn[0]);
        const int64_t r = n / gf.nn[0];
        idx[1] = (int)(r % gf.nn[1]);
        idx[2] = (int)(r / gf.nn[1]);
        int cell[3];
        for (int a = 0; a < 3; ++a) {
            if (a >= gc.dim) { cell[a] = 0; continue; }
            int m = idx[a] / 2;
            if (m > gc.nc[a] - 1) m = gc.nc[a] - 1;
            cell[a] = m;
        }
        T acc[4] = {T(0), T(0), T(0), T(0)};
        for (int c2 = 0; c2 <= (gc.dim == 3 ? 1 : 0); ++c2) {
            const int K = cell[2] + c2;
            const T wk = gc.dim == 3 ? bp1w<T>(idx[2], K, gc.nc[2]) : T(1);
            if (wk == T(0)) continue;
            for (int b = 0; b <= 1; ++b) {
                const int J = cell[1] + b;
                const T wj = bp1w<T>(idx[1], J, gc.nc[1]);
                if (wj == T(0)) continue;
                for (int a = 0; a <= 1; ++a) {
                    const int I = cell[0] + a;
                    const T wi = bp1w<T>(idx[0], I, gc.nc[0]);
                    if (wi == T(0)) continue;
                    const T w = wi * wj * wk;
                    const int64_t cn = (int64_t)I + (int64_t)gc.nn[0] * ((int64_t)J + (int64_t)gc.nn[1] * K);
                    for (int c = 0; c <= gc.dim; ++c) acc[c] += w * ec[c * gc.n_nodes + cn];
                }
            }
        }
        const uint8_t m = F.mask[n];
        for (int c = 0; c <= gf.dim; ++c)
            if (!belim(m, c, gf.dim, PHI_BITS_ALL)) xf[c * gf.n_nodes + n] += acc[c];
    }
}

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ double bwarp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double bblock_sum(double v) {
    __shared__ double sh[32];
    v = bwarp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (w == 0) {
        r = l < (int)(blockDim.x >> 5) ? sh[l] : 0.0;
        r = bwarp_sum(r);
    }
    return r;   // valid in thread 0
}

// per-instance dots over the u and phi blocks: part[(inst * P + blk) * 2 + b]
template <typename T>
__global__ void kb_dots2_partial(const BLevel* __restrict__ L, int sa, int sb, double* __restrict__ part) {
    const BLevel& d = L[blockIdx.y];
    double su = 0.0, sp = 0.0;
    if (bon(d)) {
        const int64_t nd = n_dofs(d.g), nu = d.g.n_nodes * d.g.dim;
        const T* a = bvec<T>(d, sa);
        const T* b = bvec<T>(d, sb);
        BSTRIDE(i, nd) {
            const double v = (double)a[i] * (double)b[i];
            if (i < nu) su += v; else sp += v;
        }
    }
    su = bblock_sum(su);
    sp = bblock_sum(sp);
    if (threadIdx.x == 0) {
        part[((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * 2] = su;
        part[((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * 2 + 1] = sp;
    }
}
__global__ void kb_dots2_final(const double* __restrict__ part, int P, double* __restrict__ out) {
    double su = 0.0, sp = 0.0;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        su += part[((int64_t)blockIdx.x * P + i) * 2];
        sp += part[((int64_t)blockIdx.x * P + i) * 2 + 1];
    }
    su = bblock_sum(su);
    sp = bblock_sum(sp);
    if (threadIdx.x == 0) {
        out[2 * blockIdx.x] = su;
        out[2 * blockIdx.x + 1] = sp;
    }
}

// FGMRES on the finest levels: h[inst * ldh + j] = V_j . w for j < k (two stages)
// <V_j, w> for j < k, eight basis vectors per pass over w (their sums kept in registers)
// k < 0: k = (*kcol) + 1, the column counter of the batch (captured Arnoldi steps)
__global__ void kb_multidot_partial(const BLevel* __restrict__ L, int k, const int* __restrict__ kcol, int sw,
                                    double* __restrict__ part, int kmax) {
    constexpr int G = 8;
    const BLevel& d = L[blockIdx.y];
    if (k < 0) k = *kcol + 1;
    const bool on = bon(d);
    const int64_t nd = on ? n_dofs(d.g) : 0;
    const double* w = on ? bvec<double>(d, sw) : nullptr;
    const double* V = on ? bvec<double>(d, bsel(BV_KV, 0)) : nullptr;
    for (int j0 = 0; j0 < k; j0 += G) {
        const int kk = min(G, k - j0);
        double s[G];
#pragma unroll
        for (int t = 0; t < G; ++t) s[t] = 0.0;
        if (on) {
            BSTRIDE(i, nd) {
                const double wi = w[i];
#pragma unroll
                for (int t = 0; t < G; ++t)
                    if (t < kk) s[t] += V[(int64_t)(j0 + t) * nd + i] * wi;
            }
        }
        for (int t = 0; t < kk; ++t) {
            const double v = bblock_sum(s[t]);
            if (threadIdx.x == 0) part[((int64_t)blockIdx.y * kmax + j0 + t) * gridDim.x + blockIdx.x] = v;
        }
    }
}
__global__ void kb_multidot_final(const double* __restrict__ part, int P, int k, const int* __restrict__ kcol, int kmax,
                                  double* __restrict__ h, int ldh) {
    const int wid = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (k < 0) k = *kcol + 1;
    for (int j = wid; j < k; j += nw) {
        double s = 0.0;
        for (int i = l; i < P; i += 32) s += part[((int64_t)blockIdx.x * kmax + j) * P + i];
        s = bwarp_sum(s);
        if (l == 0) h[(int64_t)blockIdx.x * ldh + j] = s;
    }
}
__global__ void kb_multi_axpy(const BLevel* __restrict__ L, int k, const int* __restrict__ kcol,
                              const double* __restrict__ h, int ldh, int sw) {
    const BLevel& d = L[blockIdx.y];
    if (!bon(d)) return;
    if (k < 0) k = *kcol + 1;
    const int64_t nd = n_dofs(d.g);
    double* w = bvec<double>(d, sw);
    const double* hh = h + (int64_t)blockIdx.y * ldh;
    const double* V = bvec<double>(d, bsel(BV_KV, 0));
    BSTRIDE(i, nd) {
        double s = w[i];
        for (int j = 0; j < k; ++j) s -= hh[j] * V[(int64_t)j * nd + i];
        w[i] = s;
    }
}
__global__ void kb_norm_partial(const BLevel* __restrict__ L, int sw, double* __restrict__ part) {
    const BLevel& d = L[blockIdx.y];
    double s = 0.0;
    if (bon(d)) {
        const int64_t nd = n_dofs(d.g);
        const double* w = bvec<double>(d, sw);
        BSTRIDE(i, nd) s += w[i] * w[i];
    }
    s = bblock_sum(s);
    if (threadIdx.x == 0) part[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = s;
}
__global__ void kb_norm_final(const double* __restrict__ part, int P, double* __restrict__ out) {
    double s = 0.0;
    for (int i = threadIdx.x; i < P; i += blockDim.x) s += part[(int64_t)blockIdx.x * P + i];
    s = bblock_sum(s);
    if (threadIdx.x == 0) out[blockIdx.x] = sqrt(s);
}
// x += Z y_inst
// kk (nullable): per-instance k
__global__ void kb_gemv_add(const BLevel* __restrict__ L, int k, const int* __restrict__ kk, const double* __restrict__ y,
                            int ldy, int sx) {
    const BLevel& d = L[blockIdx.y];
    if (!bon(d)) return;
    if (kk) k = kk[blockIdx.y];
    const int64_t nd = n_dofs(d.g);
    double* x = bvec<double>(d, sx);
    const double* yy = y + (int64_t)blockIdx.y * ldy;
    const double* Z = bvec<double>(d, bsel(BV_KZ, 0));
    BSTRIDE(i, nd) {
        double s = x[i];
        for (int j = 0; j < k; ++j) s += yy[j] * Z[(int64_t)j * nd + i];
        x[i] = s;
    }
}

// ---------------------------------------------------------------- CG pieces
// per-instance r -= alpha q; z = dinv r   (alpha2[inst*2 + b])
template <typename T>
__global__ void kb_cg_r(const BLevel* __restrict__ L, int sr, int sq, int sz, const double* __restrict__ alpha2) {
    const BLevel& d = L[blockIdx.y];
    if (!bon(d)) return;
    const int64_t nd = n_dofs(d.g), nu = d.g.n_nodes * d.g.dim;
    const T au = (T)alpha2[2 * blockIdx.y], ap = (T)alpha2[2 * blockIdx.y + 1];
    T* r = bvec<T>(d, sr);
    const T* q = bvec<T>(d, sq);
    T* z = bvec<T>(d, sz);
    const T* dinv = sizeof(T) == 8 ? (const T*)d.dinv64 : (const T*)d.dinv32;
    BSTRIDE(i, nd) {
        const T ri = r[i] - (i < nu ? au : ap) * q[i];
        r[i] = ri;
        z[i] = dinv[i] * ri;
    }
}
template <typename T>
__global__ void kb_cg_p(const BLevel* __restrict__ L, int sp, int sz, const double* __restrict__ beta2) {
    const BLevel& d = L[blockIdx.y];
    if (!bon(d)) return;
    const int64_t nd = n_dofs(d.g), nu = d.g.n_nodes * d.g.dim;
    const T bu = (T)beta2[2 * blockIdx.y], bp = (T)beta2[2 * blockIdx.y + 1];
    T* p = bvec<T>(d, sp);
    const T* z = bvec<T>(d, sz);
    BSTRIDE(i, nd) p[i] = z[i] + (i < nu ? bu : bp) * p[i];
}
__device__ __forceinline__ uint64_t bsplitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
template <typename T>
__global__ void kb_start_vector(const BLevel* __restrict__ L, int sv, const uint64_t* __restrict__ seeds, int level) {
    const BLevel& d = L[blockIdx.y];
    if (!bon(d)) return;
    const int64_t nn = d.g.n_nodes, nd = n_dofs(d.g);
    T* v = bvec<T>(d, sv);
    const uint64_t seed = seeds[blockIdx.y];
    BSTRIDE(i, nd) {
        const int c = dof_comp(i, nn);
        const uint64_t key = seed + (uint64_t)level * (1ull << 40) + (uint64_t)i;
        const double u = (double)(bsplitmix64(key) >> 11) * 0x1.0p-53;
        v[i] = belim(d.mask[i - c * nn], c, d.g.dim, PHI_BITS_ALL) ? T(0) : T(2.0 * u - 1.0);
    }
}

// ---------------------------------------------------------------- launchers
static dim3 bgrid(int blocks, int n) { return dim3(blocks, n, 1); }

template <typename T>
cudaError_t bl_init_masked(const BLevel* L, int n, int blocks, int sx, int sy, int phi_bits, T v, cudaStream_t s) {
    kb_init_masked<T><<<bgrid(blocks, n), kT, 0, s>>>(L, sx, sy, phi_bits, v);
    return count_launch(cudaGetLastError());
}
template <typename T>
cudaError_t bl_cheb(const BLevel* L, int n, int blocks, int sr, int st, int sd, int sx, const double* coef, int first,
                    cudaStream_t s, int stn) {
    kb_cheb<T><<<bgrid(blocks, n), kT, 0, s>>>(L, sr, st, sd, sx, coef, first, stn);
    return count_launch(cudaGetLastError());
}
template <typename T>
cudaError_t bl_sub(const BLevel* L, int n, int blocks, int sa, int sb, int sc, cudaStream_t s) {
    kb_sub<T><<<bgrid(blocks, n), kT, 0, s>>>(L, sa, sb, sc);
    return count_launch(cudaGetLastError());
}
template <typename T>
cudaError_t bl_copy(const BLevel* L, int n, int blocks, int ss, int sd, int block, cudaStream_t s) {
    kb_copy<T><<<bgrid(blocks, n), kT, 0, s>>>(L, ss, sd, block);
    return count_launch(cudaGetLastError());
}
template <typename Ti, typename To>
cudaError_t bl_convert(const BLevel* L, int n, int blocks, int ss, int sd, int mode, cudaStream_t s) {
    kb_convert<Ti, To><<<bgrid(blocks, n), kT, 0, s>>>(L, ss, sd, mode);
    return count_launch(cudaGetLastError());
}
cudaError_t bl_axpby64(const BLevel* L, int n, int blocks, const double* a, int sx, double b, int sy, int invert_a,
                       cudaStream_t s) {
    kb_axpby64<<<bgrid(blocks, n), kT, 0, s>>>(L, a, sx, b, sy, invert_a);
    return count_launch(cudaGetLastError());
}
template <typename T>
cudaError_t bl_restrict(const BLevel* Lc, const BLevel* Lf, int n, int blocks, int sf, int sc, cudaStream_t s) {
    kb_restrict<T><<<bgrid(blocks, n), kT, 0, s>>>(Lc, Lf, sf, sc);
    return count_launch(cudaGetLastError());
}
template <typename T>
cudaError_t bl_prolongate_add(const BLevel* Lc, const BLevel* Lf, int n, int blocks, int sc, int sf, cudaStream_t s) {
    kb_prolongate_add<T><<<bgrid(blocks, n), kT, 0, s>>>(Lc, Lf, sc, sf);
    return count_launch(cudaGetLastError());
}
template <typename T>
cudaError_t bl_dots2(const BLevel* L, int n, int sa, int sb, double* part, double* out, cudaStream_t s) {
    kb_dots2_partial<T><<<bgrid(kBPartials, n), kT, 0, s>>>(L, sa, sb, part);
    count_launch(cudaGetLastError());
    kb_dots2_final<<<n, kT, 0, s>>>(part, kBPartials, out);
    return count_launch(cudaGetLastError());
}
cudaError_t bl_multidot(const BLevel* L, int n, int k, int sw, double* part, int kmax, double* h, int ldh,
                        cudaStream_t s, const int* kcol) {
    kb_multidot_partial<<<bgrid(kBPartials, n), kT, 0, s>>>(L, k, kcol, sw, part, kmax);
    count_launch(cudaGetLastError());
    kb_multidot_final<<<n, 1024, 0, s>>>(part, kBPartials, k, kcol, kmax, h, ldh);
    return count_launch(cudaGetLastError());
}
cudaError_t bl_multi_axpy(const BLevel* L, int n, int blocks, int k, const double* h, int ldh, int sw, cudaStream_t s,
                          const int* kcol) {
    kb_multi_axpy<<<bgrid(blocks, n), kT, 0, s>>>(L, k, kcol, h, ldh, sw);
    return count_launch(cudaGetLastError());
}
cudaError_t bl_norm(const BLevel* L, int n, int sw, double* part, double* out, cudaStream_t s) {
    kb_norm_partial<<<bgrid(kBPartials, n), kT, 0, s>>>(L, sw, part);
    count_launch(cudaGetLastError());
    kb_norm_final<<<n, kT, 0, s>>>(part, kBPartials, out);
    return count_launch(cudaGetLastError());
}
cudaError_t bl_gemv_add(const BLevel* L, int n, int blocks, int k, const double* y, int ldy, int sx, cudaStream_t s,
                        const int* kk) {
    kb_gemv_add<<<bgrid(blocks, n), kT, 0, s>>>(L, k, kk, y, ldy, sx);
    return count_launch(cudaGetLastError());
}
template <typename T>
cudaError_t bl_cg_r(const BLevel* L, int n, int blocks, int sr, int sq, int sz, const double* alpha2, cudaStream_t s) {
    kb_cg_r<T><<<bgrid(blocks, n), kT, 0, s>>>(L, sr, sq, sz, alpha2);
    return count_launch(cudaGetLastError());
}
template <typename T>
cudaError_t bl_cg_p(const BLevel* L, int n, int blocks, int sp, int sz, const double* beta2, cudaStream_t s) {
    kb_cg_p<T><<<bgrid(blocks, n), kT, 0, s>>>(L, sp, sz, beta2);
    return count_launch(cudaGetLastError());
}
template <typename T>
cudaError_t bl_start_vector(const BLevel* L, int n, int blocks, int sv, const uint64_t* seeds, int level,
                            cudaStream_t s) {
    kb_start_vector<T><<<bgrid(blocks, n), kT, 0, s>>>(L, sv, seeds, level);
    return count_launch(cudaGetLastError());
}

#define PFF_INST(T)                                                                                              \
    template cudaError_t bl_init_masked<T>(const BLevel*, int, int, int, int, int, T, cudaStream_t);             \
    template cudaError_t bl_cheb<T>(const BLevel*, int, int, int, int, int, int, const double*, int, cudaStream_t, int); \
    template cudaError_t bl_sub<T>(const BLevel*, int, int, int, int, int, cudaStream_t);                        \
    template cudaError_t bl_copy<T>(const BLevel*, int, int, int, int, int, cudaStream_t);                       \
    template cudaError_t bl_restrict<T>(const BLevel*, const BLevel*, int, int, int, int, cudaStream_t);         \
    template cudaError_t bl_prolongate_add<T>(const BLevel*, const BLevel*, int, int, int, int, cudaStream_t);   \
    template cudaError_t bl_dots2<T>(const BLevel*, int, int, int, double*, double*, cudaStream_t);              \
    template cudaError_t bl_cg_r<T>(const BLevel*, int, int, int, int, int, const double*, cudaStream_t);        \
    template cudaError_t bl_cg_p<T>(const BLevel*, int, int, int, int, const double*, cudaStream_t);             \
    template cudaError_t bl_start_vector<T>(const BLevel*, int, int, int, const uint64_t*, int, cudaStream_t);
PFF_INST(float)
PFF_INST(double)
#undef PFF_INST
template cudaError_t bl_convert<double, float>(const BLevel*, int, int, int, int, int, cudaStream_t);
template cudaError_t bl_convert<float, double>(const BLevel*, int, int, int, int, int, cudaStream_t);
template cudaError_t bl_convert<double, double>(const BLevel*, int, int, int, int, int, cudaStream_t);

}  // namespace pff
