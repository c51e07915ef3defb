// Vector, transfer, reduction and bookkeeping kernels of the pff library.
//
//  - state restriction to coarse levels by coincident nodes (Sec. 4.2),
//  - canonical transfers of nested Q1/Q2 grids (Sec. 3.2): prolongation = nodal interpolation
//    of the coarse function, restriction = its transpose,
//  - Chebyshev-Jacobi update (Saad, Iterative Methods, Algorithm 12.1, on D^-1 A),
//  - deterministic two-stage reductions (fixed grid, fixed summation order),
//  - SplitMix64 counter-based start vector (Steele, Lea, Flood 2014),
//  - lumped Gauss-Lobatto mass and active-set decision (Algorithm 1, steps 1-4).
#include "pff_df64.cuh"
#include "pff_internal.cuh"

namespace pff {

static constexpr int kThreads = 256;
static constexpr int kRedBlocks = 304;   // 2 x 152 SMs; fixed so partial-sum order is fixed

static int grid_for(int64_t n) {
    int64_t b = (n + kThreads - 1) / kThreads;
    if (b > 152 * 32) b = 152 * 32;
    if (b < 1) b = 1;
    return (int)b;
}

#define GRID_STRIDE(i, n) \
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

__device__ __forceinline__ void node_ijk(const Geom& g, int64_t node, int& i, int& j, int& k) {
    i = (int)(node % g.nn[0]);
    const int64_t r = node / g.nn[0];
    j = (int)(r % g.nn[1]);
    k = (int)(r / g.nn[1]);
}

__device__ __forceinline__ int64_t node_id(const Geom& g, int i, int j, int k) {
    return (int64_t)i + (int64_t)g.nn[0] * ((int64_t)j + (int64_t)g.nn[1] * k);
}

// ---------------------------------------------------------------- state restriction
// Coincident-node injection of U, phi~ and the masks (Sec. 4.2).  On Q2 levels phi~ of a coarse node
// is the maximum of the fine phi~ over the fine nodes at most one lattice step away along every axis
// (the 3^d block around the coincident node, cut at the boundary): the Q2 field's values at edge, face
// and cell-centre nodes, which injection drops, keep the coarse cells as stiff as the fine ones.  Q1
// levels take the same maximum when phi_max_q1 is set (an option beyond the paper).
__global__ void k_restrict_state(Geom gc, Geom gf, const double* __restrict__ Uf, const double* __restrict__ ptf,
                                 const uint8_t* __restrict__ maskf, double* __restrict__ Uc,
                                 double* __restrict__ ptc, uint8_t* __restrict__ maskc, bool phi_max_q1) {
    GRID_STRIDE(n, gc.n_nodes) {
        int i, j, k;
        node_ijk(gc, n, i, j, k);
        const int fk0 = gc.dim == 3 ? 2 * k : 0;
        const int64_t f = node_id(gf, 2 * i, 2 * j, fk0);
        for (int c = 0; c <= gc.dim; ++c) Uc[c * gc.n_nodes + n] = Uf[c * gf.n_nodes + f];
        maskc[n] = maskf[f];
        double p = ptf[f];
        if (gc.deg == 2 || phi_max_q1) {
            const int k0 = gc.dim == 3 ? max(fk0 - 1, 0) : 0, k1 = gc.dim == 3 ? min(fk0 + 1, gf.nn[2] - 1) : 0;
            const int j0 = max(2 * j - 1, 0), j1 = min(2 * j + 1, gf.nn[1] - 1);
            const int i0 = max(2 * i - 1, 0), i1 = min(2 * i + 1, gf.nn[0] - 1);
            for (int kk = k0; kk <= k1; ++kk)
                for (int jj = j0; jj <= j1; ++jj)
                    for (int ii = i0; ii <= i1; ++ii) p = fmax(p, ptf[node_id(gf, ii, jj, kk)]);
        }
        ptc[n] = p;
    }
}

cudaError_t launch_restrict_state(const Geom& gc, const Geom& gf, const double* Uf, const double* ptf,
                                  const uint8_t* maskf, double* Uc, double* ptc, uint8_t* maskc, bool phi_max_q1, cudaStream_t s) {
    k_restrict_state<<<grid_for(gc.n_nodes), kThreads, 0, s>>>(gc, gf, Uf, ptf, maskf, Uc, ptc, maskc, phi_max_q1);
    return count_launch(cudaGetLastError());
}

__global__ void k_cast_f64_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
    GRID_STRIDE(i, n) b[i] = (float)a[i];
}
__global__ void k_cast_f32_f64(const float* __restrict__ a, double* __restrict__ b, int64_t n) {
    GRID_STRIDE(i, n) b[i] = (double)a[i];
}
cudaError_t launch_cast_f64_f32(const double* a, float* b, int64_t n, cudaStream_t s) {
    k_cast_f64_f32<<<grid_for(n), kThreads, 0, s>>>(a, b, n);
    return count_launch(cudaGetLastError());
}
cudaError_t launch_cast_f32_f64(const float* a, double* b, int64_t n, cudaStream_t s) {
    k_cast_f32_f64<<<grid_for(n), kThreads, 0, s>>>(a, b, n);
    return count_launch(cudaGetLastError());
}

// ---------------------------------------------------------------- masks
__global__ void k_face_mask(Geom g, unsigned faces, const uint8_t* __restrict__ extra, uint8_t* __restrict__ mask) {
    const uint8_t ubits = (uint8_t)(g.dim == 3 ? MASK_U_ALL : (PFF_MASK_UX | PFF_MASK_UY));
    GRID_STRIDE(n, g.n_nodes) {
        int idx[3];
        node_ijk(g, n, idx[0], idx[1], idx[2]);
        bool on = false;
        for (int a = 0; a < g.dim; ++a) {
            if ((faces >> (2 * a)) & 1u) on |= idx[a] == 0;
            if ((faces >> (2 * a + 1)) & 1u) on |= idx[a] == g.nn[a] - 1;
        }
        uint8_t m = on ? ubits : 0;
        if (extra) m |= (uint8_t)(extra[n] & (ubits | PFF_MASK_PHI_DIR));
        mask[n] = m;
    }
}
cudaError_t launch_face_mask(const Geom& g, unsigned faces, const uint8_t* extra, uint8_t* mask, cudaStream_t s) {
    k_face_mask<<<grid_for(g.n_nodes), kThreads, 0, s>>>(g, faces, extra, mask);
    return count_launch(cudaGetLastError());
}

__global__ void k_set_active(int64_t n, const uint8_t* __restrict__ act, uint8_t* __restrict__ mask) {
    GRID_STRIDE(i, n) mask[i] = (uint8_t)((mask[i] & ~PFF_MASK_ACTIVE) | (act[i] ? PFF_MASK_ACTIVE : 0));
}
__global__ void k_get_active(int64_t n, const uint8_t* __restrict__ mask, uint8_t* __restrict__ act) {
    GRID_STRIDE(i, n) act[i] = (mask[i] & PFF_MASK_ACTIVE) ? 1 : 0;
}
cudaError_t launch_set_active(const Geom& g, const uint8_t* active, uint8_t* mask, cudaStream_t s) {
    k_set_active<<<grid_for(g.n_nodes), kThreads, 0, s>>>(g.n_nodes, active, mask);
    return count_launch(cudaGetLastError());
}
cudaError_t launch_get_active(const Geom& g, const uint8_t* mask, uint8_t* active, cudaStream_t s) {
    k_get_active<<<grid_for(g.n_nodes), kThreads, 0, s>>>(g.n_nodes, mask, active);
    return count_launch(cudaGetLastError());
}

__device__ __forceinline__ bool elim_dof(uint8_t m, int c, int dim) {
    return c < dim ? ((m >> c) & 1) != 0 : (m & PHI_BITS_ALL) != 0;
}

// ---------------------------------------------------------------- transfers
// 1D weight of coarse basis function I at fine node i: the fine node lies in coarse cell
// m = min(i / (2 deg), nc - 1) at local coordinate t = (i - 2 deg m) / (2 deg); the weight is
// the Lagrange basis L_a(t) of local node a = I - deg m (0 outside the cell).
template <typename T>
__device__ __forceinline__ T p1w(int i, int I, int deg, int nc) {
    int m = i / (2 * deg);
    if (m > nc - 1) m = nc - 1;
    const int a = I - deg * m;
    if (a < 0 || a > deg) return T(0);
    const T t = T(i - 2 * deg * m) / T(2 * deg);
    if (deg == 1) return a == 0 ? T(1) - t : t;
    if (a == 0) return (T(1) - t) * (T(1) - T(2) * t);
    if (a == 1) return T(4) * t * (T(1) - t);
    return t * (T(2) * t - T(1));
}

template <typename T>
__global__ void k_restrict(Geom gc, Geom gf, const T* __restrict__ rf, T* __restrict__ rc,
                           const uint8_t* __restrict__ maskc) {
    const int deg = gc.deg, R = 2 * deg - 1;
    GRID_STRIDE(n, gc.n_nodes) {
        int I, J, K;
        node_ijk(gc, n, I, J, K);
        const uint8_t m = maskc[n];
        T acc[4] = {T(0), T(0), T(0), T(0)};
        const int k0 = gc.dim == 3 ? max(0, 2 * K - R) : 0, k1 = gc.dim == 3 ? min(gf.nn[2] - 1, 2 * K + R) : 0;
        const int j0 = max(0, 2 * J - R), j1 = min(gf.nn[1] - 1, 2 * J + R);
        const int i0 = max(0, 2 * I - R), i1 = min(gf.nn[0] - 1, 2 * I + R);
        for (int k = k0; k <= k1; ++k) {
            const T wk = gc.dim == 3 ? p1w<T>(k, K, deg, gc.nc[2]) : T(1);
            if (wk == T(0)) continue;
            for (int j = j0; j <= j1; ++j) {
                const T wj = p1w<T>(j, J, deg, gc.nc[1]);
                if (wj == T(0)) continue;
                for (int i = i0; i <= i1; ++i) {
                    const T wi = p1w<T>(i, I, deg, gc.nc[0]);
                    if (wi == T(0)) continue;
                    const T w = wi * wj * wk;
                    const int64_t f = node_id(gf, i, j, k);
                    for (int c = 0; c <= gc.dim; ++c) acc[c] += w * rf[c * gf.n_nodes + f];
                }
            }
        }
        for (int c = 0; c <= gc.dim; ++c) rc[c * gc.n_nodes + n] = elim_dof(m, c, gc.dim) ? T(0) : acc[c];
    }
}

template <typename T>
__global__ void k_prolongate_add(Geom gc, Geom gf, const T* __restrict__ ec, T* __restrict__ xf,
                                 const uint8_t* __restrict__ maskf) {
    const int deg = gc.deg;
    GRID_STRIDE(n, gf.n_nodes) {
        int idx[3];
        node_ijk(gf, n, idx[0], idx[1], idx[2]);
        int cell[3];
        T t[3];
        for (int a = 0; a < 3; ++a) {
            if (a >= gc.dim) { cell[a] = 0; t[a] = T(0); continue; }
            int m = idx[a] / (2 * deg);
            if (m > gc.nc[a] - 1) m = gc.nc[a] - 1;
            cell[a] = m;
            t[a] = T(idx[a] - 2 * deg * m);
        }
        T acc[4] = {T(0), T(0), T(0), T(0)};
        const int kz = gc.dim == 3 ? deg : 0;
        for (int c2 = 0; c2 <= kz; ++c2) {
            const int K = deg * cell[2] + c2;
            const T wk = gc.dim == 3 ? p1w<T>(idx[2], K, deg, gc.nc[2]) : T(1);
            if (wk == T(0)) continue;
            for (int b = 0; b <= deg; ++b) {
                const int J = deg * cell[1] + b;
                const T wj = p1w<T>(idx[1], J, deg, gc.nc[1]);
                if (wj == T(0)) continue;
                for (int a = 0; a <= deg; ++a) {
                    const int I = deg * cell[0] + a;
                    const T wi = p1w<T>(idx[0], I, deg, gc.nc[0]);
                    if (wi == T(0)) continue;
                    const T w = wi * wj * wk;
                    const int64_t cn = node_id(gc, I, J, K);
                    for (int c = 0; c <= gc.dim; ++c) acc[c] += w * ec[c * gc.n_nodes + cn];
                }
            }
        }
        const uint8_t m = maskf[n];
        for (int c = 0; c <= gf.dim; ++c)
            if (!elim_dof(m, c, gf.dim)) xf[c * gf.n_nodes + n] += acc[c];
    }
}

template <typename T>
cudaError_t launch_restrict(const Geom& gc, const Geom& gf, const T* rf, T* rc, const uint8_t* maskc, cudaStream_t s) {
    k_restrict<T><<<grid_for(gc.n_nodes), kThreads, 0, s>>>(gc, gf, rf, rc, maskc);
    return count_launch(cudaGetLastError());
}
template <typename T>
cudaError_t launch_prolongate_add(const Geom& gc, const Geom& gf, const T* ec, T* xf, const uint8_t* maskf,
                                  cudaStream_t s) {
    k_prolongate_add<T><<<grid_for(gf.n_nodes), kThreads, 0, s>>>(gc, gf, ec, xf, maskf);
    return count_launch(cudaGetLastError());
}
template cudaError_t launch_restrict<double>(const Geom&, const Geom&, const double*, double*, const uint8_t*,
                                             cudaStream_t);
template cudaError_t launch_restrict<float>(const Geom&, const Geom&, const float*, float*, const uint8_t*,
                                            cudaStream_t);
template cudaError_t launch_prolongate_add<double>(const Geom&, const Geom&, const double*, double*, const uint8_t*,
                                                   cudaStream_t);
template cudaError_t launch_prolongate_add<float>(const Geom&, const Geom&, const float*, float*, const uint8_t*,
                                                  cudaStream_t);

// ---------------------------------------------------------------- elementwise
template <typename T>
__global__ void k_invert(T* d, int64_t n) {
    GRID_STRIDE(i, n) d[i] = T(1) / d[i];
}
template <typename T>
cudaError_t launch_invert_diag(T* d, int64_t n, cudaStream_t s) {
    k_invert<T><<<grid_for(n), kThreads, 0, s>>>(d, n);
    return count_launch(cudaGetLastError());
}
template cudaError_t launch_invert_diag<double>(double*, int64_t, cudaStream_t);
template cudaError_t launch_invert_diag<float>(float*, int64_t, cudaStream_t);

// Chebyshev step on D^-1 A (Saad, Alg. 12.1), per block b (u or phi):
//   first = 1:  d = c2[b] * dinv * r,  x = d                 (d_0 = z_0 / theta)
//   first = 2:  d = c2[b] * dinv * r,  x += d
//   first = 0:  r -= t;  d = c1[b] d + c2[b] dinv r;  x += d
// With tn != nullptr the update also writes the preset of the next operator apply t = G d into tn
// (d on eliminated rows, 0 elsewhere), so that apply need not launch its own preset.
template <typename T>
__global__ void k_cheb_update(int64_t nn, int dim, T* __restrict__ r, const T* t, T* __restrict__ d,
                              const T* __restrict__ dinv, T* __restrict__ x, T c1u, T c1p, T c2u, T c2p, int first,
                              const uint8_t* __restrict__ mask, T* tn) {
    const int64_t nd = nn * (dim + 1);
    const int64_t nu = nn * dim;
    GRID_STRIDE(i, nd) {
        const bool u = i < nu;
        const T c1 = u ? c1u : c1p, c2 = u ? c2u : c2p;
        T di;
        if (first) {
            di = c2 * dinv[i] * r[i];
            x[i] = first == 1 ? di : x[i] + di;
        } else {
            const T ri = r[i] - t[i];
            r[i] = ri;
            di = c1 * d[i] + c2 * dinv[i] * ri;
            x[i] += di;
        }
        d[i] = di;
        if (tn) {
            const int c = dof_comp(i, nn);
            tn[i] = elim_dof(mask[i - c * nn], c, dim) ? di : T(0);
        }
    }
}
template <typename T>
cudaError_t launch_cheb_update(const Geom& g, T* r, const T* t, T* d, const T* dinv, T* x, double c1u, double c1p,
                               double c2u, double c2p, int first, cudaStream_t s, const uint8_t* mask, T* tn) {
    k_cheb_update<T><<<grid_for(n_dofs(g)), kThreads, 0, s>>>(g.n_nodes, g.dim, r, t, d, dinv, x, (T)c1u, (T)c1p,
                                                              (T)c2u, (T)c2p, first, mask, tn);
    return count_launch(cudaGetLastError());
}
template cudaError_t launch_cheb_update<double>(const Geom&, double*, const double*, double*, const double*, double*,
                                                double, double, double, double, int, cudaStream_t, const uint8_t*,
                                                double*);
template cudaError_t launch_cheb_update<float>(const Geom&, float*, const float*, float*, const float*, float*,
                                               double, double, double, double, int, cudaStream_t, const uint8_t*,
                                               float*);

template <typename T>
__global__ void k_axpby(int64_t n, T a, const T* __restrict__ x, T b, T* __restrict__ y) {
    GRID_STRIDE(i, n) y[i] = a * x[i] + b * y[i];
}
template <typename T>
cudaError_t launch_axpby(int64_t n, double a, const T* x, double b, T* y, cudaStream_t s) {
    k_axpby<T><<<grid_for(n), kThreads, 0, s>>>(n, (T)a, x, (T)b, y);
    return count_launch(cudaGetLastError());
}
template cudaError_t launch_axpby<double>(int64_t, double, const double*, double, double*, cudaStream_t);
template cudaError_t launch_axpby<float>(int64_t, double, const float*, double, float*, cudaStream_t);

template <typename T>
__global__ void k_sub(int64_t n, const T* __restrict__ a, const T* __restrict__ b, T* __restrict__ c) {
    GRID_STRIDE(i, n) c[i] = a[i] - b[i];
}
template <typename T>
cudaError_t launch_sub(int64_t n, const T* a, const T* b, T* c, cudaStream_t s) {
    k_sub<T><<<grid_for(n), kThreads, 0, s>>>(n, a, b, c);
    return count_launch(cudaGetLastError());
}
template cudaError_t launch_sub<double>(int64_t, const double*, const double*, double*, cudaStream_t);
template cudaError_t launch_sub<float>(int64_t, const float*, const float*, float*, cudaStream_t);

template <typename T>
__global__ void k_copy_block(int64_t nn, int dim, int block, const T* __restrict__ src, T* __restrict__ dst) {
    const int64_t nd = nn * (dim + 1), nu = nn * dim;
    GRID_STRIDE(i, nd) {
        const bool in = block == 0 ? i < nu : i >= nu;
        dst[i] = in ? src[i] : T(0);
    }
}
template <typename T>
cudaError_t launch_copy_block(const Geom& g, int block, const T* src, T* dst, cudaStream_t s) {
    k_copy_block<T><<<grid_for(n_dofs(g)), kThreads, 0, s>>>(g.n_nodes, g.dim, block, src, dst);
    return count_launch(cudaGetLastError());
}
template cudaError_t launch_copy_block<double>(const Geom&, int, const double*, double*, cudaStream_t);
template cudaError_t launch_copy_block<float>(const Geom&, int, const float*, float*, cudaStream_t);

// dst = free ? src : 0   (free_only = 1)   or   dst = eliminated ? src : dst  (free_only = 0)
template <typename T>
__global__ void k_mask_copy(int64_t nn, int dim, const uint8_t* __restrict__ mask, const T* __restrict__ src,
                            T* __restrict__ dst, int free_only) {
    const int64_t nd = nn * (dim + 1);
    GRID_STRIDE(i, nd) {
        const int c = dof_comp(i, nn);
        const bool e = elim_dof(mask[i - c * nn], c, dim);
        if (free_only) dst[i] = e ? T(0) : src[i];
        else if (e) dst[i] = src[i];
    }
}
template <typename T>
cudaError_t launch_mask_copy(const Geom& g, const uint8_t* mask, const T* src, T* dst, int free_only,
                             cudaStream_t s) {
    k_mask_copy<T><<<grid_for(n_dofs(g)), kThreads, 0, s>>>(g.n_nodes, g.dim, mask, src, dst, free_only);
    return count_launch(cudaGetLastError());
}
template cudaError_t launch_mask_copy<double>(const Geom&, const uint8_t*, const double*, double*, int, cudaStream_t);
template cudaError_t launch_mask_copy<float>(const Geom&, const uint8_t*, const float*, float*, int, cudaStream_t);

// ---------------------------------------------------------------- reductions
int dot_partials() { return kRedBlocks; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block sum of two values; result valid in thread 0.
__device__ __forceinline__ void block_sum2(double& a, double& b) {
    __shared__ double sa[32], sb[32];
    a = warp_sum(a);
    b = warp_sum(b);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { sa[w] = a; sb[w] = b; }
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        a = l < nw ? sa[l] : 0.0;
        b = l < nw ? sb[l] : 0.0;
        a = warp_sum(a);
        b = warp_sum(b);
    }
    __syncthreads();
}

// FP32 vectors: the product of two floats is exact as a double-float pair (FMA) and the per-thread
// sums run in double-float on the FP32 pipes (FP64 arithmetic issues at 1/64 of the FP32 rate on
// GB300, which made these reductions FP64-bound); FP64 vectors: plain FP64.
template <typename T>
__global__ void k_block_dots_partial(int64_t nn, int dim, const T* __restrict__ a, const T* __restrict__ b,
                                     const T* __restrict__ w, double* __restrict__ part) {
    const int64_t nd = nn * (dim + 1), nu = nn * dim;
    double su = 0.0, sp = 0.0;
    if constexpr (sizeof(T) == 4) {
        // four elements per iteration so that each thread keeps several loads in flight
        constexpr int U = 4;
        df64 fu = df_make(0.f, 0.f), fp = df_make(0.f, 0.f);
        const int64_t stride = (int64_t)gridDim.x * blockDim.x;
        for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < nd; i0 += U * stride) {
            float x[U], y[U], z[U];
#pragma unroll
            for (int r = 0; r < U; ++r) {
                const int64_t i = i0 + r * stride;
                x[r] = i < nd ? a[i] : 0.f;
                y[r] = i < nd ? b[i] : 0.f;
                z[r] = (w && i < nd) ? w[i] : 1.f;
            }
#pragma unroll
            for (int r = 0; r < U; ++r) {
                const int64_t i = i0 + r * stride;
                const float pr = __fmul_rn(x[r], y[r]);
                df64 v = df_make(pr, __fmaf_rn(x[r], y[r], -pr));
                if (w) v = v * df_make(z[r], 0.f);
                if (i < nu) fu = fu + v; else fp = fp + v;
            }
        }
        su = df_to_double(fu);
        sp = df_to_double(fp);
    } else {
        GRID_STRIDE(i, nd) {
            double v = (double)a[i] * (double)b[i];
            if (w) v *= (double)w[i];
            if (i < nu) su += v; else sp += v;
        }
    }
    block_sum2(su, sp);
    if (threadIdx.x == 0) { part[2 * blockIdx.x] = su; part[2 * blockIdx.x + 1] = sp; }
}

__global__ void k_sum_partials2(const double* __restrict__ part, int nparts, double* __restrict__ out) {
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) { a += part[2 * i]; b += part[2 * i + 1]; }
    block_sum2(a, b);
    if (threadIdx.x == 0) { out[0] = a; out[1] = b; }
}

template <typename T>
cudaError_t launch_block_dots(const Geom& g, const T* a, const T* b, const T* w, double* scratch, double* out,
                              cudaStream_t s) {
    k_block_dots_partial<T><<<kRedBlocks, kThreads, 0, s>>>(g.n_nodes, g.dim, a, b, w, scratch);
    count_launch(cudaGetLastError());
    k_sum_partials2<<<1, kThreads, 0, s>>>(scratch, kRedBlocks, out);
    return count_launch(cudaGetLastError());
}
template cudaError_t launch_block_dots<double>(const Geom&, const double*, const double*, const double*, double*,
                                               double*, cudaStream_t);
template cudaError_t launch_block_dots<float>(const Geom&, const float*, const float*, const float*, double*, double*,
                                              cudaStream_t);

// ---------------------------------------------------------------- SplitMix64 start vector
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

template <typename T>
__global__ void k_start_vector(int64_t nn, int dim, const uint8_t* __restrict__ mask, uint64_t seed, int level,
                               T* __restrict__ v) {
    const int64_t nd = nn * (dim + 1);
    GRID_STRIDE(i, nd) {
        const int c = dof_comp(i, nn);
        const uint64_t key = seed + (uint64_t)level * (1ull << 40) + (uint64_t)i;
        const double u = (double)(splitmix64(key) >> 11) * 0x1.0p-53;
        v[i] = elim_dof(mask[i - c * nn], c, dim) ? T(0) : T(2.0 * u - 1.0);
    }
}
template <typename T>
cudaError_t launch_start_vector(const Geom& g, const uint8_t* mask, uint64_t seed, int level, T* v, cudaStream_t s) {
    k_start_vector<T><<<grid_for(n_dofs(g)), kThreads, 0, s>>>(g.n_nodes, g.dim, mask, seed, level, v);
    return count_launch(cudaGetLastError());
}
template cudaError_t launch_start_vector<double>(const Geom&, const uint8_t*, uint64_t, int, double*, cudaStream_t);
template cudaError_t launch_start_vector<float>(const Geom&, const uint8_t*, uint64_t, int, float*, cudaStream_t);

// ---------------------------------------------------------------- CG pieces (per-block scalars)
// alpha2[b] per block: r -= alpha q; z = dinv r
template <typename T>
__global__ void k_cg_update_r(int64_t nn, int dim, T* __restrict__ r, const T* __restrict__ q,
                              const T* __restrict__ dinv, T* __restrict__ z, const double* __restrict__ alpha2) {
    const int64_t nd = nn * (dim + 1), nu = nn * dim;
    const T au = (T)alpha2[0], ap = (T)alpha2[1];
    GRID_STRIDE(i, nd) {
        const T al = i < nu ? au : ap;
        const T ri = r[i] - al * q[i];
        r[i] = ri;
        z[i] = dinv[i] * ri;
    }
}
template <typename T>
__global__ void k_cg_update_p(int64_t nn, int dim, T* __restrict__ p, const T* __restrict__ z,
                              const double* __restrict__ beta2) {
    const int64_t nd = nn * (dim + 1), nu = nn * dim;
    const T bu = (T)beta2[0], bp = (T)beta2[1];
    GRID_STRIDE(i, nd) p[i] = z[i] + (i < nu ? bu : bp) * p[i];
}
template <typename T>
cudaError_t launch_cg_update_r(const Geom& g, T* r, const T* q, const T* dinv, T* z, const double* alpha2,
                               cudaStream_t s) {
    k_cg_update_r<T><<<grid_for(n_dofs(g)), kThreads, 0, s>>>(g.n_nodes, g.dim, r, q, dinv, z, alpha2);
    return count_launch(cudaGetLastError());
}
template <typename T>
cudaError_t launch_cg_update_p(const Geom& g, T* p, const T* z, const double* beta2, cudaStream_t s) {
    k_cg_update_p<T><<<grid_for(n_dofs(g)), kThreads, 0, s>>>(g.n_nodes, g.dim, p, z, beta2);
    return count_launch(cudaGetLastError());
}
template cudaError_t launch_cg_update_r<double>(const Geom&, double*, const double*, const double*, double*,
                                                const double*, cudaStream_t);
template cudaError_t launch_cg_update_r<float>(const Geom&, float*, const float*, const float*, float*,
                                               const double*, cudaStream_t);
template cudaError_t launch_cg_update_p<double>(const Geom&, double*, const double*, const double*, cudaStream_t);
template cudaError_t launch_cg_update_p<float>(const Geom&, float*, const float*, const double*, cudaStream_t);

// ---------------------------------------------------------------- lumped mass and active set
// Gauss-Lobatto lumping on a uniform tensor grid: the nodal weight is the product over axes of
// the 1D lumped weights (Q1: h/2 per adjacent cell; Q2: h/6 at cell vertices, 2h/3 at
// midpoints), summed over the cells that share the node.
// Gauss-Lobatto lumped mass: sum over the domain cells around the node of |K| times the product of
// the 1D Lobatto weights (1/2, 1/2 for Q1; 1/6, 2/3, 1/6 for Q2) of the node's position in the cell.
__global__ void k_lumped_mass(Geom g, double* __restrict__ M) {
    GRID_STRIDE(n, g.n_nodes) {
        int idx[3];
        node_ijk(g, n, idx[0], idx[1], idx[2]);
        int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
        for (int a = 0; a < g.dim; ++a) {
            // cells c with deg c <= idx <= deg c + deg
            lo[a] = idx[a] >= g.deg ? (idx[a] - 1) / g.deg : 0;
            hi[a] = min(g.nc[a] - 1, idx[a] / g.deg);
        }
        double w = 0.0;
        for (int ck = lo[2]; ck <= hi[2]; ++ck)
            for (int cj = lo[1]; cj <= hi[1]; ++cj)
                for (int ci = lo[0]; ci <= hi[0]; ++ci) {
                    const int64_t cell = (int64_t)ci + (int64_t)g.nc[0] * ((int64_t)cj + (int64_t)g.nc[1] * ck);
                    if (!cell_in(g, cell)) continue;
                    const int c3[3] = {ci, cj, ck};
                    double wc = 1.0;
                    for (int a = 0; a < g.dim; ++a) {
                        const int loc = idx[a] - g.deg * c3[a];
                        const double wa = g.deg == 1 ? 0.5 : (loc == 1 ? 2.0 / 3.0 : 1.0 / 6.0);
                        wc *= wa * g.h[a];
                    }
                    w += wc;
                }
        M[n] = w;
    }
}

// domain masks: a coarse cell is in the domain if any of its children is
__global__ void k_coarsen_cell_mask(Geom gc, Geom gf, const uint8_t* __restrict__ mf, uint8_t* __restrict__ mc) {
    GRID_STRIDE(c, gc.n_cells) {
        const int i = (int)(c % gc.nc[0]), j = (int)((c / gc.nc[0]) % gc.nc[1]), k = (int)(c / ((int64_t)gc.nc[0] * gc.nc[1]));
        const int kz = gc.dim == 3 ? 2 : 1;
        uint8_t any = 0;
        for (int dk = 0; dk < kz; ++dk)
            for (int dj = 0; dj < 2; ++dj)
                for (int di = 0; di < 2; ++di)
                    any |= mf[(int64_t)(2 * i + di) + (int64_t)gf.nc[0] * ((int64_t)(2 * j + dj) + (int64_t)gf.nc[1] * (kz == 2 ? 2 * k + dk : 0))] != 0;
        mc[c] = any;
    }
}
cudaError_t launch_coarsen_cell_mask(const Geom& gc, const Geom& gf, const uint8_t* mf, uint8_t* mc, cudaStream_t s) {
    k_coarsen_cell_mask<<<grid_for(gc.n_cells), kThreads, 0, s>>>(gc, gf, mf, mc);
    return count_launch(cudaGetLastError());
}

// nodes on no cell of the domain: every component fixed (identity rows)
__global__ void k_outside_nodes(Geom g, uint8_t* __restrict__ mask) {
    GRID_STRIDE(n, g.n_nodes) {
        int idx[3];
        node_ijk(g, n, idx[0], idx[1], idx[2]);
        int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
        for (int a = 0; a < g.dim; ++a) {
            lo[a] = idx[a] >= g.deg ? (idx[a] - 1) / g.deg : 0;
            hi[a] = min(g.nc[a] - 1, idx[a] / g.deg);
        }
        bool in = false;
        for (int ck = lo[2]; ck <= hi[2]; ++ck)
            for (int cj = lo[1]; cj <= hi[1]; ++cj)
                for (int ci = lo[0]; ci <= hi[0]; ++ci)
                    in = in || cell_in(g, (int64_t)ci + (int64_t)g.nc[0] * ((int64_t)cj + (int64_t)g.nc[1] * ck));
        if (!in) mask[n] |= (uint8_t)((g.dim == 3 ? MASK_U_ALL : (PFF_MASK_UX | PFF_MASK_UY)) | PFF_MASK_PHI_DIR);
    }
}
cudaError_t launch_outside_nodes(const Geom& g, uint8_t* mask, cudaStream_t s) {
    k_outside_nodes<<<grid_for(g.n_nodes), kThreads, 0, s>>>(g, mask);
    return count_launch(cudaGetLastError());
}
cudaError_t launch_lumped_mass(const Geom& g, double* M, cudaStream_t s) {
    k_lumped_mass<<<grid_for(g.n_nodes), kThreads, 0, s>>>(g, M);
    return count_launch(cudaGetLastError());
}

// active iff R_phi / M + c (phi - phi_old) > threshold  (Algorithm 1, step 3); counts[0] = |A|,
// counts[1] = nodes whose membership changed.
__global__ void k_active_set(Geom g, const double* __restrict__ R, const double* __restrict__ M,
                             const double* __restrict__ U, const double* __restrict__ phi_old, double c,
                             double thr, int tie_scale, uint8_t* __restrict__ mask, int* __restrict__ counts) {
    const int64_t nn = g.n_nodes;
    int na = 0, nch = 0;
    GRID_STRIDE(n, nn) {
        const uint8_t m = mask[n];
        // prescribed phi (phi Dirichlet, nodes outside the domain) never enters the active set
        const bool fixed = (m & PFF_MASK_PHI_DIR) != 0 || !(M[n] > 0.0);
        const double lam = fixed ? 0.0 : R[g.dim * nn + n] / M[n];
        const double v = lam + c * (U[g.dim * nn + n] - phi_old[n]);
        const bool act = !fixed && (tie_scale ? v * M[n] : v) > thr;
        const bool was = (m & PFF_MASK_ACTIVE) != 0;
        mask[n] = (uint8_t)((m & ~PFF_MASK_ACTIVE) | (act ? PFF_MASK_ACTIVE : 0));
        na += act;
        nch += act != was;
    }
    for (int o = 16; o > 0; o >>= 1) {
        na += __shfl_xor_sync(0xffffffffu, na, o);
        nch += __shfl_xor_sync(0xffffffffu, nch, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&counts[0], na);
        atomicAdd(&counts[1], nch);
    }
}
cudaError_t launch_active_set(const Geom& g, const double* R, const double* M, const double* U,
                              const double* phi_old, double c, double threshold, int tie_scale, uint8_t* mask,
                              int* counts, cudaStream_t s) {
    k_active_set<<<grid_for(g.n_nodes), kThreads, 0, s>>>(g, R, M, U, phi_old, c, threshold, tie_scale, mask, counts);
    return count_launch(cudaGetLastError());
}

// U_c(n) = g_c(n) on the displacement DoFs clamped by the mask (Dirichlet bits): the state takes the
// prescribed boundary values, so that the Newton increments vanish there (Algorithm 1 with
// inhomogeneous Dirichlet data)
__global__ void k_lift_dirichlet(Geom g, const uint8_t* __restrict__ mask, const double* __restrict__ ud,
                                 double* __restrict__ U) {
    const int64_t nn = g.n_nodes, nu = nn * g.dim;
    GRID_STRIDE(i, nu) {
        const int c = dof_comp(i, nn);
        if ((mask[i - c * nn] >> c) & 1) U[i] = ud[i];
    }
}
cudaError_t launch_lift_dirichlet(const Geom& g, const uint8_t* mask, const double* ud, double* U, cudaStream_t s) {
    k_lift_dirichlet<<<grid_for((int64_t)g.dim * g.n_nodes), kThreads, 0, s>>>(g, mask, ud, U);
    return count_launch(cudaGetLastError());
}

// delta = phi_old - phi on active phi DoFs, 0 elsewhere
__global__ void k_active_delta(Geom g, const double* __restrict__ U, const double* __restrict__ phi_old,
                               const uint8_t* __restrict__ mask, double* __restrict__ delta) {
    const int64_t nn = g.n_nodes, nd = nn * (g.dim + 1), nu = nn * g.dim;
    GRID_STRIDE(i, nd) {
        double v = 0.0;
        if (i >= nu) {
            const int64_t n = i - nu;
            if (mask[n] & PFF_MASK_ACTIVE) v = phi_old[n] - U[i];
        }
        delta[i] = v;
    }
}
cudaError_t launch_active_delta(const Geom& g, const double* U, const double* phi_old, const uint8_t* mask,
                                double* delta, cudaStream_t s) {
    k_active_delta<<<grid_for(n_dofs(g)), kThreads, 0, s>>>(g, U, phi_old, mask, delta);
    return count_launch(cudaGetLastError());
}

// Sum of one component of R over the nodes of one boundary face (axis, side), one CTA of 256
// threads, fixed summation order.  Sec. 5: L_y is the y-traction integrated over a boundary part,
// which for the discrete solution is the sum of the residual A(U)(phi_i e_y) over the face nodes.
__global__ void k_face_sum(Geom g, int axis, int side, int comp, const double* __restrict__ R,
                           double* __restrict__ out) {
    __shared__ double sm[256];
    const int64_t nface = g.n_nodes / g.nn[axis];
    const int b1 = axis == 0 ? 1 : 0, b2 = axis == 2 ? 1 : 2;
    const int64_t fixed = side ? g.nn[axis] - 1 : 0;
    const double* Rc = R + (int64_t)comp * g.n_nodes;
    double acc = 0.0;
    for (int64_t m = threadIdx.x; m < nface; m += blockDim.x) {
        int64_t idx[3];
        idx[axis] = fixed;
        idx[b1] = m % g.nn[b1];
        idx[b2] = m / g.nn[b1];
        acc += Rc[idx[0] + (int64_t)g.nn[0] * (idx[1] + (int64_t)g.nn[1] * idx[2])];
    }
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sm[0];
}
cudaError_t launch_face_sum(const Geom& g, int axis, int side, int comp, const double* R, double* out,
                            cudaStream_t s) {
    k_face_sum<<<1, 256, 0, s>>>(g, axis, side, comp, R, out);
    return count_launch(cudaGetLastError());
}

// Per-cell modulus factor of the next coarser level: mean of the 2^d children, fixed order.
__global__ void k_coarsen_cells(Geom gc, Geom gf, const double* __restrict__ sf, double* __restrict__ sc) {
    GRID_STRIDE(c, gc.n_cells) {
        const int i = (int)(c % gc.nc[0]), j = (int)((c / gc.nc[0]) % gc.nc[1]), k = (int)(c / ((int64_t)gc.nc[0] * gc.nc[1]));
        double acc = 0.0;
        const int kz = gc.dim == 3 ? 2 : 1;
        for (int dk = 0; dk < kz; ++dk)
            for (int dj = 0; dj < 2; ++dj)
                for (int di = 0; di < 2; ++di)
                    acc += sf[(int64_t)(2 * i + di) + (int64_t)gf.nc[0] * ((int64_t)(2 * j + dj) + (int64_t)gf.nc[1] * (kz == 2 ? 2 * k + dk : 0))];
        sc[c] = acc / (double)(kz * 4);
    }
}
cudaError_t launch_coarsen_cells(const Geom& gc, const Geom& gf, const double* sf, double* sc, cudaStream_t s) {
    k_coarsen_cells<<<grid_for(gc.n_cells), kThreads, 0, s>>>(gc, gf, sf, sc);
    return count_launch(cudaGetLastError());
}

// counts entries that are not finite and positive
__global__ void k_count_nonpositive(int64_t n, const double* __restrict__ v, int* __restrict__ bad) {
    int local = 0;
    GRID_STRIDE(i, n) {
        const double x = v[i];
        if (!(x > 0.0) || !isfinite(x)) ++local;
    }
    if (local) atomicAdd(bad, local);
}
cudaError_t launch_count_nonpositive(int64_t n, const double* v, int* bad, cudaStream_t s) {
    k_count_nonpositive<<<grid_for(n), kThreads, 0, s>>>(n, v, bad);
    return count_launch(cudaGetLastError());
}

// time-lagged phi~ of Sec. 2.3: clamp(2 phi^{n-1} - phi^{n-2}, 0, 1); phi^{n-1} without phi^{n-2}
__global__ void k_extrapolate(int64_t n, const double* __restrict__ p1, const double* __restrict__ p2,
                              double* __restrict__ out) {
    GRID_STRIDE(i, n) {
        double v = p1[i];
        if (p2) v = fmin(fmax(2.0 * v - p2[i], 0.0), 1.0);
        out[i] = v;
    }
}
cudaError_t launch_extrapolate(int64_t n, const double* phi_nm1, const double* phi_nm2, double* out,
                               cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_extrapolate<<<grid_for(n), kThreads, 0, s>>>(n, phi_nm1, phi_nm2, out);
    return count_launch(cudaGetLastError());
}

// R~ = R - t on free rows; phi_old - phi on active rows; 0 on Dirichlet rows (Algorithm 1, step 4)
__global__ void k_newton_rhs(Geom g, const double* __restrict__ R, const double* __restrict__ t,
                             const double* __restrict__ U, const double* __restrict__ phi_old,
                             const uint8_t* __restrict__ mask, double* __restrict__ Rt) {
    const int64_t nn = g.n_nodes, nd = nn * (g.dim + 1);
    GRID_STRIDE(i, nd) {
        const int c = dof_comp(i, nn);
        const int64_t n = i - c * nn;
        const uint8_t m = mask[n];
        double v;
        if (c < g.dim) v = ((m >> c) & 1) ? 0.0 : R[i] - t[i];
        else if (m & PFF_MASK_ACTIVE) v = phi_old[n] - U[i];
        else if (m & PFF_MASK_PHI_DIR) v = 0.0;
        else v = R[i] - t[i];
        Rt[i] = v;
    }
}
cudaError_t launch_newton_rhs(const Geom& g, const double* R, const double* t, const double* U,
                              const double* phi_old, const uint8_t* mask, double* Rt, cudaStream_t s) {
    k_newton_rhs<<<grid_for(n_dofs(g)), kThreads, 0, s>>>(g, R, t, U, phi_old, mask, Rt);
    return count_launch(cudaGetLastError());
}

// ---------------------------------------------------------------- FGMRES kernels
// h[j] = V_j . w for j < k (two stages, fixed order); V column-major with leading dim ld.
// Partial dots <V_j, w> for j < k: each thread reads w once per group of 8 basis vectors and keeps
// the group's 8 sums in registers; per-CTA partials in a fixed order (deterministic).
constexpr int kMultiDotGroup = 8, kMultiDotThreads = 512;
__global__ void __launch_bounds__(kMultiDotThreads) k_multidot_partial(int64_t n, const double* __restrict__ V, int64_t ld,
                                                                      int k, const double* __restrict__ w,
                                                                      double* __restrict__ part) {
    __shared__ double sh[kMultiDotGroup][kMultiDotThreads / 32];
    const int wid = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int j0 = 0; j0 < k; j0 += kMultiDotGroup) {
        const int kk = min(kMultiDotGroup, k - j0);
        double s[kMultiDotGroup];
#pragma unroll
        for (int t = 0; t < kMultiDotGroup; ++t) s[t] = 0.0;
        GRID_STRIDE(i, n) {
            const double wi = w[i];
#pragma unroll
            for (int t = 0; t < kMultiDotGroup; ++t)
                if (t < kk) s[t] += V[(int64_t)(j0 + t) * ld + i] * wi;
        }
#pragma unroll
        for (int t = 0; t < kMultiDotGroup; ++t) {
            const double v = warp_sum(s[t]);
            if (l == 0) sh[t][wid] = v;
        }
        __syncthreads();
        if (wid == 0) {
            for (int t = 0; t < kk; ++t) {
                const double v = warp_sum(l < nw ? sh[t][l] : 0.0);
                if (l == 0) part[(int64_t)(j0 + t) * gridDim.x + blockIdx.x] = v;
            }
        }
        __syncthreads();
    }
}
__global__ void k_multidot_final(const double* __restrict__ part, int nparts, int k, double* __restrict__ h) {
    // one warp per output
    const int wid = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int j = wid; j < k; j += nw) {
        double s = 0.0;
        for (int i = l; i < nparts; i += 32) s += part[(int64_t)j * nparts + i];
        s = warp_sum(s);
        if (l == 0) h[j] = s;
    }
}
cudaError_t launch_multidot(int64_t n, const double* V, int64_t ld, int k, const double* w, double* scratch,
                            double* h, cudaStream_t s) {
    k_multidot_partial<<<kRedBlocks, kMultiDotThreads, 0, s>>>(n, V, ld, k, w, scratch);
    count_launch(cudaGetLastError());
    k_multidot_final<<<1, 1024, 0, s>>>(scratch, kRedBlocks, k, h);
    return count_launch(cudaGetLastError());
}

__global__ void k_multi_axpy(int64_t n, const double* __restrict__ V, int64_t ld, int k, const double* __restrict__ h,
                             double* __restrict__ w) {
    GRID_STRIDE(i, n) {
        double s = w[i];
        for (int j = 0; j < k; ++j) s -= h[j] * V[j * ld + i];
        w[i] = s;
    }
}
cudaError_t launch_multi_axpy(int64_t n, const double* V, int64_t ld, int k, const double* h, double* w,
                              cudaStream_t s) {
    k_multi_axpy<<<grid_for(n), kThreads, 0, s>>>(n, V, ld, k, h, w);
    return count_launch(cudaGetLastError());
}

__global__ void k_norm2_partial(int64_t n, const double* __restrict__ w, double* __restrict__ part) {
    double s = 0.0, d = 0.0;
    GRID_STRIDE(i, n) s += w[i] * w[i];
    block_sum2(s, d);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}
__global__ void k_norm2_final(const double* __restrict__ part, int nparts, double* __restrict__ out) {
    double s = 0.0, d = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += part[i];
    block_sum2(s, d);
    if (threadIdx.x == 0) out[0] = sqrt(s);
}
cudaError_t launch_norm2(int64_t n, const double* w, double* scratch, double* out, cudaStream_t s) {
    k_norm2_partial<<<kRedBlocks, kThreads, 0, s>>>(n, w, scratch);
    count_launch(cudaGetLastError());
    k_norm2_final<<<1, kThreads, 0, s>>>(scratch, kRedBlocks, out);
    return count_launch(cudaGetLastError());
}

__global__ void k_scale_copy(int64_t n, const double* __restrict__ w, const double* __restrict__ nrm,
                             double* __restrict__ v) {
    const double nv = nrm[0];
    const double inv = nv > 0.0 ? 1.0 / nv : 0.0;
    GRID_STRIDE(i, n) v[i] = w[i] * inv;
}
cudaError_t launch_scale_copy(int64_t n, const double* w, const double* nrm, double* v, cudaStream_t s) {
    k_scale_copy<<<grid_for(n), kThreads, 0, s>>>(n, w, nrm, v);
    return count_launch(cudaGetLastError());
}

__global__ void k_gemv_add(int64_t n, const double* __restrict__ Z, int64_t ld, int k, const double* __restrict__ y,
                           double* __restrict__ x) {
    GRID_STRIDE(i, n) {
        double s = x[i];
        for (int j = 0; j < k; ++j) s += y[j] * Z[j * ld + i];
        x[i] = s;
    }
}
cudaError_t launch_gemv_add(int64_t n, const double* Z, int64_t ld, int k, const double* y, double* x,
                            cudaStream_t s) {
    k_gemv_add<<<grid_for(n), kThreads, 0, s>>>(n, Z, ld, k, y, x);
    return count_launch(cudaGetLastError());
}

}  // namespace pff
