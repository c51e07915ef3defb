// Q1 fast path of the level operator (Sec. 4.1, 4.2), dim 2 and 3.
//
// 1) k_q1_linearize_cell (3D) / k_q1_linearize<2> (double-float, once per state and level): for
//    every cell and Gauss point q the state enters the Jacobian only through
//      c0 = w g_kappa(phi~)                                   (G_uu: c0 sigma(du) : e(w))
//      Sp = w [2 f (1-k) phi sigma(u) + 2 p phi I]            (G_phiu: Sp : e(du) psi)
//      c1 = w [2 f (1-k) E_s(u) + 2 p div u + Gc/eps]         (G_phiphi mass part)
//    (w = Gauss weight x |K|).  They are stored per level as FP32 and as df64 pairs, cell
//    fastest, so the applies read them coalesced.
// 2) The applies y = G~ x from x and the stored coefficients, in FP32 (V-cycle operators) or df64
//    (FP64-accurate operators): k_q1_apply_cell<S> (3D levels of at least 100,000 cells: one
//    thread per cell, Gauss-point derivatives in shared memory, global atomics),
//    k_q1_apply_direct (one thread per cell and Gauss point) and k_q1_apply<DIM, S> (one thread
//    per cell, shared-memory gather) elsewhere.
// 3) The residual -A(U) (k_q1_residual_cell in 3D, k_q1_resdiag<2, 0>) and the operator
//    diagonal (k_q1_resdiag<DIM, 1>), in df64.
//
// Sum factorisation for Q1 on a uniform cell (the tensor-product structure of Sec. 4.1): the 2^d
// nodal values of a field map to 2^d "modal" coefficients m_k = sum_n prod_{a in k}(2 n_a - 1) v_n
// by d butterfly stages (a, b) -> (a + b, b - a).  In reference coordinates xi in [-1,1]^d the
// field is 2^-d sum_k m_k xi^k, so at the Gauss points xi = sigma g (g = 1/sqrt 3, sigma in
// {-1,1}^d) values and gradients are sums of scaled m_k with sign patterns sigma^k, and the
// transposed (integration) step is the same butterfly run backwards.  All sign patterns are
// compile-time constants after unrolling.
#include <cstring>

#include "pff_df64.cuh"
#include "pff_split.cuh"
#include "pff_internal.cuh"
#include "pff_q1.cuh"
#include "pff_batch.cuh"

namespace pff {

constexpr int popc(int x) { return x == 0 ? 0 : (x & 1) + popc(x >> 1); }
// sigma^k at Gauss point q: product over a in k of (+1 if bit a of q set else -1)
constexpr int sgn(int k, int q) { return (popc(k & ~q) & 1) ? -1 : 1; }

template <int DIM>
struct Q1Dims {
    static constexpr int NV = 1 << DIM;        // nodes = Gauss points = modal coefficients
    static constexpr int NC = DIM + 1;
    static constexpr int NK = DIM == 3 ? 8 : 5; // stored coefficients per Gauss point
    static constexpr int NS = DIM == 3 ? 6 : 3; // symmetric tensor components
    // Miehe split: symmetric Voigt tangent K (upper triangle), Sp, c1 per Gauss point
    static constexpr int NKK = NS * (NS + 1) / 2;
    static constexpr int NKS = NKK + NS + 1;
};

// upper-triangle position of (a, b) in a symmetric NS x NS matrix stored row by row
template <int NS>
__host__ __device__ constexpr int ut_idx(int a, int b) {
    return a <= b ? a * NS - a * (a - 1) / 2 + (b - a) : b * NS - b * (b - 1) / 2 + (a - b);
}

// symmetric index helpers: (i,j) -> 0..NS-1 with diagonal first: 3D xx yy zz xy xz yz; 2D xx yy xy
template <int DIM>
__host__ __device__ constexpr int sidx(int i, int j) {
    if (i == j) return i;
    if (DIM == 2) return 2;
    const int a = i < j ? i : j, b = i < j ? j : i;
    return a == 0 ? (b == 1 ? 3 : 4) : 5;
}

// Butterfly transforms over d stages, in place.
template <int DIM, typename S>
__device__ __forceinline__ void fwd(S* v) {
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
        for (int i = 0; i < (1 << DIM); ++i)
            if (!(i & (1 << a))) {
                const S p = v[i], q = v[i | (1 << a)];
                v[i] = p + q;
                v[i | (1 << a)] = q - p;
            }
}
// inv<3> when v[0] == 0: its first pair (0, v1) becomes (-v1, v1) without additions
template <typename S>
__device__ __forceinline__ void inv3_v0_zero(S* v) {
    v[0] = -v[1];
#pragma unroll
    for (int i = 2; i < 8; i += 2) {
        const S p = v[i], q = v[i + 1];
        v[i] = p - q;
        v[i + 1] = p + q;
    }
#pragma unroll
    for (int a = 1; a < 3; ++a)
#pragma unroll
        for (int i = 0; i < 8; ++i)
            if (!(i & (1 << a))) {
                const S p = v[i], q = v[i | (1 << a)];
                v[i] = p - q;
                v[i | (1 << a)] = p + q;
            }
}
template <int DIM, typename S>
__device__ __forceinline__ void inv(S* v) {
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
        for (int i = 0; i < (1 << DIM); ++i)
            if (!(i & (1 << a))) {
                const S p = v[i], q = v[i | (1 << a)];
                v[i] = p - q;
                v[i | (1 << a)] = p + q;
            }
}

// ------------------------------------------------------------------ linearisation data (df64)
// Constants of the linearisation as (hi, lo) float pairs, computed once on the host.
struct LinConsts {
    float2 cv[4];        // g^j / 2^d: modal coefficient -> Gauss-point value
    float2 cg[3][3];     // g^j 2 / (h_d 2^d): modal coefficient -> Gauss-point derivative along d
    float2 w;            // Gauss weight x |K|
    float2 omk, kap;     // 1 - kappa, kappa
    float2 f2k;          // 2 f (1 - kappa)
    float2 p2;           // 2 p
    float2 gce;          // Gc / eps
    float2 mu, lam;      // Lame coefficients (scaled per cell by a varying modulus)
};

__device__ __forceinline__ df64 dfc(float2 v) { return df_make(v.x, v.y); }
// exact scaling by a power of two
__device__ __forceinline__ df64 df_scale(df64 a, float s) { return df_make(a.hi * s, a.lo * s); }
__device__ __forceinline__ float df_scale(float a, float s) { return a * s; }
// hi + lo renormalised so that hi is the float nearest to the value
__device__ __forceinline__ df64 df_renorm(df64 a) { return df_two_sum(a.hi, a.lo); }

// For every cell and Gauss point q the state enters the Jacobian through c0, Sp and c1 (header
// comment).  Values at the Gauss points come from the modal coefficients by one inverse butterfly
// (v_q = sum_k sigma^k(q) cv[|k|] m_k); a Q1 derivative along d does not vary along d, so its 2^(d-1)
// distinct values come from a butterfly over the other axes.  All arithmetic in df64.
template <int DIM>
__global__ void __launch_bounds__(128) k_q1_linearize(Geom g, LinConsts k, const double* __restrict__ U,
                                                      const double* __restrict__ pt, float* __restrict__ q32,
                                                      float2* __restrict__ q64) {
    using D = Q1Dims<DIM>;
    constexpr int NV = D::NV, NK = D::NK, NH = NV / 2;
    const int64_t nc = g.n_cells, nn = g.n_nodes;
    const df64 w = dfc(k.w), omk = dfc(k.omk), kap = dfc(k.kap), f2k = dfc(k.f2k), p2 = dfc(k.p2);
    const df64 gce = dfc(k.gce);
    for (int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cell < nc;
         cell += (int64_t)gridDim.x * blockDim.x) {
        if (!cell_in(g, cell)) continue;
        int ci[3] = {0, 0, 0};
        int64_t r = cell;
        for (int a = 0; a < DIM; ++a) { ci[a] = (int)(r % g.nc[a]); r /= g.nc[a]; }
        const int64_t n0 = (int64_t)ci[0] + (int64_t)g.nn[0] * ((int64_t)ci[1] + (int64_t)g.nn[1] * ci[2]);
        const df64 sE = g.es ? df_from_double(g.es[cell]) : df_make(1.f, 0.f);
        const df64 cmu = dfc(k.mu) * sE, clam = dfc(k.lam) * sE;
        // Gauss-point values of phi and phi~
        df64 vphi[NV], vpt[NV];
#pragma unroll
        for (int n = 0; n < NV; ++n) {
            const int64_t node = n0 + (n & 1) + (int64_t)g.nn[0] * (((n >> 1) & 1) + (DIM == 3 ? (int64_t)g.nn[1] * ((n >> 2) & 1) : 0));
            vphi[n] = df_from_double(U[DIM * nn + node]);
            vpt[n] = df_from_double(pt[node]);
        }
        fwd<DIM>(vphi);
        fwd<DIM>(vpt);
#pragma unroll
        for (int m = 0; m < NV; ++m) {
            vphi[m] = vphi[m] * dfc(k.cv[popc(m)]);
            vpt[m] = vpt[m] * dfc(k.cv[popc(m)]);
        }
        inv<DIM>(vphi);
        inv<DIM>(vpt);
        // displacement derivatives: gd[c][d][j], j = Gauss-point index without bit d
        df64 gd[DIM][DIM][NH];
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
            df64 m_[NV];
#pragma unroll
            for (int n = 0; n < NV; ++n) {
                const int64_t node = n0 + (n & 1) + (int64_t)g.nn[0] * (((n >> 1) & 1) + (DIM == 3 ? (int64_t)g.nn[1] * ((n >> 2) & 1) : 0));
                m_[n] = df_from_double(U[c * nn + node]);
            }
            fwd<DIM>(m_);
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
                int j = 0;
#pragma unroll
                for (int kp = 0; kp < NV; ++kp) {
                    if (kp & (1 << d)) continue;
                    gd[c][d][j] = m_[kp | (1 << d)] * dfc(k.cg[d][popc(kp)]);
                    ++j;
                }
                inv<DIM - 1>(gd[c][d]);
#pragma unroll
                for (int jj = 0; jj < NH; ++jj) gd[c][d][jj] = df_renorm(gd[c][d][jj]);
            }
        }
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            df64 gu[DIM][DIM];
#pragma unroll
            for (int c = 0; c < DIM; ++c)
#pragma unroll
                for (int d = 0; d < DIM; ++d) {
                    const int jq = (q & ((1 << d) - 1)) | ((q >> (d + 1)) << d);   // q without bit d
                    gu[c][d] = gd[c][d][jq];
                }
            df64 e[DIM][DIM], tr = gu[0][0], ee = gu[0][0] * gu[0][0];
#pragma unroll
            for (int i = 0; i < DIM; ++i) {
                e[i][i] = gu[i][i];
                if (i > 0) { tr = tr + gu[i][i]; ee = ee + gu[i][i] * gu[i][i]; }
#pragma unroll
                for (int jx = i + 1; jx < DIM; ++jx) {
                    e[i][jx] = df_scale(gu[i][jx] + gu[jx][i], 0.5f);
                    e[jx][i] = e[i][jx];
                    ee = ee + df_scale(e[i][jx] * e[i][jx], 2.f);
                }
            }
            tr = df_renorm(tr);
            const df64 Es = df_scale(clam * tr * tr, 0.5f) + cmu * ee;
            const df64 phi = df_renorm(vphi[q]), ptv = df_renorm(vpt[q]);
            df64 vals[NK];
            vals[0] = w * (omk * ptv * ptv + kap) * sE;
            const df64 a1 = f2k * phi, b1 = p2 * phi;
            const df64 ltr = clam * tr;
#pragma unroll
            for (int i = 0; i < DIM; ++i)
#pragma unroll
                for (int jx = i; jx < DIM; ++jx) {
                    df64 sig = df_scale(cmu * e[i][jx], 2.f);
                    if (i == jx) sig = sig + ltr;
                    df64 v = a1 * sig;
                    if (i == jx) v = v + b1;
                    vals[1 + sidx<DIM>(i, jx)] = w * v;
                }
            vals[NK - 1] = w * (f2k * Es + p2 * tr + gce);
#pragma unroll
            for (int kk = 0; kk < NK; ++kk) {
                const df64 v = df_renorm(vals[kk]);
                const int64_t idx = (int64_t)(q * NK + kk) * nc + cell;
                q32[idx] = v.hi;
                q64[idx] = make_float2(v.hi, v.lo);
            }
        }
    }
}

static float2 split_pair(double d);

template <typename K>
static void fill_lin_consts(const Geom& g, const Phys& ph, K& k) {
    const int NV = 1 << g.dim;
    const double gpt = 1.0 / sqrt(3.0);
    const double gp[4] = {1.0, gpt, gpt * gpt, gpt * gpt * gpt};
    for (int j = 0; j < 4; ++j) k.cv[j] = split_pair(gp[j] / NV);
    for (int d = 0; d < 3; ++d)
        for (int j = 0; j < 3; ++j) k.cg[d][j] = split_pair(d < g.dim ? gp[j] * 2.0 / (g.h[d] * NV) : 0.0);
    double vol = 1.0;
    for (int d = 0; d < g.dim; ++d) vol *= g.h[d];
    k.w = split_pair(vol / NV);
    k.omk = split_pair(1.0 - ph.kappa);
    k.kap = split_pair(ph.kappa);
    k.f2k = split_pair(2.0 * ph.f * (1.0 - ph.kappa));
    k.p2 = split_pair(2.0 * ph.p);
    k.gce = split_pair(ph.Gc / ph.eps);
    k.mu = split_pair(ph.mu);
    k.lam = split_pair(ph.lam);
}

static cudaError_t launch_linearize_cell(const Geom& g, const LinConsts& k, const double* U, const double* pt,
                                         float* q32, float2* q64, cudaStream_t s);

cudaError_t launch_q1_linearize(const Geom& g, const Phys& ph, const double* U, const double* pt, float* q32,
                                float2* q64, cudaStream_t s) {
    LinConsts k;
    fill_lin_consts(g, ph, k);
    if (g.dim == 3) return launch_linearize_cell(g, k, U, pt, q32, q64, s);
    int64_t blocks = (g.n_cells + 127) / 128;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_q1_linearize<2><<<(int)blocks, 128, 0, s>>>(g, k, U, pt, q32, q64);
    return count_launch(cudaGetLastError());
}

// ------------------------------------------------------------------ linearisation data, Miehe split
// With the split (Sec. 2.1) the displacement block is no longer isotropic: per Gauss point the
// tangent of g(phi~) sigma^+ + sigma^- is stored as a symmetric Voigt matrix K (engineering shear
// strains, upper triangle), together with Sp = w [2 f (1-k) phi sigma^+(u) + 2 p phi I] and
// c1 = w [2 f (1-k) E_s^+ + 2 p div u + Gc/eps].  Native FP64 (eigen-decompositions); once per state.
template <int DIM>
__global__ void __launch_bounds__(128) k_q1_linearize_split(Geom g, Phys ph, const double* __restrict__ U,
                                                            const double* __restrict__ pt, double gpt,
                                                            float* __restrict__ q32, float2* __restrict__ q64) {
    using D = Q1Dims<DIM>;
    constexpr int NV = D::NV, NS = D::NS, NKK = D::NKK, NKS = D::NKS;
    const int64_t nc = g.n_cells, nn = g.n_nodes;
    double vol = 1.0;
    for (int a = 0; a < DIM; ++a) vol *= g.h[a];
    const double w = vol / NV;
    double gp[DIM + 1];
    gp[0] = 1.0;
    for (int j = 1; j <= DIM; ++j) gp[j] = gp[j - 1] * gpt;
    // Voigt index -> tensor indices (diagonal first, then xy xz yz / xy)
    const int vi[6] = {0, 1, DIM == 3 ? 2 : 0, 0, 0, 1}, vj[6] = {0, 1, DIM == 3 ? 2 : 1, 1, 2, 2};
    for (int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cell < nc;
         cell += (int64_t)gridDim.x * blockDim.x) {
        if (!cell_in(g, cell)) continue;
        int ci[3] = {0, 0, 0};
        int64_t r = cell;
        for (int a = 0; a < DIM; ++a) { ci[a] = (int)(r % g.nc[a]); r /= g.nc[a]; }
        const double sE = g.es ? g.es[cell] : 1.0;
        const double cmu = ph.mu * sE, clam = ph.lam * sE;
        double mu_[DIM][NV], mphi[NV], mpt[NV];
#pragma unroll
        for (int n = 0; n < NV; ++n) {
            const int i = ci[0] + (n & 1), j = ci[1] + ((n >> 1) & 1), k = DIM == 3 ? ci[2] + ((n >> 2) & 1) : 0;
            const int64_t node = (int64_t)i + (int64_t)g.nn[0] * ((int64_t)j + (int64_t)g.nn[1] * k);
#pragma unroll
            for (int c = 0; c < DIM; ++c) mu_[c][n] = U[c * nn + node];
            mphi[n] = U[DIM * nn + node];
            mpt[n] = pt[node];
        }
#pragma unroll
        for (int c = 0; c < DIM; ++c) fwd<DIM>(mu_[c]);
        fwd<DIM>(mphi);
        fwd<DIM>(mpt);
        for (int q = 0; q < NV; ++q) {
            double e3[3][3] = {{0.0}}, phi = 0.0, ptv = 0.0, tr = 0.0;
            for (int k = 0; k < NV; ++k) {
                const double sc = sgn(k, q) * gp[popc(k)] / NV;
                phi += sc * mphi[k];
                ptv += sc * mpt[k];
            }
            double gu[DIM][DIM];
            for (int c = 0; c < DIM; ++c)
                for (int d = 0; d < DIM; ++d) {
                    double acc = 0.0;
                    for (int kp = 0; kp < NV; ++kp) {
                        if (kp & (1 << d)) continue;
                        acc += sgn(kp, q) * gp[popc(kp)] * mu_[c][kp | (1 << d)];
                    }
                    gu[c][d] = acc * (2.0 / (g.h[d] * NV));
                }
            for (int i = 0; i < DIM; ++i)
                for (int j = 0; j < DIM; ++j) e3[i][j] = 0.5 * (gu[i][j] + gu[j][i]);
            for (int i = 0; i < DIM; ++i) tr += e3[i][i];
            double sp[3][3], Esp;
            SplitEig<double> se;
            split_stress(cmu, clam, DIM, e3, sp, Esp, se);
            const double gk = (1.0 - ph.kappa) * ptv * ptv + ph.kappa;
            double vals[NKS];
            for (int b = 0; b < NS; ++b) {
                // unit engineering strain b: e_ii = 1 or e_ij = e_ji = 1/2
                double E[3][3] = {{0.0}}, cp[3][3];
                if (vi[b] == vj[b]) E[vi[b]][vi[b]] = 1.0;
                else { E[vi[b]][vj[b]] = 0.5; E[vj[b]][vi[b]] = 0.5; }
                split_tangent(cmu, clam, DIM, se, E, cp);
                const double trE = vi[b] == vj[b] ? 1.0 : 0.0;
                for (int a = b; a < NS; ++a) {
                    const int i = vi[a], j = vj[a];
                    const double full = 2.0 * cmu * E[i][j] + (i == j ? clam * trE : 0.0);
                    vals[ut_idx<NS>(b, a)] = w * (full - (1.0 - gk) * cp[i][j]);
                }
            }
            for (int a = 0; a < NS; ++a) {
                const int i = vi[a], j = vj[a];
                vals[NKK + a] = w * (2.0 * ph.f * (1.0 - ph.kappa) * phi * sp[i][j] + (i == j ? 2.0 * ph.p * phi : 0.0));
            }
            vals[NKS - 1] = w * (2.0 * ph.f * (1.0 - ph.kappa) * Esp + 2.0 * ph.p * tr + ph.Gc / ph.eps);
            for (int k = 0; k < NKS; ++k) {
                const int64_t idx = (int64_t)(q * NKS + k) * nc + cell;
                const float hi = __double2float_rn(vals[k]);
                q32[idx] = hi;
                q64[idx] = make_float2(hi, __double2float_rn(vals[k] - (double)hi));
            }
        }
    }
}

cudaError_t launch_q1_linearize_split(const Geom& g, const Phys& ph, const double* U, const double* pt, float* q32,
                                      float2* q64, cudaStream_t s) {
    const double gpt = 1.0 / sqrt(3.0);
    int64_t blocks = (g.n_cells + 127) / 128;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    if (g.dim == 3) k_q1_linearize_split<3><<<(int)blocks, 128, 0, s>>>(g, ph, U, pt, gpt, q32, q64);
    else k_q1_linearize_split<2><<<(int)blocks, 128, 0, s>>>(g, ph, U, pt, gpt, q32, q64);
    return count_launch(cudaGetLastError());
}

// ------------------------------------------------------------------ modal apply
template <int DIM, typename S>
struct Q1Tile;
template <> struct Q1Tile<3, float> { static constexpr int TX = 16, TY = 4, TZ = 2, MINB = 4; };
template <> struct Q1Tile<3, df64> { static constexpr int TX = 8, TY = 4, TZ = 4, MINB = 1; };
template <> struct Q1Tile<2, float> { static constexpr int TX = 16, TY = 16, TZ = 1, MINB = 2; };
template <> struct Q1Tile<2, df64> { static constexpr int TX = 16, TY = 8, TZ = 1, MINB = 1; };

template <typename S>
__device__ __forceinline__ S cpair(float2 v);
template <>
__device__ __forceinline__ float cpair<float>(float2 v) { return v.x; }
template <>
__device__ __forceinline__ df64 cpair<df64>(float2 v) { return df_make(v.x, v.y); }

static float2 split_pair(double d) {
    const float hi = (float)d;
    return make_float2(hi, (float)(d - (double)hi));
}

Q1Consts make_q1_consts(const Geom& g, const Phys& ph) {
    Q1Consts k;
    const int dim = g.dim, NV = 1 << dim;
    const double gpt = 1.0 / sqrt(3.0);
    const double gp[4] = {1.0, gpt, gpt * gpt, gpt * gpt * gpt};
    for (int j = 0; j <= 3; ++j) k.cv[j] = split_pair(gp[j] / NV);
    for (int d = 0; d < 3; ++d)
        for (int j = 0; j < 3; ++j) k.cg[d][j] = split_pair(d < dim ? gp[j] * 2.0 / (g.h[d] * NV) : 0.0);
    double vol = 1.0;
    for (int d = 0; d < dim; ++d) vol *= g.h[d];
    k.mu = split_pair(ph.mu);
    k.mu2 = split_pair(2.0 * ph.mu);
    k.lam = split_pair(ph.lam);
    k.gcew = split_pair(ph.Gc * ph.eps * vol / NV);
    for (int kk = 0; kk < 8; ++kk) {
        double acc = 0.0;
        for (int d = 0; d < dim; ++d) {
            if (kk >= NV || !(kk & (1 << d))) continue;
            int pc = 0;
            for (int b = 0; b < dim; ++b) pc += (kk >> b) & 1;
            const double c = gp[pc - 1] * 2.0 / (g.h[d] * NV);
            acc += c * c;
        }
        k.gk[kk] = split_pair(ph.Gc * ph.eps * vol * acc);   // 2^d (Gc eps vol / 2^d) sum cg^2
    }
    k.g2 = split_pair(0.5 * gpt);
    k.al = split_pair(0.5 * (1.0 + gpt));
    k.be = split_pair(0.5 * (1.0 - gpt));
    for (int d = 0; d < 3; ++d) k.ih[d] = split_pair(d < dim ? 1.0 / g.h[d] : 0.0);
    return k;
}

template <typename S>
struct QData;
template <> struct QData<float> {
    using type = float;
    __device__ static __forceinline__ float get(const float* p, int64_t i) { return __ldg(p + i); }
};
template <> struct QData<df64> {
    using type = float2;
    __device__ static __forceinline__ df64 get(const float2* p, int64_t i) {
        const float2 v = __ldg(p + i);
        return df_make(v.x, v.y);
    }
};

// Miehe split: flux of the displacement block at one Gauss point, sigma = K eps with the stored
// symmetric Voigt tangent K (upper triangle at base + ut_idx * stride) and the engineering strain
// eps of the gradient g_ of du.
template <int DIM, typename S, typename QT>
__device__ __forceinline__ void split_flux(const QT* qd, int64_t base, int64_t stride, const S (&g_)[DIM][DIM],
                                           S (&fu)[DIM][DIM]) {
    constexpr int NS = Q1Dims<DIM>::NS;
    S ev[NS], sv[NS];
#pragma unroll
    for (int i = 0; i < DIM; ++i)
#pragma unroll
        for (int j = i; j < DIM; ++j) ev[sidx<DIM>(i, j)] = (i == j) ? g_[i][i] : g_[i][j] + g_[j][i];
#pragma unroll
    for (int a = 0; a < NS; ++a) sv[a] = Scalar<S>::zero();
#pragma unroll
    for (int a = 0; a < NS; ++a)
#pragma unroll
        for (int b = a; b < NS; ++b) {
            const S kab = QData<S>::get(qd, base + (int64_t)ut_idx<NS>(a, b) * stride);
            sv[a] = sv[a] + kab * ev[b];
            if (a != b) sv[b] = sv[b] + kab * ev[a];
        }
#pragma unroll
    for (int i = 0; i < DIM; ++i)
#pragma unroll
        for (int j = i; j < DIM; ++j) {
            fu[i][j] = sv[sidx<DIM>(i, j)];
            fu[j][i] = fu[i][j];
        }
}

// kg: the Gauss-point scalings in global memory (batched launches), nullptr to read them from the
// kernel parameters (a.k).  SPLIT: Gauss-point data of the Miehe split (K, Sp, c1).
template <int DIM, typename S, bool BLOCKDIAG, bool SPLIT = false>
__device__ __forceinline__ void q1_apply_tile(const Q1ApplyArgs<typename Scalar<S>::storage, typename QData<S>::type>& a,
                                              int bx, int by, int bz, const Q1Consts* __restrict__ kg = nullptr) {
    using T = Q1Tile<DIM, S>;
    using D = Q1Dims<DIM>;
    using St = typename Scalar<S>::storage;
    constexpr int NV = D::NV, NC = D::NC, NK = SPLIT ? D::NKS : D::NK, SPO = SPLIT ? D::NKK : 1;
    constexpr int NCELL = T::TX * T::TY * T::TZ;
    constexpr int NTX = T::TX + 1, NTY = T::TY + 1, NTZ = DIM == 3 ? T::TZ + 1 : 1;
    constexpr int NT = NTX * NTY * NTZ;

    __shared__ S sx[NC * NT];
    __shared__ S sel[NV * NC * NCELL];
    __shared__ uint8_t smask[NT];

    const Geom& g = a.g;
    const int ci0 = bx * T::TX, cj0 = by * T::TY, ck0 = DIM == 3 ? bz * T::TZ : 0;
    const int64_t nn = g.n_nodes;

    for (int t = threadIdx.x; t < NT; t += blockDim.x) {
        const int ti = t % NTX, tj = (t / NTX) % NTY, tk = t / (NTX * NTY);
        const int gi = ci0 + ti, gj = cj0 + tj, gk = ck0 + tk;
        const bool in = gi < g.nn[0] && gj < g.nn[1] && gk < g.nn[2];
        const int64_t gn = in ? (int64_t)gi + (int64_t)g.nn[0] * ((int64_t)gj + (int64_t)g.nn[1] * gk) : 0;
        const uint8_t m = in ? a.mask[gn] : 0;
        smask[t] = m;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const bool el = c < DIM ? ((m >> c) & 1) != 0 : (m & a.phi_bits) != 0;
            sx[c * NT + t] = (in && !el) ? Scalar<S>::load(a.x[c * nn + gn]) : Scalar<S>::zero();
        }
    }
    __syncthreads();

    const int cell = threadIdx.x;
    const int li = cell % T::TX, lj = (cell / T::TX) % T::TY, lk = cell / (T::TX * T::TY);
    const bool valid = (ci0 + li < g.nc[0]) && (cj0 + lj < g.nc[1]) && (DIM == 2 || ck0 + lk < g.nc[2]) &&
                       cell_in(g, (int64_t)(ci0 + li) + (int64_t)g.nc[0] * ((int64_t)(cj0 + lj) + (int64_t)g.nc[1] * (ck0 + lk)));
    if (valid) {
        const int64_t gid = (int64_t)(ci0 + li) + (int64_t)g.nc[0] * ((int64_t)(cj0 + lj) + (int64_t)g.nc[1] * (ck0 + lk));
        const int tb = li + NTX * (lj + NTY * lk);
        // Gauss-point scalings read straight from the kernel parameters or global memory (a local
        // copy indexed in the unrolled loops ended up in local memory)
        auto cv = [&](int j) { return cpair<S>(kg ? kg->cv[j] : a.k.cv[j]); };
        auto cg = [&](int d, int j) { return cpair<S>(kg ? kg->cg[d][j] : a.k.cg[d][j]); };
        const S mu2 = cpair<S>(a.k.mu2), lam = cpair<S>(a.k.lam);

        const S mu = cpair<S>(a.k.mu);

        // ======== pass 1: displacement rows (G_uu) and the coupling term of the phi rows.
        // A Q1 derivative along d does not vary along d: its 2^(d-1) Gauss-point values come from an
        // inverse butterfly over the other axes; integration against the test-function derivatives
        // is the transposed (forward) butterfly of the Gauss-point fluxes summed in pairs along d.
        constexpr int NH = NV / 2;
        S cpl[NV];
        {
            S gd[DIM][DIM][NH];
#pragma unroll
            for (int c = 0; c < DIM; ++c) {
                S v[NV];
#pragma unroll
                for (int n = 0; n < NV; ++n) {
                    const int off = (n & 1) + NTX * (((n >> 1) & 1) + NTY * (DIM == 3 ? (n >> 2) & 1 : 0));
                    v[n] = sx[c * NT + tb + off];
                }
                fwd<DIM>(v);
#pragma unroll
                for (int d = 0; d < DIM; ++d) {
                    int j = 0;
#pragma unroll
                    for (int kp = 0; kp < NV; ++kp) {
                        if (kp & (1 << d)) continue;
                        gd[c][d][j] = v[kp | (1 << d)] * cg(d, popc(kp));
                        ++j;
                    }
                    inv<DIM - 1>(gd[c][d]);
                }
            }
            S ps[DIM][DIM][NH];
#pragma unroll
            for (int c = 0; c < DIM; ++c)
#pragma unroll
                for (int d = 0; d < DIM; ++d)
#pragma unroll
                    for (int j = 0; j < NH; ++j) ps[c][d][j] = Scalar<S>::zero();
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                S g_[DIM][DIM];
#pragma unroll
                for (int c = 0; c < DIM; ++c)
#pragma unroll
                    for (int d = 0; d < DIM; ++d) g_[c][d] = gd[c][d][(q & ((1 << d) - 1)) | ((q >> (d + 1)) << d)];
                S fs[DIM][DIM];
                if constexpr (SPLIT) split_flux<DIM, S>(a.qd, (int64_t)(q * NK) * g.n_cells + gid, g.n_cells, g_, fs);
                const S c0 = SPLIT ? Scalar<S>::zero() : QData<S>::get(a.qd, (int64_t)(q * NK + 0) * g.n_cells + gid);
                S tr = g_[0][0];
#pragma unroll
                for (int i = 1; i < DIM; ++i) tr = tr + g_[i][i];
                const S ltr = lam * tr;
                S cp = Scalar<S>::zero();
                if constexpr (!BLOCKDIAG) {
#pragma unroll
                    for (int i = 0; i < DIM; ++i)
#pragma unroll
                        for (int j = i; j < DIM; ++j) {
                            const S sp = QData<S>::get(a.qd, (int64_t)(q * NK + SPO + sidx<DIM>(i, j)) * g.n_cells + gid);
                            cp = cp + sp * ((i == j) ? g_[i][i] : g_[i][j] + g_[j][i]);   // Sp : e(du)
                        }
                }
                cpl[q] = cp;
#pragma unroll
                for (int i = 0; i < DIM; ++i)
#pragma unroll
                    for (int j = i; j < DIM; ++j) {
                        // c0 sigma(du)_ij with sigma = 2 mu e + lambda tr I and 2 e_ij = du_i,j + du_j,i
                        const S sg = (i == j) ? mu2 * g_[i][i] + ltr : mu * (g_[i][j] + g_[j][i]);
                        const S f = SPLIT ? fs[i][j] : c0 * sg;
                        const int ji = (q & ((1 << j) - 1)) | ((q >> (j + 1)) << j);
                        ps[i][j][ji] = ps[i][j][ji] + f;
                        if (i != j) {
                            const int jj = (q & ((1 << i) - 1)) | ((q >> (i + 1)) << i);
                            ps[j][i][jj] = ps[j][i][jj] + f;
                        }
                    }
            }
#pragma unroll
            for (int c = 0; c < DIM; ++c) {
#pragma unroll
                for (int d = 0; d < DIM; ++d) fwd<DIM - 1>(ps[c][d]);
                S Y[NV];
#pragma unroll
                for (int k = 0; k < NV; ++k) {
                    S acc = Scalar<S>::zero();
#pragma unroll
                    for (int d = 0; d < DIM; ++d) {
                        if (!(k & (1 << d))) continue;
                        const int kp = k & ~(1 << d);
                        const int j = (kp & ((1 << d) - 1)) | ((kp >> (d + 1)) << d);   // kp without bit d
                        acc = acc + ps[c][d][j] * cg(d, popc(kp));
                    }
                    Y[k] = acc;
                }
                inv<DIM>(Y);
#pragma unroll
                for (int n = 0; n < NV; ++n) sel[(n * NC + c) * NCELL + cell] = Y[n];
            }
        }
        // ======== pass 2: phase-field rows.  Values at the Gauss points by an inverse butterfly;
        // the gradient-gradient term is diagonal in modal coefficients (factor 2^d).
        {
            S v[NV];
#pragma unroll
            for (int n = 0; n < NV; ++n) {
                const int off = (n & 1) + NTX * (((n >> 1) & 1) + NTY * (DIM == 3 ? (n >> 2) & 1 : 0));
                v[n] = sx[DIM * NT + tb + off];
            }
            fwd<DIM>(v);
            S F[NV];
#pragma unroll
            for (int k = 0; k < NV; ++k) F[k] = v[k] * cv(popc(k));
            inv<DIM>(F);
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                const S c1 = QData<S>::get(a.qd, (int64_t)(q * NK + NK - 1) * g.n_cells + gid);
                F[q] = c1 * F[q] + cpl[q];
            }
            fwd<DIM>(F);
            S Y[NV];
            Y[0] = F[0] * cv(0);
            // gradient-gradient term: diagonal in modal coefficients, factor gk
#pragma unroll
            for (int k = 1; k < NV; ++k) Y[k] = F[k] * cv(popc(k)) + v[k] * cpair<S>(kg ? kg->gk[k] : a.k.gk[k]);
            inv<DIM>(Y);
#pragma unroll
            for (int n = 0; n < NV; ++n) sel[(n * NC + DIM) * NCELL + cell] = Y[n];
        }
    } else {
#pragma unroll
        for (int k = 0; k < NV * NC; ++k) sel[k * NCELL + cell] = Scalar<S>::zero();
    }
    __syncthreads();

    // ---- node gather (fixed order over the tile's cells), one global add per tile node
    for (int t = threadIdx.x; t < NT; t += blockDim.x) {
        const int ti = t % NTX, tj = (t / NTX) % NTY, tk = t / (NTX * NTY);
        const int gi = ci0 + ti, gj = cj0 + tj, gk = ck0 + tk;
        if (!(gi < g.nn[0] && gj < g.nn[1] && gk < g.nn[2])) continue;
        const int64_t gn = (int64_t)gi + (int64_t)g.nn[0] * ((int64_t)gj + (int64_t)g.nn[1] * gk);
        const uint8_t m = smask[t];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const bool el = c < DIM ? ((m >> c) & 1) != 0 : (m & a.phi_bits) != 0;
            if (el) continue;
            S s = Scalar<S>::zero();
#pragma unroll
            for (int dk = 0; dk < (DIM == 3 ? 2 : 1); ++dk) {
                const int ck = tk - dk;
                if (DIM == 3 && (ck < 0 || ck >= T::TZ)) continue;
#pragma unroll
                for (int dj = 0; dj < 2; ++dj) {
                    const int cj = tj - dj;
                    if (cj < 0 || cj >= T::TY) continue;
#pragma unroll
                    for (int di = 0; di < 2; ++di) {
                        const int cx = ti - di;
                        if (cx < 0 || cx >= T::TX) continue;
                        const int n = di + 2 * dj + 4 * dk;
                        s = s + sel[(n * NC + c) * NCELL + cx + T::TX * (cj + T::TY * (DIM == 3 ? ck : 0))];
                    }
                }
            }
            atomicAdd(&a.y[c * nn + gn], Scalar<S>::store(s));
        }
    }
}

// ------------------------------------------------------------------ lane apply
// One thread per (cell, node) = (cell, Gauss point): 2^d lanes of a warp form a cell.  Lane n
// holds node n's value and, after one shuffle butterfly per axis e, the value at Gauss point
// n: along e the pair (a, b) becomes ((1+g)/2 a + (1-g)/2 b, (1-g)/2 a + (1+g)/2 b), written
// per lane as (v + p)/2 + (g/2)(v - p) with p the partner's value; the derivative channel of axis
// e is s_e (v - p) / h_e (s_e = +1 on the upper side).  Integration runs the transposed
// butterflies in reverse axis order: the interpolation matrix is symmetric, and the derivative
// stage transposes to s_e (f + p) / h_e.
template <typename S>
__device__ __forceinline__ S shfl_xor(S v, int m);
template <>
__device__ __forceinline__ float shfl_xor<float>(float v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
template <>
__device__ __forceinline__ df64 shfl_xor<df64>(df64 v, int m) {
    return df_make(__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m));
}
__device__ __forceinline__ float half_of(float v) { return 0.5f * v; }
__device__ __forceinline__ df64 half_of(df64 v) { return df_make(0.5f * v.hi, 0.5f * v.lo); }

template <int DIM, typename S>
struct LaneConst {
    S g2;           // g / 2
    S al, be;       // (1 + g) / 2, (1 - g) / 2: interpolation weights of the near and far node
    S ih[DIM];      // 1 / h_e
};

// value (if WANT_VAL) and gradient at this lane's Gauss point from this lane's nodal value
template <int DIM, typename S, bool WANT_VAL>
__device__ __forceinline__ void lane_eval(S v, int n, const LaneConst<DIM, S>& k, S& val, S (&grad)[DIM]) {
#pragma unroll
    for (int e = 0; e < DIM; ++e) {
        // derivative channels of earlier axes are interpolated along e
#pragma unroll
        for (int d = 0; d < e; ++d) {
            const S p = shfl_xor(grad[d], 1 << e);
            grad[d] = k.al * grad[d] + k.be * p;
        }
        const S p = shfl_xor(v, 1 << e);
        const S diff = v - p;
        grad[e] = ((n >> e) & 1) ? diff * k.ih[e] : -(diff * k.ih[e]);
        if (WANT_VAL || e + 1 < DIM) v = k.al * v + k.be * p;
    }
    if (WANT_VAL) val = v;
}

// transposed: fluxes on the test function value (fv, if HAS_VAL) and gradient (fg) at this
// lane's Gauss point -> contribution to this lane's node
template <int DIM, typename S, bool HAS_VAL>
__device__ __forceinline__ S lane_integrate(S fv, S (&fg)[DIM], int n, const LaneConst<DIM, S>& k) {
    S tv = fv;
#pragma unroll
    for (int e = DIM - 1; e >= 0; --e) {
        const S pd = shfl_xor(fg[e], 1 << e);
        const S td = ((n >> e) & 1) ? (fg[e] + pd) * k.ih[e] : -((fg[e] + pd) * k.ih[e]);
        if (HAS_VAL || e + 1 < DIM) {
            const S p = shfl_xor(tv, 1 << e);
            tv = k.al * tv + k.be * p + td;
        } else {
            tv = td;
        }
#pragma unroll
        for (int d = 0; d < e; ++d) {
            const S p = shfl_xor(fg[d], 1 << e);
            fg[d] = k.al * fg[d] + k.be * p;
        }
    }
    return tv;
}

template <int DIM>
struct LaneTile;
template <> struct LaneTile<3> { static constexpr int TX = 4, TY = 4, TZ = 2; };
template <> struct LaneTile<2> { static constexpr int TX = 8, TY = 8, TZ = 1; };

template <int DIM, typename S, bool BLOCKDIAG>
__device__ __forceinline__ void q1_apply_lanes_tile(
    const Q1ApplyArgs<typename Scalar<S>::storage, typename QData<S>::type>& a, int bx, int by, int bz) {
    using T = LaneTile<DIM>;
    using D = Q1Dims<DIM>;
    constexpr int NV = D::NV, NC = D::NC, NK = D::NK;
    constexpr int NCELL = T::TX * T::TY * T::TZ;
    constexpr int NTX = T::TX + 1, NTY = T::TY + 1, NTZ = DIM == 3 ? T::TZ + 1 : 1;
    constexpr int NT = NTX * NTY * NTZ;
    static_assert(NCELL * NV == 256, "one CTA = 256 lanes");

    __shared__ S sx[NC * NT];
    __shared__ S sel[NV * NC * NCELL];
    __shared__ uint8_t smask[NT];

    const Geom& g = a.g;
    const int ci0 = bx * T::TX, cj0 = by * T::TY, ck0 = DIM == 3 ? bz * T::TZ : 0;
    const int64_t nn = g.n_nodes;
    for (int t = threadIdx.x; t < NT; t += blockDim.x) {
        const int ti = t % NTX, tj = (t / NTX) % NTY, tk = t / (NTX * NTY);
        const int gi = ci0 + ti, gj = cj0 + tj, gk = ck0 + tk;
        const bool in = gi < g.nn[0] && gj < g.nn[1] && gk < g.nn[2];
        const int64_t gn = in ? (int64_t)gi + (int64_t)g.nn[0] * ((int64_t)gj + (int64_t)g.nn[1] * gk) : 0;
        const uint8_t m = in ? a.mask[gn] : 0;
        smask[t] = m;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const bool el = c < DIM ? ((m >> c) & 1) != 0 : (m & a.phi_bits) != 0;
            sx[c * NT + t] = (in && !el) ? Scalar<S>::load(a.x[c * nn + gn]) : Scalar<S>::zero();
        }
    }
    __syncthreads();

    const int cell = threadIdx.x / NV, n = threadIdx.x % NV;
    const int li = cell % T::TX, lj = (cell / T::TX) % T::TY, lk = cell / (T::TX * T::TY);
    const bool valid = (ci0 + li < g.nc[0]) && (cj0 + lj < g.nc[1]) && (DIM == 2 || ck0 + lk < g.nc[2]) &&
                       cell_in(g, (int64_t)(ci0 + li) + (int64_t)g.nc[0] * ((int64_t)(cj0 + lj) + (int64_t)g.nc[1] * (ck0 + lk)));
    // every lane runs the shuffles; invalid cells work on zeros and are not stored
    const int tnode = (li + (n & 1)) + NTX * ((lj + ((n >> 1) & 1)) + NTY * (DIM == 3 ? lk + ((n >> 2) & 1) : 0));
    const int64_t gid = valid ? (int64_t)(ci0 + li) + (int64_t)g.nc[0] * ((int64_t)(cj0 + lj) + (int64_t)g.nc[1] * (ck0 + lk)) : 0;
    LaneConst<DIM, S> k;
    k.g2 = cpair<S>(a.k.g2);
    k.al = cpair<S>(a.k.al);
    k.be = cpair<S>(a.k.be);
#pragma unroll
    for (int d = 0; d < DIM; ++d) k.ih[d] = cpair<S>(a.k.ih[d]);
    const S mu = cpair<S>(a.k.mu), mu2 = cpair<S>(a.k.mu2);
    const S lam = cpair<S>(a.k.lam), gcew = cpair<S>(a.k.gcew);

    // displacement gradients at Gauss point n
    S gd[DIM][DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
        S dummy;
        lane_eval<DIM, S, false>(sx[c * NT + tnode], n, k, dummy, gd[c]);
    }
    S dphi, gphi[DIM];
    lane_eval<DIM, S, true>(sx[DIM * NT + tnode], n, k, dphi, gphi);
    const int64_t qbase = (int64_t)(n * NK) * g.n_cells + gid;
    const S c0 = valid ? QData<S>::get(a.qd, qbase) : Scalar<S>::zero();
    const S c1 = valid ? QData<S>::get(a.qd, qbase + (int64_t)(NK - 1) * g.n_cells) : Scalar<S>::zero();
    S tr = gd[0][0];
#pragma unroll
    for (int i = 1; i < DIM; ++i) tr = tr + gd[i][i];
    const S ltr = lam * tr;
    S fu[DIM][DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i)
#pragma unroll
        for (int j = i; j < DIM; ++j) {
            const S sg = (i == j) ? mu2 * gd[i][i] + ltr : mu * (gd[i][j] + gd[j][i]);
            const S f = c0 * sg;
            fu[i][j] = f;
            fu[j][i] = f;
        }
    S fp = c1 * dphi;
    if constexpr (!BLOCKDIAG) {
#pragma unroll
        for (int i = 0; i < DIM; ++i)
#pragma unroll
            for (int j = i; j < DIM; ++j) {
                const S sp = valid ? QData<S>::get(a.qd, qbase + (int64_t)(1 + sidx<DIM>(i, j)) * g.n_cells)
                                   : Scalar<S>::zero();
                fp = fp + sp * ((i == j) ? gd[i][i] : gd[i][j] + gd[j][i]);
            }
    }
    S out[NC];
#pragma unroll
    for (int c = 0; c < DIM; ++c) out[c] = lane_integrate<DIM, S, false>(Scalar<S>::zero(), fu[c], n, k);
    S fg[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) fg[d] = gcew * gphi[d];
    out[DIM] = lane_integrate<DIM, S, true>(fp, fg, n, k);
#pragma unroll
    for (int c = 0; c < NC; ++c) sel[(n * NC + c) * NCELL + cell] = valid ? out[c] : Scalar<S>::zero();
    __syncthreads();

    for (int t = threadIdx.x; t < NT; t += blockDim.x) {
        const int ti = t % NTX, tj = (t / NTX) % NTY, tk = t / (NTX * NTY);
        const int gi = ci0 + ti, gj = cj0 + tj, gk = ck0 + tk;
        if (!(gi < g.nn[0] && gj < g.nn[1] && gk < g.nn[2])) continue;
        const int64_t gn = (int64_t)gi + (int64_t)g.nn[0] * ((int64_t)gj + (int64_t)g.nn[1] * gk);
        const uint8_t m = smask[t];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const bool el = c < DIM ? ((m >> c) & 1) != 0 : (m & a.phi_bits) != 0;
            if (el) continue;
            S sum = Scalar<S>::zero();
#pragma unroll
            for (int dk = 0; dk < (DIM == 3 ? 2 : 1); ++dk) {
                const int ck = tk - dk;
                if (DIM == 3 && (ck < 0 || ck >= T::TZ)) continue;
#pragma unroll
                for (int dj = 0; dj < 2; ++dj) {
                    const int cj = tj - dj;
                    if (cj < 0 || cj >= T::TY) continue;
#pragma unroll
                    for (int di = 0; di < 2; ++di) {
                        const int cx = ti - di;
                        if (cx < 0 || cx >= T::TX) continue;
                        const int nl = di + 2 * dj + 4 * dk;
                        sum = sum + sel[(nl * NC + c) * NCELL + cx + T::TX * (cj + T::TY * (DIM == 3 ? ck : 0))];
                    }
                }
            }
            atomicAdd(&a.y[c * nn + gn], Scalar<S>::store(sum));
        }
    }
}

// Lane apply without shared memory: every lane reads its node's x from global memory (neighbour
// cells hit the caches) and adds its contribution to y with one atomic per component; no CTA
// barrier.  Same arithmetic as q1_apply_lanes_tile.
template <int DIM, typename S, bool BLOCKDIAG, bool SPLIT = false>
__device__ __forceinline__ void q1_direct_tile(const Q1ApplyArgs<typename Scalar<S>::storage, typename QData<S>::type>& a,
                                               int bx, int by, int bz) {
    using T = LaneTile<DIM>;
    using D = Q1Dims<DIM>;
    constexpr int NV = D::NV, NC = D::NC, NK = SPLIT ? D::NKS : D::NK, SPO = SPLIT ? D::NKK : 1;
    const Geom& g = a.g;
    const int ci0 = bx * T::TX, cj0 = by * T::TY, ck0 = DIM == 3 ? bz * T::TZ : 0;
    const int64_t nn = g.n_nodes;
    const int cell = threadIdx.x / NV, n = threadIdx.x % NV;
    const int li = cell % T::TX, lj = (cell / T::TX) % T::TY, lk = cell / (T::TX * T::TY);
    const bool valid = (ci0 + li < g.nc[0]) && (cj0 + lj < g.nc[1]) && (DIM == 2 || ck0 + lk < g.nc[2]) &&
                       cell_in(g, (int64_t)(ci0 + li) + (int64_t)g.nc[0] * ((int64_t)(cj0 + lj) + (int64_t)g.nc[1] * (ck0 + lk)));
    const int gi = ci0 + li + (n & 1), gj = cj0 + lj + ((n >> 1) & 1), gk = DIM == 3 ? ck0 + lk + ((n >> 2) & 1) : 0;
    const int64_t gn = valid ? (int64_t)gi + (int64_t)g.nn[0] * ((int64_t)gj + (int64_t)g.nn[1] * gk) : 0;
    const int64_t gid = valid ? (int64_t)(ci0 + li) + (int64_t)g.nc[0] * ((int64_t)(cj0 + lj) + (int64_t)g.nc[1] * (ck0 + lk)) : 0;
    const uint8_t m = valid ? a.mask[gn] : 0;
    bool el[NC];
    S xv[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        el[c] = c < DIM ? ((m >> c) & 1) != 0 : (m & a.phi_bits) != 0;
        xv[c] = (valid && !el[c]) ? Scalar<S>::load(a.x[c * nn + gn]) : Scalar<S>::zero();
    }
    LaneConst<DIM, S> k;
    k.g2 = cpair<S>(a.k.g2);
    k.al = cpair<S>(a.k.al);
    k.be = cpair<S>(a.k.be);
#pragma unroll
    for (int d = 0; d < DIM; ++d) k.ih[d] = cpair<S>(a.k.ih[d]);
    const S mu = cpair<S>(a.k.mu), mu2 = cpair<S>(a.k.mu2);
    const S lam = cpair<S>(a.k.lam), gcew = cpair<S>(a.k.gcew);
    S gd[DIM][DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
        S dummy;
        lane_eval<DIM, S, false>(xv[c], n, k, dummy, gd[c]);
    }
    S dphi, gphi[DIM];
    lane_eval<DIM, S, true>(xv[DIM], n, k, dphi, gphi);
    const int64_t qbase = (int64_t)(n * NK) * g.n_cells + gid;
    const S c0 = (valid && !SPLIT) ? QData<S>::get(a.qd, qbase) : Scalar<S>::zero();
    const S c1 = valid ? QData<S>::get(a.qd, qbase + (int64_t)(NK - 1) * g.n_cells) : Scalar<S>::zero();
    S tr = gd[0][0];
#pragma unroll
    for (int i = 1; i < DIM; ++i) tr = tr + gd[i][i];
    const S ltr = lam * tr;
    S fu[DIM][DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i)
#pragma unroll
        for (int j = i; j < DIM; ++j) {
            const S sg = (i == j) ? mu2 * gd[i][i] + ltr : mu * (gd[i][j] + gd[j][i]);
            const S f = c0 * sg;
            fu[i][j] = f;
            fu[j][i] = f;
        }
    if constexpr (SPLIT) {
        if (valid) split_flux<DIM, S>(a.qd, qbase, g.n_cells, gd, fu);
    }
    S fp = c1 * dphi;
    if constexpr (!BLOCKDIAG) {
#pragma unroll
        for (int i = 0; i < DIM; ++i)
#pragma unroll
            for (int j = i; j < DIM; ++j) {
                const S sp = valid ? QData<S>::get(a.qd, qbase + (int64_t)(SPO + sidx<DIM>(i, j)) * g.n_cells)
                                   : Scalar<S>::zero();
                fp = fp + sp * ((i == j) ? gd[i][i] : gd[i][j] + gd[j][i]);
            }
    }
    S out[NC];
#pragma unroll
    for (int c = 0; c < DIM; ++c) out[c] = lane_integrate<DIM, S, false>(Scalar<S>::zero(), fu[c], n, k);
    S fg[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) fg[d] = gcew * gphi[d];
    out[DIM] = lane_integrate<DIM, S, true>(fp, fg, n, k);
    if (valid) {
#pragma unroll
        for (int c = 0; c < NC; ++c)
            if (!el[c]) atomicAdd(&a.y[c * nn + gn], Scalar<S>::store(out[c]));
    }
}

template <int DIM, typename S, bool BLOCKDIAG, bool SPLIT = false>
__global__ void __launch_bounds__(256) k_q1_apply_direct(Q1ApplyArgs<typename Scalar<S>::storage, typename QData<S>::type> a) {
    q1_direct_tile<DIM, S, BLOCKDIAG, SPLIT>(a, blockIdx.x, blockIdx.y, blockIdx.z);
}

template <int DIM, typename S, bool BLOCKDIAG, bool SPLIT = false>
__global__ void __launch_bounds__(Q1Tile<DIM, S>::TX * Q1Tile<DIM, S>::TY * Q1Tile<DIM, S>::TZ, Q1Tile<DIM, S>::MINB)
k_q1_apply(Q1ApplyArgs<typename Scalar<S>::storage, typename QData<S>::type> a) {
    q1_apply_tile<DIM, S, BLOCKDIAG, SPLIT>(a, blockIdx.x, blockIdx.y, blockIdx.z);
}

template <int DIM, typename S, bool BLOCKDIAG>
__global__ void __launch_bounds__(256) k_q1_apply_lanes(Q1ApplyArgs<typename Scalar<S>::storage, typename QData<S>::type> a) {
    q1_apply_lanes_tile<DIM, S, BLOCKDIAG>(a, blockIdx.x, blockIdx.y, blockIdx.z);
}

// ------------------------------------------------------------------ per-cell apply
// One thread per cell (df64 for the FP64-accurate operator, or FP32), modal form (3D).  After the modal transform of a displacement
// component, the 4 distinct Gauss-point values of each derivative (c, d) go to shared memory, so
// only the flux accumulators stay in registers through the Gauss-point loop (about 100
// registers: four 128-thread CTAs per SM, limited by the 53 KB of shared memory each); the
// accumulators then return to the same shared slots and each component's element vector is added
// to y with FP64 atomics (no element buffer, no node gather, one CTA barrier).  The per-component
// stages are loops, not unrolled, to keep the code small (the fully unrolled form stalled on
// instruction fetch).  Arithmetic as in q1_apply_tile.
struct CellTile { static constexpr int TX = 16, TY = 4, TZ = 2; };

// The work of one CTA: tile (bx, by, bz) of the level; K: the Gauss-point scalings (kernel
// parameters, or the instance's descriptor in a batched launch); cell_smem: the dynamic shared
// memory of cell_smem_bytes<S>().
template <typename S, bool BLOCKDIAG>
__device__ __forceinline__ void q1_cell_tile(const Q1ApplyArgs<typename Scalar<S>::storage, typename QData<S>::type>& a,
                                             const Q1Consts& K, int bx, int by, int bz, unsigned char* cell_smem) {
    using T = CellTile;
    constexpr int NV = 8, NC = 4, NH = 4, NK = Q1Dims<3>::NK;
    constexpr int NCELL = T::TX * T::TY * T::TZ;
    constexpr int NTX = T::TX + 1, NTY = T::TY + 1, NTZ = T::TZ + 1;
    constexpr int NT = NTX * NTY * NTZ;
    static_assert(NCELL == 128, "launch bounds assume 128 cells per CTA");

    // dynamic shared memory (above the 48 KB static limit): nodal x, derivatives / flux sums
    // [(c * 3 + d) * 4 + class][cell], phi-row Gauss-point values [q][cell], node masks
    S* sx = reinterpret_cast<S*>(cell_smem);
    S* sgrad = sx + NC * NT;
    S* sfq = sgrad + 9 * NH * NCELL;
    uint8_t* smask = reinterpret_cast<uint8_t*>(sfq + NV * NCELL);

    const Geom& g = a.g;
    const int ci0 = bx * T::TX, cj0 = by * T::TY, ck0 = bz * T::TZ;
    const int64_t nn = g.n_nodes;
    for (int t = threadIdx.x; t < NT; t += NCELL) {
        const int ti = t % NTX, tj = (t / NTX) % NTY, tk = t / (NTX * NTY);
        const int gi = ci0 + ti, gj = cj0 + tj, gk = ck0 + tk;
        const bool in = gi < g.nn[0] && gj < g.nn[1] && gk < g.nn[2];
        const int64_t gn = in ? (int64_t)gi + (int64_t)g.nn[0] * ((int64_t)gj + (int64_t)g.nn[1] * gk) : 0;
        const uint8_t m = in ? a.mask[gn] : 0;
        smask[t] = m;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const bool el = c < 3 ? ((m >> c) & 1) != 0 : (m & a.phi_bits) != 0;
            sx[c * NT + t] = (in && !el) ? load_cvt<S>(a.x[c * nn + gn]) : Scalar<S>::zero();
        }
    }
    __syncthreads();

    const int cell = threadIdx.x;
    const int li = cell % T::TX, lj = (cell / T::TX) % T::TY, lk = cell / (T::TX * T::TY);
    const int gi = ci0 + li, gj = cj0 + lj, gk = ck0 + lk;
    if (gi >= g.nc[0] || gj >= g.nc[1] || gk >= g.nc[2] || gk >= a.kz_end) return;
    const int64_t gid = (int64_t)gi + (int64_t)g.nc[0] * ((int64_t)gj + (int64_t)g.nc[1] * gk);
    if (!cell_in(g, gid)) return;
    const int tb = li + NTX * (lj + NTY * lk);
    auto tnode = [&](int n) { return tb + (n & 1) + NTX * (((n >> 1) & 1) + NTY * ((n >> 2) & 1)); };
    auto cls = [](int q, int d) { return (q & ((1 << d) - 1)) | ((q >> (d + 1)) << d); };   // q without bit d
    auto cv = [&](int j) { return cpair<S>(K.cv[j]); };
    auto cg = [&](int d, int j) { return cpair<S>(K.cg[d][j]); };
    const S mu = cpair<S>(K.mu), lam = cpair<S>(K.lam);

    // displacement derivatives at the Gauss points -> shared memory
#pragma unroll (sizeof(S) == 4 ? 3 : 1)
    for (int c = 0; c < 3; ++c) {
        S v[NV];
#pragma unroll
        for (int n = 0; n < NV; ++n) v[n] = sx[c * NT + tnode(n)];
        fwd<3>(v);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            S t[NH];
#pragma unroll
            for (int j = 0; j < NH; ++j) {
                const int kp = ((j >> d) << (d + 1)) | (j & ((1 << d) - 1));   // j with a zero bit d inserted
                t[j] = v[kp | (1 << d)] * cg(d, popc(kp));
            }
            inv<2>(t);
#pragma unroll
            for (int j = 0; j < NH; ++j) sgrad[((c * 3 + d) * NH + j) * NCELL + cell] = t[j];
        }
    }
    // phi at the Gauss points -> shared memory
    {
        S v[NV], fq[NV];
#pragma unroll
        for (int n = 0; n < NV; ++n) v[n] = sx[3 * NT + tnode(n)];
        fwd<3>(v);
#pragma unroll
        for (int k = 0; k < NV; ++k) fq[k] = v[k] * cv(popc(k));
        inv<3>(fq);
#pragma unroll
        for (int q = 0; q < NV; ++q) sfq[q * NCELL + cell] = fq[q];
    }

    // flux sums per (c, d, class); each sum starts at its first Gauss point (the one with bit d of
    // q clear), so no addition with zero is spent
    S ps[3][3][NH];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        S g_[3][3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int d = 0; d < 3; ++d) g_[c][d] = sgrad[((c * 3 + d) * NH + cls(q, d)) * NCELL + cell];
        const int64_t qb = (int64_t)(q * NK) * g.n_cells + gid;
        const S c0 = QData<S>::get(a.qd, qb);
        // c0 sigma(du): c0 mu (du_i,j + du_j,i) off the diagonal, 2 c0 mu du_i,i + c0 lambda div du on it
        const S c0m = c0 * mu, c0m2 = df_scale(c0m, 2.f);
        const S c0lt = (c0 * lam) * (g_[0][0] + g_[1][1] + g_[2][2]);
        S cp = Scalar<S>::zero();
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = i; j < 3; ++j) {
                const S e2 = (i == j) ? g_[i][i] : g_[i][j] + g_[j][i];   // 2 e_ij off the diagonal
                if constexpr (!BLOCKDIAG) {
                    const S sp = QData<S>::get(a.qd, qb + (int64_t)(1 + sidx<3>(i, j)) * g.n_cells);
                    cp = (i == 0 && j == 0) ? sp * e2 : cp + sp * e2;   // Sp : e(du)
                }
                const S f = (i == j) ? c0m2 * e2 + c0lt : c0m * e2;
                S& pj = ps[i][j][cls(q, j)];
                pj = ((q >> j) & 1) ? pj + f : f;
                if (i != j) {
                    S& pi = ps[j][i][cls(q, i)];
                    pi = ((q >> i) & 1) ? pi + f : f;
                }
            }
        const S c1 = QData<S>::get(a.qd, qb + (int64_t)(NK - 1) * g.n_cells);
        if constexpr (BLOCKDIAG) sfq[q * NCELL + cell] = c1 * sfq[q * NCELL + cell];
        else sfq[q * NCELL + cell] = c1 * sfq[q * NCELL + cell] + cp;
    }
    // flux sums back to this cell's shared slots (the derivatives are no longer needed)
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int j = 0; j < NH; ++j) sgrad[((c * 3 + d) * NH + j) * NCELL + cell] = ps[c][d][j];

    const int64_t gn0 = (int64_t)gi + (int64_t)g.nn[0] * ((int64_t)gj + (int64_t)g.nn[1] * gk);
    auto noff = [&](int n) {
        return (int64_t)(n & 1) + (int64_t)g.nn[0] * (((n >> 1) & 1) + (int64_t)g.nn[1] * ((n >> 2) & 1));
    };
#pragma unroll (sizeof(S) == 4 ? 3 : 1)
    for (int c = 0; c < 3; ++c) {
        S p[3][NH];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
#pragma unroll
            for (int j = 0; j < NH; ++j) p[d][j] = sgrad[((c * 3 + d) * NH + j) * NCELL + cell];
            fwd<2>(p[d]);
        }
        S Y[NV];
        Y[0] = Scalar<S>::zero();
#pragma unroll
        for (int k = 1; k < NV; ++k) {
            const int d0 = (k & 1) ? 0 : ((k & 2) ? 1 : 2);   // lowest axis in k
            S acc = p[d0][cls(k & ~(1 << d0), d0)] * cg(d0, popc(k) - 1);
#pragma unroll
            for (int d = d0 + 1; d < 3; ++d) {
                if (!(k & (1 << d))) continue;
                const int kp = k & ~(1 << d);
                acc = acc + p[d][cls(kp, d)] * cg(d, popc(kp));
            }
            Y[k] = acc;
        }
        inv3_v0_zero(Y);
        typename Scalar<S>::storage* yc = a.y + c * nn + gn0;
#pragma unroll
        for (int n = 0; n < NV; ++n)
            if (!((smask[tnode(n)] >> c) & 1)) atomicAdd(yc + noff(n), Scalar<S>::store(Y[n]));
    }
    {
        S v[NV], fq[NV];
#pragma unroll
        for (int n = 0; n < NV; ++n) {
            v[n] = sx[3 * NT + tnode(n)];
            fq[n] = sfq[n * NCELL + cell];
        }
        fwd<3>(v);
        fwd<3>(fq);
        S Y[NV];
        Y[0] = fq[0] * cv(0);
#pragma unroll
        for (int k = 1; k < NV; ++k) Y[k] = fq[k] * cv(popc(k)) + v[k] * cpair<S>(K.gk[k]);
        inv<3>(Y);
#pragma unroll
        for (int n = 0; n < NV; ++n)
            if (!(smask[tnode(n)] & a.phi_bits)) atomicAdd(&a.y[3 * nn + gn0 + noff(n)], Scalar<S>::store(Y[n]));
    }
}

template <typename S, bool BLOCKDIAG>
__global__ void __launch_bounds__(128, sizeof(S) == 8 ? 3 : 4)
k_q1_apply_cell(Q1ApplyArgs<typename Scalar<S>::storage, typename QData<S>::type> a) {
    extern __shared__ __align__(16) unsigned char cell_smem[];
    q1_cell_tile<S, BLOCKDIAG>(a, a.k, blockIdx.x, blockIdx.y, blockIdx.z + a.tz0, cell_smem);
}

// ---- batched: one launch over the tiles of all instances of a level
template <int DIM, typename S, bool LANES>
struct TileOf {
    static constexpr int TX = LANES ? LaneTile<DIM>::TX : Q1Tile<DIM, S>::TX;
    static constexpr int TY = LANES ? LaneTile<DIM>::TY : Q1Tile<DIM, S>::TY;
    static constexpr int TZ = LANES ? LaneTile<DIM>::TZ : Q1Tile<DIM, S>::TZ;
};

// instance of flattened tile b: the last i with tile_start[i] <= b
__device__ __forceinline__ int tile_instance(const int* __restrict__ tile_start, int n, int b) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tile_start[mid] <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Persistent: each CTA loops over the flattened tiles of all instances of a level (stride gridDim.x);
// instances switched off (BLevel::on) are skipped.
template <int DIM, typename S, bool BLOCKDIAG, bool LANES>
__global__ void __launch_bounds__(LANES ? 256 : Q1Tile<DIM, S>::TX * Q1Tile<DIM, S>::TY * Q1Tile<DIM, S>::TZ,
                                  LANES ? 1 : Q1Tile<DIM, S>::MINB)
k_q1_apply_batched(const BLevel* __restrict__ L, const int* __restrict__ tile_start, int n, int sx, int sy,
                   int phi_bits) {
    using St = typename Scalar<S>::storage;
    using QT = typename QData<S>::type;
    using TT = TileOf<DIM, S, LANES>;
    const int total = tile_start[n];
    for (int b = blockIdx.x; b < total; b += gridDim.x) {
        const int i = tile_instance(tile_start, n, b);
        const BLevel& d = L[i];
        if (bon(d)) {
            Q1ApplyArgs<St, QT> a;
            a.g = d.g;
            a.qd = sizeof(St) == 8 ? reinterpret_cast<const QT*>(d.qpd64) : reinterpret_cast<const QT*>(d.qpd32);
            a.x = bvec<St>(d, sx);
            a.y = bvec<St>(d, sy);
            a.mask = d.mask;
            a.phi_bits = phi_bits;
            a.k = d.k;
            const int local = b - tile_start[i];
            const int tx = (d.g.nc[0] + TT::TX - 1) / TT::TX, ty = (d.g.nc[1] + TT::TY - 1) / TT::TY;
            const int bx = local % tx, by = (local / tx) % ty, bz = local / (tx * ty);
            if constexpr (LANES) q1_direct_tile<DIM, S, BLOCKDIAG>(a, bx, by, bz);   // atomic lanes, no barrier
            else q1_apply_tile<DIM, S, BLOCKDIAG>(a, bx, by, bz, &d.k);
        }
        if constexpr (!LANES) __syncthreads();   // the next tile reuses the shared-memory stage
    }
}

int q1_tiles(const Geom& g, bool fp64, bool lanes) {
    int TX, TY, TZ;
    if (g.dim == 3) {
        if (lanes) { TX = LaneTile<3>::TX; TY = LaneTile<3>::TY; TZ = LaneTile<3>::TZ; }
        else if (fp64) { TX = Q1Tile<3, df64>::TX; TY = Q1Tile<3, df64>::TY; TZ = Q1Tile<3, df64>::TZ; }
        else { TX = Q1Tile<3, float>::TX; TY = Q1Tile<3, float>::TY; TZ = Q1Tile<3, float>::TZ; }
    } else {
        if (lanes) { TX = LaneTile<2>::TX; TY = LaneTile<2>::TY; TZ = 1; }
        else if (fp64) { TX = Q1Tile<2, df64>::TX; TY = Q1Tile<2, df64>::TY; TZ = 1; }
        else { TX = Q1Tile<2, float>::TX; TY = Q1Tile<2, float>::TY; TZ = 1; }
    }
    const int tz = g.dim == 3 ? (g.nc[2] + TZ - 1) / TZ : 1;
    return ((g.nc[0] + TX - 1) / TX) * ((g.nc[1] + TY - 1) / TY) * tz;
}

template <int DIM, typename S, bool BD, bool LANES>
static void launch_b(const BLevel* L, const int* ts, int n, int grid, int sx, int sy, int pb, cudaStream_t s) {
    constexpr int threads = LANES ? 256 : Q1Tile<DIM, S>::TX * Q1Tile<DIM, S>::TY * Q1Tile<DIM, S>::TZ;
    k_q1_apply_batched<DIM, S, BD, LANES><<<grid, threads, 0, s>>>(L, ts, n, sx, sy, pb);
}

template <typename S>
static constexpr size_t cell_smem_bytes() {
    using T = CellTile;
    constexpr int NCELL = T::TX * T::TY * T::TZ, NT = (T::TX + 1) * (T::TY + 1) * (T::TZ + 1);
    return sizeof(S) * (4 * NT + 9 * 4 * NCELL + 8 * NCELL) + NT;
}

// Batched per-cell apply (3D): one launch over the 16x4x2-cell tiles of all instances of a level,
// the instance found from the tile prefix; the tile work of k_q1_apply_cell with the instance's
// Gauss-point scalings read from its descriptor.
template <typename S, bool BLOCKDIAG>
__global__ void __launch_bounds__(128, 4)
k_q1_apply_batched_cell(const BLevel* __restrict__ L, const int* __restrict__ tile_start, int n, int sx, int sy,
                        int phi_bits) {
    using St = typename Scalar<S>::storage;
    using QT = typename QData<S>::type;
    extern __shared__ __align__(16) unsigned char cell_smem[];
    const int total = tile_start[n];
    for (int b = blockIdx.x; b < total; b += gridDim.x) {
        const int i = tile_instance(tile_start, n, b);
        const BLevel& d = L[i];
        if (bon(d)) {
            Q1ApplyArgs<St, QT> a;
            a.g = d.g;
            a.qd = sizeof(St) == 8 ? reinterpret_cast<const QT*>(d.qpd64) : reinterpret_cast<const QT*>(d.qpd32);
            a.x = bvec<St>(d, sx);
            a.y = bvec<St>(d, sy);
            a.mask = d.mask;
            a.phi_bits = phi_bits;
            const int local = b - tile_start[i];
            const int tx = (d.g.nc[0] + CellTile::TX - 1) / CellTile::TX, ty = (d.g.nc[1] + CellTile::TY - 1) / CellTile::TY;
            q1_cell_tile<S, BLOCKDIAG>(a, d.k, local % tx, (local / tx) % ty, local / (tx * ty), cell_smem);
        }
        __syncthreads();   // the next tile reuses the shared-memory stage
    }
}

// dynamic shared memory above 48 KB needs the attribute once per device (before any stream capture)
template <typename S, bool BD>
static cudaError_t batched_cell_attr() {
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (!(dev >= 0 && dev < 64 && done[dev])) {
        e = cudaFuncSetAttribute(k_q1_apply_batched_cell<S, BD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)cell_smem_bytes<S>());
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) done[dev] = true;
    }
    return cudaSuccess;
}

cudaError_t q1_batched_prepare() {
    cudaError_t e = batched_cell_attr<df64, false>();
    if (e == cudaSuccess) e = batched_cell_attr<df64, true>();
    if (e == cudaSuccess) e = batched_cell_attr<float, false>();
    if (e == cudaSuccess) e = batched_cell_attr<float, true>();
    return e;
}

int q1_batched_ctas_per_sm(int dim, bool fp64, bool cell) {
    int nb = 0;
    cudaError_t e;
    if (cell && dim == 3) {
        if (fp64) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_q1_apply_batched_cell<df64, false>, 128,
                                                                    cell_smem_bytes<df64>());
        else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_q1_apply_batched_cell<float, false>, 128,
                                                               cell_smem_bytes<float>());
    } else if (dim == 3) {
        if (fp64) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_q1_apply_batched<3, df64, false, true>, 256, 0);
        else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_q1_apply_batched<3, float, false, false>,
                                                               Q1Tile<3, float>::TX * Q1Tile<3, float>::TY * Q1Tile<3, float>::TZ, 0);
    } else {
        if (fp64) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_q1_apply_batched<2, df64, false, true>, 256, 0);
        else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_q1_apply_batched<2, float, false, false>,
                                                               Q1Tile<2, float>::TX * Q1Tile<2, float>::TY, 0);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return nb > 0 ? nb : 1;
}

template <typename S, bool BD>
static cudaError_t launch_batched_cell(const BLevel* L, const int* ts, int n, int grid, int sx, int sy, int pb,
                                       cudaStream_t s) {
    cudaError_t e = batched_cell_attr<S, BD>();
    if (e != cudaSuccess) return e;
    k_q1_apply_batched_cell<S, BD><<<grid, CellTile::TX * CellTile::TY * CellTile::TZ, cell_smem_bytes<S>(), s>>>(
        L, ts, n, sx, sy, pb);
    return count_launch(cudaGetLastError());
}

bool q1_cell_tiles_match_f32() {
    return CellTile::TX == Q1Tile<3, float>::TX && CellTile::TY == Q1Tile<3, float>::TY &&
           CellTile::TZ == Q1Tile<3, float>::TZ;
}

cudaError_t launch_q1_apply_batched(int dim, bool fp64, bool blockdiag, bool lanes, const BLevel* L, int n,
                                    const int* tile_start, int total_tiles, int sx, int sy, int phi_bits,
                                    cudaStream_t s, bool cell, int max_ctas) {
    if (total_tiles <= 0) return cudaSuccess;
    if (max_ctas > 0 && total_tiles > max_ctas) total_tiles = max_ctas;   // persistent grid
    if (cell && dim == 3) {
        if (fp64) return blockdiag ? launch_batched_cell<df64, true>(L, tile_start, n, total_tiles, sx, sy, phi_bits, s)
                                   : launch_batched_cell<df64, false>(L, tile_start, n, total_tiles, sx, sy, phi_bits, s);
        return blockdiag ? launch_batched_cell<float, true>(L, tile_start, n, total_tiles, sx, sy, phi_bits, s)
                         : launch_batched_cell<float, false>(L, tile_start, n, total_tiles, sx, sy, phi_bits, s);
    }
#define PFF_B(D, S, BD, LN) launch_b<D, S, BD, LN>(L, tile_start, n, total_tiles, sx, sy, phi_bits, s)
    if (dim == 3) {
        if (fp64) {
            if (lanes) { if (blockdiag) PFF_B(3, df64, true, true); else PFF_B(3, df64, false, true); }
            else { if (blockdiag) PFF_B(3, df64, true, false); else PFF_B(3, df64, false, false); }
        } else {
            if (lanes) { if (blockdiag) PFF_B(3, float, true, true); else PFF_B(3, float, false, true); }
            else { if (blockdiag) PFF_B(3, float, true, false); else PFF_B(3, float, false, false); }
        }
    } else {
        if (fp64) {
            if (lanes) { if (blockdiag) PFF_B(2, df64, true, true); else PFF_B(2, df64, false, true); }
            else { if (blockdiag) PFF_B(2, df64, true, false); else PFF_B(2, df64, false, false); }
        } else {
            if (lanes) { if (blockdiag) PFF_B(2, float, true, true); else PFF_B(2, float, false, true); }
            else { if (blockdiag) PFF_B(2, float, true, false); else PFF_B(2, float, false, false); }
        }
    }
#undef PFF_B
    return count_launch(cudaGetLastError());
}

template <typename S, bool BD>
static cudaError_t launch_lanes_dim(const Q1ApplyArgs<typename Scalar<S>::storage, typename QData<S>::type>& a,
                                    cudaStream_t s, bool direct) {
    if (a.g.dim == 3) {
        using T = LaneTile<3>;
        dim3 grid((a.g.nc[0] + T::TX - 1) / T::TX, (a.g.nc[1] + T::TY - 1) / T::TY, (a.g.nc[2] + T::TZ - 1) / T::TZ);
        if (direct) k_q1_apply_direct<3, S, BD><<<grid, 256, 0, s>>>(a);
        else k_q1_apply_lanes<3, S, BD><<<grid, 256, 0, s>>>(a);
    } else {
        using T = LaneTile<2>;
        dim3 grid((a.g.nc[0] + T::TX - 1) / T::TX, (a.g.nc[1] + T::TY - 1) / T::TY, 1);
        if (direct) k_q1_apply_direct<2, S, BD><<<grid, 256, 0, s>>>(a);
        else k_q1_apply_lanes<2, S, BD><<<grid, 256, 0, s>>>(a);
    }
    return count_launch(cudaGetLastError());
}

template <typename S, bool BD>
static cudaError_t launch_apply_dim(const Q1ApplyArgs<typename Scalar<S>::storage, typename QData<S>::type>& a,
                                   cudaStream_t s) {
    if (a.g.dim == 3) {
        using T = Q1Tile<3, S>;
        dim3 grid((a.g.nc[0] + T::TX - 1) / T::TX, (a.g.nc[1] + T::TY - 1) / T::TY, (a.g.nc[2] + T::TZ - 1) / T::TZ);
        k_q1_apply<3, S, BD><<<grid, T::TX * T::TY * T::TZ, 0, s>>>(a);
    } else {
        using T = Q1Tile<2, S>;
        dim3 grid((a.g.nc[0] + T::TX - 1) / T::TX, (a.g.nc[1] + T::TY - 1) / T::TY, 1);
        k_q1_apply<2, S, BD><<<grid, T::TX * T::TY, 0, s>>>(a);
    }
    return count_launch(cudaGetLastError());
}

template <typename St, typename QT>
static void fill_consts(Q1ApplyArgs<St, QT>& a, const Phys& ph) {
    a.k = make_q1_consts(a.g, ph);
}

// opt in to the dynamic shared memory of k_q1_apply_cell (once per instantiation and device)
template <typename S, bool BD>
static cudaError_t cell_prepare() {
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(k_q1_apply_cell<S, BD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)cell_smem_bytes<S>());
    if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
    return e;
}

template <typename S, bool BD>
static cudaError_t launch_cell(const Q1ApplyArgs<typename Scalar<S>::storage, typename QData<S>::type>& a,
                               cudaStream_t s) {
    using T = CellTile;
    const Geom& g = a.g;
    const cudaError_t e = cell_prepare<S, BD>();
    if (e != cudaSuccess) return e;
    dim3 grid((g.nc[0] + T::TX - 1) / T::TX, (g.nc[1] + T::TY - 1) / T::TY, (g.nc[2] + T::TZ - 1) / T::TZ);
    k_q1_apply_cell<S, BD><<<grid, T::TX * T::TY * T::TZ, cell_smem_bytes<S>(), s>>>(a);
    return count_launch(cudaGetLastError());
}

int q1_cell_tile_z() { return CellTile::TZ; }

cudaError_t launch_q1_apply64_slab(const Geom& g, const Phys& ph, const float2* qd, const double* x, double* y,
                                   const uint8_t* mask, int phi_bits, int kz0, int kz1, cudaStream_t s) {
    using T = CellTile;
    if (g.dim != 3 || kz0 % T::TZ != 0 || kz0 < 0 || kz1 > g.nc[2] || kz1 <= kz0) return cudaErrorInvalidValue;
    Q1ApplyArgs<double, float2> a;
    a.g = g;
    a.qd = qd;
    a.x = x;
    a.y = y;
    a.mask = mask;
    a.phi_bits = phi_bits;
    fill_consts(a, ph);
    a.tz0 = kz0 / T::TZ;
    a.kz_end = kz1;
    const cudaError_t e = cell_prepare<df64, false>();
    if (e != cudaSuccess) return e;
    dim3 grid((g.nc[0] + T::TX - 1) / T::TX, (g.nc[1] + T::TY - 1) / T::TY, (kz1 - kz0 + T::TZ - 1) / T::TZ);
    k_q1_apply_cell<df64, false><<<grid, T::TX * T::TY * T::TZ, cell_smem_bytes<df64>(), s>>>(a);
    return count_launch(cudaGetLastError());
}

cudaError_t launch_q1_apply64(const Geom& g, const Phys& ph, const float2* qd, const double* x, double* y,
                              const uint8_t* mask, int phi_bits, bool blockdiag, bool lanes, cudaStream_t s,
                              bool direct, bool cell) {
    Q1ApplyArgs<double, float2> a;
    a.g = g;
    a.qd = qd;
    a.x = x;
    a.y = y;
    a.mask = mask;
    a.phi_bits = phi_bits;
    fill_consts(a, ph);
    if (cell && g.dim == 3) return blockdiag ? launch_cell<df64, true>(a, s) : launch_cell<df64, false>(a, s);
    if (lanes || direct)
        return blockdiag ? launch_lanes_dim<df64, true>(a, s, direct) : launch_lanes_dim<df64, false>(a, s, direct);
    return blockdiag ? launch_apply_dim<df64, true>(a, s) : launch_apply_dim<df64, false>(a, s);
}

cudaError_t launch_q1_apply32(const Geom& g, const Phys& ph, const float* qd, const float* x, float* y,
                              const uint8_t* mask, int phi_bits, bool blockdiag, bool lanes, cudaStream_t s,
                              bool direct, bool cell) {
    Q1ApplyArgs<float, float> a;
    a.g = g;
    a.qd = qd;
    a.x = x;
    a.y = y;
    a.mask = mask;
    a.phi_bits = phi_bits;
    fill_consts(a, ph);
    if (cell && g.dim == 3) return blockdiag ? launch_cell<float, true>(a, s) : launch_cell<float, false>(a, s);
    if (lanes || direct)
        return blockdiag ? launch_lanes_dim<float, true>(a, s, direct) : launch_lanes_dim<float, false>(a, s, direct);
    return blockdiag ? launch_apply_dim<float, true>(a, s) : launch_apply_dim<float, false>(a, s);
}

// Miehe split (Gauss-point tangent K): FP64-accurate operator as atomic lanes, FP32 per cell
template <typename S, bool BD, typename A>
static cudaError_t launch_split_dim(const A& a, cudaStream_t s) {
    if constexpr (sizeof(typename Scalar<S>::storage) == 8) {
        if (a.g.dim == 3) {
            using T = LaneTile<3>;
            dim3 grid((a.g.nc[0] + T::TX - 1) / T::TX, (a.g.nc[1] + T::TY - 1) / T::TY, (a.g.nc[2] + T::TZ - 1) / T::TZ);
            k_q1_apply_direct<3, S, BD, true><<<grid, 256, 0, s>>>(a);
        } else {
            using T = LaneTile<2>;
            dim3 grid((a.g.nc[0] + T::TX - 1) / T::TX, (a.g.nc[1] + T::TY - 1) / T::TY, 1);
            k_q1_apply_direct<2, S, BD, true><<<grid, 256, 0, s>>>(a);
        }
    } else {
        if (a.g.dim == 3) {
            using T = Q1Tile<3, S>;
            dim3 grid((a.g.nc[0] + T::TX - 1) / T::TX, (a.g.nc[1] + T::TY - 1) / T::TY, (a.g.nc[2] + T::TZ - 1) / T::TZ);
            k_q1_apply<3, S, BD, true><<<grid, T::TX * T::TY * T::TZ, 0, s>>>(a);
        } else {
            using T = Q1Tile<2, S>;
            dim3 grid((a.g.nc[0] + T::TX - 1) / T::TX, (a.g.nc[1] + T::TY - 1) / T::TY, 1);
            k_q1_apply<2, S, BD, true><<<grid, T::TX * T::TY, 0, s>>>(a);
        }
    }
    return count_launch(cudaGetLastError());
}

cudaError_t launch_q1_apply_split64(const Geom& g, const Phys& ph, const float2* qd, const double* x, double* y,
                                    const uint8_t* mask, int phi_bits, bool blockdiag, cudaStream_t s) {
    Q1ApplyArgs<double, float2> a;
    a.g = g;
    a.qd = qd;
    a.x = x;
    a.y = y;
    a.mask = mask;
    a.phi_bits = phi_bits;
    fill_consts(a, ph);
    return blockdiag ? launch_split_dim<df64, true>(a, s) : launch_split_dim<df64, false>(a, s);
}

cudaError_t launch_q1_apply_split32(const Geom& g, const Phys& ph, const float* qd, const float* x, float* y,
                                    const uint8_t* mask, int phi_bits, bool blockdiag, cudaStream_t s) {
    Q1ApplyArgs<float, float> a;
    a.g = g;
    a.qd = qd;
    a.x = x;
    a.y = y;
    a.mask = mask;
    a.phi_bits = phi_bits;
    fill_consts(a, ph);
    return blockdiag ? launch_split_dim<float, true>(a, s) : launch_split_dim<float, false>(a, s);
}

// ------------------------------------------------------------------ residual and diagonal (FP64)
// Residual -A(U) of Eq. (semilinear) (OP 0) and diagonal of G~ (OP 1) for Q1 levels.  Same tile
// and fixed-order gather as the applies.  The residual evaluates the state from the nodal
// values in modal form; the diagonal uses the stored Gauss-point coefficients c0, c1 and the
// squared shape gradients, which on a uniform cell depend only on n xor q:
// (d_d N_n(q))^2 = h_d^-2 prod_{e != d} A(n,q,e), N_n(q)^2 = prod_e A(n,q,e), with
// A = ((1 + g)/2)^2 if node n and Gauss point q lie on the same side in direction e, else
// ((1 - g)/2)^2.
// Diagonal weights per m = n xor q (node n, Gauss point q), Q1, as (hi, lo) pairs:
//   A[c][m] = mu Ws + (mu + lambda) W_c,  P[m] = prod_e a_e,  Wg[m] = Gc eps w Ws,
// with a_e = ((1 + g)/2)^2 if bit e of m is clear else ((1 - g)/2)^2, W_d = a-product over e != d
// divided by h_d^2 and Ws = sum_d W_d.  (Phi_n at q is prod_e ((1 +- g)/2); its derivative along d is
// +-1/h_d times the product over the other axes.)
struct DiagConsts {
    float2 A[3][8];
    float2 P[8];
    float2 Wg[8];
};

// Residual constants: the linearisation constants plus p and 2 w Gc eps (pair sum of a gradient flux).
struct ResConsts {
    float2 cv[4], cg[3][3];
    float2 w, omk, kap, f2k, p2, gce, mu, lam;
    float2 p, wgce2;
};

namespace {
template <int DIM>
struct RDTile;
template <> struct RDTile<3> { static constexpr int TX = 8, TY = 4, TZ = 4; };
template <> struct RDTile<2> { static constexpr int TX = 16, TY = 8, TZ = 1; };
}  // namespace

template <int DIM, int OP>
__global__ void __launch_bounds__(RDTile<DIM>::TX * RDTile<DIM>::TY * RDTile<DIM>::TZ)
k_q1_resdiag(Geom g, ResConsts rk, DiagConsts dk, const double* __restrict__ U, const double* __restrict__ pt,
             const float2* __restrict__ q64, const uint8_t* __restrict__ mask, double* __restrict__ y) {
    using T = RDTile<DIM>;
    using D = Q1Dims<DIM>;
    constexpr int NV = D::NV, NC = D::NC, NK = D::NK, NH = NV / 2;
    constexpr int NCELL = T::TX * T::TY * T::TZ;
    constexpr int NTX = T::TX + 1, NTY = T::TY + 1, NTZ = DIM == 3 ? T::TZ + 1 : 1;
    constexpr int NT = NTX * NTY * NTZ;
    constexpr int NS = OP == 0 ? NC + 1 : 1;   // staged fields: U and phi~ (residual only)
    __shared__ double sv[NS * NT];
    __shared__ double sel[NV * NC * NCELL];

    const int ci0 = blockIdx.x * T::TX, cj0 = blockIdx.y * T::TY, ck0 = DIM == 3 ? blockIdx.z * T::TZ : 0;
    const int64_t nn = g.n_nodes;
    if constexpr (OP == 0) {
        for (int t = threadIdx.x; t < NT; t += blockDim.x) {
            const int ti = t % NTX, tj = (t / NTX) % NTY, tk = t / (NTX * NTY);
            const int gi = ci0 + ti, gj = cj0 + tj, gk = ck0 + tk;
            const bool in = gi < g.nn[0] && gj < g.nn[1] && gk < g.nn[2];
            const int64_t gn = in ? (int64_t)gi + (int64_t)g.nn[0] * ((int64_t)gj + (int64_t)g.nn[1] * gk) : 0;
#pragma unroll
            for (int c = 0; c < NC; ++c) sv[c * NT + t] = in ? U[c * nn + gn] : 0.0;
            sv[NC * NT + t] = in ? pt[gn] : 0.0;
        }
        __syncthreads();
    }
    const int cell = threadIdx.x;
    const int li = cell % T::TX, lj = (cell / T::TX) % T::TY, lk = cell / (T::TX * T::TY);
    const bool valid = (ci0 + li < g.nc[0]) && (cj0 + lj < g.nc[1]) && (DIM == 2 || ck0 + lk < g.nc[2]) &&
                       cell_in(g, (int64_t)(ci0 + li) + (int64_t)g.nc[0] * ((int64_t)(cj0 + lj) + (int64_t)g.nc[1] * (ck0 + lk)));
    double el[NV][NC];
#pragma unroll
    for (int n = 0; n < NV; ++n)
#pragma unroll
        for (int c = 0; c < NC; ++c) el[n][c] = 0.0;
    if (valid) {
        const int64_t gid = (int64_t)(ci0 + li) + (int64_t)g.nc[0] * ((int64_t)(cj0 + lj) + (int64_t)g.nc[1] * (ck0 + lk));
        if constexpr (OP == 1) {
            // diag G~: for node n and Gauss point q the element weights depend on m = n xor q only
            // (host tables); c0 and c1 are the stored df64 coefficients.
            df64 acc[NV][NC];
#pragma unroll
            for (int n = 0; n < NV; ++n)
#pragma unroll
                for (int c = 0; c < NC; ++c) acc[n][c] = df_make(0.f, 0.f);
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                const float2 a0 = q64[(int64_t)(q * NK + 0) * g.n_cells + gid];
                const float2 a1 = q64[(int64_t)(q * NK + NK - 1) * g.n_cells + gid];
                const df64 c0 = df_make(a0.x, a0.y), c1 = df_make(a1.x, a1.y);
#pragma unroll
                for (int n = 0; n < NV; ++n) {
                    const int m = n ^ q;
#pragma unroll
                    for (int c = 0; c < DIM; ++c) acc[n][c] = acc[n][c] + c0 * dfc(dk.A[c][m]);
                    acc[n][DIM] = acc[n][DIM] + c1 * dfc(dk.P[m]) + dfc(dk.Wg[m]);
                }
            }
#pragma unroll
            for (int n = 0; n < NV; ++n)
#pragma unroll
                for (int c = 0; c < NC; ++c) el[n][c] = df_to_double(acc[n][c]);
        } else {
            // -A(U) in df64 (Eq. (semilinear)): u-rows (g(phi~) sigma(u) + phi~^2 p I) : grad Phi,
            // phi-rows (f g'(phi) E_s + 2 phi p div u - Gc/eps (1 - phi)) Phi + Gc eps grad phi . grad Phi.
            // Gauss-point values by inverse butterflies; integration by the transposed (forward)
            // butterflies; a Q1 derivative is constant along its own axis.
            const df64 sE = g.es ? df_from_double(g.es[gid]) : df_make(1.f, 0.f);
            const df64 cmu = dfc(rk.mu) * sE, clam = dfc(rk.lam) * sE;
            const df64 w = dfc(rk.w), omk = dfc(rk.omk), kap = dfc(rk.kap), f2k = dfc(rk.f2k), p2 = dfc(rk.p2);
            const int tb = li + NTX * (lj + NTY * lk);
            auto off = [](int n) { return (n & 1) + NTX * (((n >> 1) & 1) + NTY * (DIM == 3 ? (n >> 2) & 1 : 0)); };
            df64 vphi[NV], vpt[NV];
#pragma unroll
            for (int n = 0; n < NV; ++n) {
                vphi[n] = df_from_double(sv[DIM * NT + tb + off(n)]);
                vpt[n] = df_from_double(sv[NC * NT + tb + off(n)]);
            }
            fwd<DIM>(vphi);
            fwd<DIM>(vpt);
            df64 Hp[DIM][NH];       // phi-row gradient part, already integrated
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
                int jj = 0;
#pragma unroll
                for (int kp = 0; kp < NV; ++kp) {
                    if (kp & (1 << d)) continue;
                    Hp[d][jj] = vphi[kp | (1 << d)] * dfc(rk.cg[d][popc(kp)]);
                    ++jj;
                }
                // the flux -w Gc eps dphi/dx_d is constant along d (the pair sum over q doubles it,
                // wgce2 = 2 w Gc eps); integrating it over the other axes is the forward butterfly of
                // the inverse one, i.e. a factor 2^(d-1)
#pragma unroll
                for (int t = 0; t < NH; ++t) Hp[d][t] = df_scale(Hp[d][t] * dfc(rk.wgce2), -(float)NH);
            }
#pragma unroll
            for (int m = 0; m < NV; ++m) {
                vphi[m] = vphi[m] * dfc(rk.cv[popc(m)]);
                vpt[m] = vpt[m] * dfc(rk.cv[popc(m)]);
            }
            inv<DIM>(vphi);
            inv<DIM>(vpt);
            df64 gd[DIM][DIM][NH];
#pragma unroll
            for (int c = 0; c < DIM; ++c) {
                df64 m_[NV];
#pragma unroll
                for (int n = 0; n < NV; ++n) m_[n] = df_from_double(sv[c * NT + tb + off(n)]);
                fwd<DIM>(m_);
#pragma unroll
                for (int d = 0; d < DIM; ++d) {
                    int jj = 0;
#pragma unroll
                    for (int kp = 0; kp < NV; ++kp) {
                        if (kp & (1 << d)) continue;
                        gd[c][d][jj] = m_[kp | (1 << d)] * dfc(rk.cg[d][popc(kp)]);
                        ++jj;
                    }
                    inv<DIM - 1>(gd[c][d]);
#pragma unroll
                    for (int t = 0; t < NH; ++t) gd[c][d][t] = df_renorm(gd[c][d][t]);
                }
            }
            df64 ps[DIM][DIM][NH], fv[NV];
#pragma unroll
            for (int c = 0; c < DIM; ++c)
#pragma unroll
                for (int d = 0; d < DIM; ++d)
#pragma unroll
                    for (int t = 0; t < NH; ++t) ps[c][d][t] = df_make(0.f, 0.f);
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                df64 gu[DIM][DIM];
#pragma unroll
                for (int c = 0; c < DIM; ++c)
#pragma unroll
                    for (int d = 0; d < DIM; ++d) gu[c][d] = gd[c][d][(q & ((1 << d) - 1)) | ((q >> (d + 1)) << d)];
                df64 e[DIM][DIM], tr = gu[0][0], ee = gu[0][0] * gu[0][0];
#pragma unroll
                for (int a = 0; a < DIM; ++a) {
                    e[a][a] = gu[a][a];
                    if (a > 0) { tr = tr + gu[a][a]; ee = ee + gu[a][a] * gu[a][a]; }
#pragma unroll
                    for (int b = a + 1; b < DIM; ++b) {
                        e[a][b] = df_scale(gu[a][b] + gu[b][a], 0.5f);
                        e[b][a] = e[a][b];
                        ee = ee + df_scale(e[a][b] * e[a][b], 2.f);
                    }
                }
                tr = df_renorm(tr);
                const df64 Es = df_scale(clam * tr * tr, 0.5f) + cmu * ee;
                const df64 phi = df_renorm(vphi[q]), ptv = df_renorm(vpt[q]);
                const df64 gk = omk * ptv * ptv + kap;
                const df64 wg = w * gk, wp = w * ptv * ptv * dfc(rk.p);
                const df64 ltr = clam * tr;
#pragma unroll
                for (int a = 0; a < DIM; ++a)
#pragma unroll
                    for (int b = 0; b < DIM; ++b) {
                        df64 sg = df_scale(cmu * e[a][b], 2.f);
                        if (a == b) sg = sg + ltr;
                        df64 f = wg * sg;
                        if (a == b) f = f + wp;
                        const int jq = (q & ((1 << b) - 1)) | ((q >> (b + 1)) << b);
                        ps[a][b][jq] = ps[a][b][jq] - f;
                    }
                // value part of the phi rows: -w (f g'(phi) E_s + 2 p phi tr - Gc/eps (1 - phi))
                const df64 one_m = df_make(1.f, 0.f) - phi;
                fv[q] = w * (dfc(rk.gce) * one_m - f2k * phi * Es - p2 * phi * tr);
            }
#pragma unroll
            for (int c = 0; c < DIM; ++c)
#pragma unroll
                for (int d = 0; d < DIM; ++d) fwd<DIM - 1>(ps[c][d]);
            fwd<DIM>(fv);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                df64 Y[NV];
#pragma unroll
                for (int kk = 0; kk < NV; ++kk) {
                    df64 acc = (c == DIM) ? fv[kk] * dfc(rk.cv[popc(kk)]) : df_make(0.f, 0.f);
#pragma unroll
                    for (int d = 0; d < DIM; ++d) {
                        if (!(kk & (1 << d))) continue;
                        const int kp = kk & ~(1 << d);
                        const int jj = (kp & ((1 << d) - 1)) | ((kp >> (d + 1)) << d);
                        acc = acc + (c < DIM ? ps[c][d][jj] : Hp[d][jj]) * dfc(rk.cg[d][popc(kp)]);
                    }
                    Y[kk] = acc;
                }
                inv<DIM>(Y);
#pragma unroll
                for (int n = 0; n < NV; ++n) el[n][c] = df_to_double(Y[n]);
            }
        }
    }
#pragma unroll
    for (int n = 0; n < NV; ++n)
#pragma unroll
        for (int c = 0; c < NC; ++c) sel[(n * NC + c) * NCELL + cell] = el[n][c];
    __syncthreads();
    for (int t = threadIdx.x; t < NT; t += blockDim.x) {
        const int ti = t % NTX, tj = (t / NTX) % NTY, tk = t / (NTX * NTY);
        const int gi = ci0 + ti, gj = cj0 + tj, gk = ck0 + tk;
        if (!(gi < g.nn[0] && gj < g.nn[1] && gk < g.nn[2])) continue;
        const int64_t gn = (int64_t)gi + (int64_t)g.nn[0] * ((int64_t)gj + (int64_t)g.nn[1] * gk);
        const uint8_t m = OP == 1 ? mask[gn] : 0;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            if (OP == 1 && (c < DIM ? ((m >> c) & 1) != 0 : (m & PHI_BITS_ALL) != 0)) continue;
            double s = 0.0;
#pragma unroll
            for (int dk = 0; dk < (DIM == 3 ? 2 : 1); ++dk) {
                const int ck = tk - dk;
                if (DIM == 3 && (ck < 0 || ck >= T::TZ)) continue;
#pragma unroll
                for (int dj = 0; dj < 2; ++dj) {
                    const int cj = tj - dj;
                    if (cj < 0 || cj >= T::TY) continue;
#pragma unroll
                    for (int di = 0; di < 2; ++di) {
                        const int cx = ti - di;
                        if (cx < 0 || cx >= T::TX) continue;
                        const int n = di + 2 * dj + 4 * dk;
                        s += sel[(n * NC + c) * NCELL + cx + T::TX * (cj + T::TY * (DIM == 3 ? ck : 0))];
                    }
                }
            }
            atomicAdd(&y[c * nn + gn], s);
        }
    }
}

// Residual -A(U) in 3D, one thread per cell in df64 with the layout of k_q1_apply_cell: U and phi~
// staged in shared memory as df64, the 4 distinct Gauss-point values of each displacement
// derivative and the Gauss-point values of phi and phi~ in per-cell shared slots, the 36 flux
// sums in registers, element vectors added to R with FP64 atomics.  Arithmetic as in the residual
// branch of k_q1_resdiag (which serves 2D).
__global__ void __launch_bounds__(128, 3)
k_q1_residual_cell(Geom g, ResConsts rk, const double* __restrict__ U, const double* __restrict__ pt,
                   double* __restrict__ y) {
    using T = CellTile;
    constexpr int NV = 8, NC = 4, NH = 4;
    constexpr int NCELL = T::TX * T::TY * T::TZ;
    constexpr int NTX = T::TX + 1, NTY = T::TY + 1, NTZ = T::TZ + 1;
    constexpr int NT = NTX * NTY * NTZ;
    extern __shared__ __align__(16) unsigned char res_smem[];
    df64* sv = reinterpret_cast<df64*>(res_smem);   // [field][node]: u_x, u_y, u_z, phi, phi~
    df64* sgrad = sv + 5 * NT;                      // [(c * 3 + d) * 4 + class][cell]
    df64* sq = sgrad + 9 * NH * NCELL;              // [q][cell]: phi(q) then the phi-row flux; [8 + q]: phi~(q)

    const int ci0 = blockIdx.x * T::TX, cj0 = blockIdx.y * T::TY, ck0 = blockIdx.z * T::TZ;
    const int64_t nn = g.n_nodes;
    for (int t = threadIdx.x; t < NT; t += NCELL) {
        const int ti = t % NTX, tj = (t / NTX) % NTY, tk = t / (NTX * NTY);
        const int gi = ci0 + ti, gj = cj0 + tj, gk = ck0 + tk;
        const bool in = gi < g.nn[0] && gj < g.nn[1] && gk < g.nn[2];
        const int64_t gn = in ? (int64_t)gi + (int64_t)g.nn[0] * ((int64_t)gj + (int64_t)g.nn[1] * gk) : 0;
#pragma unroll
        for (int c = 0; c < NC; ++c) sv[c * NT + t] = in ? df_from_double(U[c * nn + gn]) : df_make(0.f, 0.f);
        sv[NC * NT + t] = in ? df_from_double(pt[gn]) : df_make(0.f, 0.f);
    }
    __syncthreads();

    const int cell = threadIdx.x;
    const int li = cell % T::TX, lj = (cell / T::TX) % T::TY, lk = cell / (T::TX * T::TY);
    const int gi = ci0 + li, gj = cj0 + lj, gk = ck0 + lk;
    if (gi >= g.nc[0] || gj >= g.nc[1] || gk >= g.nc[2]) return;
    const int64_t gid = (int64_t)gi + (int64_t)g.nc[0] * ((int64_t)gj + (int64_t)g.nc[1] * gk);
    if (!cell_in(g, gid)) return;
    const int tb = li + NTX * (lj + NTY * lk);
    auto tnode = [&](int n) { return tb + (n & 1) + NTX * (((n >> 1) & 1) + NTY * ((n >> 2) & 1)); };
    auto cls = [](int q, int d) { return (q & ((1 << d) - 1)) | ((q >> (d + 1)) << d); };
    auto cg = [&](int d, int j) { return dfc(rk.cg[d][j]); };
    auto cv = [&](int j) { return dfc(rk.cv[j]); };
    const df64 sE = g.es ? df_from_double(g.es[gid]) : df_make(1.f, 0.f);
    const df64 cmu = dfc(rk.mu) * sE, clam = dfc(rk.lam) * sE;

    // phi rows: the gradient part (integrated: constant along its axis) and phi, phi~ at the
    // Gauss points
    df64 Hp[3][NH];
    {
        df64 vphi[NV], vpt[NV];
#pragma unroll
        for (int n = 0; n < NV; ++n) {
            vphi[n] = sv[3 * NT + tnode(n)];
            vpt[n] = sv[4 * NT + tnode(n)];
        }
        fwd<3>(vphi);
        fwd<3>(vpt);
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int j = 0; j < NH; ++j) {
                const int kp = ((j >> d) << (d + 1)) | (j & ((1 << d) - 1));
                Hp[d][j] = df_scale(vphi[kp | (1 << d)] * cg(d, popc(kp)) * dfc(rk.wgce2), -(float)NH);
            }
#pragma unroll
        for (int m = 0; m < NV; ++m) {
            vphi[m] = vphi[m] * cv(popc(m));
            vpt[m] = vpt[m] * cv(popc(m));
        }
        inv<3>(vphi);
        inv<3>(vpt);
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            sq[q * NCELL + cell] = vphi[q];
            sq[(NV + q) * NCELL + cell] = vpt[q];
        }
    }
    // displacement derivatives at the Gauss points
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        df64 m_[NV];
#pragma unroll
        for (int n = 0; n < NV; ++n) m_[n] = sv[c * NT + tnode(n)];
        fwd<3>(m_);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            df64 t[NH];
#pragma unroll
            for (int j = 0; j < NH; ++j) {
                const int kp = ((j >> d) << (d + 1)) | (j & ((1 << d) - 1));
                t[j] = m_[kp | (1 << d)] * cg(d, popc(kp));
            }
            inv<2>(t);
#pragma unroll
            for (int j = 0; j < NH; ++j) sgrad[((c * 3 + d) * NH + j) * NCELL + cell] = df_renorm(t[j]);
        }
    }

    const df64 w = dfc(rk.w), omk = dfc(rk.omk), kap = dfc(rk.kap), f2k = dfc(rk.f2k), p2 = dfc(rk.p2);
    df64 ps[3][3][NH];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        df64 gu[3][3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int d = 0; d < 3; ++d) gu[c][d] = sgrad[((c * 3 + d) * NH + cls(q, d)) * NCELL + cell];
        df64 e[3][3], tr = gu[0][0], ee = gu[0][0] * gu[0][0];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            e[a][a] = gu[a][a];
            if (a > 0) { tr = tr + gu[a][a]; ee = ee + gu[a][a] * gu[a][a]; }
#pragma unroll
            for (int b = a + 1; b < 3; ++b) {
                e[a][b] = df_scale(gu[a][b] + gu[b][a], 0.5f);
                e[b][a] = e[a][b];
                ee = ee + df_scale(e[a][b] * e[a][b], 2.f);
            }
        }
        tr = df_renorm(tr);
        const df64 Es = df_scale(clam * tr * tr, 0.5f) + cmu * ee;
        const df64 phi = df_renorm(sq[q * NCELL + cell]), ptv = df_renorm(sq[(NV + q) * NCELL + cell]);
        const df64 gk = omk * ptv * ptv + kap;
        const df64 wg = w * gk, wp = w * ptv * ptv * dfc(rk.p);
        const df64 ltr = clam * tr;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = a; b < 3; ++b) {
                df64 sg = df_scale(cmu * e[a][b], 2.f);
                if (a == b) sg = sg + ltr;
                df64 f = wg * sg;
                if (a == b) f = f + wp;
                df64& pb = ps[a][b][cls(q, b)];
                pb = ((q >> b) & 1) ? pb - f : -f;
                if (a != b) {
                    df64& pa = ps[b][a][cls(q, a)];
                    pa = ((q >> a) & 1) ? pa - f : -f;
                }
            }
        // value part of the phi rows: -w (f g'(phi) E_s + 2 p phi tr - Gc/eps (1 - phi))
        const df64 one_m = df_make(1.f, 0.f) - phi;
        sq[q * NCELL + cell] = w * (dfc(rk.gce) * one_m - f2k * phi * Es - p2 * phi * tr);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int j = 0; j < NH; ++j) sgrad[((c * 3 + d) * NH + j) * NCELL + cell] = ps[c][d][j];

    const int64_t gn0 = (int64_t)gi + (int64_t)g.nn[0] * ((int64_t)gj + (int64_t)g.nn[1] * gk);
    auto noff = [&](int n) {
        return (int64_t)(n & 1) + (int64_t)g.nn[0] * (((n >> 1) & 1) + (int64_t)g.nn[1] * ((n >> 2) & 1));
    };
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        df64 p[3][NH];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
#pragma unroll
            for (int j = 0; j < NH; ++j) p[d][j] = sgrad[((c * 3 + d) * NH + j) * NCELL + cell];
            fwd<2>(p[d]);
        }
        df64 Y[NV];
        Y[0] = df_make(0.f, 0.f);
#pragma unroll
        for (int k = 1; k < NV; ++k) {
            const int d0 = (k & 1) ? 0 : ((k & 2) ? 1 : 2);
            df64 acc = p[d0][cls(k & ~(1 << d0), d0)] * cg(d0, popc(k) - 1);
#pragma unroll
            for (int d = d0 + 1; d < 3; ++d) {
                if (!(k & (1 << d))) continue;
                const int kp = k & ~(1 << d);
                acc = acc + p[d][cls(kp, d)] * cg(d, popc(kp));
            }
            Y[k] = acc;
        }
        inv3_v0_zero(Y);
        double* yc = y + c * nn + gn0;
#pragma unroll
        for (int n = 0; n < NV; ++n) atomicAdd(yc + noff(n), df_to_double(Y[n]));
    }
    {
        df64 fv[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) fv[q] = sq[q * NCELL + cell];
        fwd<3>(fv);
        df64 Y[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            df64 acc = fv[k] * cv(popc(k));
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (!(k & (1 << d))) continue;
                const int kp = k & ~(1 << d);
                acc = acc + Hp[d][cls(kp, d)] * cg(d, popc(kp));
            }
            Y[k] = acc;
        }
        inv<3>(Y);
#pragma unroll
        for (int n = 0; n < NV; ++n) atomicAdd(&y[3 * nn + gn0 + noff(n)], df_to_double(Y[n]));
    }
}

static constexpr size_t residual_cell_smem_bytes() {
    using T = CellTile;
    constexpr int NCELL = T::TX * T::TY * T::TZ, NT = (T::TX + 1) * (T::TY + 1) * (T::TZ + 1);
    return sizeof(df64) * (5 * NT + 9 * 4 * NCELL + 16 * NCELL);
}

// Gauss-point linearisation data in 3D with the tile layout of k_q1_apply_cell: U and phi~ staged
// in shared memory as df64 (one conversion per tile node), the displacement derivatives at the
// Gauss points in per-cell shared slots; one thread per cell writes its 8 x NK coefficients.
// Arithmetic as in k_q1_linearize (which serves 2D).
__global__ void __launch_bounds__(128, 4)
k_q1_linearize_cell(Geom g, LinConsts k, const double* __restrict__ U, const double* __restrict__ pt,
                    float* __restrict__ q32, float2* __restrict__ q64) {
    using T = CellTile;
    constexpr int NV = 8, NC = 4, NH = 4, NK = Q1Dims<3>::NK;
    constexpr int NCELL = T::TX * T::TY * T::TZ;
    constexpr int NTX = T::TX + 1, NTY = T::TY + 1, NTZ = T::TZ + 1;
    constexpr int NT = NTX * NTY * NTZ;
    extern __shared__ __align__(16) unsigned char lin_smem[];
    df64* sv = reinterpret_cast<df64*>(lin_smem);   // [field][node]: u_x, u_y, u_z, phi, phi~
    df64* sgrad = sv + 5 * NT;                      // [(c * 3 + d) * 4 + class][cell]

    const int ci0 = blockIdx.x * T::TX, cj0 = blockIdx.y * T::TY, ck0 = blockIdx.z * T::TZ;
    const int64_t nn = g.n_nodes, nc = g.n_cells;
    for (int t = threadIdx.x; t < NT; t += NCELL) {
        const int ti = t % NTX, tj = (t / NTX) % NTY, tk = t / (NTX * NTY);
        const int gi = ci0 + ti, gj = cj0 + tj, gk = ck0 + tk;
        const bool in = gi < g.nn[0] && gj < g.nn[1] && gk < g.nn[2];
        const int64_t gn = in ? (int64_t)gi + (int64_t)g.nn[0] * ((int64_t)gj + (int64_t)g.nn[1] * gk) : 0;
#pragma unroll
        for (int c = 0; c < NC; ++c) sv[c * NT + t] = in ? df_from_double(U[c * nn + gn]) : df_make(0.f, 0.f);
        sv[NC * NT + t] = in ? df_from_double(pt[gn]) : df_make(0.f, 0.f);
    }
    __syncthreads();

    const int cell = threadIdx.x;
    const int li = cell % T::TX, lj = (cell / T::TX) % T::TY, lk = cell / (T::TX * T::TY);
    const int gi = ci0 + li, gj = cj0 + lj, gk = ck0 + lk;
    if (gi >= g.nc[0] || gj >= g.nc[1] || gk >= g.nc[2]) return;
    const int64_t gid = (int64_t)gi + (int64_t)g.nc[0] * ((int64_t)gj + (int64_t)g.nc[1] * gk);
    if (!cell_in(g, gid)) return;
    const int tb = li + NTX * (lj + NTY * lk);
    auto tnode = [&](int n) { return tb + (n & 1) + NTX * (((n >> 1) & 1) + NTY * ((n >> 2) & 1)); };
    auto cls = [](int q, int d) { return (q & ((1 << d) - 1)) | ((q >> (d + 1)) << d); };
    const df64 sE = g.es ? df_from_double(g.es[gid]) : df_make(1.f, 0.f);
    const df64 cmu = dfc(k.mu) * sE, clam = dfc(k.lam) * sE;

    // Gauss-point values of phi and phi~
    df64 vphi[NV], vpt[NV];
#pragma unroll
    for (int n = 0; n < NV; ++n) {
        vphi[n] = sv[3 * NT + tnode(n)];
        vpt[n] = sv[4 * NT + tnode(n)];
    }
    fwd<3>(vphi);
    fwd<3>(vpt);
#pragma unroll
    for (int m = 0; m < NV; ++m) {
        vphi[m] = vphi[m] * dfc(k.cv[popc(m)]);
        vpt[m] = vpt[m] * dfc(k.cv[popc(m)]);
    }
    inv<3>(vphi);
    inv<3>(vpt);
    // displacement derivatives at the Gauss points
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        df64 m_[NV];
#pragma unroll
        for (int n = 0; n < NV; ++n) m_[n] = sv[c * NT + tnode(n)];
        fwd<3>(m_);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            df64 t[NH];
#pragma unroll
            for (int j = 0; j < NH; ++j) {
                const int kp = ((j >> d) << (d + 1)) | (j & ((1 << d) - 1));
                t[j] = m_[kp | (1 << d)] * dfc(k.cg[d][popc(kp)]);
            }
            inv<2>(t);
#pragma unroll
            for (int j = 0; j < NH; ++j) sgrad[((c * 3 + d) * NH + j) * NCELL + cell] = df_renorm(t[j]);
        }
    }
    const df64 w = dfc(k.w), omk = dfc(k.omk), kap = dfc(k.kap), f2k = dfc(k.f2k), p2 = dfc(k.p2);
    const df64 gce = dfc(k.gce);
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        df64 gu[3][3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int d = 0; d < 3; ++d) gu[c][d] = sgrad[((c * 3 + d) * NH + cls(q, d)) * NCELL + cell];
        df64 e[3][3], tr = gu[0][0], ee = gu[0][0] * gu[0][0];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            e[i][i] = gu[i][i];
            if (i > 0) { tr = tr + gu[i][i]; ee = ee + gu[i][i] * gu[i][i]; }
#pragma unroll
            for (int jx = i + 1; jx < 3; ++jx) {
                e[i][jx] = df_scale(gu[i][jx] + gu[jx][i], 0.5f);
                e[jx][i] = e[i][jx];
                ee = ee + df_scale(e[i][jx] * e[i][jx], 2.f);
            }
        }
        tr = df_renorm(tr);
        const df64 Es = df_scale(clam * tr * tr, 0.5f) + cmu * ee;
        const df64 phi = df_renorm(vphi[q]), ptv = df_renorm(vpt[q]);
        df64 vals[NK];
        vals[0] = w * (omk * ptv * ptv + kap) * sE;
        const df64 a1 = f2k * phi, b1 = p2 * phi;
        const df64 ltr = clam * tr;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int jx = i; jx < 3; ++jx) {
                df64 sig = df_scale(cmu * e[i][jx], 2.f);
                if (i == jx) sig = sig + ltr;
                df64 v = a1 * sig;
                if (i == jx) v = v + b1;
                vals[1 + sidx<3>(i, jx)] = w * v;
            }
        vals[NK - 1] = w * (f2k * Es + p2 * tr + gce);
#pragma unroll
        for (int kk = 0; kk < NK; ++kk) {
            const df64 v = df_renorm(vals[kk]);
            const int64_t idx = (int64_t)(q * NK + kk) * nc + gid;
            q32[idx] = v.hi;
            q64[idx] = make_float2(v.hi, v.lo);
        }
    }
}

static constexpr size_t linearize_cell_smem_bytes() {
    using T = CellTile;
    constexpr int NCELL = T::TX * T::TY * T::TZ, NT = (T::TX + 1) * (T::TY + 1) * (T::TZ + 1);
    return sizeof(df64) * (5 * NT + 9 * 4 * NCELL);
}

static cudaError_t launch_linearize_cell(const Geom& g, const LinConsts& k, const double* U, const double* pt,
                                         float* q32, float2* q64, cudaStream_t s) {
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (!(dev >= 0 && dev < 64 && done[dev])) {
        e = cudaFuncSetAttribute(k_q1_linearize_cell, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)linearize_cell_smem_bytes());
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) done[dev] = true;
    }
    using T = CellTile;
    dim3 grid((g.nc[0] + T::TX - 1) / T::TX, (g.nc[1] + T::TY - 1) / T::TY, (g.nc[2] + T::TZ - 1) / T::TZ);
    k_q1_linearize_cell<<<grid, T::TX * T::TY * T::TZ, linearize_cell_smem_bytes(), s>>>(g, k, U, pt, q32, q64);
    return count_launch(cudaGetLastError());
}

static ResConsts make_res_consts(const Geom& g, const Phys& ph) {
    ResConsts k;
    fill_lin_consts(g, ph, k);
    double vol = 1.0;
    for (int d = 0; d < g.dim; ++d) vol *= g.h[d];
    k.p = split_pair(ph.p);
    k.wgce2 = split_pair(2.0 * ph.Gc * ph.eps * vol / (1 << g.dim));
    return k;
}

static DiagConsts make_diag_consts(const Geom& g, const Phys& ph) {
    DiagConsts k;
    memset(&k, 0, sizeof(k));
    const int dim = g.dim, NV = 1 << dim;
    const double gpt = 1.0 / sqrt(3.0);
    const double Ap = 0.25 * (1.0 + gpt) * (1.0 + gpt), Am = 0.25 * (1.0 - gpt) * (1.0 - gpt);
    double vol = 1.0;
    for (int d = 0; d < dim; ++d) vol *= g.h[d];
    const double gcew = ph.Gc * ph.eps * vol / NV;
    for (int m = 0; m < NV; ++m) {
        double P = 1.0, Wd[3] = {0.0, 0.0, 0.0}, Ws = 0.0;
        for (int e = 0; e < dim; ++e) P *= (m >> e) & 1 ? Am : Ap;
        for (int d = 0; d < dim; ++d) {
            double f = 1.0 / (g.h[d] * g.h[d]);
            for (int e = 0; e < dim; ++e)
                if (e != d) f *= (m >> e) & 1 ? Am : Ap;
            Wd[d] = f;
            Ws += f;
        }
        for (int c = 0; c < dim; ++c) k.A[c][m] = split_pair(ph.mu * Ws + (ph.mu + ph.lam) * Wd[c]);
        k.P[m] = split_pair(P);
        k.Wg[m] = split_pair(gcew * Ws);
    }
    return k;
}

template <int OP>
static cudaError_t launch_resdiag(const Geom& g, const Phys& ph, const double* U, const double* pt,
                                  const float2* q64, const uint8_t* mask, double* y, cudaStream_t s) {
    const DiagConsts dk = make_diag_consts(g, ph);
    const ResConsts rk = make_res_consts(g, ph);
    if constexpr (OP == 0) {
        if (g.dim != 3) {
            using T = RDTile<2>;
            dim3 grid((g.nc[0] + T::TX - 1) / T::TX, (g.nc[1] + T::TY - 1) / T::TY, 1);
            k_q1_resdiag<2, 0><<<grid, T::TX * T::TY, 0, s>>>(g, rk, dk, U, pt, q64, mask, y);
            return count_launch(cudaGetLastError());
        }
        static bool done[64] = {};
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (!(dev >= 0 && dev < 64 && done[dev])) {
            e = cudaFuncSetAttribute(k_q1_residual_cell, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)residual_cell_smem_bytes());
            if (e != cudaSuccess) return e;
            if (dev >= 0 && dev < 64) done[dev] = true;
        }
        using T = CellTile;
        dim3 grid((g.nc[0] + T::TX - 1) / T::TX, (g.nc[1] + T::TY - 1) / T::TY, (g.nc[2] + T::TZ - 1) / T::TZ);
        k_q1_residual_cell<<<grid, T::TX * T::TY * T::TZ, residual_cell_smem_bytes(), s>>>(g, rk, U, pt, y);
        return count_launch(cudaGetLastError());
    } else if (g.dim == 3) {
        using T = RDTile<3>;
        dim3 grid((g.nc[0] + T::TX - 1) / T::TX, (g.nc[1] + T::TY - 1) / T::TY, (g.nc[2] + T::TZ - 1) / T::TZ);
        k_q1_resdiag<3, OP><<<grid, T::TX * T::TY * T::TZ, 0, s>>>(g, rk, dk, U, pt, q64, mask, y);
    } else {
        using T = RDTile<2>;
        dim3 grid((g.nc[0] + T::TX - 1) / T::TX, (g.nc[1] + T::TY - 1) / T::TY, 1);
        k_q1_resdiag<2, OP><<<grid, T::TX * T::TY, 0, s>>>(g, rk, dk, U, pt, q64, mask, y);
    }
    return count_launch(cudaGetLastError());
}

cudaError_t launch_q1_residual(const Geom& g, const Phys& ph, const double* U, const double* pt, double* R,
                               cudaStream_t s) {
    return launch_resdiag<0>(g, ph, U, pt, nullptr, nullptr, R, s);
}
cudaError_t launch_q1_diagonal(const Geom& g, const Phys& ph, const float2* q64, const uint8_t* mask, double* d,
                               cudaStream_t s) {
    return launch_resdiag<1>(g, ph, nullptr, nullptr, q64, mask, d, s);
}

// ------------------------------------------------------------------ energies (Sec. 5)
// bulk = int g(phi) E_s(e(u)) + phi^2 p div u, crack = int Gc/2 ((1 - phi)^2 / eps + eps |grad phi|^2)
// per cell in FP64 at the Gauss points; per-CTA partials (fixed grid) summed in a fixed order.
constexpr int kEnergyBlocks = 304;

template <int DIM>
__global__ void k_q1_energy(Geom g, Phys ph, const double* __restrict__ U, double gpt, double* __restrict__ part) {
    constexpr int NV = 1 << DIM;
    const int64_t nn = g.n_nodes;
    double vol = 1.0;
    for (int a = 0; a < DIM; ++a) vol *= g.h[a];
    const double w = vol / NV;
    double gp[DIM + 1];
    gp[0] = 1.0;
    for (int j = 1; j <= DIM; ++j) gp[j] = gp[j - 1] * gpt;
    double eb = 0.0, ec = 0.0;
    for (int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cell < g.n_cells;
         cell += (int64_t)gridDim.x * blockDim.x) {
        if (!cell_in(g, cell)) continue;
        int ci[3] = {0, 0, 0};
        int64_t r = cell;
        for (int a = 0; a < DIM; ++a) { ci[a] = (int)(r % g.nc[a]); r /= g.nc[a]; }
        const double sE = g.es ? g.es[cell] : 1.0;
        double m_[DIM + 1][NV];
#pragma unroll
        for (int n = 0; n < NV; ++n) {
            const int i = ci[0] + (n & 1), j = ci[1] + ((n >> 1) & 1), k = DIM == 3 ? ci[2] + ((n >> 2) & 1) : 0;
            const int64_t node = (int64_t)i + (int64_t)g.nn[0] * ((int64_t)j + (int64_t)g.nn[1] * k);
#pragma unroll
            for (int c = 0; c <= DIM; ++c) m_[c][n] = U[c * nn + node];
        }
#pragma unroll
        for (int c = 0; c <= DIM; ++c) fwd<DIM>(m_[c]);
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double gr[DIM + 1][DIM], phi = 0.0;
#pragma unroll
            for (int k = 0; k < NV; ++k) phi += sgn(k, q) * gp[popc(k)] / NV * m_[DIM][k];
#pragma unroll
            for (int c = 0; c <= DIM; ++c)
#pragma unroll
                for (int d = 0; d < DIM; ++d) {
                    double acc = 0.0;
#pragma unroll
                    for (int kp = 0; kp < NV; ++kp) {
                        if (kp & (1 << d)) continue;
                        acc += sgn(kp, q) * gp[popc(kp)] * m_[c][kp | (1 << d)];
                    }
                    gr[c][d] = acc * (2.0 / (g.h[d] * NV));
                }
            double tr = 0.0, ee = 0.0, gg = 0.0;
#pragma unroll
            for (int i = 0; i < DIM; ++i) tr += gr[i][i];
#pragma unroll
            for (int i = 0; i < DIM; ++i)
#pragma unroll
                for (int j = 0; j < DIM; ++j) {
                    const double eij = 0.5 * (gr[i][j] + gr[j][i]);
                    ee += eij * eij;
                }
#pragma unroll
            for (int d = 0; d < DIM; ++d) gg += gr[DIM][d] * gr[DIM][d];
            const double Es = sE * (0.5 * ph.lam * tr * tr + ph.mu * ee);
            double Esp = Es;
            if (ph.split) {   // Miehe split: g(phi) E_s^+ + (E_s - E_s^+)
                double e3[3][3], sp[3][3];
                SplitEig<double> se;
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j) e3[i][j] = (i < DIM && j < DIM) ? 0.5 * (gr[i][j] + gr[j][i]) : 0.0;
                split_stress(sE * ph.mu, sE * ph.lam, DIM, e3, sp, Esp, se);
            }
            const double gk = (1.0 - ph.kappa) * phi * phi + ph.kappa;
            eb += w * (gk * Esp + (Es - Esp) + phi * phi * ph.p * tr);
            ec += w * 0.5 * ph.Gc * ((1.0 - phi) * (1.0 - phi) / ph.eps + ph.eps * gg);
        }
    }
    __shared__ double sb[32], sc[32];
    for (int o = 16; o > 0; o >>= 1) {
        eb += __shfl_xor_sync(0xffffffffu, eb, o);
        ec += __shfl_xor_sync(0xffffffffu, ec, o);
    }
    const int wid = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { sb[wid] = eb; sc[wid] = ec; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tb = 0.0, tc = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { tb += sb[i]; tc += sc[i]; }
        part[2 * blockIdx.x] = tb;
        part[2 * blockIdx.x + 1] = tc;
    }
}

__global__ void k_energy_sum(const double* __restrict__ part, int n, double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double b = 0.0, c = 0.0;
        for (int i = 0; i < n; ++i) { b += part[2 * i]; c += part[2 * i + 1]; }
        out[0] = b;
        out[1] = c;
    }
}

cudaError_t launch_q1_energies(const Geom& g, const Phys& ph, const double* U, double* part, double* out,
                               cudaStream_t s) {
    const double gpt = 1.0 / sqrt(3.0);
    if (g.dim == 3) k_q1_energy<3><<<kEnergyBlocks, 128, 0, s>>>(g, ph, U, gpt, part);
    else k_q1_energy<2><<<kEnergyBlocks, 128, 0, s>>>(g, ph, U, gpt, part);
    count_launch(cudaGetLastError());
    k_energy_sum<<<1, 32, 0, s>>>(part, kEnergyBlocks, out);
    return count_launch(cudaGetLastError());
}

}  // namespace pff
