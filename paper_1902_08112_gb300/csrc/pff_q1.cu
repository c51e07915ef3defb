// Q1 fast path of the level operator (Sec. 4.1, 4.2), dim 2 and 3.
//
// 1) k_q1_linearize (FP64, once per state and level): for every cell and Gauss point q the
//    state enters the Jacobian only through
//      c0 = w g_kappa(phi~)                                   (G_uu: c0 sigma(du) : e(w))
//      Sp = w [2 f (1-k) phi sigma(u) + 2 p phi I]            (G_phiu: Sp : e(du) psi)
//      c1 = w [2 f (1-k) E_s(u) + 2 p div u + Gc/eps]         (G_phiphi mass part)
//    (w = Gauss weight x |K|).  They are stored per level as FP32 and as df64 pairs, cell
//    fastest, so the applies read them coalesced.
// 2) k_q1_apply<DIM, S> (S = float for the FP32 V-cycle operators, S = df64 for the
//    FP64-accurate operators): y = G~ x from x and the stored coefficients.
//
// Sum factorisation for Q1 on a uniform cell (the tensor-product structure of Sec. 4.1): the 2^d
// nodal values of a field map to 2^d "modal" coefficients m_k = sum_n prod_{a in k}(2 n_a - 1) v_n
// by d butterfly stages (a, b) -> (a + b, b - a).  In reference coordinates xi in [-1,1]^d the
// field is 2^-d sum_k m_k xi^k, so at the Gauss points xi = sigma g (g = 1/sqrt 3, sigma in
// {-1,1}^d) values and gradients are sums of scaled m_k with sign patterns sigma^k, and the
// transposed (integration) step is the same butterfly run backwards.  All sign patterns are
// compile-time constants after unrolling.
#include "pff_df64.cuh"
#include "pff_internal.cuh"
#include "pff_q1.cuh"

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
};

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

// ------------------------------------------------------------------ linearisation data (FP64)
template <int DIM>
__global__ void k_q1_linearize(Geom g, Phys ph, const double* __restrict__ U, const double* __restrict__ pt,
                               float* __restrict__ q32, float2* __restrict__ q64, double gpt) {
    using D = Q1Dims<DIM>;
    constexpr int NV = D::NV, NK = D::NK;
    const int64_t nc = g.n_cells, nn = g.n_nodes;
    double vol = 1.0;
    for (int a = 0; a < DIM; ++a) vol *= g.h[a];
    const double w = vol / NV;
    double gp[DIM + 1];
    gp[0] = 1.0;
    for (int j = 1; j <= DIM; ++j) gp[j] = gp[j - 1] * gpt;
    for (int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cell < nc;
         cell += (int64_t)gridDim.x * blockDim.x) {
        int ci[3] = {0, 0, 0};
        int64_t r = cell;
        for (int a = 0; a < DIM; ++a) { ci[a] = (int)(r % g.nc[a]); r /= g.nc[a]; }
        int64_t node[NV];
#pragma unroll
        for (int n = 0; n < NV; ++n) {
            const int i = ci[0] + (n & 1), j = ci[1] + ((n >> 1) & 1), k = DIM == 3 ? ci[2] + ((n >> 2) & 1) : 0;
            node[n] = (int64_t)i + (int64_t)g.nn[0] * ((int64_t)j + (int64_t)g.nn[1] * k);
        }
        double mu_[DIM][NV], mphi[NV], mpt[NV];
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
#pragma unroll
            for (int n = 0; n < NV; ++n) mu_[c][n] = U[c * nn + node[n]];
            fwd<DIM>(mu_[c]);
        }
#pragma unroll
        for (int n = 0; n < NV; ++n) { mphi[n] = U[DIM * nn + node[n]]; mpt[n] = pt[node[n]]; }
        fwd<DIM>(mphi);
        fwd<DIM>(mpt);
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double gu[DIM][DIM], phi = 0.0, ptv = 0.0;
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                const double s = sgn(k, q) * gp[popc(k)] / NV;
                phi += s * mphi[k];
                ptv += s * mpt[k];
            }
#pragma unroll
            for (int c = 0; c < DIM; ++c)
#pragma unroll
                for (int d = 0; d < DIM; ++d) {
                    double acc = 0.0;
#pragma unroll
                    for (int kp = 0; kp < NV; ++kp) {
                        if (kp & (1 << d)) continue;
                        acc += sgn(kp, q) * gp[popc(kp)] * mu_[c][kp | (1 << d)];
                    }
                    gu[c][d] = acc * (2.0 / (g.h[d] * NV));
                }
            double e[DIM][DIM], tr = 0.0, ee = 0.0;
#pragma unroll
            for (int i = 0; i < DIM; ++i)
#pragma unroll
                for (int j = 0; j < DIM; ++j) e[i][j] = 0.5 * (gu[i][j] + gu[j][i]);
#pragma unroll
            for (int i = 0; i < DIM; ++i) tr += e[i][i];
#pragma unroll
            for (int i = 0; i < DIM; ++i)
#pragma unroll
                for (int j = 0; j < DIM; ++j) ee += e[i][j] * e[i][j];
            const double Es = 0.5 * ph.lam * tr * tr + ph.mu * ee;
            const double gk = (1.0 - ph.kappa) * ptv * ptv + ph.kappa;
            double vals[NK];
            vals[0] = w * gk;
            const double a1 = 2.0 * ph.f * (1.0 - ph.kappa) * phi, b1 = 2.0 * ph.p * phi;
#pragma unroll
            for (int i = 0; i < DIM; ++i)
#pragma unroll
                for (int j = i; j < DIM; ++j) {
                    const double sig = 2.0 * ph.mu * e[i][j] + (i == j ? ph.lam * tr : 0.0);
                    vals[1 + sidx<DIM>(i, j)] = w * (a1 * sig + (i == j ? b1 : 0.0));
                }
            vals[NK - 1] = w * (2.0 * ph.f * (1.0 - ph.kappa) * Es + 2.0 * ph.p * tr + ph.Gc / ph.eps);
#pragma unroll
            for (int k = 0; k < NK; ++k) {
                const int64_t idx = (int64_t)(q * NK + k) * nc + cell;
                q32[idx] = (float)vals[k];
                const float hi = __double2float_rn(vals[k]);
                q64[idx] = make_float2(hi, __double2float_rn(vals[k] - (double)hi));
            }
        }
    }
}

cudaError_t launch_q1_linearize(const Geom& g, const Phys& ph, const double* U, const double* pt, float* q32,
                                float2* q64, cudaStream_t s) {
    const double gpt = 1.0 / sqrt(3.0);
    int64_t blocks = (g.n_cells + 127) / 128;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    if (g.dim == 3) k_q1_linearize<3><<<(int)blocks, 128, 0, s>>>(g, ph, U, pt, q32, q64, gpt);
    else k_q1_linearize<2><<<(int)blocks, 128, 0, s>>>(g, ph, U, pt, q32, q64, gpt);
    return count_launch(cudaGetLastError());
}

// ------------------------------------------------------------------ modal apply
template <int DIM, typename S>
struct Q1Tile;
template <> struct Q1Tile<3, float> { static constexpr int TX = 8, TY = 8, TZ = 4; };
template <> struct Q1Tile<3, df64> { static constexpr int TX = 8, TY = 4, TZ = 4; };
template <> struct Q1Tile<2, float> { static constexpr int TX = 16, TY = 16, TZ = 1; };
template <> struct Q1Tile<2, df64> { static constexpr int TX = 16, TY = 8, TZ = 1; };

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

template <int DIM, typename S, bool BLOCKDIAG>
__global__ void __launch_bounds__(Q1Tile<DIM, S>::TX * Q1Tile<DIM, S>::TY * Q1Tile<DIM, S>::TZ)
k_q1_apply(Q1ApplyArgs<typename Scalar<S>::storage, typename QData<S>::type> a) {
    using T = Q1Tile<DIM, S>;
    using D = Q1Dims<DIM>;
    using St = typename Scalar<S>::storage;
    constexpr int NV = D::NV, NC = D::NC, NK = D::NK;
    constexpr int NCELL = T::TX * T::TY * T::TZ;
    constexpr int NTX = T::TX + 1, NTY = T::TY + 1, NTZ = DIM == 3 ? T::TZ + 1 : 1;
    constexpr int NT = NTX * NTY * NTZ;

    __shared__ S sx[NC * NT];
    __shared__ S sel[NV * NC * NCELL];
    __shared__ uint8_t smask[NT];

    const Geom& g = a.g;
    const int ci0 = blockIdx.x * T::TX, cj0 = blockIdx.y * T::TY, ck0 = DIM == 3 ? blockIdx.z * T::TZ : 0;
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
    const bool valid = (ci0 + li < g.nc[0]) && (cj0 + lj < g.nc[1]) && (DIM == 2 || ck0 + lk < g.nc[2]);
    if (valid) {
        const int64_t gid = (int64_t)(ci0 + li) + (int64_t)g.nc[0] * ((int64_t)(cj0 + lj) + (int64_t)g.nc[1] * (ck0 + lk));
        const int tb = li + NTX * (lj + NTY * lk);
        S cv[DIM + 1], cg[DIM][DIM];
#pragma unroll
        for (int j = 0; j <= DIM; ++j) cv[j] = Scalar<S>::from_double(a.cv[j]);
#pragma unroll
        for (int d = 0; d < DIM; ++d)
#pragma unroll
            for (int j = 0; j < DIM; ++j) cg[d][j] = Scalar<S>::from_double(a.cg[d][j]);
        const S mu2 = Scalar<S>::from_double(2.0 * a.mu), lam = Scalar<S>::from_double(a.lam);
        const S gcew = Scalar<S>::from_double(a.gcew);

        const S mu = Scalar<S>::from_double(a.mu);

        // ======== pass 1: displacement rows (G_uu) and the coupling term of the phi rows
        S cpl[NV];
        {
            S G[DIM][DIM][NV / 2];     // G[c][d][j]: gradient-form coefficients, j = masks without bit d
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
                        G[c][d][j] = v[kp | (1 << d)] * cg[d][popc(kp)];
                        ++j;
                    }
                }
            }
            S H[DIM][DIM][NV / 2];
#pragma unroll
            for (int c = 0; c < DIM; ++c)
#pragma unroll
                for (int d = 0; d < DIM; ++d)
#pragma unroll
                    for (int j = 0; j < NV / 2; ++j) H[c][d][j] = Scalar<S>::zero();
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                S gd[DIM][DIM];
#pragma unroll
                for (int c = 0; c < DIM; ++c)
#pragma unroll
                    for (int d = 0; d < DIM; ++d) {
                        S acc = Scalar<S>::zero();
                        int j = 0;
#pragma unroll
                        for (int kp = 0; kp < NV; ++kp) {
                            if (kp & (1 << d)) continue;
                            acc = (sgn(kp, q) > 0) ? acc + G[c][d][j] : acc - G[c][d][j];
                            ++j;
                        }
                        gd[c][d] = acc;
                    }
                const S c0 = QData<S>::get(a.qd, (int64_t)(q * NK + 0) * g.n_cells + gid);
                S tr = gd[0][0];
#pragma unroll
                for (int i = 1; i < DIM; ++i) tr = tr + gd[i][i];
                const S ltr = lam * tr;
                S fu[DIM][DIM];
#pragma unroll
                for (int i = 0; i < DIM; ++i)
#pragma unroll
                    for (int j = i; j < DIM; ++j) {
                        // c0 sigma(du)_ij with sigma = 2 mu e + lambda tr I and 2 e_ij = du_i,j + du_j,i
                        const S sg = (i == j) ? mu2 * gd[i][i] + ltr : mu * (gd[i][j] + gd[j][i]);
                        const S f = c0 * sg;
                        fu[i][j] = f;
                        fu[j][i] = f;
                    }
                S cp = Scalar<S>::zero();
                if constexpr (!BLOCKDIAG) {
#pragma unroll
                    for (int i = 0; i < DIM; ++i)
#pragma unroll
                        for (int j = i; j < DIM; ++j) {
                            const S sp = QData<S>::get(a.qd, (int64_t)(q * NK + 1 + sidx<DIM>(i, j)) * g.n_cells + gid);
                            cp = cp + sp * ((i == j) ? gd[i][i] : gd[i][j] + gd[j][i]);   // Sp : e(du)
                        }
                }
                cpl[q] = cp;
#pragma unroll
                for (int c = 0; c < DIM; ++c)
#pragma unroll
                    for (int d = 0; d < DIM; ++d) {
                        int j = 0;
#pragma unroll
                        for (int kp = 0; kp < NV; ++kp) {
                            if (kp & (1 << d)) continue;
                            H[c][d][j] = (sgn(kp, q) > 0) ? H[c][d][j] + fu[c][d] : H[c][d][j] - fu[c][d];
                            ++j;
                        }
                    }
            }
#pragma unroll
            for (int c = 0; c < DIM; ++c) {
                S Y[NV];
#pragma unroll
                for (int k = 0; k < NV; ++k) {
                    S acc = Scalar<S>::zero();
#pragma unroll
                    for (int d = 0; d < DIM; ++d) {
                        if (!(k & (1 << d))) continue;
                        const int kp = k & ~(1 << d);
                        const int j = (kp & ((1 << d) - 1)) | ((kp >> (d + 1)) << d);   // kp without bit d
                        acc = acc + H[c][d][j] * cg[d][popc(kp)];
                    }
                    Y[k] = acc;
                }
                inv<DIM>(Y);
#pragma unroll
                for (int n = 0; n < NV; ++n) sel[(n * NC + c) * NCELL + cell] = Y[n];
            }
        }
        // ======== pass 2: phase-field rows (G_phiphi and the stored coupling)
        {
            S v[NV];
#pragma unroll
            for (int n = 0; n < NV; ++n) {
                const int off = (n & 1) + NTX * (((n >> 1) & 1) + NTY * (DIM == 3 ? (n >> 2) & 1 : 0));
                v[n] = sx[DIM * NT + tb + off];
            }
            fwd<DIM>(v);
            S Mp[NV], Gp[DIM][NV / 2];
#pragma unroll
            for (int k = 0; k < NV; ++k) Mp[k] = v[k] * cv[popc(k)];
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
                int j = 0;
#pragma unroll
                for (int kp = 0; kp < NV; ++kp) {
                    if (kp & (1 << d)) continue;
                    Gp[d][j] = v[kp | (1 << d)] * cg[d][popc(kp)];
                    ++j;
                }
            }
            S F[NV], Hp[DIM][NV / 2];
#pragma unroll
            for (int k = 0; k < NV; ++k) F[k] = Scalar<S>::zero();
#pragma unroll
            for (int d = 0; d < DIM; ++d)
#pragma unroll
                for (int j = 0; j < NV / 2; ++j) Hp[d][j] = Scalar<S>::zero();
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                S dphi = Scalar<S>::zero();
#pragma unroll
                for (int k = 0; k < NV; ++k) dphi = (sgn(k, q) > 0) ? dphi + Mp[k] : dphi - Mp[k];
                const S c1 = QData<S>::get(a.qd, (int64_t)(q * NK + NK - 1) * g.n_cells + gid);
                const S fp = c1 * dphi + cpl[q];
#pragma unroll
                for (int k = 0; k < NV; ++k) F[k] = (sgn(k, q) > 0) ? F[k] + fp : F[k] - fp;
#pragma unroll
                for (int d = 0; d < DIM; ++d) {
                    S gph = Scalar<S>::zero();
                    int j = 0;
#pragma unroll
                    for (int kp = 0; kp < NV; ++kp) {
                        if (kp & (1 << d)) continue;
                        gph = (sgn(kp, q) > 0) ? gph + Gp[d][j] : gph - Gp[d][j];
                        ++j;
                    }
                    const S fg = gcew * gph;
                    j = 0;
#pragma unroll
                    for (int kp = 0; kp < NV; ++kp) {
                        if (kp & (1 << d)) continue;
                        Hp[d][j] = (sgn(kp, q) > 0) ? Hp[d][j] + fg : Hp[d][j] - fg;
                        ++j;
                    }
                }
            }
            S Y[NV];
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                S acc = F[k] * cv[popc(k)];
#pragma unroll
                for (int d = 0; d < DIM; ++d) {
                    if (!(k & (1 << d))) continue;
                    const int kp = k & ~(1 << d);
                    const int j = (kp & ((1 << d) - 1)) | ((kp >> (d + 1)) << d);
                    acc = acc + Hp[d][j] * cg[d][popc(kp)];
                }
                Y[k] = acc;
            }
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
    const int dim = a.g.dim, NV = 1 << dim;
    const double gpt = 1.0 / sqrt(3.0);
    double gp[4] = {1.0, gpt, gpt * gpt, gpt * gpt * gpt};
    for (int j = 0; j <= 3; ++j) a.cv[j] = gp[j] / NV;
    for (int d = 0; d < 3; ++d)
        for (int j = 0; j < 3; ++j) a.cg[d][j] = d < dim ? gp[j] * 2.0 / (a.g.h[d] * NV) : 0.0;
    double vol = 1.0;
    for (int d = 0; d < dim; ++d) vol *= a.g.h[d];
    a.mu = ph.mu;
    a.lam = ph.lam;
    a.gcew = ph.Gc * ph.eps * vol / NV;
}

cudaError_t launch_q1_apply64(const Geom& g, const Phys& ph, const float2* qd, const double* x, double* y,
                              const uint8_t* mask, int phi_bits, bool blockdiag, cudaStream_t s) {
    Q1ApplyArgs<double, float2> a;
    a.g = g;
    a.qd = qd;
    a.x = x;
    a.y = y;
    a.mask = mask;
    a.phi_bits = phi_bits;
    fill_consts(a, ph);
    return blockdiag ? launch_apply_dim<df64, true>(a, s) : launch_apply_dim<df64, false>(a, s);
}

cudaError_t launch_q1_apply32(const Geom& g, const Phys& ph, const float* qd, const float* x, float* y,
                              const uint8_t* mask, int phi_bits, bool blockdiag, cudaStream_t s) {
    Q1ApplyArgs<float, float> a;
    a.g = g;
    a.qd = qd;
    a.x = x;
    a.y = y;
    a.mask = mask;
    a.phi_bits = phi_bits;
    fill_consts(a, ph);
    return blockdiag ? launch_apply_dim<float, true>(a, s) : launch_apply_dim<float, false>(a, s);
}

}  // namespace pff
