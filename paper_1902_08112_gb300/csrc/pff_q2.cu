// Q2 fast path of the level operator on 3D levels (Sec. 4.1: sum factorisation of the tensor-product
// element; Q2 is an extension of the paper's Q1 discretisation).
//
// One warp per cell: lane l = a + 3 b + 9 c (l < 27) stands for node (a, b, c) of the cell and for
// Gauss point (a, b, c) of the 3-point rule.  Values and gradients at the Gauss points come from the
// nodal values in three 1D stages (x, then y, then z), each a 3 x 3 contraction whose inputs are
// exchanged by warp shuffles; integration against the test functions runs the transposed stages in
// the opposite order.  A lane adds its node's result to y with one FP64 (or FP32) atomic per
// component.  No shared-memory staging, no CTA barrier.  Lanes 27..31 follow node/point (0, 0, 0)
// so that every shuffle reads a live lane, and store nothing.
//
// 1) k_q2_linearize (double-float, once per state and level): per cell and Gauss point the state
//    enters the Jacobian through c0 = w g_kappa(phi~), Sp = w [2 f (1-k) phi sigma(u) + 2 p phi I],
//    c1 = w [2 f (1-k) E_s(u) + 2 p div u + Gc/eps] (w = Gauss weight x |K|, the per-cell modulus
//    factor folded into c0, sigma and E_s), stored as FP32 and as df64 pairs at
//    [(cell * 8 + k) * 27 + q] (Gauss point fastest: a warp reads 27 consecutive entries).
// 2) k_q2_apply<S, BLOCKDIAG> (S = df64: FP64-accurate operator; S = float: V-cycle operator).
#include "pff_df64.cuh"
#include "pff_internal.cuh"
#include "pff_q1.cuh"

namespace pff {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kNQ = 27, kNK = 8;
constexpr int kWarpsPerCta = 8;

template <typename S>
__device__ __forceinline__ S shfl(S v, int src);
template <>
__device__ __forceinline__ float shfl<float>(float v, int src) { return __shfl_sync(kFull, v, src); }
template <>
__device__ __forceinline__ df64 shfl<df64>(df64 v, int src) {
    return df_make(__shfl_sync(kFull, v.hi, src), __shfl_sync(kFull, v.lo, src));
}
template <typename S>
__device__ __forceinline__ S pair(float2 v);
template <>
__device__ __forceinline__ float pair<float>(float2 v) { return v.x; }
template <>
__device__ __forceinline__ df64 pair<df64>(float2 v) { return df_make(v.x, v.y); }
__device__ __forceinline__ float2 to_pair(df64 v) { return make_float2(v.hi, v.lo); }
// exact scaling by a power of two; hi + lo renormalised so that hi is the float nearest to the value
__device__ __forceinline__ df64 df_scale(df64 a, float s) { return df_make(a.hi * s, a.lo * s); }
__device__ __forceinline__ df64 df_renorm(df64 a) { return df_two_sum(a.hi, a.lo); }

// symmetric index: xx yy zz xy xz yz
__host__ __device__ constexpr int sym3(int i, int j) {
    return i == j ? i : ((i < j ? i : j) == 0 ? ((i < j ? j : i) == 1 ? 3 : 4) : 5);
}

}  // namespace

// 1D tables of the 3-point rule on [0,1] (node k, point q): value N[k][q], derivative along axis d
// divided by h_d, D[d][k][q]; Gauss weight x |K| per point; host-prepared float pairs.
struct Q2Consts {
    float2 N[3][3];
    float2 D[3][3][3];
    float2 w[27];
    float2 gcew[27];      // Gc eps w (phi gradient-gradient term)
    float2 mu, lam, mu2;
    // linearisation
    float2 omk, kap, f2k, p2, gce;
};

static float2 q2_split(double d) {
    const float hi = (float)d;
    return make_float2(hi, (float)(d - (double)hi));
}

Q2Consts make_q2_consts(const Geom& g, const Phys& ph) {
    Q2Consts k;
    const double r = std::sqrt(3.0 / 5.0);
    const double xq[3] = {0.5 * (1.0 - r), 0.5, 0.5 * (1.0 + r)};
    const double wq[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
    for (int q = 0; q < 3; ++q) {
        const double t = xq[q];
        const double Nv[3] = {2.0 * t * t - 3.0 * t + 1.0, 4.0 * t - 4.0 * t * t, 2.0 * t * t - t};
        const double Dv[3] = {4.0 * t - 3.0, 4.0 - 8.0 * t, 4.0 * t - 1.0};
        for (int n = 0; n < 3; ++n) {
            k.N[n][q] = q2_split(Nv[n]);
            for (int d = 0; d < 3; ++d) k.D[d][n][q] = q2_split(Dv[n] / g.h[d]);
        }
    }
    const double vol = g.h[0] * g.h[1] * g.h[2];
    for (int q = 0; q < 27; ++q) {
        const double w = wq[q % 3] * wq[(q / 3) % 3] * wq[q / 9] * vol;
        k.w[q] = q2_split(w);
        k.gcew[q] = q2_split(ph.Gc * ph.eps * w);
    }
    k.mu = q2_split(ph.mu);
    k.lam = q2_split(ph.lam);
    k.mu2 = q2_split(2.0 * ph.mu);
    k.omk = q2_split(1.0 - ph.kappa);
    k.kap = q2_split(ph.kappa);
    k.f2k = q2_split(2.0 * ph.f * (1.0 - ph.kappa));
    k.p2 = q2_split(2.0 * ph.p);
    k.gce = q2_split(ph.Gc / ph.eps);
    return k;
}

namespace {

struct LaneXYZ {
    int a, b, c;
    bool live;
};
__device__ __forceinline__ LaneXYZ lane_xyz() {
    const int l = threadIdx.x & 31;
    LaneXYZ L;
    L.live = l < kNQ;
    const int m = L.live ? l : 0;
    L.a = m % 3;
    L.b = (m / 3) % 3;
    L.c = m / 9;
    return L;
}

// 1D tables staged in shared memory (lanes index them by their own coordinate)
struct Q2Tab {
    float2 N[9];      // [k * 3 + q]
    float2 D[27];     // [(d * 3 + k) * 3 + q]
};
__device__ __forceinline__ void q2_stage_tables(Q2Tab& t, const Q2Consts& K) {
    for (int i = threadIdx.x; i < 36; i += blockDim.x) {
        if (i < 9) t.N[i] = K.N[i / 3][i % 3];
        else t.D[i - 9] = K.D[(i - 9) / 9][((i - 9) / 3) % 3][(i - 9) % 3];
    }
}
#define TN(k, q) tab.N[(k) * 3 + (q)]
#define TD(d, k, q) tab.D[((d) * 3 + (k)) * 3 + (q)]

// Gauss-point value (want_val) and gradient of the field whose nodal value this lane holds
template <typename S, bool WANT_VAL>
__device__ __forceinline__ void q2_interp(S v, const LaneXYZ& L, const Q2Tab& tab, S& val, S (&gr)[3]) {
    S xn = Scalar<S>::zero(), xd = Scalar<S>::zero();
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const S vk = shfl(v, k + 3 * L.b + 9 * L.c);
        const S n = pair<S>(TN(k, L.a)), d = pair<S>(TD(0, k, L.a));
        xn = k == 0 ? n * vk : xn + n * vk;
        xd = k == 0 ? d * vk : xd + d * vk;
    }
    S ynn = Scalar<S>::zero(), ynd = Scalar<S>::zero(), ydn = Scalar<S>::zero();
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int src = L.a + 3 * k + 9 * L.c;
        const S a = shfl(xn, src), b = shfl(xd, src);
        const S n = pair<S>(TN(k, L.b)), d = pair<S>(TD(1, k, L.b));
        ynn = k == 0 ? n * a : ynn + n * a;
        ynd = k == 0 ? d * a : ynd + d * a;
        ydn = k == 0 ? n * b : ydn + n * b;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int src = L.a + 3 * L.b + 9 * k;
        const S a = shfl(ynn, src), b = shfl(ynd, src), c = shfl(ydn, src);
        const S n = pair<S>(TN(k, L.c)), d = pair<S>(TD(2, k, L.c));
        if (WANT_VAL) val = k == 0 ? n * a : val + n * a;
        gr[2] = k == 0 ? d * a : gr[2] + d * a;
        gr[1] = k == 0 ? n * b : gr[1] + n * b;
        gr[0] = k == 0 ? n * c : gr[0] + n * c;
    }
}

// integration against the test functions of this lane's node: sum over the Gauss points of
// f0 N_node + f . grad N_node (has_f0 = false: f0 = 0)
template <typename S, bool HAS_F0>
__device__ __forceinline__ S q2_integrate(S f0, const S (&f)[3], const LaneXYZ& L, const Q2Tab& tab) {
    S z0 = Scalar<S>::zero(), zx = Scalar<S>::zero(), zy = Scalar<S>::zero();
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int src = L.a + 3 * L.b + 9 * k;
        const S n = pair<S>(TN(L.c, k)), d = pair<S>(TD(2, L.c, k));
        const S fz = shfl(f[2], src), fx = shfl(f[0], src), fy = shfl(f[1], src);
        S t = d * fz;
        if (HAS_F0) t = t + n * shfl(f0, src);
        z0 = k == 0 ? t : z0 + t;
        zx = k == 0 ? n * fx : zx + n * fx;
        zy = k == 0 ? n * fy : zy + n * fy;
    }
    S y0 = Scalar<S>::zero(), yx = Scalar<S>::zero();
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int src = L.a + 3 * k + 9 * L.c;
        const S n = pair<S>(TN(L.b, k)), d = pair<S>(TD(1, L.b, k));
        const S t = n * shfl(z0, src) + d * shfl(zy, src);
        y0 = k == 0 ? t : y0 + t;
        const S u = n * shfl(zx, src);
        yx = k == 0 ? u : yx + u;
    }
    S r = Scalar<S>::zero();
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int src = k + 3 * L.b + 9 * L.c;
        const S t = pair<S>(TN(L.a, k)) * shfl(y0, src) + pair<S>(TD(0, L.a, k)) * shfl(yx, src);
        r = k == 0 ? t : r + t;
    }
    return r;
}

__device__ __forceinline__ int64_t q2_node(const Geom& g, int64_t cell, const LaneXYZ& L) {
    const int ci = (int)(cell % g.nc[0]);
    const int64_t r = cell / g.nc[0];
    const int cj = (int)(r % g.nc[1]), ck = (int)(r / g.nc[1]);
    return (int64_t)(2 * ci + L.a) + (int64_t)g.nn[0] * ((int64_t)(2 * cj + L.b) + (int64_t)g.nn[1] * (2 * ck + L.c));
}

}  // namespace

// ---------------------------------------------------------------- linearisation data
// One warp per cell (warp-stride over the cells of the level); double-float arithmetic; values that
// come out of sums with cancellation (Gauss-point gradients and values) are renormalised before the
// products that follow.
__global__ void __launch_bounds__(32 * kWarpsPerCta)
k_q2_linearize(Geom g, Q2Consts K, const double* __restrict__ U, const double* __restrict__ pt, float* __restrict__ q32,
               float2* __restrict__ q64) {
    __shared__ Q2Tab tab;
    q2_stage_tables(tab, K);
    __syncthreads();
    const LaneXYZ L = lane_xyz();
    const int lane = threadIdx.x & 31, q = L.live ? lane : 0;
    const int64_t nn = g.n_nodes;
    const int64_t stride = (int64_t)gridDim.x * kWarpsPerCta;
    for (int64_t cell = (int64_t)blockIdx.x * kWarpsPerCta + (threadIdx.x >> 5); cell < g.n_cells; cell += stride) {
        if (!cell_in(g, cell)) continue;                      // uniform across the warp
        const int64_t gn = q2_node(g, cell, L);
        df64 gu[3][3], dummy;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            q2_interp<df64, false>(df_from_double(U[c * nn + gn]), L, tab, dummy, gu[c]);
#pragma unroll
            for (int d = 0; d < 3; ++d) gu[c][d] = df_renorm(gu[c][d]);
        }
        df64 phi, ptv, gtmp[3];
        q2_interp<df64, true>(df_from_double(U[3 * nn + gn]), L, tab, phi, gtmp);
        q2_interp<df64, true>(df_from_double(pt[gn]), L, tab, ptv, gtmp);
        phi = df_renorm(phi);
        ptv = df_renorm(ptv);
        const df64 sE = g.es ? df_from_double(g.es[cell]) : df_make(1.f, 0.f);
        const df64 cmu = pair<df64>(K.mu) * sE, clam = pair<df64>(K.lam) * sE;
        const df64 w = pair<df64>(K.w[q]);
        df64 e[3][3], tr = gu[0][0], ee = gu[0][0] * gu[0][0];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            e[i][i] = gu[i][i];
            if (i > 0) {
                tr = tr + gu[i][i];
                ee = ee + gu[i][i] * gu[i][i];
            }
#pragma unroll
            for (int j = i + 1; j < 3; ++j) {
                e[i][j] = df_scale(gu[i][j] + gu[j][i], 0.5f);
                e[j][i] = e[i][j];
                ee = ee + df_scale(e[i][j] * e[i][j], 2.f);
            }
        }
        tr = df_renorm(tr);
        const df64 Es = df_scale(clam * tr * tr, 0.5f) + cmu * ee;
        df64 vals[kNK];
        vals[0] = w * (pair<df64>(K.omk) * ptv * ptv + pair<df64>(K.kap)) * sE;
        const df64 a1 = pair<df64>(K.f2k) * phi, b1 = pair<df64>(K.p2) * phi, ltr = clam * tr;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = i; j < 3; ++j) {
                df64 sig = df_scale(cmu * e[i][j], 2.f);
                if (i == j) sig = sig + ltr;
                df64 v = a1 * sig;
                if (i == j) v = v + b1;
                vals[1 + sym3(i, j)] = w * v;
            }
        vals[kNK - 1] = w * (pair<df64>(K.f2k) * Es + pair<df64>(K.p2) * tr + pair<df64>(K.gce));
        if (L.live) {
#pragma unroll
            for (int k = 0; k < kNK; ++k) {
                const df64 v = df_renorm(vals[k]);
                const int64_t idx = (cell * kNK + k) * kNQ + lane;
                q32[idx] = v.hi;
                q64[idx] = make_float2(v.hi, v.lo);
            }
        }
    }
}

// ---------------------------------------------------------------- apply
template <typename S>
struct Q2Data;
template <>
struct Q2Data<float> {
    using type = float;
    __device__ static __forceinline__ float get(const float* p, int64_t i) { return __ldg(p + i); }
};
template <>
struct Q2Data<df64> {
    using type = float2;
    __device__ static __forceinline__ df64 get(const float2* p, int64_t i) {
        const float2 v = __ldg(p + i);
        return df_make(v.x, v.y);
    }
};

template <typename S>
struct Q2ApplyArgs {
    Geom g;
    const typename Q2Data<S>::type* qd;
    const typename Scalar<S>::storage* x;
    typename Scalar<S>::storage* y;
    const uint8_t* mask;
    int phi_bits;
    Q2Consts k;
};

// y += G~ x on the free rows of a 3D Q2 level (eliminated rows preset by the caller, eliminated
// columns read as 0).  BLOCKDIAG drops the coupling G_phiu (operator of the smoother blocks).
template <typename S, bool BLOCKDIAG>
__global__ void __launch_bounds__(32 * kWarpsPerCta) k_q2_apply(Q2ApplyArgs<S> a) {
    __shared__ Q2Tab tab;
    q2_stage_tables(tab, a.k);
    __syncthreads();
    const Geom& g = a.g;
    const LaneXYZ L = lane_xyz();
    const int lane = threadIdx.x & 31, q = L.live ? lane : 0;
    const int64_t nn = g.n_nodes;
    const S mu = pair<S>(a.k.mu), mu2 = pair<S>(a.k.mu2), lam = pair<S>(a.k.lam);
    const S gcew = pair<S>(a.k.gcew[q]);
    const int64_t stride = (int64_t)gridDim.x * kWarpsPerCta;
    for (int64_t cell = (int64_t)blockIdx.x * kWarpsPerCta + (threadIdx.x >> 5); cell < g.n_cells; cell += stride) {
        if (!cell_in(g, cell)) continue;                      // uniform across the warp
        const int64_t gn = q2_node(g, cell, L);
        const uint8_t m = a.mask[gn];
        // Gauss-point gradients of the displacement components and value/gradient of phi
        S gd[3][3], dphi, gphi[3], dummy;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const bool el = ((m >> c) & 1) != 0;
            const S xv = el ? Scalar<S>::zero() : load_cvt<S>(a.x[c * nn + gn]);
            q2_interp<S, false>(xv, L, tab, dummy, gd[c]);
        }
        {
            const bool el = (m & a.phi_bits) != 0;
            const S xv = el ? Scalar<S>::zero() : load_cvt<S>(a.x[3 * nn + gn]);
            q2_interp<S, true>(xv, L, tab, dphi, gphi);
        }
        const int64_t qb = cell * kNK * kNQ + q;
        const S c0 = Q2Data<S>::get(a.qd, qb);
        const S c1 = Q2Data<S>::get(a.qd, qb + (kNK - 1) * kNQ);
        // displacement rows: c0 sigma(du) (symmetric flux on grad w)
        const S c0m = c0 * mu, c0m2 = c0 * mu2;
        const S c0lt = (c0 * lam) * (gd[0][0] + gd[1][1] + gd[2][2]);
        S fu[3][3];
        S cp = Scalar<S>::zero();
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = i; j < 3; ++j) {
                const S e2 = (i == j) ? gd[i][i] : gd[i][j] + gd[j][i];
                fu[i][j] = (i == j) ? c0m2 * e2 + c0lt : c0m * e2;
                fu[j][i] = fu[i][j];
                if constexpr (!BLOCKDIAG) {
                    const S sp = Q2Data<S>::get(a.qd, qb + (1 + sym3(i, j)) * kNQ);
                    cp = (i == 0 && j == 0) ? sp * e2 : cp + sp * e2;     // Sp : e(du)
                }
            }
        // phi rows: (c1 dphi + Sp : e(du)) psi + Gc eps w grad dphi . grad psi
        const S f0 = BLOCKDIAG ? c1 * dphi : c1 * dphi + cp;
        S fg[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) fg[d] = gcew * gphi[d];
        typename Scalar<S>::storage* y = a.y;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const S r = q2_integrate<S, false>(Scalar<S>::zero(), fu[c], L, tab);
            if (L.live && !((m >> c) & 1)) atomicAdd(&y[c * nn + gn], Scalar<S>::store(r));
        }
        const S r = q2_integrate<S, true>(f0, fg, L, tab);
        if (L.live && !(m & a.phi_bits)) atomicAdd(&y[3 * nn + gn], Scalar<S>::store(r));
    }
}

static int q2_grid(int64_t n_cells) {
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t need = (n_cells + kWarpsPerCta - 1) / kWarpsPerCta;
    const int64_t cap = (int64_t)sms * 8;      // 8 resident CTAs of 8 warps per SM
    return (int)std::max<int64_t>(1, std::min(need, cap));
}

cudaError_t launch_q2_linearize(const Geom& g, const Phys& ph, const double* U, const double* pt, float* q32,
                                float2* q64, cudaStream_t s) {
    if (g.dim != 3 || g.deg != 2) return cudaErrorInvalidValue;
    k_q2_linearize<<<q2_grid(g.n_cells), 32 * kWarpsPerCta, 0, s>>>(g, make_q2_consts(g, ph), U, pt, q32, q64);
    return count_launch(cudaGetLastError());
}

template <typename S, typename St, typename QT>
static cudaError_t launch_q2(const Geom& g, const Phys& ph, const QT* qd, const St* x, St* y, const uint8_t* mask,
                             int phi_bits, bool blockdiag, cudaStream_t s) {
    if (g.dim != 3 || g.deg != 2) return cudaErrorInvalidValue;
    Q2ApplyArgs<S> a;
    a.g = g;
    a.qd = qd;
    a.x = x;
    a.y = y;
    a.mask = mask;
    a.phi_bits = phi_bits;
    a.k = make_q2_consts(g, ph);
    const int grid = q2_grid(g.n_cells);
    if (blockdiag) k_q2_apply<S, true><<<grid, 32 * kWarpsPerCta, 0, s>>>(a);
    else k_q2_apply<S, false><<<grid, 32 * kWarpsPerCta, 0, s>>>(a);
    return count_launch(cudaGetLastError());
}

cudaError_t launch_q2_apply64(const Geom& g, const Phys& ph, const float2* qd, const double* x, double* y,
                              const uint8_t* mask, int phi_bits, bool blockdiag, cudaStream_t s) {
    return launch_q2<df64>(g, ph, qd, x, y, mask, phi_bits, blockdiag, s);
}
cudaError_t launch_q2_apply32(const Geom& g, const Phys& ph, const float* qd, const float* x, float* y,
                              const uint8_t* mask, int phi_bits, bool blockdiag, cudaStream_t s) {
    return launch_q2<float>(g, ph, qd, x, y, mask, phi_bits, blockdiag, s);
}

}  // namespace pff
