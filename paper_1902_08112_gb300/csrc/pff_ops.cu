// Matrix-free cell operators on uniform Q1/Q2 levels (Sec. 4.1 and 4.2 of the paper):
//   OP_APPLY            y = G~_l(U_l) x        (Jacobian of Eq. (semilinear), phi~ frozen)
//   OP_APPLY_BLOCKDIAG  y = blockdiag(G_uu, G_phiphi) x   (operator of the smoother blocks)
//   OP_RESIDUAL         y = -A(U)              (residual of Eq. (semilinear))
//   OP_DIAGONAL         y = diag(G~_l)         (Jacobi diagonal, remark in Sec. 4.1)
//
// Work layout: one CTA owns a tile of cells; the nodal values of x, U and phi~ of the tile
// (with the shared boundary layer) are staged in shared memory, one thread evaluates one
// cell at all (deg+1)^d Gauss points and writes its element vector to shared memory; then
// each tile node sums the contributions of the tile's cells around it in a fixed order and
// adds the sum to the global output (nodes on tile borders receive one add per tile).
// Eliminated columns are zeroed while staging; eliminated rows are preset by
// launch_init_masked (y = x for the apply, 1 for the diagonal) and skipped here.
#include "pff_internal.cuh"
#include "pff_split.cuh"

namespace pff {

template <int DIM, int DEG>
struct TileCfg;
template <>
struct TileCfg<2, 1> { static constexpr int TX = 16, TY = 16, TZ = 1; };
template <>
struct TileCfg<2, 2> { static constexpr int TX = 8, TY = 8, TZ = 1; };
template <>
struct TileCfg<3, 1> { static constexpr int TX = 8, TY = 8, TZ = 4; };
template <>
struct TileCfg<3, 2> { static constexpr int TX = 4, TY = 4, TZ = 4; };

constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

__device__ __forceinline__ bool eliminated(uint8_t m, int c, int dim, int u_bits, int phi_bits) {
    return c < dim ? (((m & u_bits) >> c) & 1) != 0 : (m & phi_bits) != 0;
}

template <int DIM, int DEG, typename T, int OP>
struct CellKernel {
    using C = TileCfg<DIM, DEG>;
    static constexpr int P = DEG + 1;
    static constexpr int NPC = ipow(P, DIM);
    static constexpr int NQ = NPC;
    static constexpr int NC = DIM + 1;
    static constexpr int NCELL = C::TX * C::TY * C::TZ;
    static constexpr int NTX = C::TX * DEG + 1;
    static constexpr int NTY = C::TY * DEG + 1;
    static constexpr int NTZ = DIM == 3 ? C::TZ * DEG + 1 : 1;
    static constexpr int NT = NTX * NTY * NTZ;
    static constexpr bool NEED_X = (OP == OP_APPLY || OP == OP_APPLY_BLOCKDIAG);
    static constexpr int NOUT = NPC * NC;
    static constexpr size_t smem_bytes() {
        return sizeof(T) * ((size_t)(NC + 1) * NT + (NEED_X ? (size_t)NC * NT : 0) + (size_t)NOUT * NCELL);
    }
};

template <int DIM, int DEG, typename T, int OP, bool SPLIT>
__global__ void __launch_bounds__(TileCfg<DIM, DEG>::TX * TileCfg<DIM, DEG>::TY * TileCfg<DIM, DEG>::TZ)
k_cell(CellArgs<T> a) {
    using K = CellKernel<DIM, DEG, T, OP>;
    using C = typename K::C;
    constexpr int P = K::P, NPC = K::NPC, NQ = K::NQ, NC = K::NC, NCELL = K::NCELL;
    constexpr int NTX = K::NTX, NTY = K::NTY, NT = K::NT;
    constexpr bool NEED_X = K::NEED_X;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sU = reinterpret_cast<T*>(smem_raw);      // [NC][NT]
    T* spt = sU + NC * NT;                        // [NT]
    T* sx = spt + NT;                             // [NC][NT] (apply only)
    T* sel = sx + (NEED_X ? NC * NT : 0);         // [NOUT][NCELL]

    const Geom& g = a.g;
    const int ci0 = blockIdx.x * C::TX, cj0 = blockIdx.y * C::TY, ck0 = (DIM == 3) ? blockIdx.z * C::TZ : 0;
    const int ni0 = ci0 * DEG, nj0 = cj0 * DEG, nk0 = ck0 * DEG;
    const int64_t nn = g.n_nodes;

    // ---- stage the tile's nodal data
    for (int t = threadIdx.x; t < NT; t += blockDim.x) {
        const int ti = t % NTX, tj = (t / NTX) % NTY, tk = t / (NTX * NTY);
        const int gi = ni0 + ti, gj = nj0 + tj, gk = nk0 + tk;
        const bool in = gi < g.nn[0] && gj < g.nn[1] && gk < g.nn[2];
        const int64_t gn = in ? (int64_t)gi + (int64_t)g.nn[0] * ((int64_t)gj + (int64_t)g.nn[1] * gk) : 0;
#pragma unroll
        for (int c = 0; c < NC; ++c) sU[c * NT + t] = in ? a.U[c * nn + gn] : T(0);
        spt[t] = in ? a.pt[gn] : T(0);
        if constexpr (NEED_X) {
            const uint8_t m = in ? a.mask[gn] : 0;
#pragma unroll
            for (int c = 0; c < NC; ++c)
                sx[c * NT + t] = (in && !eliminated(m, c, DIM, a.u_bits, a.phi_bits)) ? a.x[c * nn + gn] : T(0);
        }
    }
    for (int k = threadIdx.x; k < K::NOUT * NCELL; k += blockDim.x) sel[k] = T(0);
    __syncthreads();

    // ---- one thread per cell
    const int cell = threadIdx.x;
    if (cell < NCELL) {
        const int li = cell % C::TX, lj = (cell / C::TX) % C::TY, lk = cell / (C::TX * C::TY);
        const bool valid = (ci0 + li < g.nc[0]) && (cj0 + lj < g.nc[1]) && (DIM == 2 || ck0 + lk < g.nc[2]) &&
                           cell_in(g, (int64_t)(ci0 + li) + (int64_t)g.nc[0] * ((int64_t)(cj0 + lj) + (int64_t)g.nc[1] * (ck0 + lk)));
        if (valid) {
            const double sE = g.es ? g.es[(int64_t)(ci0 + li) + (int64_t)g.nc[0] * ((int64_t)(cj0 + lj) +
                                                    (int64_t)g.nc[1] * (ck0 + lk))] : 1.0;
            const T mu = T(a.ph.mu * sE), lam = T(a.ph.lam * sE), kap = T(a.ph.kappa), p = T(a.ph.p);
            const T Gc = T(a.ph.Gc), eps = T(a.ph.eps), ff = T(a.ph.f);
            const T one = T(1), two = T(2), half = T(0.5);
            T ih[3], vol = T(1);
#pragma unroll
            for (int d = 0; d < 3; ++d) ih[d] = T(1.0 / g.h[d]);
#pragma unroll
            for (int d = 0; d < DIM; ++d) vol *= T(g.h[d]);
            const int tbase = (DEG * li) + NTX * ((DEG * lj) + NTY * (DIM == 3 ? DEG * lk : 0));

#pragma unroll 1
            for (int q = 0; q < NQ; ++q) {
                const int qa[3] = {q % P, (q / P) % P, DIM == 3 ? q / (P * P) : 0};
                T wq = vol;
#pragma unroll
                for (int d = 0; d < DIM; ++d) wq *= T(a.tb.w1[qa[d]]);
                T Nv[3][P], Nd[3][P];
#pragma unroll
                for (int d = 0; d < 3; ++d)
#pragma unroll
                    for (int s = 0; s < P; ++s) {
                        Nv[d][s] = d < DIM ? T(a.tb.N1[s][qa[d]]) : T(1);
                        Nd[d][s] = d < DIM ? T(a.tb.D1[s][qa[d]]) * ih[d] : T(0);
                    }
                // ---- values at the quadrature point
                T gu[DIM][DIM], phi = 0, gphi[DIM], ptv = 0;
                T gdu[DIM][DIM], dphi = 0, gdphi[DIM];
#pragma unroll
                for (int i = 0; i < DIM; ++i) {
                    gphi[i] = 0;
                    gdphi[i] = 0;
#pragma unroll
                    for (int j = 0; j < DIM; ++j) { gu[i][j] = 0; gdu[i][j] = 0; }
                }
#pragma unroll
                for (int n = 0; n < NPC; ++n) {
                    const int na = n % P, nb = (n / P) % P, nc_ = DIM == 3 ? n / (P * P) : 0;
                    const T N = Nv[0][na] * Nv[1][nb] * Nv[2][nc_];
                    T G[DIM];
                    G[0] = Nd[0][na] * Nv[1][nb] * Nv[2][nc_];
                    G[1] = Nv[0][na] * Nd[1][nb] * Nv[2][nc_];
                    if constexpr (DIM == 3) G[2] = Nv[0][na] * Nv[1][nb] * Nd[2][nc_];
                    const int t = tbase + na + NTX * (nb + NTY * nc_);
#pragma unroll
                    for (int c = 0; c < DIM; ++c) {
                        const T uc = sU[c * NT + t];
#pragma unroll
                        for (int j = 0; j < DIM; ++j) gu[c][j] += uc * G[j];
                        if constexpr (NEED_X) {
                            const T xc = sx[c * NT + t];
#pragma unroll
                            for (int j = 0; j < DIM; ++j) gdu[c][j] += xc * G[j];
                        }
                    }
                    const T ph_n = sU[DIM * NT + t];
                    phi += ph_n * N;
                    if constexpr (OP == OP_RESIDUAL) {
#pragma unroll
                        for (int j = 0; j < DIM; ++j) gphi[j] += ph_n * G[j];
                    }
                    ptv += spt[t] * N;
                    if constexpr (NEED_X) {
                        const T xp = sx[DIM * NT + t];
                        dphi += xp * N;
#pragma unroll
                        for (int j = 0; j < DIM; ++j) gdphi[j] += xp * G[j];
                    }
                }
                // ---- linearisation point: strain, stress, elastic energy (Sec. 2.1)
                T eu[DIM][DIM], tru = 0;
#pragma unroll
                for (int i = 0; i < DIM; ++i)
#pragma unroll
                    for (int j = 0; j < DIM; ++j) eu[i][j] = half * (gu[i][j] + gu[j][i]);
#pragma unroll
                for (int i = 0; i < DIM; ++i) tru += eu[i][i];
                T ee = 0;
#pragma unroll
                for (int i = 0; i < DIM; ++i)
#pragma unroll
                    for (int j = 0; j < DIM; ++j) ee += eu[i][j] * eu[i][j];
                const T Es = half * lam * tru * tru + mu * ee;
                const T gt = (one - kap) * ptv * ptv + kap;   // g_kappa(phi~)
                // Miehe split (Sec. 2.1): sigma^+(u), E_s^+ and the eigen data of the tangent
                T sp3[3][3], Esp = Es;
                SplitEig<T> se;
                if constexpr (SPLIT) {
                    T e3[3][3];
#pragma unroll
                    for (int i = 0; i < 3; ++i)
#pragma unroll
                        for (int j = 0; j < 3; ++j) e3[i][j] = (i < DIM && j < DIM) ? eu[i][j] : T(0);
                    split_stress(mu, lam, DIM, e3, sp3, Esp, se);
                }

                // ---- pointwise coefficients of the test functions: fu (tensor on grad w),
                //      fphi (on psi), fgphi (on grad psi)
                T fu[DIM][DIM], fphi, fgphi[DIM];
                if constexpr (NEED_X) {
                    T ed[DIM][DIM], trd = 0;
#pragma unroll
                    for (int i = 0; i < DIM; ++i)
#pragma unroll
                        for (int j = 0; j < DIM; ++j) ed[i][j] = half * (gdu[i][j] + gdu[j][i]);
#pragma unroll
                    for (int i = 0; i < DIM; ++i) trd += ed[i][i];
                    // G_uu: g(phi~) sigma(du) : e(w); with the split g C^+ de + (C - C^+) de
                    T cpd[3][3];
                    if constexpr (SPLIT) {
                        T d3[3][3];
#pragma unroll
                        for (int i = 0; i < 3; ++i)
#pragma unroll
                            for (int j = 0; j < 3; ++j) d3[i][j] = (i < DIM && j < DIM) ? ed[i][j] : T(0);
                        split_tangent(mu, lam, DIM, se, d3, cpd);
                    }
#pragma unroll
                    for (int i = 0; i < DIM; ++i)
#pragma unroll
                        for (int j = 0; j < DIM; ++j) {
                            const T sd = two * mu * ed[i][j] + (i == j ? lam * trd : T(0));
                            if constexpr (SPLIT) fu[i][j] = wq * (sd - (one - gt) * cpd[i][j]);
                            else fu[i][j] = wq * gt * sd;
                        }
                    // G_phiphi: [2 f (1-k) E_s^+ + 2 p div u + Gc/eps] dphi psi + Gc eps grad dphi . grad psi
                    fphi = (two * ff * (one - kap) * Esp + two * p * tru + Gc / eps) * dphi;
                    if constexpr (OP == OP_APPLY) {
                        // G_phiu: 2 f (1-k) phi sigma^+(u):e(du) + 2 p phi div du
                        T su_ed = 0;
#pragma unroll
                        for (int i = 0; i < DIM; ++i)
#pragma unroll
                            for (int j = 0; j < DIM; ++j) {
                                const T sij = SPLIT ? sp3[i][j] : two * mu * eu[i][j] + (i == j ? lam * tru : T(0));
                                su_ed += sij * ed[i][j];
                            }
                        fphi += two * ff * (one - kap) * phi * su_ed + two * p * phi * trd;
                    }
                    fphi *= wq;
#pragma unroll
                    for (int j = 0; j < DIM; ++j) fgphi[j] = wq * Gc * eps * gdphi[j];
                } else if constexpr (OP == OP_RESIDUAL) {
                    // -A(U): u-rows g(phi~) sigma(u) + phi~^2 p I; phi-rows f g'(phi) E_s + 2 phi p div u
                    //        - Gc/eps (1 - phi); grad part Gc eps grad phi
#pragma unroll
                    for (int i = 0; i < DIM; ++i)
#pragma unroll
                        for (int j = 0; j < DIM; ++j) {
                            const T sij = two * mu * eu[i][j] + (i == j ? lam * tru : T(0));
                            // g(phi~) sigma^+ + sigma^- = sigma - (1 - g) sigma^+
                            const T seff = SPLIT ? sij - (one - gt) * sp3[i][j] : gt * sij;
                            fu[i][j] = -wq * (seff + (i == j ? ptv * ptv * p : T(0)));
                        }
                    fphi = -wq * (ff * two * (one - kap) * phi * Esp + two * phi * p * tru - Gc / eps * (one - phi));
#pragma unroll
                    for (int j = 0; j < DIM; ++j) fgphi[j] = -wq * Gc * eps * gphi[j];
                } else {
                    // diagonal: coefficients reused below
                    fphi = wq * (two * ff * (one - kap) * Esp + two * p * tru + Gc / eps);
#pragma unroll
                    for (int j = 0; j < DIM; ++j) fgphi[j] = wq * Gc * eps;
#pragma unroll
                    for (int i = 0; i < DIM; ++i)
#pragma unroll
                        for (int j = 0; j < DIM; ++j) fu[i][j] = wq * gt;
                }

                // ---- integrate against the test functions of the cell
#pragma unroll
                for (int n = 0; n < NPC; ++n) {
                    const int na = n % P, nb = (n / P) % P, nc_ = DIM == 3 ? n / (P * P) : 0;
                    const T N = Nv[0][na] * Nv[1][nb] * Nv[2][nc_];
                    T G[DIM];
                    G[0] = Nd[0][na] * Nv[1][nb] * Nv[2][nc_];
                    G[1] = Nv[0][na] * Nd[1][nb] * Nv[2][nc_];
                    if constexpr (DIM == 3) G[2] = Nv[0][na] * Nv[1][nb] * Nd[2][nc_];
                    if constexpr (OP == OP_DIAGONAL) {
                        T gg = 0;
#pragma unroll
                        for (int j = 0; j < DIM; ++j) gg += G[j] * G[j];
#pragma unroll
                        for (int c = 0; c < DIM; ++c) {
                            if constexpr (SPLIT) {
                                // de = sym(e_c (x) grad N): sigma(de) : de - (1 - g) C^+ de : de
                                T d3[3][3], cp3[3][3];
#pragma unroll
                                for (int i = 0; i < 3; ++i)
#pragma unroll
                                    for (int j = 0; j < 3; ++j) {
                                        T v = T(0);
                                        if (i == c && j < DIM) v += half * G[j];
                                        if (j == c && i < DIM) v += half * G[i];
                                        d3[i][j] = v;
                                    }
                                split_tangent(mu, lam, DIM, se, d3, cp3);
                                T cpdd = 0;
#pragma unroll
                                for (int i = 0; i < DIM; ++i)
#pragma unroll
                                    for (int j = 0; j < DIM; ++j) cpdd += cp3[i][j] * d3[i][j];
                                const T full = mu * (gg + G[c] * G[c]) + lam * G[c] * G[c];
                                sel[(n * NC + c) * NCELL + cell] += wq * (full - (one - gt) * cpdd);
                            } else {
                                sel[(n * NC + c) * NCELL + cell] += fu[0][0] * (mu * (gg + G[c] * G[c]) + lam * G[c] * G[c]);
                            }
                        }
                        sel[(n * NC + DIM) * NCELL + cell] += fphi * N * N + fgphi[0] * gg;
                    } else {
#pragma unroll
                        for (int c = 0; c < DIM; ++c) {
                            T s = 0;
#pragma unroll
                            for (int j = 0; j < DIM; ++j) s += fu[c][j] * G[j];
                            sel[(n * NC + c) * NCELL + cell] += s;
                        }
                        T s = fphi * N;
#pragma unroll
                        for (int j = 0; j < DIM; ++j) s += fgphi[j] * G[j];
                        sel[(n * NC + DIM) * NCELL + cell] += s;
                    }
                }
            }
        }
    }
    __syncthreads();

    // ---- node gather: fixed order over the tile's cells around each node, one global add
    const int NTZ = K::NTZ;
    for (int t = threadIdx.x; t < NT; t += blockDim.x) {
        const int ti = t % NTX, tj = (t / NTX) % NTY, tk = t / (NTX * NTY);
        const int gi = ni0 + ti, gj = nj0 + tj, gk = nk0 + tk;
        if (!(gi < g.nn[0] && gj < g.nn[1] && gk < g.nn[2])) continue;
        const int64_t gn = (int64_t)gi + (int64_t)g.nn[0] * ((int64_t)gj + (int64_t)g.nn[1] * gk);
        const uint8_t m = (OP == OP_RESIDUAL) ? 0 : a.mask[gn];
        // cells ci of the tile with DEG*ci <= ti <= DEG*ci + DEG
        const int lo_i = max(0, ti / DEG - 1), hi_i = min(C::TX - 1, ti / DEG);
        const int lo_j = max(0, tj / DEG - 1), hi_j = min(C::TY - 1, tj / DEG);
        const int lo_k = DIM == 3 ? max(0, tk / DEG - 1) : 0;
        const int hi_k = DIM == 3 ? min(C::TZ - 1, tk / DEG) : 0;
        (void)NTZ;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            if (OP != OP_RESIDUAL && eliminated(m, c, DIM, a.u_bits, a.phi_bits)) continue;
            T s = 0;
            for (int ck = lo_k; ck <= hi_k; ++ck) {
                const int oc = DIM == 3 ? tk - DEG * ck : 0;
                if (oc < 0 || oc > DEG) continue;
                for (int cj = lo_j; cj <= hi_j; ++cj) {
                    const int ob = tj - DEG * cj;
                    if (ob < 0 || ob > DEG) continue;
                    for (int ci = lo_i; ci <= hi_i; ++ci) {
                        const int oa = ti - DEG * ci;
                        if (oa < 0 || oa > DEG) continue;
                        const int n = oa + P * (ob + P * oc);
                        const int cidx = ci + C::TX * (cj + C::TY * ck);
                        s += sel[(n * NC + c) * NCELL + cidx];
                    }
                }
            }
            atomicAdd(&a.y[c * nn + gn], s);
        }
    }
}

template <int DIM, int DEG, typename T, int OP, bool SPLIT>
static cudaError_t launch_one(const CellArgs<T>& a, cudaStream_t s) {
    using K = CellKernel<DIM, DEG, T, OP>;
    using C = typename K::C;
    const size_t smem = K::smem_bytes();
    static bool attr_set = false;  // per instantiation; the attribute is per device function
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_cell<DIM, DEG, T, OP, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    dim3 grid((a.g.nc[0] + C::TX - 1) / C::TX, (a.g.nc[1] + C::TY - 1) / C::TY,
              DIM == 3 ? (a.g.nc[2] + C::TZ - 1) / C::TZ : 1);
    k_cell<DIM, DEG, T, OP, SPLIT><<<grid, K::NCELL, smem, s>>>(a);
    return count_launch(cudaGetLastError());
}

template <int DIM, int DEG, typename T>
static cudaError_t dispatch_op(int op, const CellArgs<T>& a, cudaStream_t s) {
    if (a.ph.split) {
        switch (op) {
            case OP_APPLY: return launch_one<DIM, DEG, T, OP_APPLY, true>(a, s);
            case OP_APPLY_BLOCKDIAG: return launch_one<DIM, DEG, T, OP_APPLY_BLOCKDIAG, true>(a, s);
            case OP_RESIDUAL: return launch_one<DIM, DEG, T, OP_RESIDUAL, true>(a, s);
            case OP_DIAGONAL: return launch_one<DIM, DEG, T, OP_DIAGONAL, true>(a, s);
        }
        return cudaErrorInvalidValue;
    }
    switch (op) {
        case OP_APPLY: return launch_one<DIM, DEG, T, OP_APPLY, false>(a, s);
        case OP_APPLY_BLOCKDIAG: return launch_one<DIM, DEG, T, OP_APPLY_BLOCKDIAG, false>(a, s);
        case OP_RESIDUAL: return launch_one<DIM, DEG, T, OP_RESIDUAL, false>(a, s);
        case OP_DIAGONAL: return launch_one<DIM, DEG, T, OP_DIAGONAL, false>(a, s);
    }
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_cell_op(int op, const CellArgs<T>& a, cudaStream_t s) {
    if (a.g.n_cells == 0) return cudaSuccess;
    if (a.g.dim == 2 && a.g.deg == 1) return dispatch_op<2, 1, T>(op, a, s);
    if (a.g.dim == 2 && a.g.deg == 2) return dispatch_op<2, 2, T>(op, a, s);
    if (a.g.dim == 3 && a.g.deg == 1) return dispatch_op<3, 1, T>(op, a, s);
    if (a.g.dim == 3 && a.g.deg == 2) return dispatch_op<3, 2, T>(op, a, s);
    return cudaErrorInvalidValue;
}

template cudaError_t launch_cell_op<double>(int, const CellArgs<double>&, cudaStream_t);
template cudaError_t launch_cell_op<float>(int, const CellArgs<float>&, cudaStream_t);

// ---------------------------------------------------------------- row presets
template <typename T>
__global__ void k_init_masked(int64_t nn, int dim, const uint8_t* __restrict__ mask, int u_bits,
                              int phi_bits, const T* __restrict__ x, T* __restrict__ y, T elim_val) {
    const int64_t nd = nn * (dim + 1);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nd; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = dof_comp(i, nn);
        const uint8_t m = mask[i - c * nn];
        const bool e = c < dim ? (((m & u_bits) >> c) & 1) != 0 : (m & phi_bits) != 0;
        y[i] = e ? (x ? x[i] : elim_val) : T(0);
    }
}

static int grid_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b > 152 * 32) b = 152 * 32;
    if (b < 1) b = 1;
    return (int)b;
}

template <typename T>
cudaError_t launch_init_masked(const Geom& g, const uint8_t* mask, int u_bits, int phi_bits, const T* x,
                               T* y, T elim_val, cudaStream_t s) {
    const int64_t nd = n_dofs(g);
    k_init_masked<T><<<grid_for(nd, 256), 256, 0, s>>>(g.n_nodes, g.dim, mask, u_bits, phi_bits, x, y, elim_val);
    return count_launch(cudaGetLastError());
}

// The same preset on the nodes [node0, node1) only (all components), FP64.
__global__ void k_init_masked_nodes(int64_t nn, int dim, int64_t node0, int64_t node1, const uint8_t* __restrict__ mask,
                                    int u_bits, int phi_bits, const double* __restrict__ x, double* __restrict__ y) {
    const int64_t cnt = node1 - node0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt * (dim + 1);
         t += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(t / cnt);
        const int64_t n = node0 + (t - (int64_t)c * cnt), i = (int64_t)c * nn + n;
        const uint8_t m = mask[n];
        const bool e = c < dim ? (((m & u_bits) >> c) & 1) != 0 : (m & phi_bits) != 0;
        y[i] = e ? x[i] : 0.0;
    }
}
cudaError_t launch_init_masked_nodes(const Geom& g, const uint8_t* mask, int u_bits, int phi_bits, const double* x,
                                     double* y, int64_t node0, int64_t node1, cudaStream_t s) {
    if (node1 <= node0) return cudaSuccess;
    const int64_t nd = (node1 - node0) * (g.dim + 1);
    k_init_masked_nodes<<<grid_for(nd, 256), 256, 0, s>>>(g.n_nodes, g.dim, node0, node1, mask, u_bits, phi_bits,
                                                          x, y);
    return count_launch(cudaGetLastError());
}

template cudaError_t launch_init_masked<double>(const Geom&, const uint8_t*, int, int, const double*, double*,
                                                double, cudaStream_t);
template cudaError_t launch_init_masked<float>(const Geom&, const uint8_t*, int, int, const float*, float*,
                                               float, cudaStream_t);

}  // namespace pff
