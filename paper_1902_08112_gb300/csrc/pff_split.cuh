// Miehe split of the elastic energy (Sec. 2.1): E_s^+ = lambda/2 <tr e>_+^2 + mu tr(e_+^2) with
// e_+ = sum_a <l_a>_+ n_a n_a^T over the eigenpairs (l_a, n_a) of the strain, sigma^+ = dE_s^+/de =
// lambda <tr e>_+ I + 2 mu e_+, and the tangent dsigma^+/de.  The degraded part is g(phi) E_s^+, the
// rest E_s - E_s^+ is not degraded.  Strains are 3x3 (zero rows/columns beyond dim; plane strain in
// 2D).  <x>_+ = max(0, x); its derivative H(x) is taken as 0 at x = 0.
#pragma once

#include <cuda_runtime.h>

namespace pff {

template <typename T>
struct SplitEig {
    T l[3];        // eigenvalues
    T V[3][3];     // eigenvectors in columns
    T tr;          // tr(e)
};

template <typename T>
__device__ __forceinline__ T pos_part(T x) { return x > T(0) ? x : T(0); }
template <typename T>
__device__ __forceinline__ T heaviside(T x) { return x > T(0) ? T(1) : T(0); }

// Symmetric 3x3 eigen-decomposition by cyclic Jacobi rotations (Golub and Van Loan, Matrix
// Computations, Sec. 8.5), at most 12 sweeps (quadratic convergence: a 3x3 needs about 4).
template <typename T>
__device__ void split_eig3(const T e[3][3], SplitEig<T>& s) {
    T a[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            a[i][j] = e[i][j];
            s.V[i][j] = i == j ? T(1) : T(0);
        }
    for (int sweep = 0; sweep < 12; ++sweep) {
        const T off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
        const T dia = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
        if (off == T(0) || off <= T(1e-36) * dia) break;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const int p = r == 2 ? 1 : 0, q = r == 0 ? 1 : 2;   // (0,1), (0,2), (1,2)
            if (a[p][q] == T(0)) continue;
            const T theta = (a[q][q] - a[p][p]) / (T(2) * a[p][q]);
            const T t = (theta >= T(0) ? T(1) : T(-1)) / (fabs(theta) + sqrt(theta * theta + T(1)));
            const T c = T(1) / sqrt(t * t + T(1)), sn = t * c;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const T akp = a[k][p], akq = a[k][q];
                a[k][p] = c * akp - sn * akq;
                a[k][q] = sn * akp + c * akq;
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const T apk = a[p][k], aqk = a[q][k];
                a[p][k] = c * apk - sn * aqk;
                a[q][k] = sn * apk + c * aqk;
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const T vkp = s.V[k][p], vkq = s.V[k][q];
                s.V[k][p] = c * vkp - sn * vkq;
                s.V[k][q] = sn * vkp + c * vkq;
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) s.l[i] = a[i][i];
}

// sigma^+ (3x3) and E_s^+ at the strain e; fills the eigen data for split_tangent.
template <typename T>
__device__ void split_stress(T mu, T lam, int dim, const T e[3][3], T sp[3][3], T& Esp, SplitEig<T>& s) {
    split_eig3(e, s);
    s.tr = T(0);
    for (int i = 0; i < dim; ++i) s.tr += e[i][i];
    const T trp = pos_part(s.tr);
    T ep2 = T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) ep2 += pos_part(s.l[k]) * pos_part(s.l[k]);
    Esp = T(0.5) * lam * trp * trp + mu * ep2;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            T v = T(0);
#pragma unroll
            for (int k = 0; k < 3; ++k) v += pos_part(s.l[k]) * s.V[i][k] * s.V[j][k];
            sp[i][j] = (i < dim && j < dim) ? T(2) * mu * v + (i == j ? lam * trp : T(0)) : T(0);
        }
}

// C^+ de = lambda H(tr e) tr(de) I + 2 mu sum_{a,b} theta_ab (n_a . de n_b) n_a n_b^T with
// theta_aa = H(l_a) and theta_ab = (<l_a>_+ - <l_b>_+) / (l_a - l_b) (H(l_a) when l_a = l_b): the
// derivative of the isotropic function e -> e_+.
template <typename T>
__device__ void split_tangent(T mu, T lam, int dim, const SplitEig<T>& s, const T de[3][3], T out[3][3]) {
    T dtr = T(0);
    for (int i = 0; i < dim; ++i) dtr += de[i][i];
    // de in the eigenbasis: D = V^T de V
    T D[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            T v = T(0);
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) v += s.V[i][a] * de[i][j] * s.V[j][b];
            T th;
            if (a == b || s.l[a] == s.l[b]) th = heaviside(s.l[a]);
            else th = (pos_part(s.l[a]) - pos_part(s.l[b])) / (s.l[a] - s.l[b]);
            D[a][b] = th * v;
        }
    const T vol = lam * heaviside(s.tr) * dtr;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            T v = T(0);
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) v += s.V[i][a] * D[a][b] * s.V[j][b];
            out[i][j] = (i < dim && j < dim) ? T(2) * mu * v + (i == j ? vol : T(0)) : T(0);
        }
}

}  // namespace pff
