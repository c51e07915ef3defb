// Q1 fast path: linearisation data and modal applies (see pff_q1.cu).
#pragma once

#include "pff_internal.cuh"

namespace pff {

// St: element type of x/y in global memory (float or double); QT: element type of the stored
// Gauss-point coefficients (float for the FP32 operator, float2 = df64 pair for FP64).
template <typename St, typename QT>
struct Q1ApplyArgs {
    Geom g;
    const QT* qd;            // [(q * NK + k) * n_cells + cell]
    const St* x;
    St* y;
    const uint8_t* mask;
    int phi_bits;
    double cv[4];            // g^j / 2^d
    double cg[3][3];         // g^j * 2 / (h_d 2^d)
    double mu, lam, gcew;    // Lame coefficients, Gc eps w
};

// number of stored coefficients per Gauss point and cell (c0, Sp, c1)
inline int q1_nk(int dim) { return dim == 3 ? 8 : 5; }

cudaError_t launch_q1_linearize(const Geom& g, const Phys& ph, const double* U, const double* pt, float* q32,
                                float2* q64, cudaStream_t s);
cudaError_t launch_q1_apply64(const Geom& g, const Phys& ph, const float2* qd, const double* x, double* y,
                              const uint8_t* mask, int phi_bits, bool blockdiag, cudaStream_t s);
cudaError_t launch_q1_apply32(const Geom& g, const Phys& ph, const float* qd, const float* x, float* y,
                              const uint8_t* mask, int phi_bits, bool blockdiag, cudaStream_t s);

}  // namespace pff
