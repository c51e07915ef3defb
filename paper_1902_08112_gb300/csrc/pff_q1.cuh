// Q1 fast path: linearisation data and modal applies (see pff_q1.cu).
#pragma once

#include "pff_internal.cuh"

namespace pff {

// Constants of the Q1 applies as (hi, lo) float pairs prepared on the host: the kernels use .x in
// FP32 and (x, y) as a double-float, so no FP64 instruction runs in the applies.
struct Q1Consts {
    float2 cv[4];            // g^j / 2^d
    float2 cg[3][3];         // g^j * 2 / (h_d 2^d)
    float2 mu, mu2, lam;     // Lame coefficients, 2 mu
    float2 gcew;             // Gc eps w (w = Gauss weight x |K|)
    float2 gk[8];            // 2^d Gc eps w sum_{d in k} cg[d][|k|-1]^2: the phi gradient-gradient term
                             // of modal coefficient k
    float2 g2;               // g / 2
    float2 al, be;           // (1 + g) / 2, (1 - g) / 2
    float2 ih[3];            // 1 / h_d
};
Q1Consts make_q1_consts(const Geom& g, const Phys& ph);

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
    Q1Consts k;
    int tz0 = 0;             // k_q1_apply_cell: first tile along z, and the end of the cell layers
    int kz_end = 1 << 30;    // applied (a slab of the level); the whole level by default
};

// number of stored coefficients per Gauss point and cell (c0, Sp, c1)
inline int q1_nk(int dim) { return dim == 3 ? 8 : 5; }

cudaError_t launch_q1_linearize(const Geom& g, const Phys& ph, const double* U, const double* pt, float* q32,
                                float2* q64, cudaStream_t s);
// lanes = true: one thread per (cell, Gauss point) with shuffle butterflies; false: one thread
// per cell with the modal form in registers
// The FP64-accurate per-cell apply on the cell layers [kz0, kz1) of a 3D level (kz0 a multiple
// of q1_cell_tile_z()), adding to y without presetting it.
int q1_cell_tile_z();
cudaError_t launch_q1_apply64_slab(const Geom& g, const Phys& ph, const float2* qd, const double* x, double* y,
                                   const uint8_t* mask, int phi_bits, int kz0, int kz1, cudaStream_t s);
// cell = true (3D): one thread per cell in df64 with shared-memory Gauss-point derivatives
cudaError_t launch_q1_apply64(const Geom& g, const Phys& ph, const float2* qd, const double* x, double* y,
                              const uint8_t* mask, int phi_bits, bool blockdiag, bool lanes, cudaStream_t s,
                              bool direct = false, bool cell = false);
cudaError_t launch_q1_apply32(const Geom& g, const Phys& ph, const float* qd, const float* x, float* y,
                              const uint8_t* mask, int phi_bits, bool blockdiag, bool lanes, cudaStream_t s,
                              bool direct = false, bool cell = false);

// -A(U) on a Q1 level (R zeroed by the caller) and diag(G~) on free rows (eliminated rows preset)
cudaError_t launch_q1_residual(const Geom& g, const Phys& ph, const double* U, const double* pt, double* R,
                               cudaStream_t s);
cudaError_t launch_q1_diagonal(const Geom& g, const Phys& ph, const float2* q64, const uint8_t* mask, double* d,
                               cudaStream_t s);

// bulk and crack energies of Sec. 5 at the state U (out[0] bulk, out[1] crack, device); part holds
// 2 * 304 partial sums
cudaError_t launch_q1_energies(const Geom& g, const Phys& ph, const double* U, double* part, double* out,
                               cudaStream_t s);

// Miehe split: Gauss-point tangent data (NKS coefficients per Gauss point) and the applies that use it
cudaError_t launch_q1_linearize_split(const Geom& g, const Phys& ph, const double* U, const double* pt, float* q32,
                                      float2* q64, cudaStream_t s);
cudaError_t launch_q1_apply_split64(const Geom& g, const Phys& ph, const float2* qd, const double* x, double* y,
                                    const uint8_t* mask, int phi_bits, bool blockdiag, cudaStream_t s);
cudaError_t launch_q1_apply_split32(const Geom& g, const Phys& ph, const float* qd, const float* x, float* y,
                                    const uint8_t* mask, int phi_bits, bool blockdiag, cudaStream_t s);
inline int q1_nks(int dim) { return dim == 3 ? 28 : 10; }

// Q2 fast path on 3D levels (pff_q2.cu): Gauss-point linearisation data (8 coefficients x 27 points per
// cell, [(cell * 8 + k) * 27 + q]) and the warp-per-cell sum-factorised applies (eliminated rows of y
// preset by the caller).  Miehe split and 2D Q2 use the generic kernels.
inline size_t q2_data_size(const Geom& g) { return (size_t)8 * 27 * (size_t)g.n_cells; }
cudaError_t launch_q2_linearize(const Geom& g, const Phys& ph, const double* U, const double* pt, float* q32,
                                float2* q64, cudaStream_t s);
cudaError_t launch_q2_apply64(const Geom& g, const Phys& ph, const float2* qd, const double* x, double* y,
                              const uint8_t* mask, int phi_bits, bool blockdiag, cudaStream_t s);
cudaError_t launch_q2_apply32(const Geom& g, const Phys& ph, const float* qd, const float* x, float* y,
                              const uint8_t* mask, int phi_bits, bool blockdiag, cudaStream_t s);

}  // namespace pff
