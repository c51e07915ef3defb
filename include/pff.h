/*
 * pff.h -- C ABI of the GB300 matrix-free multigrid solver for pressurised phase-field
 * fracture (Jodlbauer, Langer, Wick: "Matrix-free multigrid solvers for phase-field fracture
 * problems", arXiv 1902.08112).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Vectors are DEVICE pointers on the GPU the hierarchy was created on, caller-owned,
 *    contiguous, in the component-blocked layout [u_x | u_y | (u_z) | phi]: entry
 *    (comp, node) sits at comp * n_nodes + node, nodes lexicographic with x fastest.  The
 *    number of components is dim + 1.  FP64 vectors are double*, FP32 vectors float*.
 *  - Levels are numbered 0 (coarsest) .. n_levels-1 (finest); level -1 means the finest.
 *  - Every call is stream-ordered on the stream given at creation and asynchronous, except
 *    the calls that fill a host-side info/out struct, which synchronise that stream.
 *  - Errors are returned as pff_status; no exception, abort or device trap crosses the ABI.
 *    pff_last_error() gives a one-line description of the last failure of a hierarchy.
 *  - Node mask bits (uint8 per node): PFF_MASK_UX/UY/UZ = displacement component clamped
 *    (Dirichlet), PFF_MASK_ACTIVE = phase field in the active set, PFF_MASK_PHI_DIR = phase
 *    field clamped.  A masked (eliminated) DoF has an identity row and a zero column in every
 *    operator (Algorithm 1, step 4).
 *  - The library owns its level data, masks, preconditioner data and Krylov workspace; they
 *    are allocated once in pff_create_hierarchy and freed by pff_destroy_hierarchy.
 */
#ifndef PFF_H
#define PFF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pff_hierarchy pff_hierarchy;

typedef enum {
    PFF_OK = 0,
    PFF_EINVAL = 1,      /* bad argument (sizes, level, null pointer, unsupported option) */
    PFF_ENOMEM = 2,      /* device or host allocation failed */
    PFF_ECUDA = 3,       /* a CUDA runtime call failed */
    PFF_ENOCONV = 4,     /* iteration cap reached before the tolerance */
    PFF_ENONFINITE = 5,  /* NaN/Inf found in a residual norm or Arnoldi norm */
    PFF_ETIMEOUT = 6,    /* a bounded device-side wait ran out */
    PFF_ESTATE = 7       /* call out of order (e.g. apply before pff_set_state) */
} pff_status;

enum {
    PFF_MASK_UX = 1,
    PFF_MASK_UY = 2,
    PFF_MASK_UZ = 4,
    PFF_MASK_ACTIVE = 8,
    PFF_MASK_PHI_DIR = 16
};

/* Mesh: a uniform box [lo, hi] with n_cells[a] hexahedra (dim 3) or quadrilaterals (dim 2)
 * per axis, Q1 or Q2 Lagrange elements for u and phi (Sec. 2.4; Q2 is an extension), and a
 * nested hierarchy of n_levels uniform grids (each coarsening halves every axis, so
 * n_cells[a] must be divisible by 2^(n_levels-1)).
 * dirichlet_faces: bit 2a clamps all displacement components on the lower face of axis a,
 * bit 2a+1 on the upper face (0x3F = every face, the pressurised-crack setting of Sec. 2.1).
 * dirichlet_mask: optional HOST array of fine-level node masks (PFF_MASK_U* and PFF_MASK_PHI_DIR
 * bits) OR-ed into the face mask; NULL for none.  A PFF_MASK_PHI_DIR node keeps the phase-field
 * value of the state (it is eliminated like an active node but never enters the active set).
 * Coarse levels inherit masks from the coincident fine nodes.
 * cell_mask: optional HOST array of fine-level cells (x fastest), nonzero = in the domain, for
 * domains cut from the box such as the L-shaped panels of Sec. 5.2/5.3; NULL = the whole box.
 * Cells outside contribute nothing; nodes on no cell of the domain are fixed in every component
 * (identity rows).  A coarse cell is in the domain if any of its children is. */
typedef struct {
    int dim;
    int degree;
    int n_cells[3];
    int n_levels;
    double lo[3];
    double hi[3];
    unsigned dirichlet_faces;
    const uint8_t* dirichlet_mask;
    const uint8_t* cell_mask;
} pff_mesh;

/* Problem and solver parameters.
 *  E, nu          Young's modulus and Poisson ratio; Lame coefficients by the 3D formulas
 *                 (plane strain in 2D), as in the parameter table of Sec. 5.1.
 *  Gc, kappa, eps critical energy release rate, residual stiffness of g_kappa, phase-field
 *                 width (Problem 2.1, Sec. 2.1).
 *  pressure       constant crack pressure p (Problem 2.1).
 *  c_as, tol_as   active-set constant c and tolerance eps_as (remark after Algorithm 1:
 *                 100 and 1e-10).  tol_as also decides ties of the active-set test.
 *  phi_elastic_factor  factor f on the phi-equation elastic term f (g'(phi) E_s, psi).
 *                 1 = derivative of the bulk energy of Sec. 5 (default); 0.5 = the literal
 *                 factor printed in Eq. (semilinear).
 *  mg_precision   32: whole V-cycle in FP32 with FP32 accumulation (inside FP64 FGMRES);
 *                 64: all-FP64 V-cycle.  The coarse solve is always FP64.
 *  cheb_degree    Chebyshev degree of the smoother (Sec. 3.2.1: 4).
 *  cg_steps       CG steps of the eigenvalue estimate (Sec. 3.2.1: 10).
 *  cheb_safety, cheb_ratio  smoothing range [ratio*safety*l, safety*l] (1.2 and 1/5).
 *  coarse_rtol, coarse_maxit  Chebyshev coarse solver: steps from the Chebyshev error bound
 *                 for this reduction, capped (Sec. 3.2.2 gives neither).
 *  seed           seed of the SplitMix64 start vector of the CG eigenvalue estimate.
 *  split          0: no split of the elastic energy (E_s^+ = E_s, default); 1: Miehe split (Sec. 2.1):
 *                 E_s^+ = lambda/2 <tr e>_+^2 + mu tr(e_+^2) over the strain eigenvalues, sigma^+ its
 *                 derivative; g(phi) degrades only the + part.  Q1 levels store the Gauss-point
 *                 tangent of g sigma^+ + sigma^- (28 coefficients per Gauss point in 3D, allocated
 *                 on first use, not counted by pff_hierarchy_bytes); residuals, diagonals and Q2 use
 *                 the generic kernels; batches require 0.
 *  tie_scale      scale of the tie band of the active-set test (the paper's test is a strict
 *                 inequality; values within tol_as of zero are rounding noise and count as inactive):
 *                 0 (default): lambda_i + c (phi_i - phi_old_i) > tol_as, lambda = M^-1 R;
 *                 1: M_ii (lambda_i + c (phi_i - phi_old_i)) > tol_as, i.e. the band on the scale of the
 *                 residual entry R_i, whose rounding noise does not shrink with the lumped mass
 *                 (M_ii ~ h^d) when the mesh is refined.
 *  newton_rtol    relative tolerance of the linear solve of each pff_newton_step (1e-8).
 *  coarse_phi_max 0 (default): phi_tilde reaches the coarse Q1 levels by coincident-node injection
 *                 (Sec. 4.2); 1: on Q1 levels too, a coarse node takes the maximum of the fine
 *                 phi_tilde over the fine nodes at most one lattice step away along every axis (Q2
 *                 levels always do, see pff_set_state).  A robustness option beyond the paper: it keeps
 *                 coarse cells from turning kappa-weak where the fine cells they cover are stiff.
 *  preconditioner 0: P_full = MG(G~), the monolithic V-cycle (Sec. 3.3, default);
 *                 1: P_diag = blockdiag(MG(U~), MG(P~)) (Sec. 3.3): the coupling G_phiu is
 *                 left out of every V-cycle residual and of the coarse solve.  Batches
 *                 (pff_batch_*) require 0. */
typedef struct {
    double E, nu, Gc, kappa, eps, pressure;
    double c_as, tol_as;
    double phi_elastic_factor;
    int mg_precision;
    int cheb_degree;
    int cg_steps;
    double cheb_safety;
    double cheb_ratio;
    double coarse_rtol;
    int coarse_maxit;
    uint64_t seed;
    int preconditioner;
    int split;
    int tie_scale;
    double newton_rtol;
    int coarse_phi_max;
} pff_params;

typedef struct {
    int iterations;        /* FGMRES iterations (Arnoldi steps) */
    int converged;         /* 1 if ||b - G x|| <= rtol ||b - G x0|| */
    double res0;           /* ||b - G x0|| */
    double res_final;      /* true residual norm at exit */
} pff_solve_info;

typedef struct {
    int n_active;          /* size of the active set A_k */
    int n_changed;         /* |A_k xor A_{k-1}| */
    double res_norm;       /* ||R~_k||_2 (right-hand side of the eliminated system) */
    int converged;         /* A_k == A_{k-1} and res_norm <= tol_as (Algorithm 1) */
    pff_solve_info solve;  /* the linear solve of step 5 */
} pff_newton_info;

/* Fill *p with the defaults quoted above (E=1, nu=0.2, Gc=1, kappa=1e-10, eps=1, p=1e-3,
 * c=100, eps_as=1e-10, f=1, FP32 V-cycle, degree 4, 10 CG steps, 1.2, 0.2, 1e-6, 200, 12345,
 * P_full, no split, tie band on lambda, Newton linear tolerance 1e-8). */
void pff_default_params(pff_params* p);

/* Create the level hierarchy (Sec. 3.2 and 4.2) on the current CUDA device.  cuda_stream is a
 * cudaStream_t (NULL = legacy default stream).  Allocates all device memory the solver needs.
 * Errors: PFF_EINVAL (sizes, degree, levels), PFF_ENOMEM, PFF_ECUDA.  *out is NULL on error. */
pff_status pff_create_hierarchy(const pff_mesh* mesh, const pff_params* params, void* cuda_stream,
                                pff_hierarchy** out);

/* Device bytes pff_create_hierarchy allocates for this mesh, plus the FGMRES workspace for
 * 'restart' (0: none); -1 for an invalid mesh.  Host-only, no CUDA call: a scheduler uses it to
 * admit instances into a device-memory budget. */
int64_t pff_hierarchy_bytes(const pff_mesh* mesh, int restart);

/* Free every allocation of the hierarchy (synchronises its stream).  NULL is a no-op. */
pff_status pff_destroy_hierarchy(pff_hierarchy* h);

/* Sizes of a level: nodes, cells and nodes per axis (host outputs, any may be NULL). */
pff_status pff_level_info(const pff_hierarchy* h, int level, int64_t* n_nodes, int64_t* n_cells,
                          int nodes_per_axis[3]);

/* Replace the parameters used by later calls (same mesh).  Marks the preconditioner stale. */
pff_status pff_set_params(pff_hierarchy* h, const pff_params* params);

/* Spatially varying Young's modulus (Sec. 5.2 computes with a heterogeneous E): E = s_K E on
 * every fine cell K, i.e. mu and lambda of the cell scaled by s_K in the residual, the Jacobian,
 * the diagonal and the energies.  escale: device FP64 array of the finest level's n_cells
 * (cells lexicographic, x fastest), copied; NULL restores a uniform modulus.  Coarse levels
 * take on each cell the mean of its 2^d children.  Errors: PFF_EINVAL if a factor is not finite
 * and positive; PFF_ENOMEM.  Synchronises. */
pff_status pff_set_modulus(pff_hierarchy* h, const double* escale);

/* Kernel variant of the level operators: 0 (default) = Q1 fast path (Gauss-point linearisation
 * data precomputed per state; FP64-accurate operators evaluated in double-float arithmetic, FP32
 * operators in FP32; on 3D levels of at least 100,000 cells both run one thread per cell with the
 * Gauss-point derivatives in shared memory and add element vectors to y with global atomics; on
 * smaller levels and in 2D the FP64-accurate operators run one thread per Gauss point, each adding
 * its node's result to y with global atomics, and the FP32 operators one thread per cell with a
 * shared-memory gather), 1 = generic kernels
 * (Q1 and Q2, native FP64 or FP32, state evaluated at every apply), 2 = one thread per Gauss point
 * with a shared-memory gather in both precisions, 3 = one thread per cell in both precisions,
 * 4 = as 0 but the FP64-accurate operator gathers through shared memory, 5 = one thread per Gauss
 * point with global atomics in both precisions, 6 / 7 = as 0 with the per-cell FP64-accurate /
 * FP32 form with shared-memory derivatives on every 3D level.  3D Q2 levels run, in every variant but
 * 1, the sum-factorised Q2 applies (one warp per cell, a lane per node and Gauss point, 1D stages
 * exchanged by warp shuffles, Gauss-point linearisation data precomputed per state, double-float /
 * FP32); 2D Q2 uses the generic kernels.  Errors: PFF_EINVAL outside 0 .. 7. */
pff_status pff_set_kernel_variant(pff_hierarchy* h, int variant);

/* Set the linearisation point.  U: FP64 [u | phi] (n_dofs), phi_old: FP64 (n_nodes) = the
 * irreversibility bound, phi_tilde: FP64 (n_nodes) = the extrapolation used in the
 * displacement equation (Eq. (semilinear)).  The library copies them, restricts U and
 * phi_tilde to every coarser level by coincident nodes (Sec. 4.2), and keeps FP32 copies.  On
 * Q2 levels (an extension of the paper) phi_tilde of a coarse node is instead the maximum of the
 * fine phi_tilde over the fine nodes at most one lattice step from the coincident node along
 * every axis, so that a coarse cell is not weaker than the fine cells it covers.
 * The current active set is kept.
 * u_dirichlet (nullable): device FP64 of at least dim * n_nodes entries in the layout of U's
 * displacement blocks: prescribed displacement values on the Dirichlet DoFs (the faces of
 * pff_mesh.dirichlet_faces and the PFF_MASK_U* bits of pff_mesh.dirichlet_mask; entries elsewhere
 * are not read), as in the displacement-driven loading of the L-shaped panels (Sec. 5.2, 5.3).  The
 * stored state and, in every later pff_newton_step / pff_load_step, the caller's U take these values
 * on those DoFs, so the Newton increments vanish there (the eliminated rows of Algorithm 1, step 4,
 * stay homogeneous).  The values are copied and kept until the next pff_set_state; NULL means no
 * prescribed values (the state keeps whatever U holds on Dirichlet DoFs).
 * Errors: PFF_EINVAL (NULL U, phi_old or phi_tilde), PFF_ENOMEM. */
pff_status pff_set_state(pff_hierarchy* h, const double* U, const double* phi_old, const double* phi_tilde,
                         const double* u_dirichlet);

/* Replace the prescribed displacement values of pff_set_state (same layout and meaning; NULL removes
 * them) without resetting the state, e.g. at each step of a displacement ramp before pff_load_step.
 * The stored state takes the new values on the Dirichlet DoFs.  Errors: PFF_ENOMEM, PFF_ECUDA. */
pff_status pff_set_dirichlet_values(pff_hierarchy* h, const double* u_dirichlet);

/* Set the active set from a device array of n_nodes bytes (nonzero = active) and carry it to
 * every coarser level by coincident nodes (Sec. 4.2).  Marks the preconditioner stale. */
pff_status pff_set_active_set(pff_hierarchy* h, const uint8_t* active);

/* Copy the fine-level active indicator (0/1 bytes, n_nodes) to a device array. */
pff_status pff_get_active_set(const pff_hierarchy* h, uint8_t* active);

/* Steps 1 and 3 of Algorithm 1 at the current state: R = -A(U), lambda = M^-1 R on the phi
 * DoFs with the lumped Gauss-Lobatto mass, active iff lambda + c (phi - phi_old) > tol_as (tie_scale 1:
 * M (lambda + c (phi - phi_old)) > tol_as).
 * Installs the new active set on all levels.  Host outputs (may be NULL): the set size and
 * the number of nodes that changed.  Synchronises. */
pff_status pff_update_active_set(pff_hierarchy* h, int* n_active, int* n_changed);

/* Residual R = -A(U) of Eq. (semilinear) at the current fine state, all DoFs, no elimination
 * (FP64, device output of n_dofs). */
pff_status pff_residual(pff_hierarchy* h, double* R);

/* Bulk energy int g(phi) E_s^+(e(u)) + E_s^-(e(u)) + phi^2 p div u and crack energy
 * int Gc/2 ((1 - phi)^2 / eps + eps |grad phi|^2) of Sec. 5 at the current fine state (E_s^+ = E_s
 * without split), FP64, Q1 meshes.  out (host): [bulk, crack].  Synchronises. */
pff_status pff_energies(pff_hierarchy* h, double out[2]);

/* Boundary load of Sec. 5, L_c = int_Gamma (sigma n)_c ds over one face of the box, evaluated as
 * the reaction: the sum over the fine nodes on that face of A(U)(phi_i e_c) (Eq. (semilinear),
 * current state, no elimination), which equals the traction integral for the discrete solution.
 * face: 2a = lower face of axis a, 2a+1 = upper face; component c < dim.  out: host.
 * Synchronises.  Errors: PFF_EINVAL (face, component), PFF_ESTATE (no state). */
pff_status pff_boundary_load(pff_hierarchy* h, int face, int component, double* out);

/* Matrix-free Jacobian apply y = G~_l(U_l) x on a level (Sec. 4.1, 4.2), FP64: the level's
 * operator at its restricted state, eliminated rows give y = x, eliminated columns are
 * ignored.  x and y must not overlap.  The finest level is the Newton Jacobian G~_k. */
pff_status pff_apply_jacobian(pff_hierarchy* h, int level, const double* x, double* y);

/* The same operator evaluated in FP32 arithmetic with FP32 accumulation (V-cycle operator). */
pff_status pff_apply_jacobian_f32(pff_hierarchy* h, int level, const float* x, float* y);

/* pff_apply_jacobian with x and y in HOST memory (n_dofs doubles each, layout as above; page-
 * locked memory lets the copies overlap the computation).  On 3D levels served by the per-cell
 * kernel (variant 0: at least 100,000 cells) the level is processed in slabs of z layers, the
 * host-to-device copy of one slab, the apply of the previous one and the device-to-host copy of
 * finished nodes running concurrently on three streams; other levels copy, apply and copy back in
 * order.  Uses two library-owned device vectors of the finest level's size (allocated on first
 * use).  Synchronises.  Errors: as pff_apply_jacobian. */
pff_status pff_apply_jacobian_host(pff_hierarchy* h, int level, const double* x, double* y);

/* Diagonal of G~_l (1 on eliminated rows), computed matrix-free (remark in Sec. 4.1).
 * precision 64 -> double* d, 32 -> float* d. */
pff_status pff_diagonal(pff_hierarchy* h, int level, int precision, void* d);

/* Restricted state of a level (device outputs, any may be NULL): U_l (FP64, n_dofs_l),
 * phi_tilde_l (FP64, n_nodes_l), mask_l (uint8, n_nodes_l). */
pff_status pff_level_state(const pff_hierarchy* h, int level, double* U, double* phi_tilde,
                           uint8_t* mask);

/* Transfers between level l-1 (coarse) and l (fine), canonical for nested Q1/Q2 (Sec. 3.2):
 * restrict: r_c = P^T r_f with eliminated coarse entries set to 0;
 * prolongate_add: x_f += P e_c on the free fine entries.  precision 32 or 64. */
pff_status pff_restrict(pff_hierarchy* h, int fine_level, int precision, const void* r_fine,
                        void* r_coarse);
pff_status pff_prolongate_add(pff_hierarchy* h, int fine_level, int precision,
                              const void* e_coarse, void* x_fine);

/* Build the preconditioner at the current state and active set: level diagonals and the
 * eigenvalue bounds of 10 Jacobi-preconditioned CG steps per diagonal block (Sec. 3.2.1).
 * Called implicitly by the smoother, V-cycle and solver when stale. */
pff_status pff_setup(pff_hierarchy* h);

/* Eigenvalue estimates of D^-1 G_bb on a level (host out[4]: lmin_u, lmax_u, lmin_phi,
 * lmax_phi; synchronises). */
pff_status pff_eigen_estimates(pff_hierarchy* h, int level, double out[4]);

/* Block-diagonal Chebyshev-Jacobi smoother S_full (Sec. 3.2.1, 3.3) on level l, degree
 * cheb_degree, range [ratio*safety*l, safety*l] per block:  x <- x + S(b - G~_l x)
 * (zero_guess != 0: x <- S(b), x is output only).  Entries of b on eliminated DoFs must be
 * 0.  precision 32 or 64. */
pff_status pff_smooth(pff_hierarchy* h, int level, int precision, const void* b, void* x,
                      int zero_guess);

/* Coarse solve on level 0 (Sec. 3.2.2): Chebyshev on [0.9 lmin, 1.2 lmax] of each block, in
 * block forward-substitution order (u first, then phi with the coupling on the right), FP64. */
pff_status pff_coarse_solve(pff_hierarchy* h, const double* b, double* x);

/* One V-cycle of P_full^-1 = MG(G~) (Sec. 3.3): z ~ G~^-1 r; eliminated entries z_i = r_i.
 * Runs in params.mg_precision (FP64 in/out either way). */
pff_status pff_vcycle(pff_hierarchy* h, const double* r, double* z);

/* Right-preconditioned flexible GMRES(restart) in FP64 with the V-cycle as preconditioner:
 * solve G~ x = b from the given x (initial guess, overwritten), until
 * ||b - G~ x|| <= rtol ||b - G~ x0|| or maxit iterations.  info (host, may be NULL) is
 * filled and the call synchronises.  Returns PFF_ENOCONV at the cap, PFF_ENONFINITE on
 * NaN/Inf. */
pff_status pff_gmres_solve(pff_hierarchy* h, const double* b, double* x, double rtol, int restart,
                           int maxit, pff_solve_info* info);

/* One primal-dual active-set step (Algorithm 1) at state U (device FP64 in/out, n_dofs) with
 * the phi_old and phi_tilde of the last pff_set_state: residual, active set, elimination
 * (active rows carry phi_old - phi), FGMRES + V-cycle solve to rtol params.newton_rtol (restart 30,
 * maxit 200), U += dU.  The new U becomes the hierarchy's state. */
pff_status pff_newton_step(pff_hierarchy* h, double* U, pff_newton_info* info);

/* One incremental (load) step n of the quasi-static problem (Sec. 2.1, 2.3) solved by Algorithm 1.
 * U (device, in/out, FP64, component-blocked) holds U^{n-1} on entry and U^n on return.
 * The step sets phi_old := phi^{n-1} (the phi block of U), the pressure to 'pressure' (the rest of
 * the parameters unchanged), and the time-lagged extrapolation phi~ = clamp(2 phi^{n-1} - phi^{n-2},
 * 0, 1), or phi~ = phi^{n-1} when phi_prev (device, n_nodes, phi^{n-2}) is NULL.  It then runs
 * active-set Newton steps (pff_newton_step) until Algorithm 1's stop test holds or max_newton
 * steps ran.  The active set of the previous load step serves as A_{k-1} of the first step.
 * phi_prev must not alias U.  info (host, nullable) receives the step counts and the last step's
 * Newton info.  Errors: those of pff_newton_step; PFF_EINVAL for max_newton < 1 or a non-finite
 * pressure.  A step cap reached without convergence returns PFF_OK with info->converged = 0. */
typedef struct {
    int newton_steps;      /* active-set steps run */
    int converged;         /* 1 if Algorithm 1 stopped by its test */
    int gmres_iterations;  /* summed over the steps */
    pff_newton_info last;  /* the last step */
} pff_load_info;
pff_status pff_load_step(pff_hierarchy* h, double* U, const double* phi_prev, double pressure, int max_newton,
                         pff_load_info* info);

/* ---- Batches of independent instances (one persistent launch per level and operation across
 * instances; the batched FGMRES keeps every instance's Hessenberg matrix, Givens rotations and
 * stopping test on the device, and on a non-default stream replays its Arnoldi step -- V-cycle,
 * apply, Gram-Schmidt, norm, scalar update, for all instances at once -- from one captured CUDA graph).
 * A batch is a view over n existing hierarchies created on the same stream, all Q1 with the same
 * dimension, one mg_precision (32 or 64), preconditioner 0, split 0 and cheb_degree; instances may differ in mesh size, number of levels
 * and physical parameters.  The batch owns only descriptor tables and reduction scratch; the
 * hierarchies keep their data (a hierarchy may belong to several batches, but batches that share a
 * hierarchy must not run concurrently).  Per-instance results equal those of the single-instance
 * calls up to rounding.  restart: FGMRES restart length used by the batch (1..200). */
typedef struct pff_batch pff_batch;
pff_status pff_batch_create(int n, pff_hierarchy* const* hierarchies, int restart, pff_batch** out);
pff_status pff_batch_destroy(pff_batch* b);
/* Continuous batching: instances join and leave a live batch between calls.  n may be 0 at creation
 * (an empty batch takes its dimension, stream and options from the first submitted instance).
 * pff_batch_submit appends a compatible hierarchy (same dimension, stream, mg_precision and
 * cheb_degree; Q1, P_full, no split) at index pff_batch_size() - 1 and gives it a Krylov workspace of
 * the batch's restart length; pff_batch_retire removes the instance at 'index' (later indices move
 * down by one; the hierarchy itself is not destroyed).  The device tables, FGMRES state and captured
 * graphs are rebuilt at the next batched call (the autotuner's choices come from its process-wide
 * cache when the make-up is similar).  The per-instance arrays of the batched calls (U, rhs, x, infos)
 * follow the current order.  pff_batch_poll returns the instance's info of the last
 * pff_batch_newton_step (zeros before one).  Calls on an empty batch return PFF_ESTATE.
 * Errors: PFF_EINVAL (NULL, incompatible or duplicate instance, index out of range), PFF_ENOMEM. */
pff_status pff_batch_submit(pff_batch* b, pff_hierarchy* h, int* index);
pff_status pff_batch_retire(pff_batch* b, int index);
int pff_batch_size(const pff_batch* b);
pff_status pff_batch_poll(const pff_batch* b, int index, pff_newton_info* info);
/* Diagonals and eigenvalue bounds of every instance (batched CG estimates, Sec. 3.2.1). */
pff_status pff_batch_setup(pff_batch* b);
/* z_i ~ G~_i^-1 r_i for every instance: one V-cycle (FP32 or FP64 levels, FP64 coarse solve) run
 * in lockstep over all instances. */
pff_status pff_batch_vcycle(pff_batch* b, const double* const* r, double* const* z);
/* FGMRES(restart) of every instance to ||b_i - G~_i x_i|| <= rtol ||b_i - G~_i x0_i|| (device arrays
 * of pointers are NOT used: 'rhs' and 'x' are host arrays of n device pointers).  info: host array of
 * n entries or NULL.  Synchronises. */
pff_status pff_batch_gmres_solve(pff_batch* b, const double* const* rhs, double* const* x, double rtol,
                                 int maxit, pff_solve_info* info);
/* One active-set step (Algorithm 1) of every instance at U_i (host array of n device pointers,
 * updated in place), the linear solves batched (to the first instance's newton_rtol).  infos: host
 * array of n entries or NULL. */
pff_status pff_batch_newton_step(pff_batch* b, double* const* U, pff_newton_info* infos);
/* y_i = G~_i x_i on one level of every instance (Sec. 4.1), batched: level -1 = each instance's finest
 * level, level l >= 0 = the instance's level l (0 = coarsest; instances with fewer levels are
 * skipped and their y left untouched).  precision 64: FP64-accurate operators, x/y double*;
 * 32: FP32 operators, x/y float*.  x, y: host arrays of n device pointers (n_dofs of the
 * instance's level each).  Errors: PFF_EINVAL, PFF_ESTATE (an instance without state). */
pff_status pff_batch_apply_jacobian(pff_batch* b, int level, int precision, const void* const* x, void* const* y);
/* Kernel family of the batched level operators: 0 (default) = chosen per level (3D levels whose
 * cells over the batch reach 100,000 run the per-cell kernels with shared-memory derivatives, smaller
 * levels the Gauss-point-lane FP64-accurate and per-cell-gather FP32 kernels), 1 = the small-level
 * kernels on every level, 2 = the per-cell kernels on every 3D level.  Errors: PFF_EINVAL. */
pff_status pff_batch_set_kernel_style(pff_batch* b, int style);
/* FP32 V-cycle batches (mg_precision 32): an instance whose FGMRES solve is still above its tolerance
 * after 'iterations' iterations continues with the all-FP64 V-cycle (flexible GMRES admits a different
 * preconditioner in every iteration, so the Krylov basis built so far is kept).  In a few instances --
 * crack zones where kappa = 1e-10 leaves displacement DoFs with nearly no stiffness -- the FP32
 * V-cycle's rounding limits the achievable reduction and the solve stalls at many times the usual
 * iteration count; the switch bounds what such an instance costs the whole batch.  The decision is
 * taken on the device per instance; the batch then replays a second captured Arnoldi step whose
 * V-cycle runs in FP32 and in FP64 on the two subsets.  Default 10; 0 never switches.
 * Errors: PFF_EINVAL (negative). */
pff_status pff_batch_set_precision_switch(pff_batch* b, int iterations);
/* The V-cycle precision (32 or 64) each instance used at the end of the last batched solve (host
 * array of n ints).  Synchronises.  Errors: PFF_EINVAL, PFF_ECUDA. */
pff_status pff_batch_mg_precisions(pff_batch* b, int* precisions);
/* The autotuner's choice for one level (-1: the instances' finest levels) and precision (32 or 64):
 * style 1 = small-level kernels, 2 = per-cell kernels, 0 = not tuned (the size rule applies);
 * ctas_per_sm = the persistent grid of the batched launch in CTAs per SM (0 = one CTA per tile);
 * ms = the measured time of one apply.  With style 0 (pff_batch_set_kernel_style) the first
 * pff_batch_setup times every candidate on the batch's own data with CUDA events and keeps the
 * fastest; choices are cached for the process by dimension, precision and the binary orders of the
 * level's cells and instances.  Host outputs, any may be NULL.  Errors: PFF_EINVAL, PFF_ESTATE
 * (not tuned yet). */
pff_status pff_batch_tuning(pff_batch* b, int level, int precision, int* style, int* ctas_per_sm, double* ms);
const char* pff_batch_last_error(const pff_batch* b);

/* Kernel timing (tracing).  pff_profile(h, 1) clears the counters and starts recording CUDA
 * events on the hierarchy's stream around every level-operator launch (the preset of eliminated
 * rows plus the cell kernel); pff_profile(h, 0) stops.  pff_profile_read synchronises and
 * returns, for one class, the number of launches and their summed device time in ms.
 * Classes: PFF_PROF_APPLY64_FINE (FP64 operator on the finest level), PFF_PROF_APPLY64_COARSE
 * (FP64 operators on coarser levels), PFF_PROF_APPLY32 (FP32 operators, all levels), and
 * PFF_PROF_VCYCLE (replays of a captured V-cycle graph: the operators inside a replayed graph are
 * timed as part of the replay, not in their own classes). */
enum { PFF_PROF_APPLY64_FINE = 0, PFF_PROF_APPLY64_COARSE = 1, PFF_PROF_APPLY32 = 2, PFF_PROF_VCYCLE = 3,
       PFF_PROF_NCLASS = 4 };
pff_status pff_profile(pff_hierarchy* h, int enable);
pff_status pff_profile_read(pff_hierarchy* h, int cls, int* count, double* total_ms);

/* Allocation-free active-set decision for callers that cannot allocate device memory (for
 * example a process whose GPU memory belongs to another allocator, or code that may not call
 * cudaMalloc and so cannot create a hierarchy).  The paper has no counterpart: this is the
 * decision of pff_update_active_set (Algorithm 1, step 3: active iff
 * R_i / M_ii + c (phi_i - phi_old_i) > tol_as with the Gauss-Lobatto lumped mass M; nodes whose
 * phi is prescribed -- PFF_MASK_PHI_DIR set, or on no cell of the domain -- are never active) on
 * caller buffers, without a hierarchy and without any device allocation.
 *   mesh     the fine mesh (dim, degree, n_cells, lo, hi are used; n_levels is ignored).
 *   params   c_as, tol_as and tie_scale are used.
 *   cell_mask  device uint8, n_cells, nonzero = in the domain, or NULL for the whole box.  The
 *            lumped mass of a node sums over its domain cells only, as the hierarchy's does.
 *            mesh->cell_mask is a HOST array this call cannot read: a mesh that has one needs
 *            the same cells passed here (PFF_EINVAL otherwise).
 *   R        device FP64, n_dofs: the residual -A(U), e.g. from pff_residual.
 *   U        device FP64, n_dofs: the state [u | phi].   phi_old: device FP64, n_nodes.
 *   mask     device uint8, n_nodes, in/out: PFF_MASK_ACTIVE is rewritten, other bits kept
 *            (PFF_MASK_PHI_DIR is read, e.g. the fine mask from pff_level_state).
 *   n_active, n_changed  host outputs (may be NULL); the call synchronises cuda_stream.
 * Scratch: a file-scope device array of 2 * 65536 + 2 ints (about 512 KB) that every GPU which
 * loads the library holds until the process exits; meshes with more than 65536 * 1024 nodes
 * are rejected with PFF_EINVAL.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before any stream
 * capture.  All calls share the array, so calls that overlap on the GPU race.
 * Errors: PFF_EINVAL (NULL, bad mesh, host-only cell mask, too many nodes), PFF_ECUDA. */
pff_status pff_active_set_noalloc(const pff_mesh* mesh, const pff_params* params, const uint8_t* cell_mask,
                                  const double* R, const double* U, const double* phi_old, uint8_t* mask,
                                  int* n_active, int* n_changed, void* cuda_stream);

/* Measured FP32 fused-multiply-add rate of the current GPU in TFLOP/s (2 flops per FMA), the
 * denominator of the arithmetic roofline of the double-float operators, which run on the FP32 pipes
 * (the paper measures on CPUs and gives no counterpart).  Runs a register-only FMA kernel three
 * times on cuda_stream after a warm-up and reports the fastest; allocates and frees one small
 * device buffer; synchronises.  Errors: PFF_EINVAL (NULL), PFF_ENOMEM, PFF_ECUDA. */
pff_status pff_fp32_fma_tflops(void* cuda_stream, double* tflops);

/* Number of kernel launches this library has issued in the process so far (tracing). */
long long pff_launch_count(void);

/* Last error message of a hierarchy (never NULL; "" when none). */
const char* pff_last_error(const pff_hierarchy* h);

#ifdef __cplusplus
}
#endif

#endif /* PFF_H */
