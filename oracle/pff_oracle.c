/*
 * Plain FP64 CPU oracle for the phase-field fracture Jacobian, residual and energy.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU-baseline
 * legs of bench.py may load this library.  It shares no code with the CUDA path.
 *
 * Everything here is the plain definition, written for a reader to check against the paper:
 *   - Q1/Q2 Lagrange elements on a uniform Cartesian box (Sec. 2.4, Problem 2.2),
 *   - full tensor Gauss quadrature with (deg+1) points per axis,
 *   - the semilinear form A(U)(Phi) of Eq. (semilinear) in Sec. 2.3, no stress split
 *     (E_s^+ := E_s, Sec. 2.1), AT2 crack term,
 *   - its Newton derivative G_ij = A'(U)(Phi_i, Phi_j) with the extrapolation phi~ frozen
 *     (Sec. 2.4 and Sec. 3.3: the u-rows do not depend on delta-phi),
 *   - element-by-element assembly of a sparse (CSR) matrix, no sum factorisation,
 *   - elimination of constrained rows/columns (Algorithm 1, step 4): identity rows,
 *     zero columns,
 *   - the energy functional whose first variation is the residual (Sec. 5, bulk + crack
 *     energy), used only as a finite-difference pin,
 *   - the Gauss-Lobatto lumped mass of the remark after Algorithm 1,
 *   - optionally a Young's modulus that varies per cell (E = s_cell E_0, Sec. 5.2 uses a
 *     spatially varying E): mu and lambda of a cell are scaled by s_cell,
 *   - optionally the Miehe split of the elastic energy (Sec. 2.1): E_s^+ from the positive parts
 *     of tr(e) and of the strain eigenvalues, sigma^+ = dE_s^+/de, degraded by g while
 *     E_s^- = E_s - E_s^+ and sigma^- = sigma - sigma^+ are not.
 *
 * Notation: d = dim, comps 0..d-1 = displacement u, comp d = phase field phi.
 * DoF index = comp * n_nodes + node, node lexicographic with x fastest.
 * Mask byte per node: bit c (c < d) = u_c constrained (Dirichlet); bit 3 = phi in the active
 * set; bit 4 = phi Dirichlet.  'phi_bits' selects which of bits 3/4 constrain phi.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int dim, deg;
    int n[3];          /* cells per axis */
    double lo[3], hi[3];
    const uint8_t *cell_mask;  /* per cell: nonzero = in the domain (n_cells), NULL = the whole box */
} om_mesh;

/* Cells outside the domain (an L-shaped panel cut from its bounding box) contribute nothing. */
static int cell_in(const om_mesh *m, int64_t cell) { return !m->cell_mask || m->cell_mask[cell] != 0; }

typedef struct {
    double mu, lam;    /* Lame coefficients */
    double Gc, kappa, eps, p;
    double f;          /* factor on the phi-equation elastic term: 1 = energy consistent */
    const double *escale;  /* per cell factor on mu and lam (n_cells), NULL = uniform */
    int split;             /* 0: no split (E_s^+ = E_s); 1: Miehe split */
} om_phys;

/* The physics of one cell: mu and lam scaled by the cell's modulus factor. */
static const om_phys *cell_phys(const om_phys *ph, int64_t cell, om_phys *tmp) {
    if (!ph->escale) return ph;
    *tmp = *ph;
    tmp->mu *= ph->escale[cell];
    tmp->lam *= ph->escale[cell];
    return tmp;
}

#define MAXN 27        /* nodes per cell, Q2 in 3D */
#define MAXQ 27        /* quadrature points per cell */
#define MAXC 4         /* components */

/* ---------------------------------------------------------------- 1D building blocks */

/* Gauss-Legendre rule with npts points on [0,1] (closed forms for 2 and 3 points). */
static void gauss01(int npts, double *x, double *w) {
    if (npts == 2) {
        double a = 0.5 / sqrt(3.0);
        x[0] = 0.5 - a; x[1] = 0.5 + a;
        w[0] = 0.5; w[1] = 0.5;
    } else {
        double a = 0.5 * sqrt(0.6);
        x[0] = 0.5 - a; x[1] = 0.5; x[2] = 0.5 + a;
        w[0] = 5.0 / 18.0; w[1] = 8.0 / 18.0; w[2] = 5.0 / 18.0;
    }
}

/* Lagrange basis on the equispaced nodes t_a = a/deg of [0,1]: value and derivative. */
static void lagrange01(int deg, int a, double t, double *val, double *der) {
    double v = 1.0, dsum = 0.0;
    for (int b = 0; b <= deg; ++b) {
        if (b == a) continue;
        double ta = (double)a / deg, tb = (double)b / deg;
        v *= (t - tb) / (ta - tb);
    }
    /* derivative: sum over the factor that is differentiated */
    for (int c = 0; c <= deg; ++c) {
        if (c == a) continue;
        double ta = (double)a / deg, tc = (double)c / deg;
        double prod = 1.0 / (ta - tc);
        for (int b = 0; b <= deg; ++b) {
            if (b == a || b == c) continue;
            double tb = (double)b / deg;
            prod *= (t - tb) / (ta - tb);
        }
        dsum += prod;
    }
    *val = v;
    *der = dsum;
}

/* ---------------------------------------------------------------- mesh helpers */

static void nodes_per_axis(const om_mesh *m, int64_t nn[3]) {
    for (int a = 0; a < 3; ++a) nn[a] = (a < m->dim) ? (int64_t)m->deg * m->n[a] + 1 : 1;
}

int64_t om_n_nodes(const om_mesh *m) {
    int64_t nn[3];
    nodes_per_axis(m, nn);
    return nn[0] * nn[1] * nn[2];
}

int64_t om_n_cells(const om_mesh *m) {
    int64_t c = 1;
    for (int a = 0; a < m->dim; ++a) c *= m->n[a];
    return c;
}

static void cell_size(const om_mesh *m, double h[3]) {
    for (int a = 0; a < 3; ++a) h[a] = (a < m->dim) ? (m->hi[a] - m->lo[a]) / m->n[a] : 1.0;
}

/* Global node ids of the local nodes of cell 'cell', local order lexicographic x fastest. */
static int cell_nodes(const om_mesh *m, int64_t cell, int64_t *nodes) {
    int64_t nn[3];
    nodes_per_axis(m, nn);
    int64_t c[3] = {0, 0, 0}, rem = cell;
    for (int a = 0; a < m->dim; ++a) { c[a] = rem % m->n[a]; rem /= m->n[a]; }
    int p = m->deg + 1;
    int kz = (m->dim == 3) ? p : 1;
    int cnt = 0;
    for (int k = 0; k < kz; ++k)
        for (int j = 0; j < p; ++j)
            for (int i = 0; i < p; ++i) {
                int64_t gi = m->deg * c[0] + i, gj = m->deg * c[1] + j;
                int64_t gk = (m->dim == 3) ? m->deg * c[2] + k : 0;
                nodes[cnt++] = gi + nn[0] * (gj + nn[1] * gk);
            }
    return cnt;
}

/* Shape values N[q][n], physical gradients G[q][n][d] and weights W[q] (incl. |K|) of a cell.
 * Uniform Cartesian cells: the Jacobian is diag(h), so d/dx_a = (1/h_a) d/dt_a. */
typedef struct {
    int nq, nloc;
    double N[MAXQ][MAXN];
    double G[MAXQ][MAXN][3];
    double W[MAXQ];
} om_qpdata;

static void cell_qpdata(const om_mesh *m, om_qpdata *qd) {
    int p = m->deg + 1;
    double gx[3], gw[3], h[3];
    gauss01(p, gx, gw);
    cell_size(m, h);
    double vol = 1.0;
    for (int a = 0; a < m->dim; ++a) vol *= h[a];
    int kq = (m->dim == 3) ? p : 1;
    int q = 0;
    for (int qz = 0; qz < kq; ++qz)
        for (int qy = 0; qy < p; ++qy)
            for (int qx = 0; qx < p; ++qx) {
                int qi[3] = {qx, qy, qz};
                double w = vol;
                for (int a = 0; a < m->dim; ++a) w *= gw[qi[a]];
                qd->W[q] = w;
                int n = 0;
                for (int k = 0; k < kq; ++k)
                    for (int j = 0; j < p; ++j)
                        for (int i = 0; i < p; ++i) {
                            int li[3] = {i, j, k};
                            double v[3], dv[3];
                            for (int a = 0; a < 3; ++a) {
                                if (a < m->dim) lagrange01(m->deg, li[a], gx[qi[a]], &v[a], &dv[a]);
                                else { v[a] = 1.0; dv[a] = 0.0; }
                            }
                            qd->N[q][n] = v[0] * v[1] * v[2];
                            qd->G[q][n][0] = dv[0] / h[0] * v[1] * v[2];
                            qd->G[q][n][1] = v[0] * dv[1] / h[1] * v[2];
                            qd->G[q][n][2] = v[0] * v[1] * dv[2] / h[2];
                            ++n;
                        }
                qd->nloc = n;
                ++q;
            }
    qd->nq = q;
}

/* ---------------------------------------------------------------- pointwise physics */

/* Degradation g_kappa(phi) = (1-kappa) phi^2 + kappa (Sec. 2.1). */
static double degr(const om_phys *ph, double phi) { return (1.0 - ph->kappa) * phi * phi + ph->kappa; }

/* Strain e = sym(grad u) from a d x d displacement gradient (Sec. 2.1). */
static void strain(int d, double gu[3][3], double e[3][3]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) e[i][j] = (i < d && j < d) ? 0.5 * (gu[i][j] + gu[j][i]) : 0.0;
}

/* sigma(e) = 2 mu e + lambda tr(e) I (Sec. 2.1). */
static void stress(const om_phys *ph, int d, double e[3][3], double s[3][3]) {
    double tr = 0.0;
    for (int i = 0; i < d; ++i) tr += e[i][i];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) s[i][j] = (i < d && j < d) ? 2.0 * ph->mu * e[i][j] + (i == j ? ph->lam * tr : 0.0) : 0.0;
}

/* E_s(e) = 1/2 lambda tr(e)^2 + mu e:e (Sec. 2.1). */
static double elastic_energy(const om_phys *ph, int d, double e[3][3]) {
    double tr = 0.0, ee = 0.0;
    for (int i = 0; i < d; ++i) tr += e[i][i];
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) ee += e[i][j] * e[i][j];
    return 0.5 * ph->lam * tr * tr + ph->mu * ee;
}

/* ---------------------------------------------------------------- Miehe split (Sec. 2.1) */

/* Eigen-decomposition a = V diag(l) V^T of a symmetric 3x3 matrix by cyclic Jacobi rotations
 * (Golub and Van Loan, Matrix Computations, Sec. 8.5); the columns of V are the eigenvectors. */
static void sym_eig3(double a_in[3][3], double l[3], double V[3][3]) {
    double a[3][3];
    memcpy(a, a_in, sizeof(a));
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) V[i][j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
        double dia = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
        if (off == 0.0 || off <= 1e-36 * dia) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (a[p][q] == 0.0) continue;
                /* rotation J in the (p, q) plane that zeroes a[p][q] in J^T a J */
                double theta = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
                double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
                for (int k = 0; k < 3; ++k) {      /* a <- a J */
                    double akp = a[k][p], akq = a[k][q];
                    a[k][p] = c * akp - sn * akq;
                    a[k][q] = sn * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) {      /* a <- J^T a */
                    double apk = a[p][k], aqk = a[q][k];
                    a[p][k] = c * apk - sn * aqk;
                    a[q][k] = sn * apk + c * aqk;
                }
                for (int k = 0; k < 3; ++k) {      /* V <- V J */
                    double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - sn * vkq;
                    V[k][q] = sn * vkp + c * vkq;
                }
            }
    }
    for (int i = 0; i < 3; ++i) l[i] = a[i][i];
}

/* <x>_+ = max(0, x) and its derivative, taken as 0 at x = 0. */
static double posp(double x) { return x > 0.0 ? x : 0.0; }
static double heav(double x) { return x > 0.0 ? 1.0 : 0.0; }

typedef struct {
    double l[3], V[3][3];   /* eigenvalues and eigenvectors (columns) of e */
    double tr;              /* tr(e) */
} om_eig;

/* sigma^+ = lambda <tr e>_+ I + 2 mu e_+ and E_s^+ = lambda/2 <tr e>_+^2 + mu tr(e_+^2), with
 * e_+ = sum_a <l_a>_+ n_a n_a^T.  In 2D (plane strain) e is the 3x3 strain with e_zz = 0. */
static void miehe_split(const om_phys *ph, int d, double e[3][3], double sp[3][3], double *Esp, om_eig *E) {
    sym_eig3(e, E->l, E->V);
    E->tr = 0.0;
    for (int i = 0; i < d; ++i) E->tr += e[i][i];
    double trp = posp(E->tr), ep2 = 0.0;
    for (int a = 0; a < 3; ++a) ep2 += posp(E->l[a]) * posp(E->l[a]);
    *Esp = 0.5 * ph->lam * trp * trp + ph->mu * ep2;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double epij = 0.0;
            for (int a = 0; a < 3; ++a) epij += posp(E->l[a]) * E->V[i][a] * E->V[j][a];
            sp[i][j] = (i < d && j < d) ? 2.0 * ph->mu * epij + (i == j ? ph->lam * trp : 0.0) : 0.0;
        }
}

/* Directional derivative of sigma^+ at e in the direction de:
 *   C^+ de = lambda H(tr e) tr(de) I + 2 mu P^+(de),
 *   P^+(de) = sum_{a,b} theta_ab (n_a . de n_b) n_a n_b^T,
 * theta_aa = H(l_a), theta_ab = (<l_a>_+ - <l_b>_+) / (l_a - l_b) for l_a != l_b (H(l_a) if equal);
 * the derivative of the isotropic tensor function e -> e_+. */
static void miehe_tangent(const om_phys *ph, int d, const om_eig *E, double de[3][3], double out[3][3]) {
    double dtr = 0.0;
    for (int i = 0; i < d; ++i) dtr += de[i][i];
    double dp[3][3] = {{0}};
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double th;
            if (a == b || E->l[a] == E->l[b]) th = heav(E->l[a]);
            else th = (posp(E->l[a]) - posp(E->l[b])) / (E->l[a] - E->l[b]);
            if (th == 0.0) continue;
            double proj = 0.0;   /* n_a . de n_b */
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) proj += E->V[i][a] * de[i][j] * E->V[j][b];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) dp[i][j] += th * proj * E->V[i][a] * E->V[j][b];
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            out[i][j] = (i < d && j < d) ? 2.0 * ph->mu * dp[i][j] + (i == j ? ph->lam * heav(E->tr) * dtr : 0.0) : 0.0;
}

static double ddot(int d, double a[3][3], double b[3][3]) {
    double s = 0.0;
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) s += a[i][j] * b[i][j];
    return s;
}

/* Gradient tensor of the vector shape function N e_b: row b holds grad N. */
static void vec_shape_grad(int d, int b, const double *gN, double gv[3][3]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) gv[i][j] = (i == b && j < d) ? gN[j] : 0.0;
}

/* State of the linearisation point at one quadrature point. */
typedef struct {
    double gu[3][3];   /* grad u */
    double phi;        /* phi */
    double gphi[3];    /* grad phi */
    double pt;         /* phi~ (extrapolation) */
} om_state;

static void state_at_qp(const om_mesh *m, const om_qpdata *qd, int q, const int64_t *nodes,
                        int64_t nn, const double *U, const double *ptil, om_state *s) {
    int d = m->dim;
    memset(s, 0, sizeof(*s));
    for (int n = 0; n < qd->nloc; ++n) {
        int64_t g = nodes[n];
        for (int c = 0; c < d; ++c)
            for (int j = 0; j < d; ++j) s->gu[c][j] += U[c * nn + g] * qd->G[q][n][j];
        s->phi += U[d * nn + g] * qd->N[q][n];
        for (int j = 0; j < d; ++j) s->gphi[j] += U[d * nn + g] * qd->G[q][n][j];
        if (ptil) s->pt += ptil[g] * qd->N[q][n];
    }
}

/* ---------------------------------------------------------------- element kernels */

/* Element Jacobian Ke[(ni*nc+ci)][(nj*nc+cj)] of A'(U) with phi~ frozen:
 *   G_uu : ( g(phi~) sigma(du), e(w) )
 *   G_uphi = 0
 *   G_phiu : ( 2 f (1-k) phi sigma(u):e(du) + 2 p phi div du, psi )
 *   G_phiphi : ( [2 f (1-k) E_s(u) + 2 p div u + Gc/eps] dphi, psi ) + Gc eps (grad dphi, grad psi)
 * obtained by differentiating the semilinear form of Sec. 2.3. */
static void element_jacobian(const om_mesh *m, const om_phys *ph, const om_qpdata *qd,
                             const int64_t *nodes, int64_t nn, const double *U, const double *ptil,
                             double *Ke) {
    int d = m->dim, nc = d + 1, nl = qd->nloc, ne = nl * nc;
    memset(Ke, 0, sizeof(double) * ne * ne);
    for (int q = 0; q < qd->nq; ++q) {
        om_state s;
        state_at_qp(m, qd, q, nodes, nn, U, ptil, &s);
        double eu[3][3], su[3][3], sp[3][3], Esp;
        om_eig E;
        strain(d, s.gu, eu);
        stress(ph, d, eu, su);
        if (ph->split) miehe_split(ph, d, eu, sp, &Esp, &E);
        else { memcpy(sp, su, sizeof(sp)); Esp = elastic_energy(ph, d, eu); }
        double divu = 0.0;
        for (int i = 0; i < d; ++i) divu += s.gu[i][i];
        double gt = degr(ph, s.pt);
        double W = qd->W[q];
        for (int ni = 0; ni < nl; ++ni)
            for (int ci = 0; ci < nc; ++ci) {
                int row = ni * nc + ci;
                const double *gNi = qd->G[q][ni];
                double Ni = qd->N[q][ni];
                for (int nj = 0; nj < nl; ++nj)
                    for (int cj = 0; cj < nc; ++cj) {
                        int col = nj * nc + cj;
                        const double *gNj = qd->G[q][nj];
                        double Nj = qd->N[q][nj];
                        double val = 0.0;
                        if (ci < d && cj < d) {
                            double gi[3][3], gj[3][3], ei[3][3], ej[3][3], sj[3][3];
                            vec_shape_grad(d, ci, gNi, gi);
                            vec_shape_grad(d, cj, gNj, gj);
                            strain(d, gi, ei);
                            strain(d, gj, ej);
                            stress(ph, d, ej, sj);
                            if (ph->split) {
                                /* g C^+ de + C^- de with C^- = C - C^+ */
                                double cp[3][3];
                                miehe_tangent(ph, d, &E, ej, cp);
                                val = gt * ddot(d, cp, ei) + ddot(d, sj, ei) - ddot(d, cp, ei);
                            } else {
                                val = gt * ddot(d, sj, ei);
                            }
                        } else if (ci < d && cj == d) {
                            val = 0.0; /* phi~ frozen in the displacement equation */
                        } else if (ci == d && cj < d) {
                            double gj[3][3], ej[3][3];
                            vec_shape_grad(d, cj, gNj, gj);
                            strain(d, gj, ej);
                            double divj = gNj[cj];
                            val = (2.0 * ph->f * (1.0 - ph->kappa) * s.phi * ddot(d, sp, ej)
                                   + 2.0 * ph->p * s.phi * divj) * Ni;
                        } else {
                            double gg = 0.0;
                            for (int a = 0; a < d; ++a) gg += gNi[a] * gNj[a];
                            val = (2.0 * ph->f * (1.0 - ph->kappa) * Esp + 2.0 * ph->p * divu + ph->Gc / ph->eps) * Nj * Ni
                                  + ph->Gc * ph->eps * gg;
                        }
                        Ke[row * ne + col] += W * val;
                    }
            }
    }
}

/* Element residual Re[ni*nc+ci] = A(U)(Phi) of Eq. (semilinear), test function Phi = N_ni e_ci:
 *   u-rows  : ( g(phi~) sigma(u), e(w) ) + ( phi~^2 p, div w )
 *   phi-rows: f ( g'(phi) E_s(u), psi ) + 2 ( phi p div u, psi ) + Gc [ -(1/eps)(1-phi, psi) + eps (grad phi, grad psi) ]
 * with g'(phi) = 2 (1-k) phi. */
static void element_residual(const om_mesh *m, const om_phys *ph, const om_qpdata *qd,
                             const int64_t *nodes, int64_t nn, const double *U, const double *ptil,
                             double *Re) {
    int d = m->dim, nc = d + 1, nl = qd->nloc;
    memset(Re, 0, sizeof(double) * nl * nc);
    for (int q = 0; q < qd->nq; ++q) {
        om_state s;
        state_at_qp(m, qd, q, nodes, nn, U, ptil, &s);
        double eu[3][3], su[3][3], sp[3][3], Esp;
        om_eig E;
        strain(d, s.gu, eu);
        stress(ph, d, eu, su);
        if (ph->split) miehe_split(ph, d, eu, sp, &Esp, &E);
        else { memcpy(sp, su, sizeof(sp)); Esp = elastic_energy(ph, d, eu); }
        /* g(phi~) sigma^+ + sigma^- */
        double gt = degr(ph, s.pt);
        double seff[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) seff[i][j] = gt * sp[i][j] + (su[i][j] - sp[i][j]);
        double divu = 0.0;
        for (int i = 0; i < d; ++i) divu += s.gu[i][i];
        double W = qd->W[q];
        for (int ni = 0; ni < nl; ++ni) {
            const double *gNi = qd->G[q][ni];
            double Ni = qd->N[q][ni];
            for (int ci = 0; ci < d; ++ci) {
                double gi[3][3], ei[3][3];
                vec_shape_grad(d, ci, gNi, gi);
                strain(d, gi, ei);
                double v = ddot(d, seff, ei) + s.pt * s.pt * ph->p * gNi[ci];
                Re[ni * nc + ci] += W * v;
            }
            double gg = 0.0;
            for (int a = 0; a < d; ++a) gg += s.gphi[a] * gNi[a];
            double v = ph->f * 2.0 * (1.0 - ph->kappa) * s.phi * Esp * Ni
                       + 2.0 * s.phi * ph->p * divu * Ni
                       + ph->Gc * (-(1.0 / ph->eps) * (1.0 - s.phi) * Ni + ph->eps * gg);
            Re[ni * nc + d] += W * v;
        }
    }
}

/* Energy of one cell: g(phi) E_s(e(u)) + phi^2 p div u + Gc/2 ( (1-phi)^2/eps + eps |grad phi|^2 )
 * (bulk and crack energies of Sec. 5 with no split).  Strain computed here independently. */
static double element_energy(const om_mesh *m, const om_phys *ph, const om_qpdata *qd,
                             const int64_t *nodes, int64_t nn, const double *U) {
    int d = m->dim;
    double E = 0.0;
    for (int q = 0; q < qd->nq; ++q) {
        double gu[3][3] = {{0}}, phi = 0.0, gphi[3] = {0, 0, 0};
        for (int n = 0; n < qd->nloc; ++n) {
            int64_t g = nodes[n];
            for (int c = 0; c < d; ++c)
                for (int j = 0; j < d; ++j) gu[c][j] += U[c * nn + g] * qd->G[q][n][j];
            phi += U[d * nn + g] * qd->N[q][n];
            for (int j = 0; j < d; ++j) gphi[j] += U[d * nn + g] * qd->G[q][n][j];
        }
        double tr = 0.0, ee = 0.0, gp2 = 0.0;
        for (int i = 0; i < d; ++i) tr += gu[i][i];
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) {
                double eij = 0.5 * (gu[i][j] + gu[j][i]);
                ee += eij * eij;
            }
        for (int j = 0; j < d; ++j) gp2 += gphi[j] * gphi[j];
        double Es = 0.5 * ph->lam * tr * tr + ph->mu * ee;
        double Esp = Es;
        if (ph->split) {
            double e[3][3], sp[3][3];
            om_eig E;
            strain(d, gu, e);
            miehe_split(ph, d, e, sp, &Esp, &E);
        }
        double g = (1.0 - ph->kappa) * phi * phi + ph->kappa;
        double dens = g * Esp + (Es - Esp) + phi * phi * ph->p * tr
                      + 0.5 * ph->Gc * ((1.0 - phi) * (1.0 - phi) / ph->eps + ph->eps * gp2);
        E += qd->W[q] * dens;
    }
    return E;
}

/* ---------------------------------------------------------------- constraints */

static int is_constrained(int d, uint8_t mask, int comp, int phi_bits) {
    if (comp < d) return (mask >> comp) & 1;
    return (mask & phi_bits) != 0;
}

/* ---------------------------------------------------------------- public: vectors */

/* A(U) for all DoFs (no masking). */
void om_residual(const om_mesh *m, const om_phys *ph, const double *U, const double *ptil, double *A) {
    int64_t nn = om_n_nodes(m), nc = m->dim + 1, ncell = om_n_cells(m);
    memset(A, 0, sizeof(double) * nn * nc);
    om_qpdata *qd = malloc(sizeof(om_qpdata));
    cell_qpdata(m, qd);
    double Re[MAXN * MAXC];
    int64_t nodes[MAXN];
    for (int64_t cell = 0; cell < ncell; ++cell) {
        if (!cell_in(m, cell)) continue;
        int nl = cell_nodes(m, cell, nodes);
        om_phys pc;
        element_residual(m, cell_phys(ph, cell, &pc), qd, nodes, nn, U, ptil, Re);
        for (int n = 0; n < nl; ++n)
            for (int c = 0; c < nc; ++c) A[c * nn + nodes[n]] += Re[n * nc + c];
    }
    free(qd);
}

/* Bulk and crack energies of Sec. 5 separately (no split): out[0] = int g(phi) E_s + phi^2 p div u,
 * out[1] = int Gc/2 ( (1-phi)^2/eps + eps |grad phi|^2 ).  Evaluated with Gc = 0 and with E = p = 0
 * through element_energy, so the two parts add up to om_energy exactly in exact arithmetic. */
void om_energy_parts(const om_mesh *m, const om_phys *ph, const double *U, double *out) {
    int64_t nn = om_n_nodes(m), ncell = om_n_cells(m);
    om_qpdata *qd = malloc(sizeof(om_qpdata));
    cell_qpdata(m, qd);
    int64_t nodes[MAXN];
    om_phys bulk = *ph, crack = *ph;
    bulk.Gc = 0.0;
    crack.mu = 0.0; crack.lam = 0.0; crack.p = 0.0;
    out[0] = 0.0;
    out[1] = 0.0;
    for (int64_t cell = 0; cell < ncell; ++cell) {
        if (!cell_in(m, cell)) continue;
        cell_nodes(m, cell, nodes);
        om_phys pc;
        out[0] += element_energy(m, cell_phys(&bulk, cell, &pc), qd, nodes, nn, U);
        out[1] += element_energy(m, &crack, qd, nodes, nn, U);
    }
    free(qd);
}

double om_energy(const om_mesh *m, const om_phys *ph, const double *U) {
    int64_t nn = om_n_nodes(m), ncell = om_n_cells(m);
    om_qpdata *qd = malloc(sizeof(om_qpdata));
    cell_qpdata(m, qd);
    int64_t nodes[MAXN];
    double E = 0.0;
    for (int64_t cell = 0; cell < ncell; ++cell) {
        if (!cell_in(m, cell)) continue;
        cell_nodes(m, cell, nodes);
        om_phys pc;
        E += element_energy(m, cell_phys(ph, cell, &pc), qd, nodes, nn, U);
    }
    free(qd);
    return E;
}

/* Gauss-Lobatto lumped mass per node (remark after Algorithm 1): Lobatto points coincide
 * with the element nodes for Q1 (weights 1/2,1/2) and Q2 (weights 1/6,2/3,1/6). */
void om_lumped_mass(const om_mesh *m, double *M) {
    int64_t nn = om_n_nodes(m), ncell = om_n_cells(m);
    memset(M, 0, sizeof(double) * nn);
    double h[3];
    cell_size(m, h);
    double vol = 1.0;
    for (int a = 0; a < m->dim; ++a) vol *= h[a];
    double w1[3];
    if (m->deg == 1) { w1[0] = 0.5; w1[1] = 0.5; }
    else { w1[0] = 1.0 / 6.0; w1[1] = 2.0 / 3.0; w1[2] = 1.0 / 6.0; }
    int p = m->deg + 1, kz = (m->dim == 3) ? p : 1;
    int64_t nodes[MAXN];
    for (int64_t cell = 0; cell < ncell; ++cell) {
        if (!cell_in(m, cell)) continue;
        cell_nodes(m, cell, nodes);
        int n = 0;
        for (int k = 0; k < kz; ++k)
            for (int j = 0; j < p; ++j)
                for (int i = 0; i < p; ++i) {
                    double w = vol * w1[i] * w1[j] * (m->dim == 3 ? w1[k] : 1.0);
                    M[nodes[n++]] += w;
                }
    }
}

/* ---------------------------------------------------------------- public: sparse matrix */

/* Row structure: each row (comp, node) holds every (comp', node') with node' inside the
 * (2 deg + 1)^d box around node (clipped to the grid), sorted by column index. */
typedef struct { int64_t lo[3], w[3], cnt; } om_box;

static void row_box(const om_mesh *m, int64_t node, om_box *b) {
    int64_t nn[3];
    nodes_per_axis(m, nn);
    int64_t idx[3] = {node % nn[0], (node / nn[0]) % nn[1], node / (nn[0] * nn[1])};
    b->cnt = 1;
    for (int a = 0; a < 3; ++a) {
        int64_t lo = idx[a] - m->deg, hi = idx[a] + m->deg;
        if (lo < 0) lo = 0;
        if (hi > nn[a] - 1) hi = nn[a] - 1;
        b->lo[a] = lo;
        b->w[a] = hi - lo + 1;
        b->cnt *= b->w[a];
    }
}

/* Number of stored entries; fills indptr (size n_dofs + 1). */
int64_t om_csr_structure(const om_mesh *m, int64_t *indptr) {
    int64_t nn = om_n_nodes(m), nc = m->dim + 1;
    indptr[0] = 0;
    for (int64_t c = 0; c < nc; ++c)
        for (int64_t node = 0; node < nn; ++node) {
            om_box b;
            row_box(m, node, &b);
            int64_t r = c * nn + node;
            indptr[r + 1] = indptr[r] + nc * b.cnt;
        }
    return indptr[nc * nn];
}

static int64_t col_position(const om_mesh *m, int64_t nn, int64_t nc, const om_box *b,
                            int64_t cj, int64_t nodej) {
    int64_t nnx[3];
    nodes_per_axis(m, nnx);
    int64_t idx[3] = {nodej % nnx[0], (nodej / nnx[0]) % nnx[1], nodej / (nnx[0] * nnx[1])};
    (void)nn; (void)nc;
    int64_t off = ((idx[2] - b->lo[2]) * b->w[1] + (idx[1] - b->lo[1])) * b->w[0] + (idx[0] - b->lo[0]);
    return cj * b->cnt + off;
}

/* Assemble the eliminated Jacobian G~ (Algorithm 1, step 4) into CSR.  indptr from
 * om_csr_structure; indices/data have its length.  Constrained rows become identity rows,
 * constrained columns are zeroed. */
void om_assemble(const om_mesh *m, const om_phys *ph, const double *U, const double *ptil,
                 const uint8_t *mask, int phi_bits, const int64_t *indptr, int64_t *indices,
                 double *data) {
    int64_t nn = om_n_nodes(m), nc = m->dim + 1, ncell = om_n_cells(m);
    int64_t nnx[3];
    nodes_per_axis(m, nnx);
    /* column indices */
    for (int64_t c = 0; c < nc; ++c)
        for (int64_t node = 0; node < nn; ++node) {
            om_box b;
            row_box(m, node, &b);
            int64_t r = c * nn + node, pos = indptr[r];
            for (int64_t cj = 0; cj < nc; ++cj)
                for (int64_t k = 0; k < b.w[2]; ++k)
                    for (int64_t j = 0; j < b.w[1]; ++j)
                        for (int64_t i = 0; i < b.w[0]; ++i) {
                            int64_t nodej = (b.lo[0] + i) + nnx[0] * ((b.lo[1] + j) + nnx[1] * (b.lo[2] + k));
                            indices[pos] = cj * nn + nodej;
                            data[pos] = 0.0;
                            ++pos;
                        }
        }
    om_qpdata *qd = malloc(sizeof(om_qpdata));
    cell_qpdata(m, qd);
    int nl = qd->nloc;
    int ne = nl * (int)nc;
    double *Ke = malloc(sizeof(double) * ne * ne);
    int64_t nodes[MAXN];
    for (int64_t cell = 0; cell < ncell; ++cell) {
        if (!cell_in(m, cell)) continue;
        cell_nodes(m, cell, nodes);
        om_phys pc;
        element_jacobian(m, cell_phys(ph, cell, &pc), qd, nodes, nn, U, ptil, Ke);
        for (int ni = 0; ni < nl; ++ni) {
            om_box b;
            row_box(m, nodes[ni], &b);
            for (int ci = 0; ci < nc; ++ci) {
                int64_t r = ci * nn + nodes[ni];
                for (int nj = 0; nj < nl; ++nj)
                    for (int cj = 0; cj < nc; ++cj) {
                        int64_t pos = indptr[r] + col_position(m, nn, nc, &b, cj, nodes[nj]);
                        data[pos] += Ke[(ni * nc + ci) * ne + nj * nc + cj];
                    }
            }
        }
    }
    free(Ke);
    free(qd);
    /* elimination */
    int d = m->dim;
    for (int64_t r = 0; r < nc * nn; ++r) {
        int64_t cr = r / nn, noder = r % nn;
        int rc = is_constrained(d, mask[noder], (int)cr, phi_bits);
        for (int64_t pos = indptr[r]; pos < indptr[r + 1]; ++pos) {
            int64_t col = indices[pos];
            if (rc) { data[pos] = (col == r) ? 1.0 : 0.0; continue; }
            int64_t cc = col / nn, nodec = col % nn;
            if (is_constrained(d, mask[nodec], (int)cc, phi_bits)) data[pos] = 0.0;
        }
    }
}

/* (G~ x)_r for a list of rows, computed from the element matrices of the cells around each
 * row's node (for sampled checks on meshes too large to assemble). */
void om_apply_rows(const om_mesh *m, const om_phys *ph, const double *U, const double *ptil,
                   const uint8_t *mask, int phi_bits, const double *x, int64_t nrows,
                   const int64_t *rows, double *out) {
    int64_t nn = om_n_nodes(m), nc = m->dim + 1;
    int d = m->dim;
    int64_t nnx[3];
    nodes_per_axis(m, nnx);
    om_qpdata *qd = malloc(sizeof(om_qpdata));
    cell_qpdata(m, qd);
    int nl = qd->nloc, ne = nl * (int)nc;
    double *Ke = malloc(sizeof(double) * ne * ne);
    int64_t nodes[MAXN];
    for (int64_t t = 0; t < nrows; ++t) {
        int64_t r = rows[t], cr = r / nn, node = r % nn;
        if (is_constrained(d, mask[node], (int)cr, phi_bits)) { out[t] = x[r]; continue; }
        int64_t idx[3] = {node % nnx[0], (node / nnx[0]) % nnx[1], node / (nnx[0] * nnx[1])};
        int64_t clo[3], chi[3];
        for (int a = 0; a < 3; ++a) {
            if (a >= d) { clo[a] = 0; chi[a] = 0; continue; }
            /* cells c with deg*c <= idx <= deg*c + deg */
            int64_t lo = (idx[a] - m->deg + m->deg - 1) / m->deg; /* ceil((idx-deg)/deg) for idx>=deg */
            if (idx[a] < m->deg) lo = 0;
            int64_t hi = idx[a] / m->deg;
            if (hi > m->n[a] - 1) hi = m->n[a] - 1;
            clo[a] = lo; chi[a] = hi;
        }
        double acc = 0.0;
        for (int64_t ck = clo[2]; ck <= chi[2]; ++ck)
            for (int64_t cj = clo[1]; cj <= chi[1]; ++cj)
                for (int64_t ci = clo[0]; ci <= chi[0]; ++ci) {
                    int64_t cell = ci + m->n[0] * (cj + (d == 3 ? (int64_t)m->n[1] * ck : 0));
                    if (!cell_in(m, cell)) continue;
                    cell_nodes(m, cell, nodes);
                    int li = -1;
                    for (int n = 0; n < nl; ++n) if (nodes[n] == node) li = n;
                    if (li < 0) continue;
                    om_phys pc;
                    element_jacobian(m, cell_phys(ph, cell, &pc), qd, nodes, nn, U, ptil, Ke);
                    for (int nj = 0; nj < nl; ++nj)
                        for (int cj2 = 0; cj2 < nc; ++cj2) {
                            if (is_constrained(d, mask[nodes[nj]], cj2, phi_bits)) continue;
                            acc += Ke[(li * nc + cr) * ne + nj * nc + cj2] * x[cj2 * nn + nodes[nj]];
                        }
                }
        out[t] = acc;
    }
    free(Ke);
    free(qd);
}
