// C ABI of the pff library (declarations and contracts in include/pff.h).
#include <math.h>
#include <string.h>

#include <new>
#include <string>

#include "pff_q1.cuh"
#include "pff_solver.cuh"

using namespace pff;

static pff_status fail(pff_hierarchy* h, pff_status st, const std::string& msg) {
    if (h) h->err = msg;
    return st;
}

#define CUDA_OR_FAIL(h, expr)                                                                   \
    do {                                                                                        \
        cudaError_t e_ = (expr);                                                                \
        if (e_ != cudaSuccess) return fail(h, PFF_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define REQUIRE(h, cond, st, msg) \
    do {                          \
        if (!(cond)) return fail(h, st, msg); \
    } while (0)

extern "C" void pff_default_params(pff_params* p) {
    if (!p) return;
    p->E = 1.0;
    p->nu = 0.2;
    p->Gc = 1.0;
    p->kappa = 1e-10;
    p->eps = 1.0;
    p->pressure = 1e-3;
    p->c_as = 100.0;
    p->tol_as = 1e-10;
    p->phi_elastic_factor = 1.0;
    p->mg_precision = 32;
    p->cheb_degree = 4;
    p->cg_steps = 10;
    p->cheb_safety = 1.2;
    p->cheb_ratio = 0.2;
    p->coarse_rtol = 1e-6;
    p->coarse_maxit = 200;
    p->seed = 12345;
    p->preconditioner = 0;
    p->split = 0;
    p->tie_scale = 0;
    p->newton_rtol = 1e-8;
    p->coarse_phi_max = 0;
}

// Gauss-Legendre rule with deg+1 points mapped to [0,1] and the Lagrange basis on the
// equispaced nodes a/deg evaluated there (value and derivative).
static void make_tables(int deg, Tables& tb) {
    memset(&tb, 0, sizeof(tb));
    const int np = deg + 1;
    double xq[3], wq[3];
    if (np == 2) {
        const double r = 1.0 / sqrt(3.0);
        xq[0] = 0.5 * (1.0 - r);
        xq[1] = 0.5 * (1.0 + r);
        wq[0] = wq[1] = 0.5;
    } else {
        const double r = sqrt(3.0 / 5.0);
        xq[0] = 0.5 * (1.0 - r);
        xq[1] = 0.5;
        xq[2] = 0.5 * (1.0 + r);
        wq[0] = wq[2] = 5.0 / 18.0;
        wq[1] = 8.0 / 18.0;
    }
    for (int q = 0; q < np; ++q) {
        tb.w1[q] = wq[q];
        const double t = xq[q];
        if (deg == 1) {
            tb.N1[0][q] = 1.0 - t;
            tb.N1[1][q] = t;
            tb.D1[0][q] = -1.0;
            tb.D1[1][q] = 1.0;
        } else {
            tb.N1[0][q] = 2.0 * t * t - 3.0 * t + 1.0;
            tb.N1[1][q] = 4.0 * t - 4.0 * t * t;
            tb.N1[2][q] = 2.0 * t * t - t;
            tb.D1[0][q] = 4.0 * t - 3.0;
            tb.D1[1][q] = 4.0 - 8.0 * t;
            tb.D1[2][q] = 4.0 * t - 1.0;
        }
    }
}

static Phys make_phys(const pff_params& p) {
    Phys ph;
    ph.mu = p.E / (2.0 * (1.0 + p.nu));
    ph.lam = p.E * p.nu / ((1.0 + p.nu) * (1.0 - 2.0 * p.nu));
    ph.Gc = p.Gc;
    ph.kappa = p.kappa;
    ph.eps = p.eps;
    ph.p = p.pressure;
    ph.f = p.phi_elastic_factor;
    ph.split = p.split;
    return ph;
}

static const char* check_params(const pff_params* p) {
    if (!p) return "params is NULL";
    if (!(p->E > 0) || !(p->nu > -1.0 && p->nu < 0.5)) return "need E > 0 and -1 < nu < 0.5";
    if (!(p->eps > 0) || !(p->Gc >= 0) || !(p->kappa >= 0 && p->kappa < 1)) return "need eps > 0, Gc >= 0, 0 <= kappa < 1";
    if (p->mg_precision != 32 && p->mg_precision != 64) return "mg_precision must be 32 or 64";
    if (p->cheb_degree < 1 || p->cheb_degree > 64) return "cheb_degree must be in [1, 64]";
    if (p->cg_steps < 1 || p->cg_steps > 50) return "cg_steps must be in [1, 50]";
    if (!(p->cheb_safety > 0) || !(p->cheb_ratio > 0 && p->cheb_ratio < 1)) return "need cheb_safety > 0, 0 < cheb_ratio < 1";
    if (!(p->coarse_rtol > 0 && p->coarse_rtol < 1) || p->coarse_maxit < 1) return "need 0 < coarse_rtol < 1, coarse_maxit >= 1";
    if (p->preconditioner != 0 && p->preconditioner != 1) return "preconditioner must be 0 (P_full) or 1 (P_diag)";
    if (p->split != 0 && p->split != 1) return "split must be 0 (none) or 1 (Miehe)";
    if (p->tie_scale != 0 && p->tie_scale != 1) return "tie_scale must be 0 (lambda) or 1 (residual)";
    if (!(p->newton_rtol > 0 && p->newton_rtol < 1)) return "need 0 < newton_rtol < 1";
    if (p->coarse_phi_max != 0 && p->coarse_phi_max != 1) return "coarse_phi_max must be 0 or 1";
    return nullptr;
}

// Device memory, the library-owned streams and the events of a hierarchy (also on the error
// paths of pff_create_hierarchy, where some of them may not exist yet).
static void free_all(pff_hierarchy* h) {
    for (void* p : h->allocs) cudaFree(p);
    h->allocs.clear();
    for (cudaStream_t& st : h->lv_stream) {
        if (st) cudaStreamDestroy(st);
        st = nullptr;
    }
    for (cudaEvent_t& e : h->lv_event) {
        if (e) cudaEventDestroy(e);
        e = nullptr;
    }
    for (cudaEvent_t e : h->slab_ev) cudaEventDestroy(e);
    h->slab_ev.clear();
    if (h->cs_in) cudaStreamDestroy(h->cs_in);
    if (h->cs_out) cudaStreamDestroy(h->cs_out);
    h->cs_in = h->cs_out = nullptr;
}

template <typename T>
static cudaError_t dalloc(pff_hierarchy* h, T** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T) + 16);
    if (e != cudaSuccess) return e;
    h->allocs.push_back(q);
    *p = reinterpret_cast<T*>(q);
    return cudaMemsetAsync(q, 0, count * sizeof(T) + 16, h->stream);
}

// Gauss-point tangent storage of the Miehe split on Q1 levels (allocated when the split is first used)
static cudaError_t ensure_split_storage(pff_hierarchy* h) {
    if (!h->ph.split) return cudaSuccess;
    for (auto& L : h->lv) {
        if (L.g.deg != 1 || L.qps64) continue;
        const size_t nq = (size_t)q1_nks(L.g.dim) * (size_t)(1 << L.g.dim) * (size_t)L.g.n_cells;
        cudaError_t e = dalloc(h, &L.qps32, nq);
        if (e == cudaSuccess) e = dalloc(h, &L.qps64, nq);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

extern "C" pff_status pff_create_hierarchy(const pff_mesh* mesh, const pff_params* params, void* cuda_stream,
                                           pff_hierarchy** out) {
    if (!out) return PFF_EINVAL;
    *out = nullptr;
    if (!mesh) return PFF_EINVAL;
    if (check_params(params)) return PFF_EINVAL;
    if (mesh->dim != 2 && mesh->dim != 3) return PFF_EINVAL;
    if (mesh->degree != 1 && mesh->degree != 2) return PFF_EINVAL;
    if (mesh->n_levels < 1 || mesh->n_levels > 16) return PFF_EINVAL;
    const int div = 1 << (mesh->n_levels - 1);
    for (int a = 0; a < mesh->dim; ++a) {
        if (mesh->n_cells[a] < 1 || mesh->n_cells[a] % div != 0) return PFF_EINVAL;
        if (!(mesh->hi[a] > mesh->lo[a])) return PFF_EINVAL;
    }
    pff_hierarchy* h = new (std::nothrow) pff_hierarchy();
    if (!h) return PFF_ENOMEM;
    h->mesh = *mesh;
    h->mesh.dirichlet_mask = nullptr;
    h->prm = *params;
    h->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    h->L = mesh->n_levels;
    h->ph = make_phys(*params);
    make_tables(mesh->degree, h->tb);
    h->lv.resize(h->L);
    pff_status st = PFF_OK;
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < h->L && e == cudaSuccess; ++l) {
        Level& L = h->lv[l];
        Geom& g = L.g;
        g.dim = mesh->dim;
        g.deg = mesh->degree;
        g.es = nullptr;
        g.cm = nullptr;
        const int f = 1 << (h->L - 1 - l);
        g.n_nodes = 1;
        g.n_cells = 1;
        for (int a = 0; a < 3; ++a) {
            if (a < mesh->dim) {
                g.nc[a] = mesh->n_cells[a] / f;
                g.nn[a] = g.deg * g.nc[a] + 1;
                g.h[a] = (mesh->hi[a] - mesh->lo[a]) / g.nc[a];
            } else {
                g.nc[a] = 1;
                g.nn[a] = 1;
                g.h[a] = 1.0;
            }
            g.n_nodes *= g.nn[a];
            if (a < mesh->dim) g.n_cells *= g.nc[a];
        }
        const size_t nn = (size_t)g.n_nodes, nd = (size_t)n_dofs(g);
        if (e == cudaSuccess) e = dalloc(h, &L.mask, nn);
        if (e == cudaSuccess) e = dalloc(h, &L.U64, nd);
        if (e == cudaSuccess) e = dalloc(h, &L.pt64, nn);
        if (e == cudaSuccess) e = dalloc(h, &L.U32, nd);
        if (e == cudaSuccess) e = dalloc(h, &L.pt32, nn);
        if (e == cudaSuccess) e = dalloc(h, &L.dinv64, nd);
        if (e == cudaSuccess) e = dalloc(h, &L.dinv32, nd);
        if (e == cudaSuccess && (g.deg == 1 || g.dim == 3)) {
            // Gauss-point linearisation data of the fast paths (Q1; Q2 in 3D)
            const size_t nq = g.deg == 1 ? (size_t)q1_nk(g.dim) * (size_t)(1 << g.dim) * (size_t)g.n_cells
                                         : q2_data_size(g);
            e = dalloc(h, &L.qpd32, nq);
            if (e == cudaSuccess) e = dalloc(h, &L.qpd64, nq);
        }
        for (int k = 0; k < 6 && e == cudaSuccess; ++k) {
            float* wf = nullptr;
            double* wd = nullptr;
            e = dalloc(h, &wf, nd);
            if (e == cudaSuccess) e = dalloc(h, &wd, nd);
            L.w[0][k] = wf;
            L.w[1][k] = wd;
        }
    }
    Level& F = h->lv[h->L - 1];
    const size_t nnf = (size_t)F.g.n_nodes, ndf = (size_t)n_dofs(F.g);
    if (e == cudaSuccess) e = dalloc(h, &h->dir_mask, nnf);
    if (e == cudaSuccess) e = dalloc(h, &h->phi_old, nnf);
    if (e == cudaSuccess) e = dalloc(h, &h->lumped, nnf);
    if (e == cudaSuccess) e = dalloc(h, &h->R, ndf);
    for (int k = 0; k < 4 && e == cudaSuccess; ++k) e = dalloc(h, &h->tmp64[k], ndf);
    if (e == cudaSuccess) e = dalloc(h, &h->prev_active, nnf);
    if (e == cudaSuccess) e = dalloc(h, &h->d_counts, 16);
    if (e == cudaSuccess) e = dalloc(h, &h->d_scal, 4096);
    if (e == cudaSuccess) e = dalloc(h, &h->d_scratch, (size_t)dot_partials() * 64);
    if (e == cudaSuccess) e = dalloc(h, &h->d_scal_lv, (size_t)kLevelScal * h->L);
    if (e == cudaSuccess) e = dalloc(h, &h->d_scratch_lv, (size_t)kLevelScratch * h->L);
    for (int l = 0; l < h->L && e == cudaSuccess; ++l) e = cudaStreamCreateWithFlags(&h->lv_stream[l], cudaStreamNonBlocking);
    for (int l = 0; l <= h->L && e == cudaSuccess; ++l) e = cudaEventCreateWithFlags(&h->lv_event[l], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        st = (e == cudaErrorMemoryAllocation) ? PFF_ENOMEM : PFF_ECUDA;
        cudaGetLastError();
        free_all(h);
        delete h;
        return st;
    }
    if (e == cudaSuccess) e = ensure_split_storage(h);
    if (e != cudaSuccess) {
        st = (e == cudaErrorMemoryAllocation) ? PFF_ENOMEM : PFF_ECUDA;
        cudaGetLastError();
        free_all(h);
        delete h;
        return st;
    }
    // domain masks (cells outside an L-shaped or otherwise cut domain), finest from the host
    if (mesh->cell_mask) {
        for (int l = 0; l < h->L && e == cudaSuccess; ++l) e = dalloc(h, &h->lv[l].cm_buf, (size_t)h->lv[l].g.n_cells);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(F.cm_buf, mesh->cell_mask, (size_t)F.g.n_cells, cudaMemcpyHostToDevice, h->stream);
        for (int l = h->L - 2; l >= 0 && e == cudaSuccess; --l)
            e = launch_coarsen_cell_mask(h->lv[l].g, h->lv[l + 1].g, h->lv[l + 1].cm_buf, h->lv[l].cm_buf, h->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            free_all(h);
            delete h;
            return PFF_ECUDA;
        }
        for (auto& L : h->lv) L.g.cm = L.cm_buf;
    }
    // Dirichlet mask of the finest level (faces + optional host mask), copied to every level
    uint8_t* extra = nullptr;
    if (mesh->dirichlet_mask) {
        if (dalloc(h, &extra, nnf) != cudaSuccess ||
            cudaMemcpyAsync(extra, mesh->dirichlet_mask, nnf, cudaMemcpyHostToDevice, h->stream) != cudaSuccess) {
            free_all(h);
            delete h;
            return PFF_ECUDA;
        }
    }
    e = launch_face_mask(F.g, mesh->dirichlet_faces, extra, h->dir_mask, h->stream);
    if (e == cudaSuccess && mesh->cell_mask) e = launch_outside_nodes(F.g, h->dir_mask, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(F.mask, h->dir_mask, nnf, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess) e = propagate_state(h);
    if (e == cudaSuccess) e = launch_lumped_mass(F.g, h->lumped, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_all(h);
        delete h;
        return PFF_ECUDA;
    }
    *out = h;
    return PFF_OK;
}

extern "C" pff_status pff_destroy_hierarchy(pff_hierarchy* h) {
    if (!h) return PFF_OK;
    cudaStreamSynchronize(h->stream);
    drop_graph(h);
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    free_all(h);
    delete h;
    return PFF_OK;
}

static int resolve_level(const pff_hierarchy* h, int level) { return level < 0 ? h->L - 1 : level; }

extern "C" int64_t pff_hierarchy_bytes(const pff_mesh* mesh, int restart) {
    if (!mesh || (mesh->dim != 2 && mesh->dim != 3) || (mesh->degree != 1 && mesh->degree != 2) ||
        mesh->n_levels < 1 || mesh->n_levels > 16 || restart < 0)
        return -1;
    const int div = 1 << (mesh->n_levels - 1);
    for (int a = 0; a < mesh->dim; ++a)
        if (mesh->n_cells[a] < 1 || mesh->n_cells[a] % div != 0) return -1;
    const int64_t pad = 16;   // every allocation carries 16 spare bytes
    int64_t total = 0, nn_f = 0, nd_f = 0;
    for (int l = 0; l < mesh->n_levels; ++l) {
        const int f = 1 << (mesh->n_levels - 1 - l);
        int64_t nn = 1, nc = 1;
        for (int a = 0; a < mesh->dim; ++a) {
            nn *= (int64_t)mesh->degree * (mesh->n_cells[a] / f) + 1;
            nc *= mesh->n_cells[a] / f;
        }
        const int64_t nd = (mesh->dim + 1) * nn;
        total += (nn + pad) + (nd * 8 + pad) + (nn * 8 + pad) + (nd * 4 + pad) + (nn * 4 + pad) + (nd * 8 + pad) +
                 (nd * 4 + pad) + 6 * ((nd * 4 + pad) + (nd * 8 + pad));
        if (mesh->degree == 1 || mesh->dim == 3) {
            const int64_t nq = mesh->degree == 1 ? (int64_t)(mesh->dim == 3 ? 8 : 5) * (1 << mesh->dim) * nc
                                                 : (int64_t)8 * 27 * nc;
            total += (nq * 4 + pad) + (nq * 8 + pad);
        }
        if (mesh->cell_mask) total += nc + pad;
        nn_f = nn;
        nd_f = nd;
    }
    total += (nn_f + pad) + 2 * (nn_f * 8 + pad) + (nd_f * 8 + pad) + 4 * (nd_f * 8 + pad) + (nn_f + pad) +
             (16 * 4 + pad) + (4096 * 8 + pad) + ((int64_t)dot_partials() * 64 * 8 + pad) +
             ((int64_t)kLevelScal * mesh->n_levels * 8 + pad) + ((int64_t)kLevelScratch * mesh->n_levels * 8 + pad);
    if (restart > 0) total += ((int64_t)(restart + 1) * nd_f * 8 + pad) + ((int64_t)restart * nd_f * 8 + pad) +
                              ((int64_t)(2 * (restart + 1) + 2) * 8 + pad);
    return total;
}

extern "C" pff_status pff_level_info(const pff_hierarchy* h, int level, int64_t* n_nodes, int64_t* n_cells,
                                     int nodes_per_axis[3]) {
    if (!h) return PFF_EINVAL;
    const int l = resolve_level(h, level);
    if (l < 0 || l >= h->L) return PFF_EINVAL;
    const Geom& g = h->lv[l].g;
    if (n_nodes) *n_nodes = g.n_nodes;
    if (n_cells) *n_cells = g.n_cells;
    if (nodes_per_axis)
        for (int a = 0; a < 3; ++a) nodes_per_axis[a] = g.nn[a];
    return PFF_OK;
}

extern "C" pff_status pff_set_params(pff_hierarchy* h, const pff_params* params) {
    if (!h) return PFF_EINVAL;
    const char* why = check_params(params);
    REQUIRE(h, !why, PFF_EINVAL, why ? why : "");
    h->prm = *params;
    h->ph = make_phys(*params);
    {
        cudaError_t e = ensure_split_storage(h);
        if (e != cudaSuccess) {
            cudaGetLastError();
            h->err = "pff_set_params: no device memory for the split's Gauss-point data";
            return e == cudaErrorMemoryAllocation ? PFF_ENOMEM : PFF_ECUDA;
        }
    }
    if (h->has_state) CUDA_OR_FAIL(h, propagate_state(h));   // linearisation data depend on the physics
    h->stale = true;
    return PFF_OK;
}

extern "C" pff_status pff_set_modulus(pff_hierarchy* h, const double* escale) {
    if (!h) return PFF_EINVAL;
    drop_graph(h);
    h->stale = true;
    if (!escale) {
        for (auto& L : h->lv) L.g.es = nullptr;
    } else {
        Level& F = h->lv[h->L - 1];
        CUDA_OR_FAIL(h, cudaMemsetAsync(h->d_counts, 0, sizeof(int), h->stream));
        CUDA_OR_FAIL(h, launch_count_nonpositive(F.g.n_cells, escale, h->d_counts, h->stream));
        int bad = 0;
        CUDA_OR_FAIL(h, cudaMemcpyAsync(&bad, h->d_counts, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
        REQUIRE(h, bad == 0, PFF_EINVAL, "pff_set_modulus: factors must be finite and > 0");
        for (auto& L : h->lv)
            if (!L.es_buf) CUDA_OR_FAIL(h, dalloc(h, &L.es_buf, (size_t)L.g.n_cells));
        CUDA_OR_FAIL(h, cudaMemcpyAsync(F.es_buf, escale, sizeof(double) * F.g.n_cells, cudaMemcpyDeviceToDevice,
                                        h->stream));
        for (int l = h->L - 2; l >= 0; --l)
            CUDA_OR_FAIL(h, launch_coarsen_cells(h->lv[l].g, h->lv[l + 1].g, h->lv[l + 1].es_buf, h->lv[l].es_buf,
                                                 h->stream));
        for (auto& L : h->lv) L.g.es = L.es_buf;
    }
    if (h->has_state) CUDA_OR_FAIL(h, propagate_state(h));
    return PFF_OK;
}

extern "C" pff_status pff_set_kernel_variant(pff_hierarchy* h, int variant) {
    if (!h) return PFF_EINVAL;
    REQUIRE(h, variant >= 0 && variant <= 7, PFF_EINVAL, "variant must be 0 .. 7");
    drop_graph(h);
    h->fast_q1 = variant != 1;
    static const int style[8] = {52, 52, 3, 0, 1, 12, 52 | 64, 52 | 128};
    h->q1_style = style[variant];
    h->stale = true;
    return PFF_OK;
}

extern "C" pff_status pff_set_state(pff_hierarchy* h, const double* U, const double* phi_old,
                                    const double* phi_tilde, const double* u_dirichlet) {
    if (!h) return PFF_EINVAL;
    REQUIRE(h, U && phi_old && phi_tilde, PFF_EINVAL, "pff_set_state: NULL vector");
    Level& F = h->lv[h->L - 1];
    const size_t nn = (size_t)F.g.n_nodes, nd = (size_t)n_dofs(F.g);
    if (u_dirichlet) {
        if (!h->udir) CUDA_OR_FAIL(h, dalloc(h, &h->udir, (size_t)F.g.dim * nn));
        CUDA_OR_FAIL(h, cudaMemcpyAsync(h->udir, u_dirichlet, (size_t)F.g.dim * nn * sizeof(double),
                                        cudaMemcpyDeviceToDevice, h->stream));
        h->has_udir = true;
    } else {
        h->has_udir = false;
    }
    CUDA_OR_FAIL(h, cudaMemcpyAsync(F.U64, U, nd * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    if (h->has_udir) CUDA_OR_FAIL(h, launch_lift_dirichlet(F.g, h->dir_mask, h->udir, F.U64, h->stream));
    CUDA_OR_FAIL(h, cudaMemcpyAsync(F.pt64, phi_tilde, nn * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    CUDA_OR_FAIL(h, cudaMemcpyAsync(h->phi_old, phi_old, nn * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    CUDA_OR_FAIL(h, propagate_state(h));
    h->has_state = true;
    return PFF_OK;
}

extern "C" pff_status pff_set_dirichlet_values(pff_hierarchy* h, const double* u_dirichlet) {
    if (!h) return PFF_EINVAL;
    Level& F = h->lv[h->L - 1];
    const size_t nu = (size_t)F.g.dim * (size_t)F.g.n_nodes;
    if (!u_dirichlet) {
        h->has_udir = false;
        return PFF_OK;
    }
    if (!h->udir) CUDA_OR_FAIL(h, dalloc(h, &h->udir, nu));
    CUDA_OR_FAIL(h, cudaMemcpyAsync(h->udir, u_dirichlet, nu * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    h->has_udir = true;
    if (h->has_state) {
        CUDA_OR_FAIL(h, launch_lift_dirichlet(F.g, h->dir_mask, h->udir, F.U64, h->stream));
        h->derived_dirty = true;
        h->stale = true;
    }
    return PFF_OK;
}

extern "C" pff_status pff_set_active_set(pff_hierarchy* h, const uint8_t* active) {
    if (!h) return PFF_EINVAL;
    REQUIRE(h, active, PFF_EINVAL, "pff_set_active_set: NULL");
    Level& F = h->lv[h->L - 1];
    CUDA_OR_FAIL(h, launch_set_active(F.g, active, F.mask, h->stream));
    CUDA_OR_FAIL(h, propagate_state(h, false));
    h->active_known = true;
    return PFF_OK;
}

extern "C" pff_status pff_get_active_set(const pff_hierarchy* h, uint8_t* active) {
    if (!h || !active) return PFF_EINVAL;
    const Level& F = h->lv[h->L - 1];
    cudaError_t e = launch_get_active(F.g, F.mask, active, h->stream);
    return e == cudaSuccess ? PFF_OK : PFF_ECUDA;
}

// Steps 1 and 3 of Algorithm 1; returns counts on the host.
static pff_status update_active(pff_hierarchy* h, int* n_active, int* n_changed) {
    Level& F = h->lv[h->L - 1];
    CUDA_OR_FAIL(h, residual_fine(h, h->R));
    CUDA_OR_FAIL(h, cudaMemsetAsync(h->d_counts, 0, 2 * sizeof(int), h->stream));
    CUDA_OR_FAIL(h, launch_active_set(F.g, h->R, h->lumped, F.U64, h->phi_old, h->prm.c_as, h->prm.tol_as,
                                      h->prm.tie_scale, F.mask, h->d_counts, h->stream));
    int cnt[2] = {0, 0};
    CUDA_OR_FAIL(h, cudaMemcpyAsync(cnt, h->d_counts, sizeof(cnt), cudaMemcpyDeviceToHost, h->stream));
    CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
    if (!h->active_known) cnt[1] = cnt[0];
    h->active_known = true;
    CUDA_OR_FAIL(h, propagate_state(h, false));
    if (n_active) *n_active = cnt[0];
    if (n_changed) *n_changed = cnt[1];
    return PFF_OK;
}

extern "C" pff_status pff_update_active_set(pff_hierarchy* h, int* n_active, int* n_changed) {
    if (!h) return PFF_EINVAL;
    REQUIRE(h, h->has_state, PFF_ESTATE, "pff_update_active_set before pff_set_state");
    return update_active(h, n_active, n_changed);
}

extern "C" pff_status pff_energies(pff_hierarchy* h, double out[2]) {
    if (!h || !out) return PFF_EINVAL;
    REQUIRE(h, h->has_state, PFF_ESTATE, "pff_energies before pff_set_state");
    REQUIRE(h, h->mesh.degree == 1, PFF_EINVAL, "pff_energies supports Q1 meshes");
    Level& F = h->lv[h->L - 1];
    CUDA_OR_FAIL(h, launch_q1_energies(F.g, h->ph, F.U64, h->d_scratch, h->d_scal + 400, h->stream));
    CUDA_OR_FAIL(h, cudaMemcpyAsync(out, h->d_scal + 400, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
    return PFF_OK;
}

extern "C" pff_status pff_boundary_load(pff_hierarchy* h, int face, int component, double* out) {
    if (!h || !out) return PFF_EINVAL;
    REQUIRE(h, h->has_state, PFF_ESTATE, "pff_boundary_load before pff_set_state");
    Level& F = h->lv[h->L - 1];
    REQUIRE(h, face >= 0 && face < 2 * F.g.dim, PFF_EINVAL, "pff_boundary_load: face out of range");
    REQUIRE(h, component >= 0 && component < F.g.dim, PFF_EINVAL, "pff_boundary_load: component out of range");
    double* R = h->tmp64[3];
    CUDA_OR_FAIL(h, residual_fine(h, R));
    CUDA_OR_FAIL(h, launch_face_sum(F.g, face / 2, face % 2, component, R, h->d_scal + 402, h->stream));
    double v = 0.0;
    CUDA_OR_FAIL(h, cudaMemcpyAsync(&v, h->d_scal + 402, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
    *out = -v;    // R = -A(U): the load is the sum of A(U)(phi_i e_c) over the face nodes
    return PFF_OK;
}

extern "C" pff_status pff_residual(pff_hierarchy* h, double* R) {
    if (!h) return PFF_EINVAL;
    REQUIRE(h, R, PFF_EINVAL, "pff_residual: NULL");
    REQUIRE(h, h->has_state, PFF_ESTATE, "pff_residual before pff_set_state");
    CUDA_OR_FAIL(h, residual_fine(h, R));
    return PFF_OK;
}

template <typename T>
static pff_status apply_checked(pff_hierarchy* h, int level, const T* x, T* y) {
    if (!h) return PFF_EINVAL;
    const int l = resolve_level(h, level);
    REQUIRE(h, l >= 0 && l < h->L, PFF_EINVAL, "level out of range");
    REQUIRE(h, x && y && (const void*)x != (const void*)y, PFF_EINVAL, "apply: NULL or aliased vectors");
    REQUIRE(h, h->has_state, PFF_ESTATE, "apply before pff_set_state");
    CUDA_OR_FAIL(h, apply_level<T>(h, l, OP_APPLY, x, y, PHI_BITS_ALL));
    return PFF_OK;
}

extern "C" pff_status pff_apply_jacobian(pff_hierarchy* h, int level, const double* x, double* y) {
    return apply_checked<double>(h, level, x, y);
}

extern "C" pff_status pff_apply_jacobian_f32(pff_hierarchy* h, int level, const float* x, float* y) {
    return apply_checked<float>(h, level, x, y);
}

// y = G~_l x with x, y in host memory.  On 3D levels served by the per-cell FP64-accurate kernel
// the level is cut into slabs of z node layers and three streams overlap the host-to-device copy of
// slab s + 1, the apply of slab s and the device-to-host copy of the finished nodes.
extern "C" pff_status pff_apply_jacobian_host(pff_hierarchy* h, int level, const double* x, double* y) {
    if (!h) return PFF_EINVAL;
    const int l = resolve_level(h, level);
    REQUIRE(h, l >= 0 && l < h->L, PFF_EINVAL, "level out of range");
    REQUIRE(h, x && y && (const void*)x != (const void*)y, PFF_EINVAL, "apply: NULL or aliased vectors");
    REQUIRE(h, h->has_state, PFF_ESTATE, "apply before pff_set_state");
    Level& L = h->lv[l];
    const Geom& g = L.g;
    const int64_t nn = g.n_nodes, nd = n_dofs(g);
    cudaStream_t s = h->stream;
    if (!h->hx) {
        const int64_t nmax = n_dofs(h->lv[h->L - 1].g);
        CUDA_OR_FAIL(h, dalloc(h, &h->hx, (size_t)nmax));
        CUDA_OR_FAIL(h, dalloc(h, &h->hy, (size_t)nmax));
    }
    const bool slabs = g.dim == 3 && g.deg == 1 && h->fast_q1 && !h->ph.split &&
                       ((h->q1_style & 64) != 0 || ((h->q1_style & 16) != 0 && g.n_cells >= kCellMinCells));
    if (!slabs) {
        CUDA_OR_FAIL(h, cudaMemcpyAsync(h->hx, x, nd * sizeof(double), cudaMemcpyHostToDevice, s));
        CUDA_OR_FAIL(h, apply_level<double>(h, l, OP_APPLY, h->hx, h->hy, PHI_BITS_ALL));
        CUDA_OR_FAIL(h, cudaMemcpyAsync(y, h->hy, nd * sizeof(double), cudaMemcpyDeviceToHost, s));
        CUDA_OR_FAIL(h, cudaStreamSynchronize(s));
        return PFF_OK;
    }
    CUDA_OR_FAIL(h, refresh_state(h));
    const int TZ = q1_cell_tile_z(), ncz = g.nc[2];
    int zc = (ncz + 7) / 8;                  // about 8 slabs, each a whole number of CTA tiles
    zc = ((zc + TZ - 1) / TZ) * TZ;
    const int S = (ncz + zc - 1) / zc;
    if (!h->cs_in) {
        CUDA_OR_FAIL(h, cudaStreamCreateWithFlags(&h->cs_in, cudaStreamNonBlocking));
        CUDA_OR_FAIL(h, cudaStreamCreateWithFlags(&h->cs_out, cudaStreamNonBlocking));
    }
    while ((int)h->slab_ev.size() < 2 * S + 1) {
        cudaEvent_t e;
        CUDA_OR_FAIL(h, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        h->slab_ev.push_back(e);
    }
    cudaEvent_t* ev_in = h->slab_ev.data() + 1;
    cudaEvent_t* ev_app = ev_in + S;
    const int64_t layer = (int64_t)g.nn[0] * g.nn[1];
    auto nodes = [&](int sl, int64_t& n0, int64_t& n1) {   // node layers [sl zc, (sl + 1) zc), the last to the top
        n0 = (int64_t)sl * zc * layer;
        n1 = sl + 1 < S ? (int64_t)(sl + 1) * zc * layer : nn;
    };
    // the copies start after the library's earlier work on hx and hy
    CUDA_OR_FAIL(h, cudaEventRecord(h->slab_ev[0], s));
    CUDA_OR_FAIL(h, cudaStreamWaitEvent(h->cs_in, h->slab_ev[0], 0));
    for (int sl = 0; sl < S; ++sl) {
        int64_t n0, n1;
        nodes(sl, n0, n1);
        for (int c = 0; c <= g.dim; ++c)
            CUDA_OR_FAIL(h, cudaMemcpyAsync(h->hx + c * nn + n0, x + c * nn + n0, (n1 - n0) * sizeof(double),
                                            cudaMemcpyHostToDevice, h->cs_in));
        CUDA_OR_FAIL(h, cudaEventRecord(ev_in[sl], h->cs_in));
    }
    // slab sl's cells reach the first node layer of slab sl + 1: apply slab sl once slab sl + 1 is
    // copied and preset
    for (int sl = 0; sl <= S; ++sl) {
        if (sl < S) {
            int64_t n0, n1;
            nodes(sl, n0, n1);
            CUDA_OR_FAIL(h, cudaStreamWaitEvent(s, ev_in[sl], 0));
            CUDA_OR_FAIL(h, launch_init_masked_nodes(g, L.mask, MASK_U_ALL, PHI_BITS_ALL, h->hx, h->hy, n0, n1, s));
        }
        if (sl >= 1) {
            const int a = sl - 1, k0 = a * zc, k1 = std::min(ncz, (a + 1) * zc);
            CUDA_OR_FAIL(h, launch_q1_apply64_slab(g, h->ph, L.qpd64, h->hx, h->hy, L.mask, PHI_BITS_ALL, k0, k1, s));
            CUDA_OR_FAIL(h, cudaEventRecord(ev_app[a], s));
        }
    }
    for (int sl = 0; sl < S; ++sl) {
        int64_t n0, n1;
        nodes(sl, n0, n1);
        CUDA_OR_FAIL(h, cudaStreamWaitEvent(h->cs_out, ev_app[sl], 0));
        for (int c = 0; c <= g.dim; ++c)
            CUDA_OR_FAIL(h, cudaMemcpyAsync(y + c * nn + n0, h->hy + c * nn + n0, (n1 - n0) * sizeof(double),
                                            cudaMemcpyDeviceToHost, h->cs_out));
    }
    CUDA_OR_FAIL(h, cudaStreamSynchronize(h->cs_out));
    CUDA_OR_FAIL(h, cudaStreamSynchronize(s));
    return PFF_OK;
}

extern "C" pff_status pff_diagonal(pff_hierarchy* h, int level, int precision, void* d) {
    if (!h) return PFF_EINVAL;
    const int l = resolve_level(h, level);
    REQUIRE(h, l >= 0 && l < h->L && d, PFF_EINVAL, "pff_diagonal: bad level or NULL");
    REQUIRE(h, precision == 32 || precision == 64, PFF_EINVAL, "precision must be 32 or 64");
    REQUIRE(h, h->has_state, PFF_ESTATE, "pff_diagonal before pff_set_state");
    if (precision == 64) CUDA_OR_FAIL(h, diagonal_level<double>(h, l, (double*)d));
    else CUDA_OR_FAIL(h, diagonal_level<float>(h, l, (float*)d));
    return PFF_OK;
}

extern "C" pff_status pff_level_state(const pff_hierarchy* h, int level, double* U, double* phi_tilde,
                                      uint8_t* mask) {
    if (!h) return PFF_EINVAL;
    const int l = resolve_level(h, level);
    if (l < 0 || l >= h->L) return PFF_EINVAL;
    const Level& L = h->lv[l];
    cudaError_t e = refresh_state(const_cast<pff_hierarchy*>(h));   // logically const: derived data only
    if (e == cudaSuccess && phi_tilde)
        e = cudaMemcpyAsync(phi_tilde, L.pt64, sizeof(double) * L.g.n_nodes, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess && U) e = cudaMemcpyAsync(U, L.U64, sizeof(double) * n_dofs(L.g), cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess && mask) e = cudaMemcpyAsync(mask, L.mask, L.g.n_nodes, cudaMemcpyDeviceToDevice, h->stream);
    return e == cudaSuccess ? PFF_OK : PFF_ECUDA;
}

extern "C" pff_status pff_restrict(pff_hierarchy* h, int fine_level, int precision, const void* r_fine,
                                   void* r_coarse) {
    if (!h) return PFF_EINVAL;
    const int l = resolve_level(h, fine_level);
    REQUIRE(h, l >= 1 && l < h->L && r_fine && r_coarse, PFF_EINVAL, "pff_restrict: bad level or NULL");
    REQUIRE(h, precision == 32 || precision == 64, PFF_EINVAL, "precision must be 32 or 64");
    Level& C = h->lv[l - 1];
    Level& F = h->lv[l];
    if (precision == 64)
        CUDA_OR_FAIL(h, launch_restrict<double>(C.g, F.g, (const double*)r_fine, (double*)r_coarse, C.mask, h->stream));
    else
        CUDA_OR_FAIL(h, launch_restrict<float>(C.g, F.g, (const float*)r_fine, (float*)r_coarse, C.mask, h->stream));
    return PFF_OK;
}

extern "C" pff_status pff_prolongate_add(pff_hierarchy* h, int fine_level, int precision, const void* e_coarse,
                                         void* x_fine) {
    if (!h) return PFF_EINVAL;
    const int l = resolve_level(h, fine_level);
    REQUIRE(h, l >= 1 && l < h->L && e_coarse && x_fine, PFF_EINVAL, "pff_prolongate_add: bad level or NULL");
    REQUIRE(h, precision == 32 || precision == 64, PFF_EINVAL, "precision must be 32 or 64");
    Level& C = h->lv[l - 1];
    Level& F = h->lv[l];
    if (precision == 64)
        CUDA_OR_FAIL(h, launch_prolongate_add<double>(C.g, F.g, (const double*)e_coarse, (double*)x_fine, F.mask,
                                                      h->stream));
    else
        CUDA_OR_FAIL(h, launch_prolongate_add<float>(C.g, F.g, (const float*)e_coarse, (float*)x_fine, F.mask,
                                                     h->stream));
    return PFF_OK;
}

static pff_status ensure_setup(pff_hierarchy* h) {
    REQUIRE(h, h->has_state, PFF_ESTATE, "preconditioner needs pff_set_state first");
    if (h->stale) CUDA_OR_FAIL(h, setup(h));
    return PFF_OK;
}

extern "C" pff_status pff_setup(pff_hierarchy* h) {
    if (!h) return PFF_EINVAL;
    REQUIRE(h, h->has_state, PFF_ESTATE, "pff_setup before pff_set_state");
    CUDA_OR_FAIL(h, setup(h));
    return PFF_OK;
}

extern "C" pff_status pff_eigen_estimates(pff_hierarchy* h, int level, double out[4]) {
    if (!h || !out) return PFF_EINVAL;
    const int l = resolve_level(h, level);
    REQUIRE(h, l >= 0 && l < h->L, PFF_EINVAL, "level out of range");
    pff_status st = ensure_setup(h);
    if (st != PFF_OK) return st;
    const Level& L = h->lv[l];
    out[0] = L.lam_min[0];
    out[1] = L.lam_max[0];
    out[2] = L.lam_min[1];
    out[3] = L.lam_max[1];
    return PFF_OK;
}

extern "C" pff_status pff_smooth(pff_hierarchy* h, int level, int precision, const void* b, void* x, int zero_guess) {
    if (!h) return PFF_EINVAL;
    const int l = resolve_level(h, level);
    REQUIRE(h, l >= 0 && l < h->L && b && x && b != x, PFF_EINVAL, "pff_smooth: bad level, NULL or aliased");
    REQUIRE(h, precision == 32 || precision == 64, PFF_EINVAL, "precision must be 32 or 64");
    pff_status st = ensure_setup(h);
    if (st != PFF_OK) return st;
    if (precision == 64) CUDA_OR_FAIL(h, smooth<double>(h, l, (const double*)b, (double*)x, zero_guess));
    else CUDA_OR_FAIL(h, smooth<float>(h, l, (const float*)b, (float*)x, zero_guess));
    return PFF_OK;
}

extern "C" pff_status pff_coarse_solve(pff_hierarchy* h, const double* b, double* x) {
    if (!h) return PFF_EINVAL;
    REQUIRE(h, b && x && b != x, PFF_EINVAL, "pff_coarse_solve: NULL or aliased");
    pff_status st = ensure_setup(h);
    if (st != PFF_OK) return st;
    CUDA_OR_FAIL(h, coarse_solve(h, b, x));
    return PFF_OK;
}

extern "C" pff_status pff_vcycle(pff_hierarchy* h, const double* r, double* z) {
    if (!h) return PFF_EINVAL;
    REQUIRE(h, r && z && r != z, PFF_EINVAL, "pff_vcycle: NULL or aliased");
    pff_status st = ensure_setup(h);
    if (st != PFF_OK) return st;
    CUDA_OR_FAIL(h, vcycle(h, r, z));
    return PFF_OK;
}

static pff_status ensure_krylov(pff_hierarchy* h, int m) {
    if (h->kr_m >= m) return PFF_OK;
    const size_t n = (size_t)n_dofs(h->lv[h->L - 1].g);
    CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
    if (h->kr_V) {   // release the old workspace
        for (void* p : {(void*)h->kr_V, (void*)h->kr_Z, (void*)h->kr_h}) {
            for (auto it = h->allocs.begin(); it != h->allocs.end(); ++it)
                if (*it == p) { cudaFree(p); h->allocs.erase(it); break; }
        }
        h->kr_V = h->kr_Z = h->kr_h = nullptr;
        h->kr_m = 0;
    }
    cudaError_t e = dalloc(h, &h->kr_V, (size_t)(m + 1) * n);
    if (e == cudaSuccess) e = dalloc(h, &h->kr_Z, (size_t)m * n);
    if (e == cudaSuccess) e = dalloc(h, &h->kr_h, (size_t)2 * (m + 1) + 2);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(h, e == cudaErrorMemoryAllocation ? PFF_ENOMEM : PFF_ECUDA, "Krylov workspace allocation failed");
    }
    h->kr_m = m;
    return PFF_OK;
}

extern "C" pff_status pff_gmres_solve(pff_hierarchy* h, const double* b, double* x, double rtol, int restart,
                                      int maxit, pff_solve_info* info) {
    if (!h) return PFF_EINVAL;
    REQUIRE(h, b && x && b != x, PFF_EINVAL, "pff_gmres_solve: NULL or aliased");
    REQUIRE(h, rtol > 0 && rtol < 1 && restart >= 1 && restart <= 1000 && maxit >= 1, PFF_EINVAL,
            "pff_gmres_solve: need 0 < rtol < 1, 1 <= restart <= 1000, maxit >= 1");
    pff_status st = ensure_setup(h);
    if (st != PFF_OK) return st;
    st = ensure_krylov(h, restart);
    if (st != PFF_OK) return st;
    std::string err;
    st = fgmres(h, b, x, rtol, restart, maxit, info, err);
    if (st != PFF_OK) h->err = err;
    return st;
}

pff_status pff_internal_ensure_krylov(pff_hierarchy* h, int m) { return ensure_krylov(h, m); }

// Algorithm 1 up to the linear solve: state U, residual, active set, eliminated right-hand side
// R~ in tmp64[1] and its norm.
pff_status pff_internal_newton_prepare(pff_hierarchy* h, double* U, int* n_act, int* n_chg, double* res) {
    REQUIRE(h, U, PFF_EINVAL, "pff_newton_step: NULL");
    REQUIRE(h, h->has_state, PFF_ESTATE, "pff_newton_step before pff_set_state");
    Level& F = h->lv[h->L - 1];
    const int64_t nd = n_dofs(F.g);
    cudaStream_t s = h->stream;
    // prescribed displacements: the iterate takes the boundary values, the increments vanish there
    if (h->has_udir) CUDA_OR_FAIL(h, launch_lift_dirichlet(F.g, h->dir_mask, h->udir, U, s));
    CUDA_OR_FAIL(h, cudaMemcpyAsync(F.U64, U, nd * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CUDA_OR_FAIL(h, propagate_state(h));
    pff_status st = update_active(h, n_act, n_chg);
    if (st != PFF_OK) return st;
    // eliminated right-hand side: active rows carry phi_old - phi, their columns move right
    double* Rt = h->tmp64[1];
    double* t = h->tmp64[2];
    CUDA_OR_FAIL(h, launch_active_delta(F.g, F.U64, h->phi_old, F.mask, Rt, s));
    CUDA_OR_FAIL(h, apply_level<double>(h, h->L - 1, OP_APPLY, Rt, t, PFF_MASK_PHI_DIR));
    CUDA_OR_FAIL(h, launch_newton_rhs(F.g, h->R, t, F.U64, h->phi_old, F.mask, Rt, s));
    CUDA_OR_FAIL(h, launch_norm2(nd, Rt, h->d_scratch, h->d_scal + 300, s));
    CUDA_OR_FAIL(h, cudaMemcpyAsync(res, h->d_scal + 300, sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_OR_FAIL(h, cudaStreamSynchronize(s));
    return PFF_OK;
}

// U += dU (tmp64[2]); the new U becomes the hierarchy's state.  The coarse levels and the
// Gauss-point data follow lazily (refresh_state), so that a following Newton step, which sets the
// state again, computes them once.
pff_status pff_internal_newton_finish(pff_hierarchy* h, double* U) {
    Level& F = h->lv[h->L - 1];
    const int64_t nd = n_dofs(F.g);
    CUDA_OR_FAIL(h, launch_axpby<double>(nd, 1.0, h->tmp64[2], 1.0, U, h->stream));
    CUDA_OR_FAIL(h, cudaMemcpyAsync(F.U64, U, nd * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    h->derived_dirty = true;
    h->stale = true;
    return PFF_OK;
}

extern "C" pff_status pff_newton_step(pff_hierarchy* h, double* U, pff_newton_info* info) {
    if (!h) return PFF_EINVAL;
    int n_act = 0, n_chg = 0;
    double res = 0.0;
    pff_status st = pff_internal_newton_prepare(h, U, &n_act, &n_chg, &res);
    if (st != PFF_OK) return st;
    Level& F = h->lv[h->L - 1];
    const int64_t nd = n_dofs(F.g);
    st = ensure_setup(h);
    if (st != PFF_OK) return st;
    st = ensure_krylov(h, 30);
    if (st != PFF_OK) return st;
    double* dU = h->tmp64[2];
    CUDA_OR_FAIL(h, cudaMemsetAsync(dU, 0, nd * sizeof(double), h->stream));
    pff_solve_info si;
    memset(&si, 0, sizeof(si));
    std::string err;
    st = fgmres(h, h->tmp64[1], dU, h->prm.newton_rtol, 30, 200, &si, err);
    if (st != PFF_OK && st != PFF_ENOCONV) {
        h->err = err;
        return st;
    }
    pff_status s2 = pff_internal_newton_finish(h, U);
    if (s2 != PFF_OK) return s2;
    CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
    if (info) {
        info->n_active = n_act;
        info->n_changed = n_chg;
        info->res_norm = res;
        info->solve = si;
        info->converged = (n_chg == 0 && res <= h->prm.tol_as) ? 1 : 0;
    }
    if (st == PFF_ENOCONV) h->err = err;
    return st;
}

extern "C" pff_status pff_load_step(pff_hierarchy* h, double* U, const double* phi_prev, double pressure,
                                    int max_newton, pff_load_info* info) {
    if (!h) return PFF_EINVAL;
    REQUIRE(h, U, PFF_EINVAL, "pff_load_step: NULL U");
    REQUIRE(h, max_newton >= 1, PFF_EINVAL, "pff_load_step: max_newton must be >= 1");
    REQUIRE(h, std::isfinite(pressure), PFF_EINVAL, "pff_load_step: non-finite pressure");
    Level& F = h->lv[h->L - 1];
    const int64_t nn = F.g.n_nodes;
    cudaStream_t s = h->stream;
    h->prm.pressure = pressure;
    h->ph = make_phys(h->prm);
    h->stale = true;
    CUDA_OR_FAIL(h, cudaMemcpyAsync(h->phi_old, U + (int64_t)F.g.dim * nn, nn * sizeof(double),
                                    cudaMemcpyDeviceToDevice, s));
    CUDA_OR_FAIL(h, launch_extrapolate(nn, h->phi_old, phi_prev, F.pt64, s));
    h->has_state = true;
    pff_load_info li;
    memset(&li, 0, sizeof(li));
    pff_status st = PFF_OK;
    for (int k = 0; k < max_newton; ++k) {
        pff_newton_info ni;
        memset(&ni, 0, sizeof(ni));
        st = pff_newton_step(h, U, &ni);
        if (st != PFF_OK && st != PFF_ENOCONV) break;
        li.newton_steps = k + 1;
        li.gmres_iterations += ni.solve.iterations;
        li.last = ni;
        if (ni.converged) {
            li.converged = 1;
            break;
        }
    }
    if (info) *info = li;
    return st;
}

extern "C" pff_status pff_profile(pff_hierarchy* h, int enable) {
    if (!h) return PFF_EINVAL;
    CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
    for (auto& v : h->prof) v.clear();
    h->ev_used = 0;
    h->prof_on = enable != 0;
    return PFF_OK;
}

extern "C" pff_status pff_profile_read(pff_hierarchy* h, int cls, int* count, double* total_ms) {
    if (!h || cls < 0 || cls >= PFF_PROF_NCLASS) return PFF_EINVAL;
    CUDA_OR_FAIL(h, cudaStreamSynchronize(h->stream));
    double tot = 0.0;
    for (auto& pr : h->prof[cls]) {
        float ms = 0.f;
        CUDA_OR_FAIL(h, cudaEventElapsedTime(&ms, pr.first, pr.second));
        tot += ms;
    }
    if (count) *count = (int)h->prof[cls].size();
    if (total_ms) *total_ms = tot;
    return PFF_OK;
}

extern "C" const char* pff_last_error(const pff_hierarchy* h) {
    if (!h) return "null hierarchy";
    return h->err.c_str();
}

#include <atomic>

namespace pff {
static std::atomic<long long> g_launches{0};
cudaError_t count_launch(cudaError_t e) {
    if (e == cudaSuccess) g_launches.fetch_add(1, std::memory_order_relaxed);
    return e;
}
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }
void add_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace pff

extern "C" long long pff_launch_count(void) { return pff::launch_count(); }
