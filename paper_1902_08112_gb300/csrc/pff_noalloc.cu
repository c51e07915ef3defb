// Allocation-free variant of the active-set decision (step 3 of Algorithm 1) for callers that
// cannot allocate device memory: e.g. a host process whose GPU memory is owned by another
// allocator or pool, or code that is not allowed to call cudaMalloc at all and therefore cannot
// create a pff_hierarchy.  It runs on caller-owned buffers only; its one scratch buffer, the
// per-CTA partial counts of the deterministic count reduction, is the file-scope device array
// below, which every GPU that loads this library holds until the process exits.
#include <mutex>

#include "pff_internal.cuh"

namespace {

// One CTA per kNoAllocNodesPerCta nodes, at most kNoAllocMaxCtas CTAs: the largest fine mesh
// this entry point accepts has kNoAllocMaxCtas * kNoAllocNodesPerCta nodes (67,108,864).
constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocNodesPerCta = 1024;
constexpr int kNoAllocMaxCtas = 65536;

// [2 * cta + 0] = active nodes counted by CTA cta, [2 * cta + 1] = changed nodes,
// [2 * kNoAllocMaxCtas + 0/1] = totals.  Every slot a call reads is written earlier in the same
// call, so nothing has to start at zero; calls that overlap on the GPU share it and race.
static __device__ __align__(256) int g_noalloc_counts[2 * kNoAllocMaxCtas + 2];

std::mutex g_noalloc_mutex;
int* g_noalloc_ptr[128] = {nullptr};   // device address of the array, per device ordinal

// Gauss-Lobatto lumped mass of one node on a uniform tensor grid: the sum over the node's cells in
// the domain (cm == nullptr: every cell) of the cell's tensor weight (Q1: h/2 per axis; Q2: h/6 at
// cell vertices, 2h/3 at midpoints), in the summation order of the library's lumped-mass kernel so
// that both give the same bits.  0 for a node on no domain cell.
__device__ __forceinline__ double lumped_mass_node(const pff::Geom& g, const uint8_t* __restrict__ cm, int64_t n) {
    int idx[3];
    idx[0] = (int)(n % g.nn[0]);
    const int64_t r = n / g.nn[0];
    idx[1] = (int)(r % g.nn[1]);
    idx[2] = (int)(r / g.nn[1]);
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int a = 0; a < g.dim; ++a) {
        lo[a] = idx[a] >= g.deg ? (idx[a] - 1) / g.deg : 0;
        hi[a] = min(g.nc[a] - 1, idx[a] / g.deg);
    }
    double w = 0.0;
    for (int ck = lo[2]; ck <= hi[2]; ++ck)
        for (int cj = lo[1]; cj <= hi[1]; ++cj)
            for (int ci = lo[0]; ci <= hi[0]; ++ci) {
                const int64_t cell = (int64_t)ci + (int64_t)g.nc[0] * ((int64_t)cj + (int64_t)g.nc[1] * ck);
                if (cm && cm[cell] == 0) continue;
                const int c3[3] = {ci, cj, ck};
                double wc = 1.0;
                for (int a = 0; a < g.dim; ++a) {
                    const int loc = idx[a] - g.deg * c3[a];
                    const double wa = g.deg == 1 ? 0.5 : (loc == 1 ? 2.0 / 3.0 : 1.0 / 6.0);
                    wc *= wa * g.h[a];
                }
                w += wc;
            }
    return w;
}

__global__ void k_active_set_noalloc(pff::Geom g, const uint8_t* __restrict__ cm, const double* __restrict__ R,
                                     const double* __restrict__ U, const double* __restrict__ phi_old, double c,
                                     double thr, int tie_scale, uint8_t* __restrict__ mask, int* __restrict__ counts) {
    const int64_t nn = g.n_nodes;
    const int64_t base = (int64_t)blockIdx.x * kNoAllocNodesPerCta;
    int na = 0, nch = 0;
    for (int k = threadIdx.x; k < kNoAllocNodesPerCta; k += blockDim.x) {
        const int64_t n = base + k;
        if (n >= nn) break;
        const uint8_t m = mask[n];
        // prescribed phi (phi Dirichlet bit, nodes on no domain cell) never enters the active set
        const double M = lumped_mass_node(g, cm, n);
        const bool fixed = (m & PFF_MASK_PHI_DIR) != 0 || !(M > 0.0);
        const double lam = fixed ? 0.0 : R[g.dim * nn + n] / M;
        const double v = lam + c * (U[g.dim * nn + n] - phi_old[n]);
        const bool act = !fixed && (tie_scale ? v * M : v) > thr;
        const bool was = (m & PFF_MASK_ACTIVE) != 0;
        mask[n] = (uint8_t)((m & ~PFF_MASK_ACTIVE) | (act ? PFF_MASK_ACTIVE : 0));
        na += act;
        nch += act != was;
    }
    __shared__ int sa[kNoAllocThreads / 32], sc[kNoAllocThreads / 32];
    for (int o = 16; o > 0; o >>= 1) {
        na += __shfl_xor_sync(0xffffffffu, na, o);
        nch += __shfl_xor_sync(0xffffffffu, nch, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { sa[w] = na; sc[w] = nch; }
    __syncthreads();
    if (threadIdx.x == 0) {
        int ta = 0, tc = 0;
        for (int i = 0; i < kNoAllocThreads / 32; ++i) { ta += sa[i]; tc += sc[i]; }
        counts[2 * blockIdx.x] = ta;
        counts[2 * blockIdx.x + 1] = tc;
    }
}

// Sums the per-CTA counts in a fixed order into the two total slots.
__global__ void k_sum_counts_noalloc(int* __restrict__ counts, int nctas) {
    __shared__ long long sa[kNoAllocThreads], sc[kNoAllocThreads];
    long long a = 0, c = 0;
    for (int i = threadIdx.x; i < nctas; i += blockDim.x) { a += counts[2 * i]; c += counts[2 * i + 1]; }
    sa[threadIdx.x] = a;
    sc[threadIdx.x] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long ta = 0, tc = 0;
        for (int i = 0; i < (int)blockDim.x; ++i) { ta += sa[i]; tc += sc[i]; }
        counts[2 * kNoAllocMaxCtas] = (int)ta;
        counts[2 * kNoAllocMaxCtas + 1] = (int)tc;
    }
}

}  // namespace

extern "C" pff_status pff_active_set_noalloc(const pff_mesh* mesh, const pff_params* params, const uint8_t* cell_mask,
                                             const double* R, const double* U, const double* phi_old, uint8_t* mask,
                                             int* n_active, int* n_changed, void* cuda_stream) {
    if (!mesh || !params || !R || !U || !phi_old || !mask) return PFF_EINVAL;
    // a cut domain needs its cell mask in device memory: the host copy in the mesh cannot be read
    // by the kernel, and copying it would need a device allocation
    if (mesh->cell_mask && !cell_mask) return PFF_EINVAL;
    if (mesh->dim != 2 && mesh->dim != 3) return PFF_EINVAL;
    if (mesh->degree != 1 && mesh->degree != 2) return PFF_EINVAL;
    pff::Geom g;
    g.es = nullptr;
    g.cm = nullptr;
    g.dim = mesh->dim;
    g.deg = mesh->degree;
    g.n_nodes = 1;
    g.n_cells = 1;
    for (int a = 0; a < 3; ++a) {
        if (a < mesh->dim) {
            if (mesh->n_cells[a] < 1 || !(mesh->hi[a] > mesh->lo[a])) return PFF_EINVAL;
            g.nc[a] = mesh->n_cells[a];
            g.nn[a] = g.deg * g.nc[a] + 1;
            g.h[a] = (mesh->hi[a] - mesh->lo[a]) / g.nc[a];
        } else {
            g.nc[a] = 1;
            g.nn[a] = 1;
            g.h[a] = 1.0;
        }
        g.n_nodes *= g.nn[a];
        g.n_cells *= g.nc[a];
    }
    const int64_t nctas = (g.n_nodes + kNoAllocNodesPerCta - 1) / kNoAllocNodesPerCta;
    if (nctas > kNoAllocMaxCtas) return PFF_EINVAL;   // more nodes than the scratch array covers
    // one-time set-up per device: the device address of the scratch array
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return PFF_ECUDA;
    int* counts = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_counts) != cudaSuccess || !p) return PFF_ECUDA;
            g_noalloc_ptr[dev] = reinterpret_cast<int*>(p);
        }
        counts = g_noalloc_ptr[dev];
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    k_active_set_noalloc<<<(unsigned)nctas, kNoAllocThreads, 0, s>>>(g, cell_mask, R, U, phi_old, params->c_as,
                                                                      params->tol_as, params->tie_scale, mask, counts);
    if (cudaGetLastError() != cudaSuccess) return PFF_ECUDA;
    k_sum_counts_noalloc<<<1, kNoAllocThreads, 0, s>>>(counts, (int)nctas);
    if (cudaGetLastError() != cudaSuccess) return PFF_ECUDA;
    int tot[2] = {0, 0};
    if (cudaMemcpyAsync(tot, counts + 2 * kNoAllocMaxCtas, sizeof(tot), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return PFF_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return PFF_ECUDA;
    if (n_active) *n_active = tot[0];
    if (n_changed) *n_changed = tot[1];
    return PFF_OK;
}
