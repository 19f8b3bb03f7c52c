// fe_action_noalloc: the thread-per-cell action for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc: applications whose device memory is
// reserved up front by their own pool allocator, hosts that forbid further
// device allocations after start-up, or code paths where the implicit device
// synchronisation and the failure modes of cudaMalloc are not acceptable.  For
// them this entry point runs the same kernel as fe_action without a plan: the
// scratch the kernel needs (the tabulation block, the work-queue counters and
// the status word) lives in the file-scope device array below, which every GPU
// that loads the library holds until the process exits.  The caller passes the
// inputs (the host tabulation written by fe_tabulate, the mesh, u) and the
// output y.
//
// Every call shares the array and it keeps the last call's contents; each call
// clears the counters and the status word before it launches.  Calls whose GPU
// work overlaps in time (different streams without ordering, or several host
// threads) race on the array and must be avoided.
#include <mutex>

#include "fe_internal.h"

namespace fe {
namespace {

// Scratch layout: bytes [0, 256): status word (int32 at 0), work-queue counters
// (int32 at 16 and 20); bytes [256, 256 + kNoallocTableBytes): table block.
constexpr size_t kNoallocHeaderBytes = 256;
constexpr size_t kNoallocTableBytes = (size_t)FE_NOALLOC_TABLE_DOUBLES * sizeof(double);
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocHeaderBytes + kNoallocTableBytes];

constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_setup_mutex;

constexpr int kMaxVariants = 128;
Variant g_na_variants[kMaxVariants];
int g_na_nvariants = 0;
std::once_flag g_na_once;

void init_noalloc_registry()
{
    int n = 0;
    n += register_variants_2d_linear(g_na_variants + n, kMaxVariants - n);
    n += register_variants_2d_nh(g_na_variants + n, kMaxVariants - n);
    n += register_variants_3d(g_na_variants + n, kMaxVariants - n);
    g_na_nvariants = n;
}

const Variant *noalloc_variant(int form, int dim, int degree)
{
    std::call_once(g_na_once, init_noalloc_registry);
    for (int i = 0; i < g_na_nvariants; ++i) {
        const Variant &v = g_na_variants[i];
        if (v.form == form && v.dim == dim && v.degree == degree && v.op == 0 && v.precision == FE_PREC_FP64)
            return &v;
    }
    return nullptr;
}

// Per-device set-up, done by the first call on each device with that device
// current: the host code needs the device address of the scratch array (its
// name in host code is only a host-side stand-in).
int scratch_address(int dev, void **out)
{
    if (dev < 0 || dev >= kMaxDevices) return FE_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return FE_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return FE_OK;
}

}  // namespace
}  // namespace fe

using namespace fe;

extern "C" int fe_action_noalloc(const fe_form *form, const fe_mesh *mesh, const double *tab_host,
                                 const double *wts_host, int nq, const double *u, double *y,
                                 int *device_status, void *stream)
{
    if (!form || !mesh || !tab_host || !wts_host || !y || nq < 1) return FE_ERR_INVALID_ARG;
    const fe_mesh &m = *mesh;
    const fe_form &f = *form;
    if (m.dim < 2 || m.dim > 3 || m.degree < 1 || m.n_cells < 0 || m.n_vertices < 0 || m.n_nodes < 0)
        return FE_ERR_INVALID_ARG;
    if (m.n_cells > 0 && (!m.coords || !m.cell2vertex || !m.cell2node)) return FE_ERR_INVALID_ARG;
    if (m.dim == 2 && reinterpret_cast<uintptr_t>(m.coords) % 16 != 0) return FE_ERR_INVALID_ARG;
    if (f.kind < FE_FORM_MASS || f.kind > FE_FORM_NH_JACOBIAN) return FE_ERR_INVALID_ARG;
    if (f.precision != FE_PREC_FP64) return FE_ERR_UNSUPPORTED;
    // Only the plain atomic-scatter kernel runs here: the other plan options
    // (cells-per-CTA kernel, global tables, node-ordered scatter, block size)
    // would need plan-owned memory or another kernel, so asking for them is an
    // error rather than a silent fallback.
    if ((f.flags & ~FE_FLAG_ACCUMULATE) != 0 || f.tile_cells != 0) return FE_ERR_UNSUPPORTED;
    if (f.kind == FE_FORM_NH_JACOBIAN && !f.u_lin) return FE_ERR_INVALID_ARG;
    const int ncomp = f.kind == FE_FORM_MASS ? 1 : m.dim;
    const long long n_dofs = (long long)m.n_nodes * ncomp;
    if (n_dofs >= (1ll << 31)) return FE_ERR_INVALID_ARG;
    if (n_dofs > 0 && !u) return FE_ERR_INVALID_ARG;
    if (u == y && n_dofs > 0) return FE_ERR_INVALID_ARG;
    if (ncomp == 2 && (reinterpret_cast<uintptr_t>(u) % 16 != 0 ||
                       (f.u_lin && reinterpret_cast<uintptr_t>(f.u_lin) % 16 != 0)))
        return FE_ERR_INVALID_ARG;
    const Variant *v = noalloc_variant(f.kind, m.dim, m.degree);
    if (!v) return FE_ERR_UNSUPPORTED;

    const int n = nloc(m.dim, m.degree);
    long long tab_doubles = (long long)nq * (1 + m.dim) * n + 2ll * nq;  // table, weights twice
    tab_doubles = (tab_doubles + 1) & ~1ll;
    if (tab_doubles > FE_NOALLOC_TABLE_DOUBLES) return FE_ERR_INVALID_ARG;  // beyond the scratch
    if (!tab_zeros_hold(m.dim, n, nq, tab_host)) return FE_ERR_INVALID_ARG;  // not fe_tabulate's table
    const size_t smem = (size_t)tab_doubles * sizeof(double);

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FE_ERR_CUDA;
    void *base = nullptr;
    int rc = scratch_address(dev, &base);
    if (rc != FE_OK) return rc;
    unsigned char *scratch = static_cast<unsigned char *>(base);
    int32_t *status = reinterpret_cast<int32_t *>(scratch);
    int32_t *sched = reinterpret_cast<int32_t *>(scratch + 16);
    double *table = reinterpret_cast<double *>(scratch + kNoallocHeaderBytes);
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    // Clear the status word and the queue counters (the array keeps the last
    // call's contents), then lay the caller's [1+d][nq][n] table out as the
    // kernel's [nq][1+d][n] block followed by the weights (twice: the kernel
    // reads one copy in FP64 and one in its contraction type, here also FP64).
    if (cudaMemsetAsync(scratch, 0, kNoallocHeaderBytes, s) != cudaSuccess) return FE_ERR_CUDA;
    for (int k = 0; k <= m.dim; ++k) {
        if (cudaMemcpy2DAsync(table + (size_t)k * n, (size_t)(1 + m.dim) * n * sizeof(double),
                              tab_host + (size_t)k * nq * n, (size_t)n * sizeof(double),
                              (size_t)n * sizeof(double), (size_t)nq, cudaMemcpyHostToDevice,
                              s) != cudaSuccess)
            return FE_ERR_CUDA;
    }
    for (int copy = 0; copy < 2; ++copy) {
        if (cudaMemcpyAsync(table + (size_t)nq * (1 + m.dim) * n + (size_t)copy * nq, wts_host,
                            (size_t)nq * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess)
            return FE_ERR_CUDA;
    }
    // From page-locked host memory these copies run asynchronously and would
    // still read tab_host / wts_host after the call returns; waiting for them
    // here lets the caller reuse or free the tables as soon as the call returns,
    // whatever kind of host memory holds them.
    if (cudaStreamSynchronize(s) != cudaSuccess) return FE_ERR_CUDA;

    if (!(f.flags & FE_FLAG_ACCUMULATE) && n_dofs > 0) {
        if (cudaMemsetAsync(y, 0, (size_t)n_dofs * sizeof(double), s) != cudaSuccess) return FE_ERR_CUDA;
    }
    if (m.n_cells > 0) {
        if (allow_max_dynamic_smem(v->func) != cudaSuccess) return FE_ERR_CUDA;
        int per_sm = 0, sms = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, v->func, v->block, smem) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
        const long long want = ((long long)m.n_cells + v->block - 1) / v->block;
        const long long full = (long long)per_sm * sms;
        const int grid = (int)(want < full ? want : full);

        ActionArgs a{};
        a.coords = m.coords;
        a.c2v = m.cell2vertex;
        a.c2n = m.cell2node;
        a.u = u;
        a.u_lin = f.u_lin;
        a.y = y;
        a.mu_cell = f.mu_cell;
        a.lam_cell = f.lambda_cell;
        a.mu = f.mu;
        a.lam = f.lambda;
        a.tab = table;
        a.tab_doubles = (int32_t)tab_doubles;
        a.nq = nq;
        a.n_cells = m.n_cells;
        a.n_vertices = m.n_vertices;
        a.n_nodes = m.n_nodes;
        a.status = status;
        a.sched = sched;
        if (v->launch(a, grid, v->block, smem, s) != cudaSuccess) return FE_ERR_CUDA;
    }
    if (device_status) {
        int32_t st = 0;
        if (cudaMemcpyAsync(&st, status, sizeof(st), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return FE_ERR_CUDA;
        *device_status = st;
    }
    return FE_OK;
}
