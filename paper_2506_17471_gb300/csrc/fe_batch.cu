// Batched persistent action: many independent meshes of uneven size, degree and
// form in one persistent launch per device code.
//
// The host builds two work lists of items (problem, first cell), one per
// device code: tiles of 128 cells for the problems run by the thread-per-cell
// code, tiles of C cells for those run by the cooperative code, each list
// sorted so that the most expensive problems' items come first.  Each list is
// served by its own persistent kernel (128 threads per CTA and the registers of
// the thread-per-cell paths; 256 threads and the registers of the cooperative
// paths), so neither code runs with the other's occupancy.  A CTA pulls items
// from its list's counter and stages a problem's table block into shared memory
// only when the problem changes (one bulk async copy completing on an mbarrier
// whose phase it tracks; waits are bounded).  All outputs are zeroed by one
// multi-array kernel first; the two persistent kernels then run concurrently
// (the second on a batch-owned stream forked from and joined back to the
// caller's stream with events), and the whole can be captured in a CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "fe_coop.cuh"

namespace fe {

constexpr int kBatchBlock = 128;       // thread-per-cell code: one cell per thread
constexpr int kBatchCoopBlock = 256;   // cooperative code: the per-problem kernel's block

struct BatchProblemDev {
    ActionArgs a;        // pointers and sizes; a.tab points into the batch's table buffer
    int op, dim, degree;
    int kind;            // 0 thread-per-cell, 1 cooperative
    int coop_cells;      // cooperative tile (cells per item)
    int pad;
};

struct BatchItem {
    int problem;
    int cell0;
};

namespace {

// Bounded wait for the given mbarrier phase parity (all threads poll).
__device__ __forceinline__ bool wait_phase(uint32_t sbar, uint32_t parity)
{
    for (int it = 0; it < kWaitLimit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(sbar), "r"(parity)
            : "memory");
        if (ok) return true;
        __nanosleep(64);
    }
    return false;
}

template <int OP, int D>
__device__ __forceinline__ void run_tpc(const ActionArgs &a, int degree, const double *tab, const double *wts,
                                        int cell)
{
    const int nq = a.nq;
    const double *wts_r = wts + nq;
    (void)tab;
    // mass and elasticity take weight-folded tables (built so by fe_batch_create)
    constexpr bool WF = OP == OP_MASS || OP == OP_ELASTICITY;
    switch (degree) {
    case 1: action_cell<OP, D, 1, double, 0, WF>(a, tab, wts, wts_r, cell); break;
    case 2: action_cell<OP, D, 2, double, 0, WF>(a, tab, wts, wts_r, cell); break;
    case 3:
        if constexpr (D == 2 || OP == OP_MASS) action_cell<OP, D, 3, double, 0, WF>(a, tab, wts, wts_r, cell);
        break;
    case 4:
        if constexpr (D == 2 || OP == OP_MASS) action_cell<OP, D, 4, double, 0, WF>(a, tab, wts, wts_r, cell);
        break;
    default: break;
    }
}

template <int OP, int D>
__device__ __forceinline__ void run_coop(const BatchProblemDev &P, unsigned char *base, int cell0)
{
    constexpr int NC = OpTraits<OP, D>::NC;
    const CoopLayout L = coop_layout<double>(P.a.coop_n, P.a.nq, D, NC, P.coop_cells, 1, P.a.tab_b != nullptr);
    const CoopSmem<double> S = coop_smem<double>(base, L, P.a);
    if (L.C % 32 == 0) coop_node_order<D, double>(S, L.n, whole_cta());   // the node-major phase's order
    coop_batch<OP, D, double>(P.a, L, S, cell0, min(P.coop_cells, P.a.n_cells - cell0));
}

// CODE 0: items of thread-per-cell problems; CODE 1: items of cooperative problems.
template <int CODE>
__global__ void __launch_bounds__(CODE == 0 ? kBatchBlock : kBatchCoopBlock)
    k_action_batched(const BatchProblemDev *__restrict__ probs, const BatchItem *__restrict__ items, int n_items,
                     int32_t *sched, int32_t *status)
{
    extern __shared__ __align__(128) double smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_item;
    const uint32_t sbar = (uint32_t)__cvta_generic_to_shared(&bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sbar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    int staged = -1;
    uint32_t parity = 0;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(sched, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const BatchItem item = items[it];
        const BatchProblemDev &P = probs[item.problem];
        if (item.problem != staged) {
            // every thread has finished the previous item (barrier above)
            if (threadIdx.x == 0) {
                const uint32_t bytes = (uint32_t)P.a.tab_doubles * 8u;
                const uint32_t sdst = (uint32_t)__cvta_generic_to_shared(smem);
                const uint64_t gsrc = (uint64_t)__cvta_generic_to_global(P.a.tab);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sbar), "r"(bytes)
                             : "memory");
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        sdst),
                    "l"(gsrc), "r"(bytes), "r"(sbar)
                    : "memory");
            }
            const int ok = wait_phase(sbar, parity);
            if (!__syncthreads_and(ok)) {
                if (threadIdx.x == 0) set_status(status, FE_ERR_TIMEOUT);
                wait_phase(sbar, parity);   // let the copy land before the CTA leaves
                break;
            }
            parity ^= 1u;
            staged = item.problem;
        }
        unsigned char *base = reinterpret_cast<unsigned char *>(smem);
        if constexpr (CODE == 0) {
            const int cell = item.cell0 + (int)threadIdx.x;
            if (cell < P.a.n_cells) {
                const double *tab = smem;
                const int n = nloc(P.dim, P.degree);
                const double *wts = smem + (size_t)P.a.nq * (P.dim + 1) * n;
                if (P.dim == 2) {
                    if (P.op == OP_MASS) run_tpc<OP_MASS, 2>(P.a, P.degree, tab, wts, cell);
                    else if (P.op == OP_ELASTICITY) run_tpc<OP_ELASTICITY, 2>(P.a, P.degree, tab, wts, cell);
                    else run_tpc<OP_NH_RESIDUAL, 2>(P.a, P.degree, tab, wts, cell);
                } else {
                    if (P.op == OP_MASS) run_tpc<OP_MASS, 3>(P.a, P.degree, tab, wts, cell);
                    else if (P.op == OP_ELASTICITY) run_tpc<OP_ELASTICITY, 3>(P.a, P.degree, tab, wts, cell);
                    else run_tpc<OP_NH_RESIDUAL, 3>(P.a, P.degree, tab, wts, cell);
                }
            }
            __syncthreads();
        } else {
            if (P.dim == 2) {
                if (P.op == OP_MASS) run_coop<OP_MASS, 2>(P, base, item.cell0);
                else if (P.op == OP_ELASTICITY) run_coop<OP_ELASTICITY, 2>(P, base, item.cell0);
                else run_coop<OP_NH_RESIDUAL, 2>(P, base, item.cell0);
            } else {
                if (P.op == OP_MASS) run_coop<OP_MASS, 3>(P, base, item.cell0);
                else if (P.op == OP_ELASTICITY) run_coop<OP_ELASTICITY, 3>(P, base, item.cell0);
                else run_coop<OP_NH_RESIDUAL, 3>(P, base, item.cell0);
            }
        }
    }
    leave_queue(sched);
}

struct ZeroSpan {
    double *y;
    long long n;
};

__global__ void k_zero_many(const ZeroSpan *__restrict__ spans)
{
    const ZeroSpan s = spans[blockIdx.y];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < s.n;
         i += (long long)gridDim.x * blockDim.x)
        s.y[i] = 0.0;
}

bool tpc_available(int op, int dim, int degree)
{
    if (degree < 1 || degree > 4) return false;
    if (dim == 2) return op <= OP_NH_RESIDUAL;
    return op == OP_MASS || degree <= 2;
}

}  // namespace
}  // namespace fe

struct fe_batch {
    int count;
    fe::BatchProblemDev *d_probs = nullptr;
    fe::BatchItem *d_items = nullptr;
    fe::ZeroSpan *d_spans = nullptr;
    double *d_tables = nullptr;
    int32_t *d_words = nullptr;  // status [0]; queue counters: thread-per-cell [4..5], cooperative [6..7]
    int n_items = 0;
    int n_items_code[2] = {0, 0};   // items per device code (thread-per-cell first in d_items)
    int grid_code[2] = {0, 0};
    size_t smem_code[2] = {0, 0};
    cudaStream_t side = nullptr;    // the cooperative kernel's stream (forked from the caller's)
    cudaEvent_t fork = nullptr, join = nullptr;
    int grid = 0;
    size_t smem = 0;
    long long max_dofs = 0;
    double flops = 0.0;
    long long dofs = 0;
    std::vector<int> kinds, tiles;
};

namespace {

void batch_free(fe_batch *b)
{
    if (!b) return;
    cudaFree(b->d_probs);
    cudaFree(b->d_items);
    cudaFree(b->d_spans);
    cudaFree(b->d_tables);
    cudaFree(b->d_words);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->join) cudaEventDestroy(b->join);
    if (b->side) cudaStreamDestroy(b->side);
    delete b;
}

}  // namespace

extern "C" int fe_batch_create(const fe_batch_problem *problems, int count, fe_batch **out)
{
    using namespace fe;
    if (!problems || count < 1 || !out) return FE_ERR_INVALID_ARG;
    *out = nullptr;
    fe_batch *b = new (std::nothrow) fe_batch();
    if (!b) return FE_ERR_NO_MEMORY;
    b->count = count;
    std::vector<BatchProblemDev> probs(count);
    std::vector<std::vector<double>> blocks(count);
    std::vector<size_t> offsets(count);
    std::vector<double> cost(count);
    std::vector<ZeroSpan> spans(count);
    std::vector<size_t> staged_doubles(count), gsizes(count);
    std::vector<long long> global_off(count);
    size_t table_doubles = 0, smem = 0;
    for (int i = 0; i < count; ++i) {
        const fe_batch_problem &pb = problems[i];
        const fe_form &f = pb.form;
        const fe_mesh &m = pb.mesh;
        if (m.dim < 2 || m.dim > 3 || m.degree < 1 || m.n_cells < 0 || m.n_nodes < 0 || !pb.y ||
            (m.n_cells > 0 && (!m.coords || !m.cell2vertex || !m.cell2node || !pb.u)) ||
            f.precision != FE_PREC_FP64 || f.kind < FE_FORM_MASS || f.kind > FE_FORM_NH_RESIDUAL ||
            f.quad_degree < 0 || f.quad_degree > 40 || (f.flags & ~(uint32_t)FE_FLAG_TABLES_GLOBAL) ||
            (m.dim == 2 && reinterpret_cast<uintptr_t>(m.coords) % 16 != 0) ||
            (m.dim == 2 && f.kind != FE_FORM_MASS && reinterpret_cast<uintptr_t>(pb.u) % 16 != 0)) {
            batch_free(b);
            return FE_ERR_INVALID_ARG;
        }
        int nq = 0;
        if (fe_tabulate_scheme(m.dim, m.degree, f.quad_degree, f.quad_scheme, &nq, nullptr, nullptr, nullptr, 0) != FE_OK) {
            batch_free(b);
            return FE_ERR_INVALID_ARG;
        }
        const int n = nloc(m.dim, m.degree);
        const int ncomp = f.kind == FE_FORM_MASS ? 1 : m.dim;
        std::vector<double> pts((size_t)nq * m.dim), wts(nq), tab((size_t)(1 + m.dim) * nq * n);
        if (fe_tabulate_scheme(m.dim, m.degree, f.quad_degree, f.quad_scheme, &nq, pts.data(), wts.data(),
                               tab.data(), tab.size()) != FE_OK ||
            !tab_zeros_hold(m.dim, n, nq, tab.data())) {
            batch_free(b);
            return FE_ERR_INVALID_ARG;
        }
        int kind = pb.kernel;
        if (kind < 0) kind = tpc_available(f.kind, m.dim, m.degree) ? 0 : 1;
        if (kind == 0 && !tpc_available(f.kind, m.dim, m.degree)) {
            batch_free(b);
            return FE_ERR_UNSUPPORTED;
        }
        int C = 0;
        size_t rs, block_bytes, need;
        bool global_tab = false;
        if (kind == 1) {
            const bool gt = (f.flags & FE_FLAG_TABLES_GLOBAL) || coop_default_global<double>(n, nq, m.dim);
            // default tile: the largest that keeps two CTAs per SM, as for a single plan
            C = pb.tile_cells > 0 ? pb.tile_cells : coop_cells_for(n, nq, m.dim, ncomp, 1, sizeof(double), 100 * 1024, gt);
            const CoopLayout L = coop_layout<double>(n, nq, m.dim, ncomp, C, 1, gt);
            rs = L.rs;
            block_bytes = L.table_block_bytes;
            need = L.total;
            global_tab = L.global_tab != 0;
        } else {
            rs = (size_t)(1 + m.dim) * n;
            block_bytes = ((size_t)nq * rs * 8 + (size_t)nq * 16 + 15) & ~(size_t)15;
            need = block_bytes;
        }
        if (need > 200 * 1024) {
            batch_free(b);
            return FE_ERR_UNSUPPORTED;
        }
        smem = std::max(smem, need);
        b->smem_code[kind] = std::max(b->smem_code[kind], need);
        // staged block (table rows unless kept in global memory, then the weights
        // twice), followed for global-table problems by the phase-B [1+d][n][nq]
        // and phase-C [nq][1+d][n] tables; every piece an even number of doubles
        const size_t tdoubles = global_tab ? 0 : (size_t)nq * rs;
        const size_t gdoubles = global_tab ? (((size_t)(1 + m.dim) * n * nq + 1) & ~(size_t)1) : 0;
        std::vector<double> &blk = blocks[i];
        blk.assign(block_bytes / 8 + 2 * gdoubles, 0.0);
        // rows of point q scaled by sqrt(w_q) where the kernel expects it: the
        // cells-per-CTA linear forms (coop_weights_folded) and the thread-per-cell
        // mass and elasticity (run_tpc)
        const bool fold_w = (kind == 1 && (f.kind == FE_FORM_ELASTICITY || f.kind == FE_FORM_LAPLACE ||
                                           f.kind == FE_FORM_HELMHOLTZ || f.kind == FE_FORM_MASS)) ||
                            (kind == 0 && (f.kind == FE_FORM_ELASTICITY || f.kind == FE_FORM_MASS));
        for (int q = 0; q < nq; ++q)
            for (int k = 0; k <= m.dim; ++k)
                for (int j = 0; j < n; ++j) {
                    double t = tab[((size_t)k * nq + q) * n + j];
                    if (fold_w) t *= std::sqrt(wts[q]);
                    if (global_tab) {
                        blk[block_bytes / 8 + ((size_t)k * n + j) * nq + q] = t;
                        blk[block_bytes / 8 + gdoubles + ((size_t)q * (1 + m.dim) + k) * n + j] = t;
                    } else {
                        blk[(size_t)q * rs + (size_t)k * n + j] = t;
                    }
                }
        for (int q = 0; q < nq; ++q) {
            blk[tdoubles + q] = wts[q];
            blk[tdoubles + nq + q] = wts[q];
        }
        offsets[i] = table_doubles;
        table_doubles += blk.size();   // multiple of 2: every piece stays 16-byte aligned
        staged_doubles[i] = block_bytes / 8;
        global_off[i] = global_tab ? (long long)(block_bytes / 8) : -1;
        gsizes[i] = gdoubles;

        BatchProblemDev &P = probs[i];
        std::memset(&P, 0, sizeof(P));
        ActionArgs &a = P.a;
        a.coords = m.coords;
        a.c2v = m.cell2vertex;
        a.c2n = m.cell2node;
        a.u = pb.u;
        a.y = pb.y;
        a.mu_cell = f.mu_cell;
        a.lam_cell = f.lambda_cell;
        a.mu = f.mu;
        a.lam = f.lambda;
        a.tab_doubles = (int32_t)staged_doubles[i];
        a.nq = nq;
        a.n_cells = m.n_cells;
        a.n_vertices = m.n_vertices;
        a.n_nodes = m.n_nodes;
        a.coop_n = n;
        a.coop_cells = C;
        P.op = f.kind;
        P.dim = m.dim;
        P.degree = m.degree;
        P.kind = kind;
        P.coop_cells = C;
        b->kinds.push_back(kind);
        b->tiles.push_back(C);
        // algorithmic cost of the problem (flops of Algorithm 2), for ordering
        const double per_qp = (f.kind == FE_FORM_MASS) ? 4.0 * n : 4.0 * m.dim * m.dim * n;
        cost[i] = (double)m.n_cells * nq * per_qp;
        b->flops += cost[i];
        spans[i].y = pb.y;
        spans[i].n = (long long)m.n_nodes * ncomp;
        b->dofs += spans[i].n;
        b->max_dofs = std::max(b->max_dofs, spans[i].n);
    }
    // items: per device code, problems in decreasing cost, each problem's tiles in
    // order; the thread-per-cell list first, then the cooperative list
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    std::vector<BatchItem> items;
    for (int code = 0; code < 2; ++code)
        for (int i : order) {
            if (probs[i].kind != code) continue;
            const int tile = code == 0 ? kBatchBlock : probs[i].coop_cells;
            for (int c0 = 0; c0 < probs[i].a.n_cells; c0 += tile) items.push_back(BatchItem{i, c0});
            b->n_items_code[code] += (probs[i].a.n_cells + tile - 1) / tile;
        }
    b->n_items = (int)items.size();
    b->smem = smem;
    if (cudaMalloc(&b->d_tables, std::max<size_t>(table_doubles, 2) * 8) != cudaSuccess ||
        cudaMalloc(&b->d_probs, sizeof(BatchProblemDev) * count) != cudaSuccess ||
        cudaMalloc(&b->d_items, sizeof(BatchItem) * std::max<size_t>(items.size(), 1)) != cudaSuccess ||
        cudaMalloc(&b->d_spans, sizeof(ZeroSpan) * count) != cudaSuccess ||
        cudaMalloc(&b->d_words, 8 * sizeof(int32_t)) != cudaSuccess) {
        cudaGetLastError();
        batch_free(b);
        return FE_ERR_NO_MEMORY;
    }
    for (int i = 0; i < count; ++i) {
        probs[i].a.tab = b->d_tables + offsets[i];
        if (global_off[i] >= 0) {
            probs[i].a.tab_b = b->d_tables + offsets[i] + global_off[i];
            probs[i].a.tab_c = b->d_tables + offsets[i] + global_off[i] + gsizes[i];
        }
        probs[i].a.status = b->d_words;
        probs[i].a.sched = nullptr;   // the batched kernel uses the batch's queue
        if (cudaMemcpy(b->d_tables + offsets[i], blocks[i].data(), blocks[i].size() * 8, cudaMemcpyHostToDevice) !=
            cudaSuccess) {
            batch_free(b);
            return FE_ERR_CUDA;
        }
    }
    if (cudaMemcpy(b->d_probs, probs.data(), sizeof(BatchProblemDev) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
        (!items.empty() && cudaMemcpy(b->d_items, items.data(), sizeof(BatchItem) * items.size(),
                                      cudaMemcpyHostToDevice) != cudaSuccess) ||
        cudaMemcpy(b->d_spans, spans.data(), sizeof(ZeroSpan) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(b->d_words, 0, 8 * sizeof(int32_t)) != cudaSuccess ||
        allow_max_dynamic_smem(reinterpret_cast<const void *>(k_action_batched<0>)) != cudaSuccess ||
        allow_max_dynamic_smem(reinterpret_cast<const void *>(k_action_batched<1>)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming) != cudaSuccess) {
        batch_free(b);
        return FE_ERR_CUDA;
    }
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const void *fn[2] = {reinterpret_cast<const void *>(k_action_batched<0>),
                         reinterpret_cast<const void *>(k_action_batched<1>)};
    const int block[2] = {kBatchBlock, kBatchCoopBlock};
    b->grid = 0;
    for (int code = 0; code < 2; ++code) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn[code], block[code], b->smem_code[code]) !=
                cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        b->grid_code[code] = std::max(0, std::min(per_sm * std::max(sms, 1), b->n_items_code[code]));
        b->grid += b->grid_code[code];
    }
    *out = b;
    return FE_OK;
}

extern "C" int fe_batch_run(fe_batch *b, void *stream)
{
    using namespace fe;
    if (!b) return FE_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    long long gx = (b->max_dofs + 255) / 256;
    gx = std::max(1ll, std::min(gx, 256ll));
    k_zero_many<<<dim3((unsigned)gx, (unsigned)b->count), 256, 0, s>>>(b->d_spans);
    if (cudaGetLastError() != cudaSuccess) return FE_ERR_CUDA;
    const int n0 = b->n_items_code[0], n1 = b->n_items_code[1];
    const bool both = n0 > 0 && n1 > 0;
    // the cooperative kernel runs on the side stream, forked after the zero kernel
    if (both && (cudaEventRecord(b->fork, s) != cudaSuccess || cudaStreamWaitEvent(b->side, b->fork, 0) != cudaSuccess))
        return FE_ERR_CUDA;
    if (n1 > 0) {
        k_action_batched<1><<<b->grid_code[1], kBatchCoopBlock, b->smem_code[1], both ? b->side : s>>>(
            b->d_probs, b->d_items + n0, n1, b->d_words + 6, b->d_words);
        if (cudaGetLastError() != cudaSuccess) return FE_ERR_CUDA;
    }
    if (n0 > 0) {
        k_action_batched<0><<<b->grid_code[0], kBatchBlock, b->smem_code[0], s>>>(b->d_probs, b->d_items, n0,
                                                                                  b->d_words + 4, b->d_words);
        if (cudaGetLastError() != cudaSuccess) return FE_ERR_CUDA;
    }
    if (both && (cudaEventRecord(b->join, b->side) != cudaSuccess || cudaStreamWaitEvent(s, b->join, 0) != cudaSuccess))
        return FE_ERR_CUDA;
    return FE_OK;
}

extern "C" int fe_batch_status(fe_batch *b, int *device_status)
{
    if (!b || !device_status) return FE_ERR_INVALID_ARG;
    int32_t w[8] = {0};
    if (cudaDeviceSynchronize() != cudaSuccess) return FE_ERR_CUDA;
    if (cudaMemcpy(w, b->d_words, sizeof(w), cudaMemcpyDeviceToHost) != cudaSuccess) return FE_ERR_CUDA;
    int32_t st = w[0];
    if ((w[4] || w[5] || w[6] || w[7]) && st == FE_OK) st = FE_ERR_CUDA;
    if (cudaMemset(b->d_words, 0, sizeof(w)) != cudaSuccess) return FE_ERR_CUDA;
    *device_status = st;
    return FE_OK;
}

extern "C" int fe_batch_get_info(const fe_batch *b, fe_batch_info *info)
{
    if (!b || !info) return FE_ERR_INVALID_ARG;
    info->problems = b->count;
    info->items = b->n_items;
    info->grid_blocks = b->grid;
    info->smem_bytes = (int64_t)b->smem;
    info->dofs = b->dofs;
    info->contraction_flops = b->flops;
    return FE_OK;
}

extern "C" int fe_batch_destroy(fe_batch *b)
{
    if (!b) return FE_OK;
    cudaDeviceSynchronize();
    batch_free(b);
    return FE_OK;
}
