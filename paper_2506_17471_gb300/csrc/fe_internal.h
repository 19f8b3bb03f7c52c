// Internal declarations shared by the library's translation units.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/feaction.h"

namespace fe {

// Number of P_p Lagrange nodes on a d-simplex: C(p + d, d).
__host__ __device__ constexpr int nloc(int d, int p)
{
    return d == 1 ? p + 1 : (d == 2 ? (p + 1) * (p + 2) / 2 : (p + 1) * (p + 2) * (p + 3) / 6);
}

// Arguments of every action kernel (passed by value; lives in the kernel's
// constant parameter bank).
struct ActionArgs {
    const double *coords;     // [n_vertices][D]
    const int32_t *c2v;       // [n_cells][D+1]
    const int32_t *c2n;       // [n_cells][N]
    const double *u;          // trial DoFs (du for the Jacobian action, w for the adjoint)
    const double *u_lin;      // linearisation point (Neo-Hookean Jacobian / adjoint)
    double *y;                // output DoFs (scatter-add target)
    const double *mu_cell;    // [n_cells] or nullptr
    const double *lam_cell;   // [n_cells] or nullptr
    double *dmu;              // adjoint outputs [n_cells] (nullptr otherwise)
    double *dlam;
    double mu, lam;           // constant Lame parameters
    const double *tab;        // device table block: tab [nq][1+D][N] then wts [nq], padded
    int32_t tab_doubles;      // doubles in the table block (multiple of 2)
    int32_t nq;
    int32_t n_cells, n_vertices, n_nodes;
    int32_t *status;          // device status word (first error wins)
    int32_t *sched;           // [2] work-queue counters: next chunk, warps finished (self-resetting)
    int32_t coop_n;           // cooperative kernel: local nodes per cell
    int32_t coop_cells;       // cooperative kernel: cells per batch (of one thread group)
    int32_t coop_groups;      // cooperative kernel: independent thread groups per CTA (0/1: one)
    const void *tab_b;        // cooperative kernel, large tables: [1+D][N][nq] in global memory
    const void *tab_c;        // cooperative kernel, large tables: [nq][1+D][N] in global memory
    int32_t tc_qc;            // tensor-core kernel: quadrature points per chunk
    int32_t tc_pipes;         // tensor-core kernel: 128-cell pipelines per CTA (1, 2 or 4)
    int32_t tc_wshift;        // tensor-core kernel: staged weights are w_q 2^tc_wshift
    // Node-gather scatter (FE_FLAG_GATHER_SCATTER): when non-null the action stores
    // each cell's outputs to cell_out[cell][j][comp] (float for FP32 contractions,
    // double otherwise) instead of adding them into y; skipped cells store zeros.
    void *cell_out;
    // Hyperelastic laws: table of the logarithm (fe_log in fe_kernels.cuh) in
    // global memory, or nullptr for CUDA's log and the IEEE division.
    const double *log_tab;
    // FP32 thread-per-cell kernels: shared-memory hash slots of the scatter
    // aggregation (0: scatter each cell's updates directly)
    int32_t agg_slots;
};

// Launch function of one compiled kernel variant.
using LaunchFn = cudaError_t (*)(const ActionArgs &, int grid, int block, size_t smem,
                                 cudaStream_t stream);

struct Variant {
    int form, dim, degree;
    int op;            // 0 = action, 1 = adjoint
    int precision;     // enum fe_precision of the contractions
    int kernel_id;     // fe_plan_info.kernel
    int block;         // threads per block
    LaunchFn launch;
    const void *func;  // kernel symbol (for occupancy queries)
    // FP32 thread-per-cell mass variants: the kernel that sums the updates of
    // nodes shared by a CTA's cells in shared memory before the global scatter
    // (launched instead of func when ActionArgs::agg_slots > 0)
    const void *func_agg = nullptr;
    // thread-per-cell FP64 linear forms: the kernel takes tables whose rows of
    // point q are scaled by sqrt(w_q) (the plan builds them so)
    bool wfold = false;
};

// Raise a kernel's dynamic shared-memory limit to the device's opt-in maximum.
// The limit is an attribute of the kernel function, shared by every plan that
// uses it, so it must never be lowered to one plan's need.
inline cudaError_t allow_max_dynamic_smem(const void *func)
{
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes attr;
    e = cudaFuncGetAttributes(&attr, func);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - (int)attr.sharedSizeBytes);
}

// Registry population, one per instantiation translation unit; each appends
// its variants to out[] and returns how many it wrote (at most cap).
int register_variants_2d_linear(Variant *out, int cap);
int register_variants_2d_nh(Variant *out, int cap);
int register_variants_3d(Variant *out, int cap);
int register_variants_fold(Variant *out, int cap);
int register_variants_coop(Variant *out, int cap);
int register_variants_tc(Variant *out, int cap);
int register_variants_tc2(Variant *out, int cap);
int register_variants_tc3(Variant *out, int cap);
int register_variants_forms(Variant *out, int cap);
int register_variants_coop_forms(Variant *out, int cap);

// True when every structural zero of the reference gradient tables (the
// entries the thread-per-cell contractions skip) holds exactly 0.0 in tab,
// laid out as fe_tabulate writes it: [(1+dim)][nq][n].
bool tab_zeros_hold(int dim, int n, int nq, const double *tab);

// The table of fe_log (fe_kernels.cuh), kLogTabDoubles doubles, from the C
// library's long double logarithm.
void fill_log_table(double *t);

}  // namespace fe

// The plan object behind the opaque C handle.
struct fe_plan {
    fe_form form;
    fe_mesh mesh;
    int nq, n_loc, ncomp;
    double *d_tab;        // device table block (cooperative kernel, large tables: then the
                          // phase-B and phase-C tables follow it in the same allocation)
    const void *d_tab_b;  // cooperative kernel, large tables (else nullptr)
    const void *d_tab_c;
    int tab_doubles;
    int32_t *d_status;    // device status word
    int32_t *d_sched;     // [4] work-queue counters: forward kernel [0..1], adjoint kernel [2..3]
    fe::Variant var;      // forward action kernel
    fe::Variant adj;      // adjoint kernel (launch == nullptr if none)
    int grid_blocks;
    int adj_grid_blocks;
    size_t smem_bytes;
    int coop_cells;       // cells per batch (cooperative kernel), else 0
    int coop_groups = 1;  // cooperative kernel: thread groups per CTA, each with its own batches
    int tc_qc;            // tensor-core kernel: quadrature points per chunk, else 0
    int tc_pipes;         // tensor-core kernel: 128-cell pipelines per CTA, else 0
    int tc_wshift;        // tensor-core kernel: staged weights are w_q 2^tc_wshift
    int device;
    double flops_per_cell;
    double flops_per_cell_dense;   // the same with every gradient-table entry counted
    double bytes_min;
    // fe_action_host_pipelined: two copy streams and, per buffer pair b, the
    // events h2d done, action done, d2h done (created on first use)
    // FE_FLAG_GATHER_SCATTER: per-cell outputs and the node -> (cell*n + j) incidences
    double *d_log_tab = nullptr;   // Neo-Hookean plans: the logarithm's table (fe_log)
    int agg_slots = 0;             // FP32 thread-per-cell: shared-memory scatter aggregation slots
    void *d_cell_out = nullptr;
    int32_t *d_node_ptr = nullptr;   // [n_nodes + 1]
    int32_t *d_node_inc = nullptr;   // [incidences]
    int cell_out_f32 = 0;
    cudaStream_t pipe_h2d = nullptr, pipe_d2h = nullptr;
    cudaEvent_t pipe_ev[6] = {};
    bool pipe_ready = false;
};
