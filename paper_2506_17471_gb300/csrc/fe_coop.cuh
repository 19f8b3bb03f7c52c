// Cooperative (cells-per-CTA) action kernel for high-degree elements.
//
// Thread-per-cell keeps a cell's DoFs and outputs in registers; from about 60
// doubles of per-cell state upwards (Neo-Hookean Jacobian P6 in 2D,
// elasticity P3+ in 3D) that spills.  This kernel splits Algorithm 2's phases
// across the threads of a CTA instead, for a batch of C cells at a time (the
// role of the paper's multi-level tiling with N_c cells per work-group, Sec.
// "Multi-level Tiling"; here the whole tabulation fits in shared memory, so the
// tables are not tiled):
//   A  gather: nodes, vertex coordinates and DoFs of the batch into shared
//      memory; one thread per cell forms J^{-1}, |det J| (FP64);
//   B  evaluation + pointwise: one thread per (cell, quadrature point) computes
//      the reference gradients from the shared DoFs, maps them, evaluates the
//      pointwise form and writes e[c][q][k][comp] to shared memory;
//   C  quadrature + scatter: one thread per (cell, node) contracts e with the
//      test tabulation and scatter-adds its components with FP64 atomics.
// The degree and the rule are runtime values, so one instantiation per
// (operation, dimension, contraction type) serves every degree.
// Shared-memory strides are odd (in 8-byte words for double, 4-byte for float)
// so that threads reading consecutive quadrature points or cells hit distinct
// banks.  Tables larger than kCoopSmemTableBytes stay in global memory (L2/L1
// resident) in two layouts, [1+D][N][nq] for phase B (consecutive threads read
// consecutive quadrature points) and [nq][1+D][N] for phase C (consecutive
// nodes), so shared memory holds only the batch scratch and the weights.
// The FP64 kernel of the tetrahedral gradient forms runs the wide layout (below)
// as two independent 256-thread groups per CTA; it hands out the last, partial
// round of batches split by ranges of quadrature points (k_action_coop), and the
// FP64 linear forms take tables with the quadrature weights folded in
// (coop_weights_folded).
#pragma once

#include "fe_kernels.cuh"

namespace fe {

constexpr int kCoopBlock = 256;
// Wide layout of the FP64 kernel: one CTA of 512 threads per SM with a batch of
// C = 64 (or 32) cells, a multiple of the warp size, so that in phase C every
// warp works on one local node for 32 cells and can leave out that node's
// structurally zero derivative directions without diverging.
constexpr int kCoopWideBlock = 512;
constexpr int kCoopMaxGroups = 2;   // thread groups of the wide layout (see CtaGroup)
constexpr size_t kCoopWideSmemBytes = 224 * 1024;
constexpr size_t kCoopSmemTableBytes = 96 * 1024;   // larger tables stay in global memory
// Per-cell geometry record in shared memory: J^{-1} (D*D), |det J|, mu, lambda,
// a validity flag, and for FP64 linear elasticity 2 mu |det J|, lambda |det J|,
// mu |det J|; the stride is odd so that threads reading the records of
// consecutive cells hit distinct banks.
constexpr int kCoopGeoStride = 17;

// The FP64 linear forms (elasticity, Laplacian, Helmholtz, mass) in the
// cells-per-CTA kernel take their tables with the quadrature weights folded in,
// every row of point q scaled by sqrt(w_q) (the plan and the batch build them
// so): the evaluation then yields sqrt(w_q) times the values and reference
// gradients, the pointwise form is linear in them, and the quadrature
// contraction with the same table supplies the other sqrt(w_q), so the action is
// unchanged while the per-point weight products drop out of the FP64 work.  The
// Laplacian and Helmholtz forms keep M = |det J| J^{-1} J^{-T} in the geometry
// record in place of J^{-1}: their gradient term is then M times the reference
// gradient.
template <int OP, typename R>
__host__ __device__ constexpr bool coop_weights_folded()
{
    return (OP == OP_ELASTICITY || OP == OP_LAPLACE || OP == OP_HELMHOLTZ || OP == OP_MASS) &&
           sizeof(R) == sizeof(double);
}

// Shared-memory plan of one CTA, computed identically on host and device.
struct CoopLayout {
    int n, nq, D, NC, C, fields;
    int global_tab;   // 1: the tables stay in global memory (only the weights are staged)
    int rs;        // table row stride per quadrature point (elements), odd
    int ls;        // per-cell DoF stride (doubles), odd
    int es;        // per-(cell, q) stride of e (elements), odd
    int ecs;       // per-cell stride of e (elements), odd: threads of a warp that read
                   // the same (q, k) entry of 32 consecutive cells hit distinct banks
    size_t tab_bytes, wts_off, wtsr_off, table_block_bytes;   // the staged table block
    size_t off_l, off_e, off_nodes, off_geo, off_acc, off_order, total;
};

// Default table residency of the cells-per-CTA kernel: shared memory unless the
// table is larger than kCoopSmemTableBytes (a plan may also ask for global).
template <typename R>
__host__ __device__ inline bool coop_default_global(int n, int nq, int D)
{
    return (size_t)nq * (1 + D) * n * sizeof(R) > kCoopSmemTableBytes;
}

template <typename R>
__host__ __device__ inline CoopLayout coop_layout(int n, int nq, int D, int NC, int C, int fields,
                                                  bool global_tab)
{
    CoopLayout L;
    L.n = n;
    L.nq = nq;
    L.D = D;
    L.NC = NC;
    L.C = C;
    L.fields = fields;
    L.rs = ((1 + D) * n) | 1;
    L.ls = (fields * n * NC) | 1;
    L.es = ((D * NC > 1 + D) ? D * NC : 1 + D) | 1;   // gradient terms, or value + gradient
    L.ecs = (nq * L.es) | 1;
    L.global_tab = global_tab ? 1 : 0;
    L.tab_bytes = L.global_tab ? 0 : (size_t)nq * L.rs * sizeof(R);
    L.wts_off = (L.tab_bytes + 7) & ~(size_t)7;
    L.wtsr_off = L.wts_off + (size_t)nq * sizeof(double);
    L.table_block_bytes = (L.wtsr_off + (size_t)nq * sizeof(R) + 15) & ~(size_t)15;
    L.off_l = L.table_block_bytes;
    L.off_e = (L.off_l + (size_t)C * L.ls * sizeof(double) + 15) & ~(size_t)15;
    L.off_nodes = (L.off_e + (size_t)C * L.ecs * sizeof(R) + 15) & ~(size_t)15;
    L.off_geo = (L.off_nodes + (size_t)C * n * sizeof(int) + 15) & ~(size_t)15;
    L.off_acc = L.off_geo + (size_t)C * kCoopGeoStride * sizeof(double);
    // adjoint accumulators dmu, dlam per cell, then the quadrature phase's node order
    L.off_order = L.off_acc + (size_t)C * 2 * sizeof(double);
    L.total = (L.off_order + (size_t)n * sizeof(int) + 15) & ~(size_t)15;
    return L;
}

// Shared-memory pointers of one CTA's cooperative scratch.
template <typename R>
struct CoopSmem {
    const R *tab;
    const R *tab_b;     // global-memory tables (global_tab == 1)
    const R *tab_c;
    const double *wts;
    const R *wts_r;
    double *l;
    R *e;
    int *nodes;
    int *order;     // node-major quadrature phase: local nodes by decreasing work
    double *geo;
    double *acc;
};

template <typename R>
__device__ __forceinline__ CoopSmem<R> coop_smem(unsigned char *base, const CoopLayout &L,
                                                 const ActionArgs &a, size_t scratch_shift = 0)
{
    CoopSmem<R> S;
    S.tab = reinterpret_cast<const R *>(base);
    S.tab_b = reinterpret_cast<const R *>(a.tab_b);
    S.tab_c = reinterpret_cast<const R *>(a.tab_c);
    S.wts = reinterpret_cast<const double *>(base + L.wts_off);
    S.wts_r = reinterpret_cast<const R *>(base + L.wtsr_off);
    base += scratch_shift;   // this group's batch scratch
    S.l = reinterpret_cast<double *>(base + L.off_l);
    S.e = reinterpret_cast<R *>(base + L.off_e);
    S.nodes = reinterpret_cast<int *>(base + L.off_nodes);
    S.geo = reinterpret_cast<double *>(base + L.off_geo);
    S.acc = reinterpret_cast<double *>(base + L.off_acc);
    S.order = reinterpret_cast<int *>(base + L.off_order);
    return S;
}

// Phase B: the contribution of local node j to the reference gradients gh of
// the cell's field(s), along the directions in the bit set DIRS only.
template <int D, int FIELDS, int NC, int DIRS, typename R>
__device__ __forceinline__ void eval_node(R (&gh)[FIELDS][NC][D], const R *T, const R *TB, bool gtab,
                                          const double *lc, int n, int nq, int j)
{
    R t[D];
#pragma unroll
    for (int k = 0; k < D; ++k)
        if ((DIRS >> k) & 1)
            t[k] = gtab ? __ldg(TB + ((size_t)(k + 1) * n + j) * nq) : T[(k + 1) * n + j];
#pragma unroll
    for (int f = 0; f < FIELDS; ++f)
#pragma unroll
        for (int m = 0; m < NC; ++m) {
            const R lv = cvt<R>(lc[(f * n + j) * NC + m]);
#pragma unroll
            for (int k = 0; k < D; ++k)
                if ((DIRS >> k) & 1) gh[f][m][k] = fma(t[k], lv, gh[f][m][k]);
        }
}

// Number of multi-indices with `dims` nonnegative entries summing to at most s.
__device__ __forceinline__ int simplex_count(int dims, int s)
{
    return dims == 0 ? 1 : (dims == 1 ? s + 1 : (s + 1) * (s + 2) / 2);
}

// Directions k (bit k) along which the reference derivative of the basis
// function of local node j can be nonzero.  The node's multi-index alpha is
// recovered from j in the documented nested-loop order (alpha_1 outermost).  A
// node with alpha_0 = deg - |alpha| > 0 may vary along every direction; on the
// face alpha_0 = 0 the derivative along k vanishes identically where alpha_k = 0
// (the structural zeros of grad_zero_mask).
template <int D>
__device__ __forceinline__ int node_dirs(int deg, int j)
{
    int rem = deg, dirs = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        int t = 0;
        for (;;) {
            const int cnt = simplex_count(D - 1 - k, rem - t);
            if (j < cnt || t >= rem) break;
            j -= cnt;
            ++t;
        }
        if (t > 0) dirs |= 1 << k;
        rem -= t;
    }
    return rem > 0 ? (1 << D) - 1 : dirs;
}

// Phase C for one (cell, node): out[m] += sum_q sum_k Phi_k[q][j] e[q][m][k],
// over the directions in the bit set DIRS only.  (Splitting the sums into even
// and odd quadrature points, for twice the independent FMA chains, measured
// 0.6 % slower on elasticity P4 3D: the FP64 pipe, not the chain latency, binds;
// unrolling the point loop by 1, 3 or 4 instead of 2 moves it by under 0.2 %.)
template <int D, int NC, int DIRS, typename R>
__device__ __forceinline__ void quad_node(R (&out)[NC], const R *tab, const R *tab_c, bool gtab,
                                          const R *ec, int rs, int es, int n, int q0, int q1, int j)
{
#pragma unroll 2
    for (int q = q0; q < q1; ++q) {
        const R *T = gtab ? tab_c + (size_t)q * (D + 1) * n : tab + (size_t)q * rs;
        const R *e = ec + (size_t)q * es;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            if (!((DIRS >> k) & 1)) continue;
            const R t = gtab ? __ldg(T + (k + 1) * n + j) : T[(k + 1) * n + j];
#pragma unroll
            for (int m = 0; m < NC; ++m) out[m] = fma(t, e[m * D + k], out[m]);
        }
    }
}

// The threads that process one batch together: the whole CTA (barrier id 0, i.e.
// __syncthreads), or one of several equal groups of it, each with its own named
// barrier (ids 1, 2, ...) and its own batches, so that one group's gather phase
// overlaps another group's FP64 work and a group waiting at its barrier does not
// stop the other.
struct CtaGroup {
    int tid;    // thread index within the group
    int size;   // threads in the group (a multiple of 32)
    int bar;    // 0: the whole CTA; else the named barrier id of the group
    __device__ __forceinline__ void sync() const
    {
        if (bar == 0)
            __syncthreads();
        else
            asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(size) : "memory");
    }
};

__device__ __forceinline__ CtaGroup whole_cta()
{
    return CtaGroup{(int)threadIdx.x, (int)blockDim.x, 0};
}

// The node order of the node-major quadrature phase: local nodes by decreasing
// number of derivative directions contracted (FP64 skips the structurally zero
// ones), so that with the items dealt round-robin to the warps the lightest come
// last and the warps reach the batch's final barrier closer together.  Filled
// once per CTA (a counting sort by the direction count); ends with a barrier.
template <int D, typename R>
__device__ __forceinline__ void coop_node_order(const CoopSmem<R> &S, int n, const CtaGroup &grp)
{
    if (grp.tid == 0) {
        const int deg = lagrange_degree(D, n);
        int k = 0;
        for (int w = D; w >= 1; --w)
            for (int j = 0; j < n; ++j) {
                const int dirs = std::is_same<R, double>::value ? node_dirs<D>(deg, j) : (1 << D) - 1;
                if (__popc(dirs) == w) S.order[k++] = j;
            }
    }
    grp.sync();
}

// One batch of cells [cell0, cell0 + nb) through phases A-C by one group of
// threads (the whole CTA by default), over the quadrature points [q0, q1) (all of
// them by default; a sub-range adds that part of the quadrature sum into y, the
// rest being added by other calls: the action is linear in the sum over points).
// Must be called by every thread of the group; ends with the group's barrier.
// RANGE = false compiles the full sum (q0, q1 ignored), so that the ordinary
// batches carry no range arithmetic.
template <int OP, int D, typename R, bool RANGE = false, int KG = 4>
__device__ __forceinline__ void coop_batch(const ActionArgs &a, const CoopLayout &L, const CoopSmem<R> &S,
                                           const int cell0, const int nb, const CtaGroup grp = whole_cta(),
                                           int q0 = 0, int q1 = 0)
{
    constexpr int NC = OpTraits<OP, D>::NC;
    constexpr int FIELDS = OpTraits<OP, D>::kTwoFields ? 2 : 1;
    const int n = L.n;
    [[maybe_unused]] const int deg = lagrange_degree(D, n);   // Lagrange degree of the cell
    const int nq = L.nq;
    if constexpr (!RANGE) {
        q0 = 0;
        q1 = nq;
    }
    const int nqs = RANGE ? q1 - q0 : nq;   // quadrature points of this call
    const R *tab = S.tab;
    const double *wts = S.wts;
    const R *wts_r = S.wts_r;
    double *sl = S.l;
    R *se = S.e;
    int *snodes = S.nodes;
    double *sgeo = S.geo;
    double *sacc = S.acc;
    // ---- A: gather nodes and DoFs; geometry (one thread per cell).  Hyperelastic
    // forms in reduced precision use only gradients and store the DoFs relative to
    // the cell's first node, differenced in FP64 (see gather_dofs).
    constexpr bool kRel = !std::is_same<R, double>::value && OpTraits<OP, D>::kNonlinear;
    // The (cell, node) items are taken KG per thread at a time: all of the group's
    // node indices are loaded first, then all of its DoFs, so a thread waits for
    // two memory round trips per group instead of two per item.
    constexpr int kG = KG;
    const int a_items = nb * n;
    const int stride = grp.size;
    for (int i0 = grp.tid; i0 < a_items; i0 += kG * stride) {
        int node[kG];
        [[maybe_unused]] int node0[kG];
#pragma unroll
        for (int g = 0; g < kG; ++g) {
            const int i = i0 + g * stride;
            node[g] = -1;
            node0[g] = -1;
            if (i < a_items) {
                const int c = i / n;
                node[g] = __ldg(a.c2n + (size_t)cell0 * n + i);
                if constexpr (kRel) node0[g] = __ldg(a.c2n + (size_t)(cell0 + c) * n);
            }
        }
        double v[kG][FIELDS][NC];
#pragma unroll
        for (int g = 0; g < kG; ++g) {
            const bool ok = (unsigned)node[g] < (unsigned)a.n_nodes;
#pragma unroll
            for (int f = 0; f < FIELDS; ++f) {
                const double *src = (f == 0) ? a.u : a.u_lin;
#pragma unroll
                for (int m = 0; m < NC; ++m) v[g][f][m] = ok ? __ldg(src + (size_t)node[g] * NC + m) : 0.0;
            }
        }
#pragma unroll
        for (int g = 0; g < kG; ++g) {
            const int i = i0 + g * stride;
            if (i >= a_items) break;
            const int c = i / n, j = i - c * n;
            const bool ok = (unsigned)node[g] < (unsigned)a.n_nodes;
            if (!ok) set_status(a.status, FE_ERR_INDEX);
            snodes[c * n + j] = ok ? node[g] : -1;
            [[maybe_unused]] const bool ok0 = (unsigned)node0[g] < (unsigned)a.n_nodes;
#pragma unroll
            for (int f = 0; f < FIELDS; ++f) {
                [[maybe_unused]] const double *src = (f == 0) ? a.u : a.u_lin;
#pragma unroll
                for (int m = 0; m < NC; ++m) {
                    double x = v[g][f][m];
                    if constexpr (kRel) x = (ok && ok0) ? x - __ldg(src + (size_t)node0[g] * NC + m) : 0.0;
                    sl[c * L.ls + (f * n + j) * NC + m] = x;
                }
            }
        }
    }
    for (int c = grp.tid; c < nb; c += grp.size) {
        const int cell = cell0 + c;
        double X[D + 1][D];
        bool ok = true;
#pragma unroll
        for (int m = 0; m <= D; ++m) {
            const int v = __ldg(a.c2v + (size_t)cell * (D + 1) + m);
            ok &= (unsigned)v < (unsigned)a.n_vertices;
#pragma unroll
            for (int i = 0; i < D; ++i) X[m][i] = ok ? __ldg(a.coords + (size_t)v * D + i) : 0.0;
        }
        // a cell with an out-of-range node index contributes nothing at all (as in
        // the other kernels); its row of cell2node was just read by the gather above
        bool nodes_ok = true;
        for (int j = 0; j < n; ++j) nodes_ok &= (unsigned)__ldg(a.c2n + (size_t)cell * n + j) < (unsigned)a.n_nodes;
        double Jinv[D][D];
        const double det = cell_geometry<D>(X, Jinv);
        double *g = sgeo + c * kCoopGeoStride;
        const bool good = ok && nodes_ok && (det != 0.0) && isfinite(det);
        if (!ok || !nodes_ok) set_status(a.status, FE_ERR_INDEX);
        else if (!good) set_status(a.status, FE_ERR_BAD_MESH);
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int k = 0; k < D; ++k) g[i * D + k] = good ? Jinv[i][k] : 0.0;
        if constexpr ((OP == OP_LAPLACE || OP == OP_HELMHOLTZ) && coop_weights_folded<OP, R>()) {
            // M = |det J| J^{-1} J^{-T} (symmetric) in place of J^{-1}
            const double ad = good ? fabs(det) : 0.0;
#pragma unroll
            for (int i = 0; i < D; ++i)
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    double mk = Jinv[i][0] * Jinv[k][0];
#pragma unroll
                    for (int r = 1; r < D; ++r) mk = fma(Jinv[i][r], Jinv[k][r], mk);
                    g[i * D + k] = good ? ad * mk : 0.0;
                }
        }
        g[D * D] = good ? fabs(det) : 0.0;
        g[D * D + 1] = (OpTraits<OP, D>::kCellCoeff && a.mu_cell) ? __ldg(a.mu_cell + cell) : a.mu;
        g[D * D + 2] = (OpTraits<OP, D>::kCellCoeff && a.lam_cell) ? __ldg(a.lam_cell + cell) : a.lam;
        g[D * D + 3] = good ? 1.0 : 0.0;
        if constexpr (coop_weights_folded<OP, R>()) {
            g[D * D + 4] = 2.0 * g[D * D + 1] * g[D * D];
            g[D * D + 5] = g[D * D + 2] * g[D * D];
            g[D * D + 6] = g[D * D + 1] * g[D * D];
        }
        sacc[2 * c] = 0.0;
        sacc[2 * c + 1] = 0.0;
    }
    grp.sync();

    // ---- B: evaluation + pointwise per (cell, quadrature point)
    bool nh_ok = true;
    for (int i = grp.tid; i < nb * nqs; i += grp.size) {
        const int c = i / nqs, q = q0 + (i - c * nqs);
        const double *g = sgeo + c * kCoopGeoStride;
        const R *T = tab + (size_t)q * L.rs;
        const bool gtab = L.global_tab;
        const R *TB = S.tab_b + q;   // [k][j][q]: element (k, j) at TB[(k * n + j) * nq]
        const double *lc = sl + c * L.ls;
        R *e = se + (size_t)c * L.ecs + (size_t)q * L.es;
        const double absdet = g[D * D];
        double Jinv[D][D];
#pragma unroll
        for (int ii = 0; ii < D; ++ii)
#pragma unroll
            for (int k = 0; k < D; ++k) Jinv[ii][k] = g[ii * D + k];
        const double mu = g[D * D + 1], lam = g[D * D + 2];
        if constexpr (OP == OP_MASS) {
            R uq = R(0);
            for (int j = 0; j < n; ++j)
                uq = fma(gtab ? __ldg(TB + (size_t)j * nq) : T[j], cvt<R>(lc[j]), uq);
            if constexpr (coop_weights_folded<OP, R>())
                e[0] = uq * absdet;
            else
                e[0] = uq * (wts_r[q] * cvt<R>(absdet));
        } else {
            // reference gradients of the field(s) at q
            R gh[FIELDS][NC][D];
#pragma unroll
            for (int f = 0; f < FIELDS; ++f)
#pragma unroll
                for (int m = 0; m < NC; ++m)
#pragma unroll
                    for (int k = 0; k < D; ++k) gh[f][m][k] = R(0);
            if constexpr (std::is_same<R, double>::value) {
                // Nodes in tabulation order (alpha_1 outermost); the last node of each
                // innermost run has alpha_0 = 0, and its derivative along every
                // direction k with alpha_{k+1} = 0 vanishes identically (the structural
                // zeros of grad_zero_mask): those terms are skipped.  The branch is
                // uniform across the warp (every thread walks the same nodes).  Only
                // the FP64 kernel does this: it is bound by the FP64 pipe, while in the
                // FP32 kernel the branches cost more than the saved FMAs.
                int j = 0;
                for (int a1 = 0; a1 <= deg; ++a1) {
                    if constexpr (D == 3) {
                        for (int a2 = 0; a2 <= deg - a1; ++a2) {
                            const int a3 = deg - a1 - a2;
                            for (int c3 = 0; c3 < a3; ++c3, ++j)
                                eval_node<D, FIELDS, NC, 7>(gh, T, TB, gtab, lc, n, nq, j);
                            switch ((a1 != 0) | ((a2 != 0) << 1) | ((a3 != 0) << 2)) {
                            case 1: eval_node<D, FIELDS, NC, 1>(gh, T, TB, gtab, lc, n, nq, j); break;
                            case 2: eval_node<D, FIELDS, NC, 2>(gh, T, TB, gtab, lc, n, nq, j); break;
                            case 3: eval_node<D, FIELDS, NC, 3>(gh, T, TB, gtab, lc, n, nq, j); break;
                            case 4: eval_node<D, FIELDS, NC, 4>(gh, T, TB, gtab, lc, n, nq, j); break;
                            case 5: eval_node<D, FIELDS, NC, 5>(gh, T, TB, gtab, lc, n, nq, j); break;
                            case 6: eval_node<D, FIELDS, NC, 6>(gh, T, TB, gtab, lc, n, nq, j); break;
                            default: eval_node<D, FIELDS, NC, 7>(gh, T, TB, gtab, lc, n, nq, j); break;
                            }
                            ++j;
                        }
                    } else {
                        const int a2 = deg - a1;
                        for (int c2 = 0; c2 < a2; ++c2, ++j)
                            eval_node<D, FIELDS, NC, 3>(gh, T, TB, gtab, lc, n, nq, j);
                        switch ((a1 != 0) | ((a2 != 0) << 1)) {
                        case 1: eval_node<D, FIELDS, NC, 1>(gh, T, TB, gtab, lc, n, nq, j); break;
                        case 2: eval_node<D, FIELDS, NC, 2>(gh, T, TB, gtab, lc, n, nq, j); break;
                        default: eval_node<D, FIELDS, NC, 3>(gh, T, TB, gtab, lc, n, nq, j); break;
                        }
                        ++j;
                    }
                }
            } else {
                for (int j = 0; j < n; ++j)
                    eval_node<D, FIELDS, NC, (1 << D) - 1>(gh, T, TB, gtab, lc, n, nq, j);
            }
            if constexpr ((OP == OP_LAPLACE || OP == OP_HELMHOLTZ) && coop_weights_folded<OP, R>()) {
                // e = M grad_ref u with M = |det J| J^{-1} J^{-T} from the geometry record
                // (in place of J^{-1}) and the weight in the tables (+ |det J| u for Helmholtz)
                constexpr int kV = (OP == OP_HELMHOLTZ) ? 1 : 0;
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    R sk = Jinv[k][0] * gh[0][0][0];
#pragma unroll
                    for (int ii = 1; ii < D; ++ii) sk = fma(Jinv[k][ii], gh[0][0][ii], sk);
                    e[kV + k] = sk;
                }
                if constexpr (OP == OP_HELMHOLTZ) {
                    R uq = R(0);
                    for (int j = 0; j < n; ++j)
                        uq = fma(gtab ? __ldg(TB + (size_t)j * nq) : T[j], cvt<R>(lc[j]), uq);
                    e[0] = uq * absdet;
                }
            } else if constexpr (OP == OP_LAPLACE || OP == OP_HELMHOLTZ) {
                // e = w |det J| J^{-1} J^{-T} grad_ref u  (+ the value term for Helmholtz)
                R Jr[D][D], g[D];
                convert<D, D>(Jinv, Jr);
                const R wdet_r = wts_r[q] * cvt<R>(absdet);
                constexpr int kV = (OP == OP_HELMHOLTZ) ? 1 : 0;
#pragma unroll
                for (int ii = 0; ii < D; ++ii) {
                    R sg = R(0);
#pragma unroll
                    for (int k = 0; k < D; ++k) sg = fma(gh[0][0][k], Jr[k][ii], sg);
                    g[ii] = sg * wdet_r;
                }
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    R sk = R(0);
#pragma unroll
                    for (int ii = 0; ii < D; ++ii) sk = fma(g[ii], Jr[k][ii], sk);
                    e[kV + k] = sk;
                }
                if constexpr (OP == OP_HELMHOLTZ) {
                    R uq = R(0);
                    for (int j = 0; j < n; ++j)
                        uq = fma(gtab ? __ldg(TB + (size_t)j * nq) : T[j], cvt<R>(lc[j]), uq);
                    e[0] = uq * wdet_r;
                }
            } else if constexpr (OP == OP_SVK_RESIDUAL || OP == OP_SVK_JACOBIAN) {
                // St. Venant-Kirchhoff law in FP64; the linearisation point is the last field
                const double wdet = wts[q] * absdet;
                double ghd[D][D], G[D][D], H[D][D], P[D][D], ed[D][D];
                convert<D, D>(gh[FIELDS - 1], ghd);
                map_grad<D, double>(ghd, Jinv, G);
                if constexpr (OP == OP_SVK_JACOBIAN) {
                    convert<D, D>(gh[0], ghd);
                    map_grad<D, double>(ghd, Jinv, H);
                }
                svk_stress<D, OP == OP_SVK_JACOBIAN>(G, H, mu, lam, wdet, P);
                pull_back<D, double>(P, Jinv, ed);
#pragma unroll
                for (int m = 0; m < NC; ++m)
#pragma unroll
                    for (int k = 0; k < D; ++k) e[m * D + k] = cvt<R>(ed[m][k]);
            } else if constexpr (OP == OP_ELASTICITY) {
                R Jr[D][D], G[D][D], S[D][D], er[D][D];
                convert<D, D>(Jinv, Jr);
                map_grad<D, R>(gh[0], Jr, G);
                R tr = G[0][0];
#pragma unroll
                for (int ii = 1; ii < D; ++ii) tr += G[ii][ii];
                // mu and lambda times w_q |det J| (the weight folded into the tables
                // in FP64: the per-cell products from the geometry record)
                R smu, smu2, slt;
                if constexpr (coop_weights_folded<OP, R>()) {
                    smu2 = g[D * D + 4];
                    slt = g[D * D + 5] * tr;
                    smu = g[D * D + 6];
                } else {
                    const R wdet_r = wts_r[q] * cvt<R>(absdet);
                    smu = wdet_r * cvt<R>(mu);
                    smu2 = R(2) * smu;
                    slt = wdet_r * cvt<R>(lam) * tr;
                }
#pragma unroll
                for (int ii = 0; ii < D; ++ii) {
                    S[ii][ii] = fma(smu2, G[ii][ii], slt);
#pragma unroll
                    for (int k = ii + 1; k < D; ++k) {
                        const R s = smu * (G[ii][k] + G[k][ii]);
                        S[ii][k] = s;
                        S[k][ii] = s;
                    }
                }
                pull_back<D, R>(S, Jr, er);
#pragma unroll
                for (int m = 0; m < NC; ++m)
#pragma unroll
                    for (int k = 0; k < D; ++k) e[m * D + k] = er[m][k];
            } else {
                const double wdet = wts[q] * absdet;
                double ghd[D][D], F[D][D], C2[D][D], S[D][D], ed[D][D];
                // the field whose gradient forms F: u (residual) or u_lin (tangent)
                convert<D, D>(gh[FIELDS - 1], ghd);
                map_grad<D, double>(ghd, Jinv, F);
#pragma unroll
                for (int ii = 0; ii < D; ++ii) F[ii][ii] += 1.0;
                const double Jd = det_cof<D>(F, C2);
                nh_ok &= (Jd > 0.0);
                const double lnJ = law_log(Jd, a.log_tab);
                const double rJ = a.log_tab ? fe_rcp(Jd) : 1.0 / Jd;
                if constexpr (OP == OP_NH_RESIDUAL) {
                    const double smu = wdet * mu;
                    const double scf = wdet * fma(lam, lnJ, -mu) * rJ;
#pragma unroll
                    for (int ii = 0; ii < D; ++ii)
#pragma unroll
                        for (int k = 0; k < D; ++k) S[ii][k] = fma(smu, F[ii][k], scf * C2[ii][k]);
                } else {
                    double H[D][D], Fit[D][D], A[D][D];
                    convert<D, D>(gh[0], ghd);
                    map_grad<D, double>(ghd, Jinv, H);
                    double tr = 0.0;
#pragma unroll
                    for (int ii = 0; ii < D; ++ii)
#pragma unroll
                        for (int k = 0; k < D; ++k) {
                            Fit[ii][k] = C2[ii][k] * rJ;
                            tr = fma(Fit[ii][k], H[ii][k], tr);
                        }
#pragma unroll
                    for (int ii = 0; ii < D; ++ii)
#pragma unroll
                        for (int k = 0; k < D; ++k) {
                            double s = Fit[ii][0] * H[k][0];
#pragma unroll
                            for (int mm = 1; mm < D; ++mm) s = fma(Fit[ii][mm], H[k][mm], s);
                            A[ii][k] = s;
                        }
                    const double smu = wdet * mu;
                    const double sm2 = wdet * fma(-lam, lnJ, mu);
                    const double str = wdet * lam * tr;
#pragma unroll
                    for (int ii = 0; ii < D; ++ii)
#pragma unroll
                        for (int k = 0; k < D; ++k) {
                            double m = A[ii][0] * Fit[0][k];
#pragma unroll
                            for (int mm = 1; mm < D; ++mm) m = fma(A[ii][mm], Fit[mm][k], m);
                            S[ii][k] = fma(smu, H[ii][k], fma(sm2, m, str * Fit[ii][k]));
                        }
                    if constexpr (OP == OP_NH_ADJOINT) {
                        double amu = 0.0, alam = 0.0;
#pragma unroll
                        for (int ii = 0; ii < D; ++ii)
#pragma unroll
                            for (int k = 0; k < D; ++k) {
                                amu = fma(wdet * (F[ii][k] - Fit[ii][k]), H[ii][k], amu);
                                alam = fma(wdet * lnJ * Fit[ii][k], H[ii][k], alam);
                            }
                        atomicAdd(sacc + 2 * c, amu);       // shared-memory FP64 atomics
                        atomicAdd(sacc + 2 * c + 1, alam);
                    }
                }
                pull_back<D, double>(S, Jinv, ed);
#pragma unroll
                for (int m = 0; m < NC; ++m)
#pragma unroll
                    for (int k = 0; k < D; ++k) e[m * D + k] = cvt<R>(ed[m][k]);
            }
        }
    }
    if (!nh_ok) set_status(a.status, FE_ERR_NONFINITE);
    grp.sync();

    // ---- C: quadrature contraction + scatter per (cell, node).  With a batch of a
    // multiple of 32 cells the items are node-major (item i: node i / C, cell
    // i % C), so every warp holds one node for 32 cells and the FP64 kernel can
    // skip that node's structurally zero directions with a warp-uniform branch;
    // otherwise cell-major (consecutive threads: consecutive nodes of a cell).
    const bool store = OP != OP_NH_ADJOINT && a.cell_out;   // node-gather scatter
    const bool node_major = (L.C % 32) == 0;
    const int items = node_major ? n * L.C : nb * n;
    for (int i = grp.tid; i < items; i += grp.size) {
        int c, j;
        if (node_major) {
            const int r = i / L.C;
            c = i - r * L.C;
            j = S.order[r];          // heaviest nodes first: the last items are the light ones
            if (c >= nb) continue;   // ragged last batch
        } else {
            c = i / n;
            j = i - c * n;
        }
        const int node = snodes[c * n + j];
        if (node < 0 || sgeo[c * kCoopGeoStride + D * D + 3] == 0.0) {
            if (store) {
                R *o = static_cast<R *>(a.cell_out) + ((size_t)(cell0 + c) * n + j) * NC;
#pragma unroll
                for (int m = 0; m < NC; ++m) o[m] = R(0);
            }
            continue;
        }
        R out[NC];
#pragma unroll
        for (int m = 0; m < NC; ++m) out[m] = R(0);
        const R *ec = se + (size_t)c * L.ecs;
        const bool gtab = L.global_tab;
        if constexpr (OP == OP_MASS || OP == OP_HELMHOLTZ) {
            for (int q = q0; q < q1; ++q) {
                const R *T = gtab ? S.tab_c + (size_t)q * (D + 1) * n : tab + (size_t)q * L.rs;
                const R *e = ec + (size_t)q * L.es;
                if constexpr (OP == OP_MASS) {
                    out[0] = fma(gtab ? __ldg(T + j) : T[j], e[0], out[0]);
                } else {
                    R o = fma(gtab ? __ldg(T + j) : T[j], e[0], out[0]);
#pragma unroll
                    for (int k = 0; k < D; ++k)
                        o = fma(gtab ? __ldg(T + (k + 1) * n + j) : T[(k + 1) * n + j], e[1 + k], o);
                    out[0] = o;
                }
            }
        } else {
            constexpr int kAll = (1 << D) - 1;
            // the structural-zero skip only where the branch is warp-uniform, and
            // only in FP64 (the FP32 kernel is not bound by its FMA pipe)
            const int dirs = (std::is_same<R, double>::value && node_major) ? node_dirs<D>(deg, j) : kAll;
            const R *tc_ = S.tab_c;
            if constexpr (D == 3) {
                switch (dirs) {
                case 1: quad_node<D, NC, 1>(out, tab, tc_, gtab, ec, L.rs, L.es, n, q0, q1, j); break;
                case 2: quad_node<D, NC, 2>(out, tab, tc_, gtab, ec, L.rs, L.es, n, q0, q1, j); break;
                case 3: quad_node<D, NC, 3>(out, tab, tc_, gtab, ec, L.rs, L.es, n, q0, q1, j); break;
                case 4: quad_node<D, NC, 4>(out, tab, tc_, gtab, ec, L.rs, L.es, n, q0, q1, j); break;
                case 5: quad_node<D, NC, 5>(out, tab, tc_, gtab, ec, L.rs, L.es, n, q0, q1, j); break;
                case 6: quad_node<D, NC, 6>(out, tab, tc_, gtab, ec, L.rs, L.es, n, q0, q1, j); break;
                default: quad_node<D, NC, kAll>(out, tab, tc_, gtab, ec, L.rs, L.es, n, q0, q1, j); break;
                }
            } else {
                switch (dirs) {
                case 1: quad_node<D, NC, 1>(out, tab, tc_, gtab, ec, L.rs, L.es, n, q0, q1, j); break;
                case 2: quad_node<D, NC, 2>(out, tab, tc_, gtab, ec, L.rs, L.es, n, q0, q1, j); break;
                default: quad_node<D, NC, kAll>(out, tab, tc_, gtab, ec, L.rs, L.es, n, q0, q1, j); break;
                }
            }
        }
        if (store) {
            R *o = static_cast<R *>(a.cell_out) + ((size_t)(cell0 + c) * n + j) * NC;
#pragma unroll
            for (int m = 0; m < NC; ++m) o[m] = out[m];
        } else {
#pragma unroll
            for (int m = 0; m < NC; ++m) red_add(a.y + (size_t)node * NC + m, cvt<double>(out[m]));
        }
    }
    if constexpr (OP == OP_NH_ADJOINT) {
        for (int c = grp.tid; c < nb; c += grp.size) {
            a.dmu[cell0 + c] = sacc[2 * c];
            a.dlam[cell0 + c] = sacc[2 * c + 1];
        }
    }
    grp.sync();   // the batch's shared state is reused by the next batch
}

template <int OP, int D, typename R>
__global__ void __launch_bounds__(kCoopWideBlock, 1) k_action_coop(const ActionArgs a, const int n, const int C)
{
    constexpr int NC = OpTraits<OP, D>::NC;
    constexpr int FIELDS = OpTraits<OP, D>::kTwoFields ? 2 : 1;
    extern __shared__ __align__(128) double smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_chunks[kCoopMaxGroups], s_takes[kCoopMaxGroups];
    const CoopLayout L = coop_layout<R>(n, a.nq, D, NC, C, FIELDS, a.tab_b != nullptr);
    if (!stage_table(smem, a.tab, a.tab_doubles, &bar, a.status)) {
        leave_queue(a.sched);
        return;
    }
    // a.coop_groups groups of threads, each with its own batches and its own copy
    // of the batch scratch behind the shared table block
    const int groups = a.coop_groups > 1 ? a.coop_groups : 1;
    const int gsize = (int)blockDim.x / groups, g = (int)threadIdx.x / gsize;
    const CtaGroup grp{(int)threadIdx.x - g * gsize, gsize, groups > 1 ? 1 + g : 0};
    const CoopSmem<R> S = coop_smem<R>(reinterpret_cast<unsigned char *>(smem), L, a,
                                       (size_t)g * (L.total - L.table_block_bytes));
    if (C % 32 == 0) coop_node_order<D, R>(S, n, grp);
    int &s_chunk = s_chunks[g];
    int &s_take = s_takes[g];
    // The queue hands out units of U cells: the whole batch (U = C), or, when C is a
    // multiple of 32, 32-cell units of which a CTA takes C/32 at a time until fewer
    // than that many per CTA remain and one at a time after that, which halves (or
    // better) the last round's imbalance on meshes of a few batches per CTA.
    const int U = (C % 32 == 0) ? 32 : C;
    const int per = C / U;
    const int n_units = (a.n_cells + U - 1) / U;
    // Tail split: with one unit per take, the T units of the last, partial round
    // (T = n_units mod the number of groups) would run on T groups while the rest
    // idle for a whole unit.  When T is at most half a round, each of them is
    // handed out instead as `split` items over consecutive ranges of quadrature
    // points, so the last round costs about 1/split of a unit plus one gather.
    // Not for the adjoint (its per-cell outputs are stored, not summed) nor the
    // node-gather scatter (which stores each cell's outputs); FP64 only, whose long
    // FP64-pipe-bound units make the tail expensive (the FP32 kernels' are short).
    constexpr bool kTailSplit = OP != OP_NH_ADJOINT && std::is_same<R, double>::value;
    // gather items per thread per round trip: 6 for FP64 (headline 11.65 -> 11.62 ms
    // against 4, same 116 registers), 4 for FP32, whose kernels would spill or lose a
    // resident CTA with 6
    constexpr int kGather = std::is_same<R, double>::value ? 6 : 4;
    const int n_groups = (int)gridDim.x * groups;
    int tail = 0, split = 1;
    if (kTailSplit && per == 1 && !a.cell_out) {
        const int T = n_units % n_groups;
        if (T > 0 && 2 * T <= n_groups) {
            split = min(L.nq, n_groups / T);
            if (split > 1) tail = T;
        }
    }
    const int n_full = n_units - tail;
    const int n_items = n_full + tail * split;
    for (;;) {
        if (grp.tid == 0) {
            int take = per;
            if (per > 1 && n_units - *reinterpret_cast<volatile int32_t *>(a.sched) < per * n_groups)
                take = 1;
            s_chunk = atomicAdd(a.sched, take);
            s_take = take;
        }
        grp.sync();
        const int item = s_chunk, take = s_take;
        if (item >= n_items) break;
        if (item < n_full) {
            const int cell0 = item * U;
            coop_batch<OP, D, R, false, kGather>(a, L, S, cell0, min(take * U, a.n_cells - cell0), grp);
        } else if constexpr (kTailSplit) {
            // a tail item: one unit (take is 1 here), one range of quadrature points
            const int sub = item - n_full, part = sub % split, cell0 = (n_full + sub / split) * U;
            coop_batch<OP, D, R, true, kGather>(a, L, S, cell0, min(U, a.n_cells - cell0), grp,
                                                part * L.nq / split, (part + 1) * L.nq / split);
        }
    }
    leave_queue(a.sched);
}

template <int OP, int D, typename R>
cudaError_t launch_coop(const ActionArgs &a, int grid, int block, size_t smem, cudaStream_t s)
{
    k_action_coop<OP, D, R><<<grid, block, smem, s>>>(a, a.coop_n, a.coop_cells);
    return cudaGetLastError();
}

template <int OP, int D, typename R = double>
Variant make_coop_variant()
{
    Variant v;
    v.form = form_of(OP);
    v.dim = D;
    v.degree = 0;   // any degree
    v.op = OP == OP_NH_ADJOINT ? 1 : 0;
    v.precision = std::is_same<R, double>::value ? FE_PREC_FP64 : FE_PREC_FP32;
    v.kernel_id = 1;
    v.block = kCoopBlock;
    v.launch = &launch_coop<OP, D, R>;
    v.func = reinterpret_cast<const void *>(&k_action_coop<OP, D, R>);
    return v;
}

// Largest cell batch whose shared-memory plan fits budget (100 KB leaves room for
// two CTAs per SM); at most 64 cells, at least 1.  Host side.
inline int coop_cells_for(int n, int nq, int dim, int ncomp, int fields, size_t esz, size_t budget, bool gt)
{
    int best = 1;
    for (int C = 1; C <= 64; ++C) {
        const size_t total = esz == sizeof(float)
                                 ? coop_layout<float>(n, nq, dim, ncomp, C, fields, gt).total
                                 : coop_layout<double>(n, nq, dim, ncomp, C, fields, gt).total;
        if (total <= budget) best = C;
    }
    return best;
}

}  // namespace fe
