/*
 * feaction.h: C-ABI of the GB300 matrix-free finite element action library.
 *
 * The library computes the action y = A(u) of a variational form on an affine
 * simplex mesh without assembling A: per cell it gathers vertex coordinates and
 * DoFs through the local-to-global maps, contracts the DoFs with the tabulated
 * reference basis (values or derivatives) at the quadrature points, applies the
 * affine geometry (Jacobian, determinant, inverse) and the pointwise form,
 * contracts with the test-function tabulation and scatter-adds into y.  This is
 * the paper's Algorithm 2 (the action of the bilinear form of Eq.
 * "generalized_bilinear_form", with the quadrature sum of Eq.
 * "poisson_action_w_quadrature" and the tabulations of Eq.
 * "poisson_tabulated_values"); the forms are those of Appendix A (Mass,
 * Laplacian, Helmholtz, Elasticity, St. Venant-Kirchhoff hyperelasticity:
 * residual and Jacobian action) plus a compressible Neo-Hookean law (residual,
 * Jacobian action and adjoint with per-cell material derivatives).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Reference simplex: vertices 0, e_1, ..., e_d (d = 2 or 3).  A cell with
 *   vertices (v_0..v_d) maps xhat -> x_{v_0} + sum_k xhat_k (x_{v_k} - x_{v_0});
 *   the Jacobian J[i][k] = x_{v_k}[i] - x_{v_0}[i]; integrals use |det J|.
 * - Local P_p nodes are multi-indices alpha (alpha_k >= 0, sum <= p) at the
 *   reference points alpha/p, enumerated by nested ascending loops with alpha_1
 *   outermost and alpha_d innermost.  cell2node must list a cell's nodes in that
 *   order.
 * - Vector-valued fields (elasticity, Neo-Hookean) interleave components:
 *   DoF index = node * d + component.  Scalar fields: DoF index = node.
 * - All index arrays are int32, row-major; all real arrays are IEEE double.
 * - Device pointers are CUDA device (or managed) memory on the current device.
 *   The caller owns every array; a plan owns only its device tabulation, its
 *   device status word and its work-queue counters (allocated once, at plan
 *   creation).  No entry point allocates on the action path.
 * - Calls that take a stream enqueue work on that stream (a cudaStream_t passed
 *   as void*; NULL means the legacy default stream) and return without
 *   synchronising.  Host-detectable errors are returned immediately and nothing
 *   is enqueued; errors found by the kernels (degenerate cell, index out of
 *   range, det F <= 0) are recorded in the plan's device status word and read
 *   with fe_plan_status().  No kernel traps or asserts.
 */
#ifndef FEACTION_H
#define FEACTION_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
enum fe_status {
    FE_OK = 0,
    FE_ERR_INVALID_ARG = 1,  /* null pointer, bad size, bad enum value            */
    FE_ERR_UNSUPPORTED = 2,  /* (form, dim, degree, precision) not compiled in    */
    FE_ERR_CUDA = 3,         /* a CUDA runtime call failed                        */
    FE_ERR_BAD_MESH = 4,     /* device: det J == 0 or non-finite in some cell     */
    FE_ERR_INDEX = 5,        /* device: a cell2node / cell2vertex entry out of range */
    FE_ERR_TIMEOUT = 6,      /* device: a bounded wait gave up                    */
    FE_ERR_NO_MEMORY = 7,    /* plan creation could not allocate its tables       */
    FE_ERR_NONFINITE = 8     /* device: det F <= 0 or non-finite (Neo-Hookean)    */
};

/* Human-readable name of a status code (static storage; never NULL). */
const char *fe_status_string(int status);

/* ------------------------------------------------------------------ forms */
enum fe_form_kind {
    FE_FORM_MASS = 0,        /* a(u,v) = int u v                       (App. A, Mass)       */
    FE_FORM_ELASTICITY = 1,  /* a(u,v) = int sigma(u):eps(v), sigma = lambda tr(eps) I + 2 mu eps
                                                                         (App. A, Elasticity) */
    FE_FORM_NH_RESIDUAL = 2, /* r(u;v) = int P(F):grad v, F = I + grad u,
                                P = mu (F - F^{-T}) + lambda ln(det F) F^{-T}; nonlinear in u */
    FE_FORM_NH_JACOBIAN = 3, /* a(du,v) = d/de r(u_lin + e du; v) at e = 0: the linearisation
                                of the residual (App. A, Hyperelasticity's bilinear form)    */
    FE_FORM_LAPLACE = 4,     /* a(u,v) = int grad u . grad v, scalar     (App. A, Laplacian)  */
    FE_FORM_HELMHOLTZ = 5,   /* a(u,v) = int (grad u . grad v + u v), scalar (App. A, Helmholtz) */
    FE_FORM_SVK_RESIDUAL = 6,/* r(u;v) = int P(F):grad v, St. Venant-Kirchhoff: F = I + grad u,
                                E = (F^T F - I)/2, S = lambda tr(E) I + 2 mu E, P = F S
                                                                 (App. A, Hyperelasticity)   */
    FE_FORM_SVK_JACOBIAN = 7 /* a(du,v) = d/de r(u_lin + e du; v) at e = 0 for the
                                St. Venant-Kirchhoff residual: dP = H S + F dS, H = grad du,
                                dE = (H^T F + F^T H)/2, dS = lambda tr(dE) I + 2 mu dE       */
};

enum fe_precision {
    FE_PREC_FP64 = 0,        /* every operation in IEEE double                           */
    FE_PREC_FP32 = 1,        /* evaluation and quadrature contractions (tables, DoFs,
                                accumulators) in IEEE single with FP32 accumulation;
                                geometry (det J, J^{-1}), quadrature weights, the
                                Neo-Hookean kinematics, log det F and stress, and the
                                scatter-add stay FP64.  The linear elasticity stress is
                                evaluated in single.  Error: see fe_plan_create.        */
    FE_PREC_BF16 = 2,        /* tensor-core kernel (forms: see fe_plan_create): both contractions on
                                tcgen05 tensor cores with bfloat16 operands (tables, DoFs
                                scaled per cell by a power of two, pointwise results) and
                                FP32 accumulation in tensor memory; geometry FP64, linear
                                stress FP32, scatter-add FP64.  Any tabulated degree
                                (1-10) with at most 256 local nodes (3D P10 has 286).
                                Error: see fe_plan_create.                             */
    FE_PREC_FP16 = 3,        /* as FE_PREC_BF16 with IEEE binary16 operands (3 more
                                significand bits, smaller range; the per-cell power-of-two
                                scaling keeps the operands O(1))                        */
    FE_PREC_FP16X2 = 4,      /* tensor-core kernel with every operand split into a pair of
                                binary16 values (hi + the rounding of the remainder, ~22
                                significand bits) and three products per term (hi*hi,
                                hi*lo, lo*hi): error of the same class as FE_PREC_FP32 at
                                tensor-core speed                                       */
    FE_PREC_TF32 = 5         /* as FE_PREC_BF16 with TF32 operands (tcgen05 kind::tf32:
                                binary32 containers rounded to nearest even to 10
                                fraction bits, 8 exponent bits; 4 bytes per operand, so
                                the staged tables and operands take twice the shared
                                memory of the 16-bit types)                             */
};

/* Flags for fe_form.flags */
#define FE_FLAG_ACCUMULATE 1u  /* y += A(u) instead of y = A(u) */
#define FE_FLAG_COOPERATIVE 2u /* use the cells-per-CTA kernel even where a
                                  thread-per-cell kernel exists for the degree
                                  (it is always used where none exists)      */
#define FE_FLAG_GATHER_SCATTER 8u /* scatter without atomics: fe_action stores every
                                  cell's outputs into a plan-owned buffer and a
                                  second kernel sums, for every node, the
                                  contributions of its cells in a fixed order
                                  (node -> incident (cell, local node) list built
                                  at plan creation from a snapshot of cell2node:
                                  changing cell2node afterwards needs a new plan).
                                  Bitwise reproducible run to run.  Cost: the
                                  store-and-gather pass takes 0.74-0.96x the time
                                  of the atomic scatter on most forms, 1.36x
                                  faster for FP32 P3 mass (measured).  Plan
                                  memory: n_cells * n_loc * ncomp values (float for
                                  FE_PREC_FP32, double otherwise) plus the list.
                                  fe_action_adjoint keeps adding atomically.      */
#define FE_FLAG_TABLES_GLOBAL 4u /* cells-per-CTA kernel: keep the tabulation in
                                  global memory (L2/L1 resident, two coalesced
                                  layouts) instead of shared memory; the default
                                  does so only for tables above 96 KB          */

/* Mesh: affine simplices with P_degree Lagrange DoFs (Sec. "Background",
 * Ciarlet triple and local-to-global maps iota_T).  All pointers are device
 * pointers and must stay valid for the lifetime of every plan built on it. */
typedef struct fe_mesh {
    int32_t dim;                 /* 2 or 3                                         */
    int32_t degree;              /* Lagrange degree p >= 1                         */
    int32_t n_vertices;          /* rows of coords                                 */
    int32_t n_cells;             /* rows of cell2vertex / cell2node (may be 0)     */
    int32_t n_nodes;             /* global P_p node count (DoFs per component)     */
    const double *coords;        /* [n_vertices][dim]                              */
    const int32_t *cell2vertex;  /* [n_cells][dim+1]                               */
    const int32_t *cell2node;    /* [n_cells][C(degree+dim, dim)]                  */
} fe_mesh;

/* Form descriptor.  Coefficients: ELASTICITY uses the constants (lambda, mu);
 * the hyperelastic kinds (Neo-Hookean and St. Venant-Kirchhoff) use per-cell
 * P0 arrays mu_cell / lambda_cell (device, [n_cells]) when non-NULL, else the
 * constants.  NH_JACOBIAN and SVK_JACOBIAN linearise at u_lin (device,
 * [n_nodes*dim]); the plan keeps the pointer, so the caller may update its
 * contents between calls.  MASS, LAPLACE and HELMHOLTZ act on scalar fields
 * (ncomp = 1), the others on vector fields (ncomp = dim). */
typedef struct fe_form {
    int32_t kind;                /* enum fe_form_kind                              */
    int32_t quad_degree;         /* quadrature exactness degree q >= 0             */
    int32_t precision;           /* enum fe_precision                              */
    uint32_t flags;              /* FE_FLAG_*                                      */
    double lambda, mu;           /* constant Lame parameters                       */
    const double *lambda_cell;   /* [n_cells] or NULL                              */
    const double *mu_cell;       /* [n_cells] or NULL                              */
    const double *u_lin;         /* [n_nodes*dim] for NH_JACOBIAN / SVK_JACOBIAN,
                                    else NULL                                      */
    int32_t tile_cells;          /* cells per CTA batch of the cells-per-CTA kernel
                                    (0: the largest that leaves room for two CTAs
                                    per SM); tensor-core kernel: cells per CTA
                                    (128, 256, 512; 0 automatic); thread-per-cell
                                    kernel: threads (= cells) per block, 32, 64,
                                    96 or 128 (0: 128; others FE_ERR_UNSUPPORTED) */
    int32_t quad_scheme;         /* enum fe_quad_scheme (0: conical product)        */
} fe_form;

/* ------------------------------------------------------------------ tabulation */
/* Host function.  Quadrature rule and reference tabulation (Eq.
 * "poisson_tabulated_values"): the collapsed conical-product Gauss-Jacobi rule
 * exact to degree quad_degree with n = ceil((quad_degree+1)/2) points per
 * direction (nq = n^dim; collapsed coordinates xhat_1 = t_1,
 * xhat_2 = t_2 (1 - t_1), xhat_3 = t_3 (1 - t_1)(1 - t_2); t_1 outermost, each
 * direction ascending), and the P_degree Lagrange basis values and reference
 * derivatives at the points.
 * Outputs (host memory, caller-owned): *nq; pts [nq][dim]; wts [nq];
 * tab [(1+dim)][nq][n_loc] with row 0 the values and row k the derivative
 * d/dxhat_k.  cap is the number of doubles available in tab; pts and wts must
 * hold nq*dim and nq doubles (query with tab == NULL to get *nq only).
 * Errors: FE_ERR_INVALID_ARG (dim not 1..3, degree < 1 or > 10, quad_degree < 0
 * or > 40, cap too small). */
int fe_tabulate(int dim, int degree, int quad_degree, int *nq, double *pts, double *wts,
                double *tab, size_t cap);

/* Quadrature families (fe_form.quad_scheme). */
enum fe_quad_scheme {
    FE_QUAD_CONICAL = 0,   /* collapsed conical-product Gauss-Jacobi rule (as fe_tabulate) */
    FE_QUAD_SYMMETRIC = 1  /* fully symmetric rule (invariant under every permutation of the
                              barycentric coordinates, positive weights, interior points) of
                              the smallest tabulated degree >= quad_degree, derived at run
                              time by Gauss-Newton on the moment equations from a stated
                              orbit structure; tabulated: triangles degree 2, 4, 6, 8 (3, 6,
                              12, 16 points), tetrahedra degree 2, 5, 6 (4, 14, 24 points).  Other
                              requests fall back to FE_QUAD_CONICAL.  Points are ordered
                              lexicographically by (xhat_1, xhat_2, xhat_3).            */
};

/* fe_tabulate for either quadrature family; same outputs and errors
 * (FE_ERR_INVALID_ARG also for an unknown scheme). */
int fe_tabulate_scheme(int dim, int degree, int quad_degree, int scheme, int *nq, double *pts,
                       double *wts, double *tab, size_t cap);

/* ------------------------------------------------------------------ plans */
typedef struct fe_plan fe_plan;

/* Validates the form/mesh pair, tabulates on the host, uploads the tables to
 * the current device and selects the kernel.  Synchronous.  The plan stores
 * copies of *form and *mesh (pointers inside them are borrowed).  This is the
 * set-up that precedes Algorithm 2: the tabulations Phi of Eq.
 * "poisson_tabulated_values" and the quadrature weights are computed once per
 * (form, mesh) pair, not per cell (Sec. "Towards Discretization"), and the
 * kernel's parameters are fixed (the role of the transformation choices of
 * Sec. "Transformation Space").
 *
 * Accuracy of y = A(u) against the exact-arithmetic action (norm-wise,
 * ||y - y_exact||_inf / ||y_exact||_inf):
 *   FE_PREC_FP64  rounding level (parity with an FP64 reference to 1e-12,
 *                 except where the action itself is ill-conditioned in FP64);
 *   FE_PREC_FP32  <= 5e-5 (each contraction's forward error is at most
 *                 gamma_256 of its absolute terms; measured 1e-7 - 6e-7;
 *                 DoFs and geometry factors below 2^-126 in magnitude enter
 *                 the FP32 contractions as zero, so fields and cell volumes
 *                 must lie in binary32's normal range);
 *   FE_PREC_BF16, FE_PREC_FP16, FE_PREC_TF32  a multiple k of u16 = 2^-8 (BF16)
 *                 or 2^-11 (FP16, TF32), per form (the largest deviation measured
 *                 over the library's tests, all degrees, 2D and 3D, scaled meshes
 *                 and materials, times 1.5):
 *                   form          BF16   FP16   TF32
 *                   mass          2.25   1.5    1.25
 *                   elasticity    2.0    2.25   2.25
 *                   Laplacian     1.75   1.5    1.5
 *                   Helmholtz     1.5    1.5    1.5
 *                   NH Jacobian   4.0    6.5    4.75  (smooth linearisation
 *                                                      point rounded to 16 bits)
 *                   SVK Jacobian  1.75   2.0    2.0
 *                 e.g. elasticity in FP16 <= 2.25 x 2^-11 = 1.1e-3;
 *   FE_PREC_FP16X2 <= 5e-5 (the FP32 bound).
 *
 * Tensor-core plans (FE_PREC_BF16 / FE_PREC_FP16 / FE_PREC_FP16X2 / FE_PREC_TF32): kinds MASS, ELASTICITY,
 * LAPLACE, HELMHOLTZ, NH_JACOBIAN and SVK_JACOBIAN (the residual kinds:
 * FE_ERR_UNSUPPORTED); cell2node must be 16-byte
 * aligned (FE_ERR_INVALID_ARG otherwise); tile_cells selects the 128-cell
 * pipelines per CTA (128, 256 or 512, one thread per cell; other values
 * FE_ERR_UNSUPPORTED); 0 lets the plan take the most pipelines that fit and,
 * when fewer than four fit, 2 or 4 threads per cell (fe_plan_info reports
 * threads_per_block = 128 x pipelines x threads per cell);
 * FE_ERR_UNSUPPORTED also if the degree has more than 256
 * local nodes or the tables and operands do not fit one SM (FE_PREC_FP16X2
 * and FE_PREC_TF32 double both).
 * Errors: FE_ERR_INVALID_ARG, FE_ERR_UNSUPPORTED, FE_ERR_NO_MEMORY, FE_ERR_CUDA. */
int fe_plan_create(const fe_form *form, const fe_mesh *mesh, fe_plan **out);

/* Frees the plan's device tables and status word.  Synchronises the device.
 * NULL is accepted. */
int fe_plan_destroy(fe_plan *plan);

/* y = A(u) (or y += A(u) with FE_FLAG_ACCUMULATE), enqueued on stream: the
 * matrix-free action of Algorithm 2, y_i = sum over cells T of the quadrature
 * sum of Eq. "poisson_action_w_quadrature" for the form of the plan, gathered
 * through cell2node and scatter-added (Sec. "Towards Discretization").
 * u, y: device arrays of n_nodes * ncomp doubles (ncomp = 1 for MASS, LAPLACE
 * and HELMHOLTZ, dim otherwise); u and y must not alias.  For the Jacobian kinds
 * u is the direction du.
 * Errors: FE_ERR_INVALID_ARG before launch, FE_ERR_CUDA on a failed launch. */
int fe_action(fe_plan *plan, const double *u, double *y, void *stream);

/* Adjoint of the Neo-Hookean residual r(u; mu, lambda) (plan built with
 * kind = FE_FORM_NH_RESIDUAL and per-cell or constant Lame parameters).  The
 * residual is the hyperelastic form of Appendix A with the Neo-Hookean stress
 * in place of St. Venant-Kirchhoff's; its transpose action has the structure
 * of Algorithm 2 with the tangent dP/dF applied to grad w at each point:
 *   jtw      = J(u)^T w          (device, n_nodes*dim; overwritten unless
 *                                 FE_FLAG_ACCUMULATE)
 *   dmu[c]     = w . dr/dmu_c     = int_c (F - F^{-T}) : grad w      (device, n_cells)
 *   dlambda[c] = w . dr/dlambda_c = int_c ln(det F) F^{-T} : grad w  (device, n_cells)
 * The deformation gradient is recomputed at every quadrature point, nothing is
 * stored between the forward and the adjoint call.  J^T w is formed with the
 * fourth-order tangent dP/dF, which for a hyperelastic law has major symmetry,
 * applied to grad w.  dmu and dlambda are overwritten (one value per cell).
 * Errors: FE_ERR_UNSUPPORTED for other forms, FE_ERR_INVALID_ARG, FE_ERR_CUDA. */
int fe_action_adjoint(fe_plan *plan, const double *u, const double *w, double *jtw, double *dmu,
                      double *dlambda, void *stream);

/* End-to-end convenience: copies u_host (n_dofs doubles, ideally pinned) to the
 * caller's device buffer u_dev, runs fe_action into y_dev, copies y_dev back to
 * y_host and synchronises the stream.  Allocates nothing. */
int fe_action_host(fe_plan *plan, const double *u_host, double *y_host, double *u_dev,
                   double *y_dev, void *stream);

/* End-to-end over a sequence of n_steps independent inputs (for example the
 * right-hand sides of successive solves): y_host[i] = A(u_host[i]), i < n_steps,
 * each u_host[i] / y_host[i] a host array of n_dofs doubles (pinned for the
 * copies to be asynchronous).  The steps are pipelined through two device
 * buffer pairs u_dev[0..1], y_dev[0..1] (caller-owned, n_dofs doubles each,
 * all four distinct): the host-to-device copy of step i+1 and the
 * device-to-host copy of step i-1 run on two plan-owned copy streams while the
 * action of step i runs on `stream`, ordered by events, so the per-step time is
 * the largest of the three instead of their sum.  Every step still copies its
 * input in and its result out.  Returns after the last result has reached
 * y_host[n_steps-1] (synchronises `stream`).  The plan creates its two copy
 * streams and six events on first use and frees them in fe_plan_destroy.
 * Errors: FE_ERR_INVALID_ARG (NULL arrays, aliasing device buffers, n_steps <
 * 0), FE_ERR_CUDA. */
int fe_action_host_pipelined(fe_plan *plan, int n_steps, const double *const *u_host, double *const *y_host,
                             double *const *u_dev, double *const *y_dev, void *stream);

/* Reads and clears the plan's device status word (synchronises the device).
 * *device_status receives FE_OK or the first device-detected error; it is
 * FE_ERR_CUDA if a launch left the plan's work-queue counters inconsistent.
 *
 * Concurrency: a plan's kernels pull cells from a plan-owned work queue (two
 * counters per kernel, reset by the last warp of each launch).  Launches of the
 * same plan must therefore not overlap in time: issue them on one stream, or
 * order them with events.  Different plans are independent. */
int fe_plan_status(fe_plan *plan, int *device_status);

/* Plan facts for callers and benchmarks. */
typedef struct fe_plan_info {
    int32_t nq;               /* quadrature points per cell                        */
    int32_t n_loc;            /* local nodes per cell                              */
    int32_t ncomp;            /* components per node                               */
    int32_t kernel;           /* variant id: 0 thread-per-cell, 1 cells-per-CTA,
                                 2 tensor core (128-cell tiles)                    */
    int32_t threads_per_block;
    int32_t grid_blocks;      /* blocks launched per action                        */
    int64_t n_dofs;           /* n_nodes * ncomp                                   */
    double flops_per_cell;    /* algorithmic FP64 flops of Algorithm 2 per cell,
                                 gradient contractions counted over the structurally
                                 nonzero reference-gradient entries: d phi_alpha /
                                 dxhat_k vanishes identically when alpha_0 =
                                 alpha_k = 0 (barycentric multi-index alpha)       */
    double bytes_min;         /* roofline footprint: each DoF, coordinate and map
                                 entry counted once (Sec. "Roofline Model")         */
    double flops_per_cell_dense; /* the same counting every table entry (the
                                 paper's Ops_usable convention, Eq. "ops_usable")   */
} fe_plan_info;

int fe_plan_get_info(const fe_plan *plan, fe_plan_info *info);

/* ------------------------------------------------------------------ batched persistent action */
/* Many independent problems (meshes of uneven size, degree and form) in one
 * persistent launch.  Each problem is a FP64 MASS, ELASTICITY or NH_RESIDUAL
 * form on its own mesh with its own device input u and output y (same layouts
 * as fe_action; y is overwritten).  kernel selects the device code used for
 * the problem's tiles: -1 automatic (thread-per-cell where compiled for the
 * degree, else cells-per-CTA), 0 thread-per-cell (tiles of 128 cells), 1
 * cells-per-CTA with tile_cells cells per tile (0: the largest tile that keeps
 * two CTAs per SM, as for a single plan).
 * fe_batch_create validates, tabulates every problem, uploads the tables and
 * the cost-ordered work lists (one per device code), and allocates the
 * batch's device memory, a side stream and two events (synchronous).  Pointers
 * inside the problems are borrowed and must outlive the batch.  fe_batch_run
 * enqueues on stream a kernel that zeroes every y, then two persistent kernels
 * whose CTAs pull tiles from their work lists (a CTA restages a problem's table
 * only when the problem changes): one for the thread-per-cell problems (128
 * threads per CTA), one for the cells-per-CTA problems (256 threads) on the
 * batch's side stream, forked from and joined back to stream with events, so
 * the two run concurrently and the whole run can be captured in a CUDA graph
 * on stream.  Runs of one batch must not overlap in time.  fe_batch_status
 * reads and clears the batch's device status word (synchronises).
 * fe_batch_info: grid_blocks is the sum of the two grids, smem_bytes the
 * larger of their dynamic shared memories.
 * Errors: FE_ERR_INVALID_ARG, FE_ERR_UNSUPPORTED, FE_ERR_NO_MEMORY, FE_ERR_CUDA. */
typedef struct fe_batch_problem {
    fe_form form;
    fe_mesh mesh;
    const double *u;             /* device, n_nodes * ncomp                        */
    double *y;                   /* device, n_nodes * ncomp                        */
    int32_t kernel;              /* -1 auto, 0 thread-per-cell, 1 cells-per-CTA    */
    int32_t tile_cells;          /* cells per tile for kernel 1 (0: automatic)     */
} fe_batch_problem;

typedef struct fe_batch fe_batch;

typedef struct fe_batch_info {
    int32_t problems, items, grid_blocks, pad;
    int64_t smem_bytes;
    int64_t dofs;                /* sum of the problems' DoFs                      */
    double contraction_flops;    /* contraction flops of all problems (Ops_usable) */
} fe_batch_info;

int fe_batch_create(const fe_batch_problem *problems, int count, fe_batch **out);
int fe_batch_run(fe_batch *batch, void *stream);
int fe_batch_status(fe_batch *batch, int *device_status);
int fe_batch_get_info(const fe_batch *batch, fe_batch_info *info);
int fe_batch_destroy(fe_batch *batch);

/* ------------------------------------------------------------------ Krylov building blocks */
/* Vector kernels for conjugate gradients with FP64 iterative refinement around
 * a reduced-precision action (the action is the operator; these supply one
 * CG iteration's vector work).  All vectors are device FP64 arrays of n
 * entries; mask is NULL (every DoF free) or a device uint8 array of n entries,
 * 1 for a free DoF and 0 for a Dirichlet DoF (the masked system is
 * M A M + (I - M) with M = diag(mask)).  Every scalar stays on the device in
 * the caller's workspace ws of FE_CG_WORKSPACE_DOUBLES doubles, which must be
 * zero-filled once before first use; scalars live at ws[FE_CG_PARTIALS + s]
 * with s: 0 rr, 1 pq, 2 alpha, 3 beta, 4 rr after the update, 5..14 free slots
 * for fe_vec_dot, 15 reserved (reduction counter, self-resetting).
 * Reductions are deterministic (fixed grid, fixed summation order).  Calls
 * sharing one ws must be ordered (one stream).  All are asynchronous on stream.
 * Errors: FE_ERR_INVALID_ARG, FE_ERR_CUDA. */
#define FE_CG_PARTIALS 1024
#define FE_CG_WORKSPACE_DOUBLES (FE_CG_PARTIALS + 16)
/* r = M (b - Ax); p = r; rr = r . r */
int fe_cg_start(long long n, const double *b, const double *Ax, const uint8_t *mask, double *r,
                double *p, double *ws, void *stream);
/* q <- M q; pq = p . q; alpha = rr / pq   (q = A p from the action on entry) */
int fe_cg_direction(long long n, const double *p, double *q, const uint8_t *mask, double *ws,
                    void *stream);
/* x += alpha p; r -= alpha q; beta = (r . r) / rr; rr = r . r */
int fe_cg_update(long long n, double *x, double *r, const double *p, const double *q, double *ws,
                 void *stream);
/* p = r + beta p */
int fe_cg_new_direction(long long n, const double *r, double *p, const double *ws, void *stream);
/* y += a x (a on the host) */
int fe_vec_axpy(long long n, double a, const double *x, double *y, void *stream);
/* ws scalar slot (5..14) = (M x) . y */
int fe_vec_dot(long long n, const double *x, const double *y, const uint8_t *mask, double *ws,
               int slot, void *stream);

/* ------------------------------------------------------------------ no-allocation variant */
/* fe_action for callers that cannot allocate device memory (the paper has no
 * counterpart; this is a deployment convenience).  Such callers include
 * applications whose device memory is owned up front by their own pool
 * allocator and hosts that forbid device allocations after start-up: they
 * cannot create a plan, because fe_plan_create calls cudaMalloc for the table
 * block, the status word and the work-queue counters.
 *
 * This entry point runs the same thread-per-cell kernel as fe_action and
 * allocates nothing: no cudaMalloc, cudaFree or allocating library call.  Its
 * scratch (table block, status word, queue counters) is a file-scope device
 * array of 256 bytes plus FE_NOALLOC_TABLE_DOUBLES doubles (96 KB), which every
 * GPU that loads the library holds until the process exits.
 *   form, mesh: as for fe_plan_create (device pointers inside them).
 *   tab_host, wts_host, nq: the host tabulation exactly as fe_tabulate writes it
 *     for (mesh->dim, mesh->degree, form->quad_degree): tab [(1+dim)][nq][n_loc],
 *     wts [nq], in pageable or page-locked host memory.  The call waits for its
 *     copies of them to finish (a synchronisation of `stream`, which also waits
 *     for the work queued before the call) before it launches the kernel, so
 *     the caller may reuse or free both as soon as the call returns.
 *   form->flags: FE_FLAG_ACCUMULATE or nothing, and form->tile_cells 0; the
 *     other plan options need plan-owned memory or another kernel and are
 *     refused with FE_ERR_UNSUPPORTED.
 *   u, y: device DoF vectors as for fe_action (y is overwritten unless
 *     FE_FLAG_ACCUMULATE).
 *   device_status: NULL, or a host int that receives the device status word
 *     (FE_OK or the first device-detected error); a non-NULL pointer makes the
 *     call synchronise the stream.
 * Set-up: the first call on each device (with that device current) looks up the
 * device address of the scratch array; make that first call before any stream
 * capture.  Every call clears the status word and the counters before it
 * launches, and keeps its table in the array afterwards.  Calls whose GPU work
 * overlaps (unordered streams, several host threads) race on the shared array.
 * Errors: FE_ERR_INVALID_ARG (bad arguments, a table block larger than
 * FE_NOALLOC_TABLE_DOUBLES doubles, or a table that is not exactly 0.0 at a
 * structural zero of the reference gradients, d phi_alpha / dxhat_k with
 * alpha_0 = alpha_k = 0, which the kernel does not read), FE_ERR_UNSUPPORTED
 * (no thread-per-cell kernel for this form/dim/degree, a precision other than
 * FP64, a flag other than FE_FLAG_ACCUMULATE, tile_cells != 0), FE_ERR_CUDA. */
#define FE_NOALLOC_TABLE_DOUBLES 12288
int fe_action_noalloc(const fe_form *form, const fe_mesh *mesh, const double *tab_host,
                      const double *wts_host, int nq, const double *u, double *y,
                      int *device_status, void *stream);

/* ------------------------------------------------------------------ diagnostics */
/* Measures the device's FP64 FMA throughput with an unrolled independent-chain
 * kernel: writes the achieved FP64 GFLOP/s (an FMA counts 2) to *gflops.
 * scratch: device buffer of at least 152*8*256 doubles (results are written
 * there so the work cannot be elided).  Synchronous. */
int fe_measure_fp64_peak(double *scratch, size_t scratch_doubles, double *gflops);

/* Self-test of the mixed-precision kernels' binary64<->binary32 conversions
 * (branch-free integer bit-pattern conversions with round-to-nearest-even,
 * used instead of the hardware conversion, which issues on the slow FP64 pipe
 * of this part; values below binary32's normal range, |x| < 2^-126, become
 * signed zero) against the hardware conversions with that flush applied, over
 * the device array x [n]: count[0] += binary64->binary32 mismatches, count[1]
 * += binary32->binary64 mismatches; count is a device array of 2
 * zero-initialised uint64.  Asynchronous on stream. */
int fe_selftest_conversions(const double *x, long long n, unsigned long long *count, void *stream);

/* Device self-test of the tensor-core kernel's conversions.  The integer
 * conversions binary64 -> bfloat16 and binary64 -> binary16 (round to nearest
 * even, done without the FP64 pipe) against CUDA's __double2bfloat16 /
 * __double2half: count[0] += bfloat16 mismatches, count[1] += binary16
 * mismatches (NaN results compare equal).  The kernel's rounding pass (binary64
 * times 2^-k narrowed to binary32 by rounding to odd, then rounded by the
 * hardware's binary32 conversion) against the integer conversions bit for bit,
 * for bfloat16, binary16 and TF32 at k = 0, -5, 9, 20: count[2] += mismatches.
 * x device [n]; count device [3] unsigned 64-bit.  Asynchronous.
 * Errors: FE_ERR_INVALID_ARG, FE_ERR_CUDA. */
int fe_selftest_conversions16(const double *x, long long n, unsigned long long *count, void *stream);

/* Device self-test of the kernels' bounded waits: one CTA waits on a shared-
 * memory mbarrier that nothing ever completes, gives up after `polls` polls
 * (each followed by a ~64 ns sleep) and records FE_ERR_TIMEOUT in *status
 * (device int32, caller-owned, as a plan's status word: the first error wins).
 * The context stays usable.  Asynchronous on stream.  Errors: FE_ERR_INVALID_ARG
 * (NULL status, polls outside [1, 2^24]), FE_ERR_CUDA. */
int fe_selftest_bounded_wait(int32_t *status, int polls, void *stream);

/* Device self-test of the Neo-Hookean laws' logarithm and reciprocal: the
 * kernels evaluate log det F by Tang's table-driven method (ACM TOMS 16(4),
 * 1990: x = 2^e m, m within 2^-8 of a table point c = i/128, log x = e ln2 +
 * log c + log1p((m - c)/c) with a degree-8 Taylor polynomial) and 1/det F by
 * the approximate hardware reciprocal refined by two Newton-Raphson steps.
 * table: device buffer of FE_LOG_TABLE_DOUBLES doubles that receives the
 * logarithm's table (synchronises stream once); x [n] device; log_out[i] =
 * the kernels' log(x[i]), rcp_out[i] = their 1/x[i] (device, [n]).
 * Asynchronous on stream after the table upload.  Errors: FE_ERR_INVALID_ARG,
 * FE_ERR_CUDA. */
#define FE_LOG_TABLE_DOUBLES 370
int fe_selftest_log_rcp(const double *x, long long n, double *table, double *log_out, double *rcp_out,
                        void *stream);

/* Host function.  Rounds x[n] (host) to the 16-bit type of precision
 * (FE_PREC_BF16 or FE_PREC_FP16) to nearest even, exactly as plans round their
 * tabulation for the tensor-core kernel; bits[n] (host, caller-owned) receives
 * the bit patterns.  Errors: FE_ERR_INVALID_ARG (NULL with n > 0),
 * FE_ERR_UNSUPPORTED (another precision). */
int fe_round16(const double *x, size_t n, int precision, uint16_t *bits);

/* Host function.  Rounds x[n] (host) to TF32 to nearest even, as a TF32 plan
 * rounds its operands: from_binary32 = 0 rounds the binary64 value directly
 * (the tables and the DoFs), from_binary32 != 0 first rounds it to binary32
 * and then to TF32 (the pointwise results, which the kernel holds in
 * binary32).  bits[n] (host, caller-owned) receives the binary32 container bit
 * patterns (13 low fraction bits zero).  Errors: FE_ERR_INVALID_ARG (NULL with
 * n > 0). */
int fe_round_tf32(const double *x, size_t n, int from_binary32, uint32_t *bits);

/* ------------------------------------------------------------- mesh orderings
 * Host functions.  At low order the action is dominated by its indirect
 * gathers and scatters, whose cache behaviour depends on how close the DoFs of
 * cells processed together are in memory (Sec. "Behavior at low orders").
 * These compute locality orderings; applying them is a renumbering, not a
 * change of the operator. */

/* Cells along a Morton (Z-order) curve of their centroids (bounding box
 * quantised to 2^21 levels per axis in 3D, 2^32 in 2D; ties keep the input
 * order).  coords [n_vertices][dim], cell2vertex [n_cells][dim+1] (host);
 * perm [n_cells] (host, caller-owned) receives the old index of the k-th cell
 * of the new order.  Errors: FE_ERR_INVALID_ARG, FE_ERR_INDEX (a vertex index
 * out of range), FE_ERR_BAD_MESH (a non-finite centroid). */
int fe_order_cells_morton(int dim, int n_vertices, int n_cells, const double *coords,
                          const int32_t *cell2vertex, int32_t *perm);

/* Entities (nodes or vertices) numbered by first touch: visiting the cells in
 * the order cell_order [n_cells] (NULL: 0, 1, ...), each not yet numbered
 * entity of cell2entity [n_cells][per_cell] gets the next index; entities no
 * cell references follow in their old order.  new_of_old [n_entities] (host,
 * caller-owned) receives the new index of each old entity.  Errors:
 * FE_ERR_INVALID_ARG (bad sizes, NULL, cell_order not a permutation),
 * FE_ERR_INDEX (an index out of range). */
int fe_order_first_touch(int n_entities, int n_cells, int per_cell, const int32_t *cell2entity,
                         const int32_t *cell_order, int32_t *new_of_old);

#ifdef __cplusplus
}
#endif
#endif /* FEACTION_H */
