// C-ABI of the action library: plans, launches, status, diagnostics.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "fe_internal.h"
#include "fe_coop.cuh"
#include "fe_tc.cuh"

namespace fe {

bool tab_zeros_hold(int dim, int n, int nq, const double *tab)
{
    for (int k = 0; k < dim; ++k) {
        const uint64_t z = grad_zero_mask(dim, n, k);
        for (int j = 0; j < n && j < 64; ++j)
            if ((z >> j) & 1u)
                for (int q = 0; q < nq; ++q)
                    if (tab[((size_t)(k + 1) * nq + q) * n + j] != 0.0) return false;
    }
    return true;
}

namespace {

constexpr int kMaxVariants = 512;
Variant g_variants[kMaxVariants];
int g_nvariants = 0;
std::once_flag g_once;

void init_registry()
{
    int n = 0;
    // weight-folded thread-per-cell variants first: find_variant returns the first match
    n += register_variants_fold(g_variants + n, kMaxVariants - n);
    n += register_variants_2d_linear(g_variants + n, kMaxVariants - n);
    n += register_variants_2d_nh(g_variants + n, kMaxVariants - n);
    n += register_variants_3d(g_variants + n, kMaxVariants - n);
    n += register_variants_coop(g_variants + n, kMaxVariants - n);
    n += register_variants_tc(g_variants + n, kMaxVariants - n);
    n += register_variants_tc2(g_variants + n, kMaxVariants - n);
    n += register_variants_tc3(g_variants + n, kMaxVariants - n);
    n += register_variants_forms(g_variants + n, kMaxVariants - n);
    n += register_variants_coop_forms(g_variants + n, kMaxVariants - n);
    // a full table means some registration was cut off: serve nothing rather than
    // a silently incomplete set (every plan then fails with FE_ERR_UNSUPPORTED)
    g_nvariants = n < kMaxVariants ? n : 0;
}

// The thread-per-cell variant compiled for exactly this degree, else (or when
// forced) the cooperative variant, which serves every degree.
// The 16-bit precisions (single or split) have only the tensor-core kernel (any degree).
const Variant *find_variant(int form, int dim, int degree, int op, int precision, bool force_coop)
{
    std::call_once(g_once, init_registry);
    const Variant *coop = nullptr;
    for (int i = 0; i < g_nvariants; ++i) {
        const Variant &v = g_variants[i];
        if (v.form != form || v.dim != dim || v.op != op || v.precision != precision) continue;
        if (v.kernel_id == 2) return &v;
        if (v.kernel_id == 1) coop = &v;
        else if (v.degree == degree && !force_coop) return &v;
    }
    return coop;
}


// Tensor-core tile shape: the most 128-cell pipelines per CTA (4, 2, 1, or the
// count force_pipes asks for) whose staged tables, operands and accumulators
// fit the SM's shared memory and 512 TMEM columns, with the fewest
// quadrature-point chunks.  Returns false if nothing fits.
bool tc_choose(int n, int nq, int ncomp, int kd, int fields, size_t smem_cap, int force_pipes, int terms,
               int esz, TcLayout *out)
{
    if (n > 256 || nq < 1) return false;
    for (int pipes = kTcMaxPipes; pipes >= 1; pipes /= 2) {
        if (force_pipes && pipes != force_pipes) continue;
        for (int nch = 1; nch <= nq; ++nch) {
            const int qc = (nq + nch - 1) / nch;
            const TcLayout L = tc_layout(n, nq, ncomp, kd, fields, qc, pipes, terms, esz);
            if (L.N1p > 256 || L.N2p > 256 || L.tmem_cols > 512) continue;
            if (L.total > smem_cap || L.staged_bytes >= (1u << 20)) continue;
            *out = L;
            return true;
        }
    }
    return false;
}

// Structurally nonzero entries of the reference gradient tables of the degree-p
// basis: d * n minus the pairs (node, direction) with alpha_0 = alpha_{k+1} = 0,
// whose derivative vanishes identically (the zeros grad_zero_mask flags; counted
// here for every degree, not only for n <= 64).
int grad_nonzeros(int d, int p)
{
    int n = 0, zeros = 0;
    for (int a = 0; a <= p; ++a)
        for (int b = 0; b <= p - a; ++b)
            for (int c = 0; c <= (d == 3 ? p - a - b : 0); ++c) {
                const int alpha[4] = {p - a - b - c, a, b, c};
                for (int k = 0; k < d; ++k) zeros += (alpha[0] == 0 && alpha[k + 1] == 0);
                ++n;
            }
    return d * n - zeros;
}

// Algorithmic FP64 flops of Algorithm 2 for one cell (multiply and add count 1
// each, an FMA 2; a division or a logarithm 1).  Geometry is counted once per
// cell as in the untransformed kernel.  Eval/quad terms follow the paper's
// Ops_usable (Eq. "ops_usable"): 2 N_deriv Q n + 2 N_eval Q n, with the gradient
// terms counted over the g structurally nonzero reference-gradient entries
// (dense = true counts all d * n of them, the paper's convention).
double algorithmic_flops(int op, int d, int n, int nq, bool dense)
{
    const double geo = d == 2 ? 11.0 : 50.0;
    const double d2 = double(d) * d;
    const double g = dense ? double(d) * n : double(grad_nonzeros(d, lagrange_degree(d, n)));
    double eval = 0, pw = 0, quad = 0;
    switch (op) {
    case 0:  // mass
        eval = 2.0 * n;
        pw = 2.0;
        quad = 2.0 * n;
        break;
    case 1:  // elasticity
        eval = 2.0 * d * g;
        pw = d == 2 ? 37.0 : 115.0;
        quad = 2.0 * d * g;
        break;
    case 2:  // Neo-Hookean residual
        eval = 2.0 * d * g;
        pw = d == 2 ? 56.0 : 182.0;
        quad = 2.0 * d * g;
        break;
    case 3:  // Neo-Hookean Jacobian action
        eval = 4.0 * d * g;
        pw = d == 2 ? 105.0 : 345.0;
        quad = 2.0 * d * g;
        break;
    case 4:  // Neo-Hookean adjoint (J^T w, dmu, dlambda)
        eval = 4.0 * d * g;
        pw = d == 2 ? 131.0 : 401.0;
        quad = 2.0 * d * g;
        break;
    case 5:  // Laplacian: map (2 d^2), scale (d), pull back (2 d^2)
        eval = 2.0 * g;
        pw = 4.0 * d2 + d + 1.0;
        quad = 2.0 * g;
        break;
    case 6:  // Helmholtz: Laplacian plus the value term
        eval = 2.0 * (g + n);
        pw = 4.0 * d2 + d + 2.0;
        quad = 2.0 * (g + n);
        break;
    case 7:  // St. Venant-Kirchhoff residual: map, E, S, P = F S, pull back
        eval = 2.0 * d * g;
        pw = d == 2 ? 66.0 : 202.0;
        quad = 2.0 * d * g;
        break;
    case 8:  // St. Venant-Kirchhoff Jacobian action: two maps, E, S, dE, dS, dP, pull back
        eval = 4.0 * d * g;
        pw = d == 2 ? 129.0 : 395.0;
        quad = 2.0 * d * g;
        break;
    }
    return geo + nq * (eval + pw + quad);
}

__global__ void k_zero(double *__restrict__ y, long long n)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long n2 = n / 2;
    double2 *y2 = reinterpret_cast<double2 *>(y);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2; i += stride)
        y2[i] = make_double2(0.0, 0.0);
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) y[n - 1] = 0.0;
}

int g_num_sms = 0;

int num_sms()
{
    if (g_num_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 1;
    }
    return g_num_sms;
}

cudaError_t launch_zero(double *y, long long n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int block = 256;
    long long want = (n / 2 + block - 1) / block;
    const long long cap = (long long)num_sms() * 8;
    const int grid = (int)(want < 1 ? 1 : (want > cap ? cap : want));
    if (reinterpret_cast<uintptr_t>(y) % 16 != 0) {
        // unaligned output: plain element-wise zeroing
        return cudaMemsetAsync(y, 0, (size_t)n * sizeof(double), s);
    }
    k_zero<<<grid, block, 0, s>>>(y, n);
    return cudaGetLastError();
}

int ncomp_of(int kind, int dim)
{
    return (kind == FE_FORM_MASS || kind == FE_FORM_LAPLACE || kind == FE_FORM_HELMHOLTZ) ? 1 : dim;
}

// Internal operation of a public form kind (adjoint: see find_variant's op).
int op_of(int kind)
{
    switch (kind) {
    case FE_FORM_LAPLACE: return OP_LAPLACE;
    case FE_FORM_HELMHOLTZ: return OP_HELMHOLTZ;
    case FE_FORM_SVK_RESIDUAL: return OP_SVK_RESIDUAL;
    case FE_FORM_SVK_JACOBIAN: return OP_SVK_JACOBIAN;
    default: return kind;
    }
}

int grid_for(const Variant &v, size_t smem, int n_cells, int cells_per_cta)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, v.func, v.block, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const long long full = (long long)per_sm * num_sms();
    const long long want = ((long long)n_cells + cells_per_cta - 1) / cells_per_cta;
    long long g = want < full ? want : full;
    return (int)(g < 1 ? 1 : g);
}

__global__ void k_dfma(double *out, int iters, double b, double c)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    double a0 = 1e-3 * threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3;
    double a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6, a7 = a0 + 7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            a0 = fma(a0, b, c); a1 = fma(a1, b, c); a2 = fma(a2, b, c); a3 = fma(a3, b, c);
            a4 = fma(a4, b, c); a5 = fma(a5, b, c); a6 = fma(a6, b, c); a7 = fma(a7, b, c);
        }
    }
    out[tid] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}

// Node-gather scatter: y[node] (+)= the node's incident cell outputs, summed in
// the fixed order of the incidence list (T: the stored type; float sums in
// float, then widens exactly).
template <typename T, int NC>
__global__ void k_gather_nodes(const int32_t *__restrict__ ptr, const int32_t *__restrict__ inc,
                               const T *__restrict__ cell_out, double *__restrict__ y, int n_nodes, int accumulate)
{
    for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < n_nodes; node += gridDim.x * blockDim.x) {
        T s[NC];
#pragma unroll
        for (int m = 0; m < NC; ++m) s[m] = T(0);
        const int e = __ldg(ptr + node + 1);
        for (int k = __ldg(ptr + node); k < e; ++k) {
            const T *v = cell_out + (size_t)__ldg(inc + k) * NC;
#pragma unroll
            for (int m = 0; m < NC; ++m) s[m] += __ldg(v + m);
        }
#pragma unroll
        for (int m = 0; m < NC; ++m) {
            const double sm = cvt<double>(s[m]);
            double *dst = y + (size_t)node * NC + m;
            *dst = accumulate ? *dst + sm : sm;
        }
    }
}

template <typename T>
cudaError_t launch_gather(const fe_plan *p, double *y, cudaStream_t st)
{
    const int n = p->mesh.n_nodes;
    if (n <= 0) return cudaSuccess;
    const int block = 256;
    const int grid = std::max(1, std::min((n + block - 1) / block, num_sms() * 16));
    const int acc = (p->form.flags & FE_FLAG_ACCUMULATE) ? 1 : 0;
    const T *co = static_cast<const T *>(p->d_cell_out);
    switch (p->ncomp) {
    case 1: k_gather_nodes<T, 1><<<grid, block, 0, st>>>(p->d_node_ptr, p->d_node_inc, co, y, n, acc); break;
    case 2: k_gather_nodes<T, 2><<<grid, block, 0, st>>>(p->d_node_ptr, p->d_node_inc, co, y, n, acc); break;
    default: k_gather_nodes<T, 3><<<grid, block, 0, st>>>(p->d_node_ptr, p->d_node_inc, co, y, n, acc); break;
    }
    return cudaGetLastError();
}

// FE_FLAG_GATHER_SCATTER: node -> (cell * n_loc + j) incidences from a host
// snapshot of cell2node (cells in increasing order: the summation order), and
// the per-cell output buffer.
int build_gather(fe_plan *p)
{
    const long long nc = p->mesh.n_cells, n = p->n_loc, nn = p->mesh.n_nodes;
    if (nc * n >= (1ll << 31)) return FE_ERR_UNSUPPORTED;
    std::vector<int32_t> c2n((size_t)(nc * n));
    if (nc > 0 && cudaMemcpy(c2n.data(), p->mesh.cell2node, c2n.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        return FE_ERR_CUDA;
    std::vector<int32_t> ptr((size_t)nn + 1, 0);
    for (int32_t v : c2n)
        if (v >= 0 && v < nn) ++ptr[(size_t)v + 1];
    for (long long i = 0; i < nn; ++i) ptr[i + 1] += ptr[i];
    std::vector<int32_t> inc((size_t)ptr[nn] + 1), pos(ptr.begin(), ptr.end() - 1);
    for (long long k = 0; k < nc * n; ++k) {
        const int32_t v = c2n[k];
        if (v >= 0 && v < nn) inc[pos[v]++] = (int32_t)k;
    }
    p->cell_out_f32 = p->form.precision == FE_PREC_FP32;
    const size_t esz = p->cell_out_f32 ? sizeof(float) : sizeof(double);
    if (cudaMalloc(&p->d_cell_out, std::max<size_t>((size_t)(nc * n) * p->ncomp * esz, 16)) != cudaSuccess ||
        cudaMalloc(&p->d_node_ptr, ptr.size() * 4) != cudaSuccess ||
        cudaMalloc(&p->d_node_inc, inc.size() * 4) != cudaSuccess) {
        cudaGetLastError();
        return FE_ERR_NO_MEMORY;
    }
    if (cudaMemcpy(p->d_node_ptr, ptr.data(), ptr.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->d_node_inc, inc.data(), inc.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
        return FE_ERR_CUDA;
    return FE_OK;
}

}  // namespace
}  // namespace fe

using namespace fe;

extern "C" const char *fe_status_string(int status)
{
    switch (status) {
    case FE_OK: return "FE_OK";
    case FE_ERR_INVALID_ARG: return "FE_ERR_INVALID_ARG";
    case FE_ERR_UNSUPPORTED: return "FE_ERR_UNSUPPORTED";
    case FE_ERR_CUDA: return "FE_ERR_CUDA";
    case FE_ERR_BAD_MESH: return "FE_ERR_BAD_MESH";
    case FE_ERR_INDEX: return "FE_ERR_INDEX";
    case FE_ERR_TIMEOUT: return "FE_ERR_TIMEOUT";
    case FE_ERR_NO_MEMORY: return "FE_ERR_NO_MEMORY";
    case FE_ERR_NONFINITE: return "FE_ERR_NONFINITE";
    default: return "FE_ERR_UNKNOWN";
    }
}

// Value of a binary16 / bfloat16 bit pattern (exact), on the host.
template <typename T16>
static double small_to_double(uint16_t b)
{
    constexpr int EB = std::is_same<T16, __nv_bfloat16>::value ? 8 : 5;
    constexpr int MB = 15 - EB;
    constexpr int bias = (1 << (EB - 1)) - 1;
    const int e = (b >> MB) & ((1 << EB) - 1);
    const int mant = b & ((1 << MB) - 1);
    const double sgn = (b >> 15) ? -1.0 : 1.0;
    if (e == (1 << EB) - 1) return mant ? NAN : sgn * INFINITY;
    if (e == 0) return sgn * std::ldexp((double)mant, 1 - bias - MB);
    return sgn * std::ldexp((double)(mant | (1 << MB)), e - bias - MB);
}

// Plan of the tensor-core kernel: the staged block holds Phi (evaluation GEMM
// B operand, rows = chunk columns (q, k), K = node j) and Phi^T (quadrature
// GEMM B operand, rows = node j, K = (q, k) over all chunks) rounded to the
// operand type, in the K-major core-matrix layout, then the weights in FP64
// and FP32.
template <typename TE>
static void tc_fill_block(const TcLayout &L, int kind, const std::vector<double> &wts,
                          const std::vector<double> &tab, int wshift, std::vector<unsigned char> &blk)
{
    constexpr int esz = TcElem<TE>::kBytes;
    using Bits = typename std::conditional<esz == 4, uint32_t, uint16_t>::type;
    blk.assign(L.staged_bytes, 0);
    Bits *B1 = reinterpret_cast<Bits *>(blk.data() + L.b1_off);
    Bits *B2 = reinterpret_cast<Bits *>(blk.data() + L.b2_off);
    const size_t b1_region = (size_t)L.nch * L.N1p * L.K1p, b2_region = (size_t)L.N2p * L.K2;
    for (int ch = 0; ch < L.nch; ++ch)
        for (int ql = 0; ql < L.qc; ++ql) {
            const int q = ch * L.qc + ql;
            if (q >= L.nq) break;
            for (int k = 0; k < L.KD; ++k) {
                const int row = ch * L.N1p + ql * L.KDP + k;
                // value row first for the forms that use values, then the derivatives
                const int kt = (kind == FE_FORM_MASS || kind == FE_FORM_HELMHOLTZ) ? k : 1 + k;
                for (int j = 0; j < L.n; ++j) {
                    const double tv = tab[((size_t)kt * L.nq + q) * L.n + j];
                    if constexpr (esz == 4) {
                        const uint32_t bits = to_tf32_bits(tv);
                        B1[tc_off(row, j, L.K1p, esz)] = bits;
                        B2[tc_off(j, row, L.K2, esz)] = bits;
                    } else {
                        const uint16_t bits = to16_bits<TE>(tv);
                        B1[tc_off(row, j, L.K1p)] = bits;
                        B2[tc_off(j, row, L.K2)] = bits;
                        if (L.terms == 2) {
                            // lo term: the rounding of the remainder
                            const uint16_t lo = to16_bits<TE>(tv - small_to_double<TE>(bits));
                            B1[b1_region + tc_off(row, j, L.K1p)] = lo;
                            B2[b2_region + tc_off(j, row, L.K2)] = lo;
                        }
                    }
                }
            }
        }
    for (int q = 0; q < L.nq; ++q) {
        const double w = std::ldexp(wts[q], wshift);   // exact
        reinterpret_cast<double *>(blk.data() + L.wd_off)[q] = w;
        reinterpret_cast<float *>(blk.data() + L.wf_off)[q] = (float)w;
    }
}

static_assert(kLogTabDoubles == FE_LOG_TABLE_DOUBLES, "log table size of the header");
// the plan folds the quadrature weights into the tables exactly where the
// cells-per-CTA kernel expects them folded (FP64 linear elasticity only)
static_assert(coop_weights_folded<OP_ELASTICITY, double>() && coop_weights_folded<OP_LAPLACE, double>() &&
                  coop_weights_folded<OP_HELMHOLTZ, double>() && coop_weights_folded<OP_MASS, double>() &&
                  !coop_weights_folded<OP_ELASTICITY, float>() && !coop_weights_folded<OP_NH_RESIDUAL, double>() &&
                  !coop_weights_folded<OP_SVK_RESIDUAL, double>(),
              "table folding of the cells-per-CTA kernel");

namespace fe {
void fill_log_table(double *t)
{
    // per table point c = i/128: c, 1/c rounded, and log c split into a head on
    // the 2^-42 grid and a tail; then ln 2 split the same way (section on fe_log)
    const long double grid = 4398046511104.0L;   // 2^42
    for (int i = kLogTabFirst; i <= kLogTabLast; ++i) {
        double *e = t + 4 * (i - kLogTabFirst);
        const long double L = logl((long double)i / 128.0L);
        const long double head = nearbyintl(L * grid) / grid;
        e[0] = (double)i / 128.0;
        e[1] = 128.0 / (double)i;
        e[2] = (double)head;
        e[3] = (double)(L - head);
    }
    const long double L2 = logl(2.0L);
    const long double head2 = nearbyintl(L2 * grid) / grid;
    t[kLogTabDoubles - 2] = (double)head2;
    t[kLogTabDoubles - 1] = (double)(L2 - head2);
}
}  // namespace fe

// Shared-memory scatter aggregation: only for outputs at least this large.
// Measured on mass P3 triangles: +12 % at 4M DoFs (y = 32 MB), 1.67x at 16M DoFs
// (y = 128 MB, larger than L2, where each direct reduction reaches DRAM).
constexpr long long kAggMinOutputBytes = 16ll << 20;

// True when the mesh's numbering makes the cells of a 128-cell tile share nodes:
// four tiles spread over the mesh are copied to the host and their cell-node
// incidences must outnumber their distinct nodes by at least 1.4 (a structured
// P3 triangle mesh gives 1.66: 128 cells, 1,280 incidences, 772 distinct nodes;
// a random numbering about 1).
static bool tiles_share_nodes(const fe_mesh &m, int n)
{
    if (m.n_cells < kTpcBlock) return false;
    std::vector<int32_t> rows((size_t)kTpcBlock * n);
    long long incidences = 0, distinct = 0;
    for (int t = 0; t < 4; ++t) {
        const long long c0 = (long long)(m.n_cells - kTpcBlock) * t / 3;
        if (cudaMemcpy(rows.data(), m.cell2node + c0 * n, rows.size() * sizeof(int32_t), cudaMemcpyDeviceToHost) !=
            cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        std::sort(rows.begin(), rows.end());
        distinct += std::unique(rows.begin(), rows.end()) - rows.begin();
        incidences += (long long)rows.size();
    }
    return 5 * incidences >= 7 * distinct;
}

// Neo-Hookean plans evaluate log det F with fe_log: upload its table.
static int attach_log_table(fe_plan *p)
{
    const int k = p->form.kind;
    if (k != FE_FORM_NH_RESIDUAL && k != FE_FORM_NH_JACOBIAN) return FE_OK;
    std::vector<double> t(kLogTabDoubles);
    fill_log_table(t.data());
    if (cudaMalloc(&p->d_log_tab, t.size() * sizeof(double)) != cudaSuccess) {
        p->d_log_tab = nullptr;
        cudaGetLastError();
        return FE_ERR_NO_MEMORY;
    }
    if (cudaMemcpy(p->d_log_tab, t.data(), t.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
        return FE_ERR_CUDA;
    return FE_OK;
}

static int plan_create_tc(const fe_form &f, const fe_mesh &m, const Variant &v, int nq, int n, int ncomp,
                          const std::vector<double> &wts, const std::vector<double> &tab, fe_plan **out)
{
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return FE_ERR_CUDA;
    const int kd = f.kind == FE_FORM_MASS ? 1 : (f.kind == FE_FORM_HELMHOLTZ ? 1 + m.dim : m.dim);
    // tiles copy their cell2node block with 16-byte loads
    if (reinterpret_cast<uintptr_t>(m.cell2node) % 16 != 0) return FE_ERR_INVALID_ARG;
    // tile_cells selects the pipelines per CTA (128 cells each): 128, 256, 512, or 0 automatic
    if (f.tile_cells != 0 && f.tile_cells != kTcRows && f.tile_cells != 2 * kTcRows &&
        f.tile_cells != 4 * kTcRows)
        return FE_ERR_UNSUPPORTED;
    TcLayout L;
    const int fields = (f.kind == FE_FORM_NH_JACOBIAN || f.kind == FE_FORM_SVK_JACOBIAN) ? 2 : 1;
    const int terms = f.precision == FE_PREC_FP16X2 ? 2 : 1;
    const int esz = f.precision == FE_PREC_TF32 ? 4 : 2;
    if (!tc_choose(n, nq, ncomp, kd, fields, (size_t)optin - 256, f.tile_cells / kTcRows, terms, esz, &L))
        return FE_ERR_UNSUPPORTED;
    // weights scaled by 2^wshift into [1/2, 1) at their largest, so w_q E' stays
    // in binary16's normal range for rules with very small weights
    double wmax = 0.0;
    for (double w : wts) wmax = std::max(wmax, w);
    int we = 0;
    std::frexp(wmax > 0.0 ? wmax : 1.0, &we);
    const int wshift = -we;
    std::vector<unsigned char> blk;
    if (f.precision == FE_PREC_BF16)
        tc_fill_block<__nv_bfloat16>(L, f.kind, wts, tab, wshift, blk);
    else if (f.precision == FE_PREC_TF32)
        tc_fill_block<tf32_t>(L, f.kind, wts, tab, wshift, blk);
    else
        tc_fill_block<__half>(L, f.kind, wts, tab, wshift, blk);   // binary16, single or split

    fe_plan *p = new (std::nothrow) fe_plan();
    if (!p) return FE_ERR_NO_MEMORY;
    p->form = f;
    p->mesh = m;
    p->nq = nq;
    p->n_loc = n;
    p->ncomp = ncomp;
    p->tab_doubles = (int)(L.staged_bytes / sizeof(double));
    p->var = v;
    // threads per cell: with fewer than four pipelines, 2 or 4 threads share each
    // tile row (more warps to hide the gather and scatter latency, same TMEM); a
    // forced tile_cells keeps one.  The cell's threads combine their partial
    // DoF ranges through the quadrature A-operand region, which must hold them.
    int tpc = 1;
    if (f.tile_cells == 0) {
        const bool offset = f.kind != FE_FORM_MASS && f.kind != FE_FORM_HELMHOLTZ;
        const size_t slot = 8 * (size_t)(offset ? 2 * fields * ncomp + 1 : fields + 1);
        const size_t a2_bytes = L.nodes_off - L.a2_off;
        while (L.pipes * tpc * 2 <= kTcMaxPipes && (size_t)kTcRows * tpc * 2 * slot <= a2_bytes) tpc *= 2;
    }
    p->var.block = kTcRows * L.pipes * tpc;
    p->adj = Variant{};
    p->smem_bytes = L.total;
    p->device = dev;
    p->tc_qc = L.qc;
    p->tc_pipes = L.pipes;
    p->tc_wshift = wshift;
    if (cudaMalloc(&p->d_tab, L.staged_bytes) != cudaSuccess ||
        cudaMalloc(&p->d_status, 8 * sizeof(int32_t)) != cudaSuccess) {
        cudaFree(p->d_tab);
        delete p;
        cudaGetLastError();
        return FE_ERR_NO_MEMORY;
    }
    p->d_sched = p->d_status + 4;
    if (cudaMemcpy(p->d_tab, blk.data(), L.staged_bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(p->d_status, 0, 8 * sizeof(int32_t)) != cudaSuccess || allow_max_dynamic_smem(v.func) != cudaSuccess) {
        fe_plan_destroy(p);
        return FE_ERR_CUDA;
    }
    if (const int lrc = attach_log_table(p); lrc != FE_OK) {
        fe_plan_destroy(p);
        return lrc;
    }
    // one CTA per SM (a kernel that uses tensor memory is resident alone on its SM)
    const long long tiles = ((long long)m.n_cells + kTcRows - 1) / kTcRows;
    const long long want = (tiles + L.pipes - 1) / L.pipes;
    p->grid_blocks = (int)std::max(1LL, std::min(want, (long long)num_sms()));
    p->flops_per_cell = algorithmic_flops(op_of(f.kind), m.dim, n, nq, false);
    p->flops_per_cell_dense = algorithmic_flops(op_of(f.kind), m.dim, n, nq, true);
    const double dofs = (double)m.n_nodes * ncomp;
    p->bytes_min = 2.0 * dofs * 8.0 + (double)m.n_vertices * m.dim * 8.0 + (double)m.n_cells * (n + m.dim + 1) * 4.0;
    if (f.kind == FE_FORM_NH_JACOBIAN)
        p->bytes_min += dofs * 8.0 + (f.mu_cell ? 8.0 * m.n_cells : 0.0) + (f.lambda_cell ? 8.0 * m.n_cells : 0.0);
    if (f.flags & FE_FLAG_GATHER_SCATTER) {
        const int rc = build_gather(p);
        if (rc != FE_OK) {
            fe_plan_destroy(p);
            return rc;
        }
    }
    *out = p;
    return FE_OK;
}

extern "C" int fe_plan_create(const fe_form *form, const fe_mesh *mesh, fe_plan **out)
{
    if (!form || !mesh || !out) return FE_ERR_INVALID_ARG;
    *out = nullptr;
    const fe_mesh &m = *mesh;
    const fe_form &f = *form;
    if (m.dim < 2 || m.dim > 3 || m.degree < 1 || m.n_cells < 0 || m.n_vertices < 0 || m.n_nodes < 0)
        return FE_ERR_INVALID_ARG;
    if (m.n_cells > 0 && (!m.coords || !m.cell2vertex || !m.cell2node)) return FE_ERR_INVALID_ARG;
    // 2D vertex coordinates are gathered as one 16-byte load per vertex
    if (m.dim == 2 && reinterpret_cast<uintptr_t>(m.coords) % 16 != 0) return FE_ERR_INVALID_ARG;
    if (f.kind < FE_FORM_MASS || f.kind > FE_FORM_SVK_JACOBIAN) return FE_ERR_INVALID_ARG;
    if (f.precision < FE_PREC_FP64 || f.precision > FE_PREC_TF32) return FE_ERR_UNSUPPORTED;
    const bool tc = f.precision >= FE_PREC_BF16;   // BF16, FP16, FP16X2, TF32: tensor-core kernel
    if (tc && (f.kind == FE_FORM_NH_RESIDUAL || f.kind == FE_FORM_SVK_RESIDUAL)) return FE_ERR_UNSUPPORTED;
    if (f.quad_degree < 0 || f.quad_degree > 40) return FE_ERR_INVALID_ARG;
    if ((f.kind == FE_FORM_NH_JACOBIAN || f.kind == FE_FORM_SVK_JACOBIAN) && !f.u_lin) return FE_ERR_INVALID_ARG;
    if (f.tile_cells < 0 || f.tile_cells > 4096) return FE_ERR_INVALID_ARG;
    const int ncomp = ncomp_of(f.kind, m.dim);
    if ((long long)m.n_nodes * ncomp >= (1ll << 31)) return FE_ERR_INVALID_ARG;

    const bool force_coop = (f.flags & FE_FLAG_COOPERATIVE) != 0;
    const Variant *v = find_variant(f.kind, m.dim, m.degree, 0, f.precision, force_coop);
    if (!v) return FE_ERR_UNSUPPORTED;
    const Variant *adj = (f.kind == FE_FORM_NH_RESIDUAL)
                             ? find_variant(f.kind, m.dim, m.degree, 1, f.precision, force_coop)
                             : nullptr;
    if (adj && adj->kernel_id != v->kernel_id) adj = find_variant(f.kind, m.dim, m.degree, 1, f.precision, true);

    // host tabulation -> device table block [nq][1+d][n] + wts[nq], padded to 16 B
    int nq = 0;
    if (fe_tabulate_scheme(m.dim, m.degree, f.quad_degree, f.quad_scheme, &nq, nullptr, nullptr, nullptr, 0) != FE_OK)
        return FE_ERR_INVALID_ARG;
    const int n = nloc(m.dim, m.degree);
    std::vector<double> pts((size_t)nq * m.dim), wts(nq), tab((size_t)(1 + m.dim) * nq * n);
    int rc = fe_tabulate_scheme(m.dim, m.degree, f.quad_degree, f.quad_scheme, &nq, pts.data(), wts.data(), tab.data(),
                           tab.size());
    if (rc != FE_OK) return rc;
    if (!tab_zeros_hold(m.dim, n, nq, tab.data())) return FE_ERR_INVALID_ARG;
    // table block.  Thread-per-cell: tab [nq][1+d][n] in the contraction
    // precision, padded to 8 B, the weights [nq] in double, the weights [nq] in
    // the contraction precision, padded to 16 B.  Cooperative: the same with the
    // per-point row stride padded to an odd element count, followed in shared
    // memory by the batch scratch (not staged).
    if (tc) return plan_create_tc(f, m, *v, nq, n, ncomp, wts, tab, out);
    const size_t esz = f.precision == FE_PREC_FP32 ? sizeof(float) : sizeof(double);
    const bool coop = v->kernel_id == 1;
    const int fields_max =
        (f.kind == FE_FORM_NH_JACOBIAN || f.kind == FE_FORM_SVK_JACOBIAN || (adj != nullptr)) ? 2 : 1;
    int coop_cells = 0;
    int coop_block = kCoopBlock;
    int coop_groups = 1;
    bool global_tab = false;
    size_t rs = (size_t)(1 + m.dim) * n, woff, smem, block_bytes;
    if (coop) {
        const bool gt = (f.flags & FE_FLAG_TABLES_GLOBAL) ||
                        (esz == sizeof(float) ? coop_default_global<float>(n, nq, m.dim)
                                              : coop_default_global<double>(n, nq, m.dim));
        if (f.tile_cells > 0) {
            coop_cells = f.tile_cells;
        } else if (esz == sizeof(double) && m.dim == 3 && f.kind != FE_FORM_MASS) {
            // FP64 gradient forms on tetrahedra (Helmholtz included): the wide layout
            // (one 512-thread CTA per SM) where its shared memory fits, preferably as
            // two independent 256-thread groups with 32-cell batches each (one group's
            // gather phase overlaps the other's FP64 work), else one group with 64 or
            // 32 cells.  Its quadrature phase skips the structurally zero directions
            // (14-30 % of the gradient entries of a P2-P4 tetrahedron), which outweighs
            // running one CTA per SM instead of two; on triangles (at most 7 % zeros)
            // it does not (measured: SVK P4 and NH Jacobian P6 2-3 % slower).
            const CoopLayout L32 = coop_layout<double>(n, nq, m.dim, ncomp, 32, fields_max, gt);
            if (L32.table_block_bytes + 2 * (L32.total - L32.table_block_bytes) <= kCoopWideSmemBytes) {
                coop_cells = 32;
                coop_groups = 2;
                coop_block = kCoopWideBlock;
            } else {
                for (int C : {64, 32}) {
                    if (coop_layout<double>(n, nq, m.dim, ncomp, C, fields_max, gt).total <= kCoopWideSmemBytes) {
                        coop_cells = C;
                        coop_block = kCoopWideBlock;
                        break;
                    }
                }
            }
        }
        if (coop_cells == 0) coop_cells = coop_cells_for(n, nq, m.dim, ncomp, fields_max, esz, 100 * 1024, gt);
        CoopLayout L = esz == sizeof(float) ? coop_layout<float>(n, nq, m.dim, ncomp, coop_cells, fields_max, gt)
                                            : coop_layout<double>(n, nq, m.dim, ncomp, coop_cells, fields_max, gt);
        rs = L.rs;
        woff = L.wts_off;
        block_bytes = L.table_block_bytes;
        smem = L.total + (size_t)(coop_groups - 1) * (L.total - L.table_block_bytes);
        global_tab = L.global_tab != 0;
    } else {
        woff = ((size_t)nq * rs * esz + 7) & ~(size_t)7;
        block_bytes = (woff + (size_t)nq * (sizeof(double) + esz) + 15) & ~(size_t)15;
        smem = block_bytes;
    }
    const int tab_doubles = (int)(block_bytes / sizeof(double));
    if (smem > (coop_block == kCoopWideBlock ? kCoopWideSmemBytes : (size_t)200 * 1024)) return FE_ERR_UNSUPPORTED;
    // global-memory tables of the cooperative kernel follow the staged block:
    // phase B [1+d][n][nq], then phase C [nq][1+d][n], each 16-byte aligned
    const size_t gsz = global_tab ? (((size_t)(1 + m.dim) * n * nq * esz + 15) & ~(size_t)15) : 0;
    const size_t alloc_bytes = block_bytes + 2 * gsz;
    std::vector<double> block(alloc_bytes / sizeof(double), 0.0);
    unsigned char *blk = reinterpret_cast<unsigned char *>(block.data());
    auto put = [&](size_t byte_off, size_t idx, double t) {
        if (esz == sizeof(float))
            reinterpret_cast<float *>(blk + byte_off)[idx] = (float)t;
        else
            reinterpret_cast<double *>(blk + byte_off)[idx] = t;
    };
    // FP64 linear forms in the cells-per-CTA kernel, and the thread-per-cell
    // variants that ask for it: the rows of point q scaled by sqrt(w_q)
    // (coop_weights_folded, Variant::wfold; the kernel then leaves out w_q)
    const bool fold_w = (coop && esz == sizeof(double) &&
                         (f.kind == FE_FORM_ELASTICITY || f.kind == FE_FORM_LAPLACE ||
                          f.kind == FE_FORM_HELMHOLTZ || f.kind == FE_FORM_MASS)) ||
                        (!coop && v->wfold);
    for (int q = 0; q < nq; ++q)
        for (int k = 0; k <= m.dim; ++k)
            for (int j = 0; j < n; ++j) {
                double t = tab[((size_t)k * nq + q) * n + j];
                if (fold_w) t *= std::sqrt(wts[q]);
                if (global_tab) {
                    put(block_bytes, ((size_t)k * n + j) * nq + q, t);
                    put(block_bytes + gsz, ((size_t)q * (1 + m.dim) + k) * n + j, t);
                } else {
                    put(0, (size_t)q * rs + (size_t)k * n + j, t);
                }
            }
    for (int q = 0; q < nq; ++q) {
        reinterpret_cast<double *>(blk + woff)[q] = wts[q];
        put(woff + (size_t)nq * sizeof(double), q, wts[q]);
    }

    fe_plan *p = new (std::nothrow) fe_plan();
    if (!p) return FE_ERR_NO_MEMORY;
    p->form = f;
    p->mesh = m;
    p->nq = nq;
    p->n_loc = n;
    p->ncomp = ncomp;
    p->tab_doubles = tab_doubles;
    p->var = *v;
    p->adj = adj ? *adj : Variant{};
    if (!coop && f.tile_cells > 0) {
        // thread-per-cell: tile_cells is the block size (the paper's work-group size)
        if (f.tile_cells % 32 != 0 || f.tile_cells > kTpcBlock) {
            delete p;
            return FE_ERR_UNSUPPORTED;
        }
        p->var.block = f.tile_cells;
        if (adj) p->adj.block = f.tile_cells;
    }
    if (coop) {
        p->var.block = coop_block;
        if (adj) p->adj.block = coop_block;
    }
    // FP32 thread-per-cell mass plans sum the updates of nodes shared by a CTA's
    // cells in shared memory before the global scatter, where that pays: y larger
    // than L2 and a numbering whose 128-cell tiles share nodes (not with the
    // node-ordered scatter, which stores per-cell outputs instead)
    if (!coop && v->func_agg && !(f.flags & FE_FLAG_GATHER_SCATTER) &&
        (long long)m.n_nodes * ncomp * (long long)sizeof(double) >= kAggMinOutputBytes &&
        tiles_share_nodes(m, n)) {
        p->agg_slots = agg_slots_for(n);
        smem += (size_t)p->agg_slots * sizeof(int32_t) * (1 + ncomp);
        p->var.func = v->func_agg;
    }
    p->smem_bytes = smem;
    cudaGetDevice(&p->device);
    p->coop_cells = coop_cells;
    p->coop_groups = coop_groups;
    if (cudaMalloc(&p->d_tab, alloc_bytes) != cudaSuccess ||
        cudaMalloc(&p->d_status, 8 * sizeof(int32_t)) != cudaSuccess) {
        cudaFree(p->d_tab);
        delete p;
        cudaGetLastError();
        return FE_ERR_NO_MEMORY;
    }
    p->d_sched = p->d_status + 4;  // status word, padding, then the queue counters
    p->d_tab_b = global_tab ? reinterpret_cast<unsigned char *>(p->d_tab) + block_bytes : nullptr;
    p->d_tab_c = global_tab ? reinterpret_cast<unsigned char *>(p->d_tab) + block_bytes + gsz : nullptr;
    if (cudaMemcpy(p->d_tab, block.data(), alloc_bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(p->d_status, 0, 8 * sizeof(int32_t)) != cudaSuccess) {
        fe_plan_destroy(p);
        return FE_ERR_CUDA;
    }
    if (allow_max_dynamic_smem(p->var.func) != cudaSuccess || (adj && allow_max_dynamic_smem(adj->func) != cudaSuccess)) {
        fe_plan_destroy(p);
        return FE_ERR_CUDA;
    }
    if (const int lrc = attach_log_table(p); lrc != FE_OK) {
        fe_plan_destroy(p);
        return lrc;
    }
    p->grid_blocks = grid_for(p->var, smem, m.n_cells, coop ? coop_cells * coop_groups : p->var.block);
    p->adj_grid_blocks =
        adj ? grid_for(p->adj, smem, m.n_cells, coop ? coop_cells * coop_groups : p->adj.block) : 0;
    p->flops_per_cell = algorithmic_flops(op_of(f.kind), m.dim, n, nq, false);
    p->flops_per_cell_dense = algorithmic_flops(op_of(f.kind), m.dim, n, nq, true);
    const double dofs = (double)m.n_nodes * ncomp;
    double bytes = 2.0 * dofs * 8.0 + (double)m.n_vertices * m.dim * 8.0 +
                   (double)m.n_cells * (n + m.dim + 1) * 4.0;
    const bool hyper = f.kind == FE_FORM_NH_RESIDUAL || f.kind == FE_FORM_NH_JACOBIAN ||
                       f.kind == FE_FORM_SVK_RESIDUAL || f.kind == FE_FORM_SVK_JACOBIAN;
    if (hyper) bytes += (f.mu_cell ? 8.0 * m.n_cells : 0.0) + (f.lambda_cell ? 8.0 * m.n_cells : 0.0);
    if (f.kind == FE_FORM_NH_JACOBIAN || f.kind == FE_FORM_SVK_JACOBIAN) bytes += dofs * 8.0;
    p->bytes_min = bytes;
    if (f.flags & FE_FLAG_GATHER_SCATTER) {
        const int rc = build_gather(p);
        if (rc != FE_OK) {
            fe_plan_destroy(p);
            return rc;
        }
    }
    *out = p;
    return FE_OK;
}

// Copy streams and events of fe_action_host_pipelined (null handles skipped).
static void release_pipeline(fe_plan *plan)
{
    for (cudaEvent_t &e : plan->pipe_ev) {
        if (e) cudaEventDestroy(e);
        e = nullptr;
    }
    if (plan->pipe_h2d) cudaStreamDestroy(plan->pipe_h2d);
    if (plan->pipe_d2h) cudaStreamDestroy(plan->pipe_d2h);
    plan->pipe_h2d = plan->pipe_d2h = nullptr;
    plan->pipe_ready = false;
}

extern "C" int fe_plan_destroy(fe_plan *plan)
{
    if (!plan) return FE_OK;
    cudaDeviceSynchronize();
    cudaFree(plan->d_tab);
    cudaFree(plan->d_status);
    cudaFree(plan->d_cell_out);
    cudaFree(plan->d_node_ptr);
    cudaFree(plan->d_node_inc);
    cudaFree(plan->d_log_tab);
    release_pipeline(plan);
    delete plan;
    return FE_OK;
}

static ActionArgs make_args(const fe_plan *p, const double *u, double *y)
{
    ActionArgs a{};
    a.coords = p->mesh.coords;
    a.c2v = p->mesh.cell2vertex;
    a.c2n = p->mesh.cell2node;
    a.u = u;
    a.u_lin = p->form.u_lin;
    a.y = y;
    a.mu_cell = p->form.mu_cell;
    a.lam_cell = p->form.lambda_cell;
    a.mu = p->form.mu;
    a.lam = p->form.lambda;
    a.tab = p->d_tab;
    a.tab_doubles = p->tab_doubles;
    a.nq = p->nq;
    a.n_cells = p->mesh.n_cells;
    a.n_vertices = p->mesh.n_vertices;
    a.n_nodes = p->mesh.n_nodes;
    a.status = p->d_status;
    a.sched = p->d_sched;
    a.coop_n = p->n_loc;
    a.coop_cells = p->coop_cells;
    a.coop_groups = p->coop_groups;
    a.tab_b = p->d_tab_b;
    a.tab_c = p->d_tab_c;
    a.tc_qc = p->tc_qc;
    a.tc_pipes = p->tc_pipes;
    a.tc_wshift = p->tc_wshift;
    a.cell_out = p->d_cell_out;
    a.log_tab = p->d_log_tab;
    a.agg_slots = p->agg_slots;
    return a;
}

extern "C" int fe_action(fe_plan *plan, const double *u, double *y, void *stream)
{
    if (!plan || !y) return FE_ERR_INVALID_ARG;
    const long long n = (long long)plan->mesh.n_nodes * plan->ncomp;
    if (n > 0 && !u) return FE_ERR_INVALID_ARG;
    if (u == y && n > 0) return FE_ERR_INVALID_ARG;
    if (plan->ncomp == 2 && (reinterpret_cast<uintptr_t>(u) % 16 != 0 ||
                             (plan->form.u_lin && reinterpret_cast<uintptr_t>(plan->form.u_lin) % 16 != 0)))
        return FE_ERR_INVALID_ARG;  // vector gathers of 2-component nodes load 16 B at once
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool gather = plan->d_cell_out != nullptr;
    if (!(plan->form.flags & FE_FLAG_ACCUMULATE) && !gather) {
        if (launch_zero(y, n, s) != cudaSuccess) return FE_ERR_CUDA;
    }
    ActionArgs a = make_args(plan, u, y);
    if (plan->mesh.n_cells > 0 &&
        plan->var.launch(a, plan->grid_blocks, plan->var.block, plan->smem_bytes, s) != cudaSuccess)
        return FE_ERR_CUDA;
    if (gather) {
        const cudaError_t e = plan->cell_out_f32 ? launch_gather<float>(plan, y, s) : launch_gather<double>(plan, y, s);
        if (e != cudaSuccess) return FE_ERR_CUDA;
    }
    return FE_OK;
}

extern "C" int fe_action_adjoint(fe_plan *plan, const double *u, const double *w, double *jtw, double *dmu,
                                 double *dlambda, void *stream)
{
    if (!plan || !plan->adj.launch) return plan ? FE_ERR_UNSUPPORTED : FE_ERR_INVALID_ARG;
    const long long n = (long long)plan->mesh.n_nodes * plan->ncomp;
    if (!jtw || !dmu || !dlambda || (n > 0 && (!u || !w))) return FE_ERR_INVALID_ARG;
    if (u == jtw || w == jtw) return FE_ERR_INVALID_ARG;
    if (plan->ncomp == 2 && (reinterpret_cast<uintptr_t>(u) % 16 != 0 || reinterpret_cast<uintptr_t>(w) % 16 != 0))
        return FE_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!(plan->form.flags & FE_FLAG_ACCUMULATE)) {
        if (launch_zero(jtw, n, s) != cudaSuccess) return FE_ERR_CUDA;
    }
    if (plan->mesh.n_cells == 0) return FE_OK;
    ActionArgs a = make_args(plan, w, jtw);
    a.cell_out = nullptr;   // the adjoint adds into jtw atomically
    a.u_lin = u;
    a.sched = plan->d_sched + 2;
    a.dmu = dmu;
    a.dlam = dlambda;
    if (plan->adj.launch(a, plan->adj_grid_blocks, plan->adj.block, plan->smem_bytes, s) != cudaSuccess)
        return FE_ERR_CUDA;
    return FE_OK;
}

extern "C" int fe_action_host(fe_plan *plan, const double *u_host, double *y_host, double *u_dev, double *y_dev,
                              void *stream)
{
    if (!plan || !u_host || !y_host || !u_dev || !y_dev) return FE_ERR_INVALID_ARG;
    const size_t bytes = (size_t)plan->mesh.n_nodes * plan->ncomp * sizeof(double);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(u_dev, u_host, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return FE_ERR_CUDA;
    int rc = fe_action(plan, u_dev, y_dev, stream);
    if (rc != FE_OK) return rc;
    if (cudaMemcpyAsync(y_host, y_dev, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) return FE_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return FE_ERR_CUDA;
    return FE_OK;
}

extern "C" int fe_action_host_pipelined(fe_plan *plan, int n_steps, const double *const *u_host,
                                        double *const *y_host, double *const *u_dev, double *const *y_dev,
                                        void *stream)
{
    if (!plan || n_steps < 0) return FE_ERR_INVALID_ARG;
    if (n_steps == 0) return FE_OK;
    if (!u_host || !y_host || !u_dev || !y_dev || !u_dev[0] || !u_dev[1] || !y_dev[0] || !y_dev[1])
        return FE_ERR_INVALID_ARG;
    const double *bufs[4] = {u_dev[0], u_dev[1], y_dev[0], y_dev[1]};
    for (int i = 0; i < 4; ++i)
        for (int k = i + 1; k < 4; ++k)
            if (bufs[i] == bufs[k]) return FE_ERR_INVALID_ARG;
    for (int i = 0; i < n_steps; ++i)
        if (!u_host[i] || !y_host[i]) return FE_ERR_INVALID_ARG;
    if (!plan->pipe_ready) {
        bool ok = cudaStreamCreateWithFlags(&plan->pipe_h2d, cudaStreamNonBlocking) == cudaSuccess;
        ok = ok && cudaStreamCreateWithFlags(&plan->pipe_d2h, cudaStreamNonBlocking) == cudaSuccess;
        for (cudaEvent_t &e : plan->pipe_ev) ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            release_pipeline(plan);   // whatever was created before the failure
            cudaGetLastError();
            return FE_ERR_CUDA;
        }
        plan->pipe_ready = true;
    }
    cudaStream_t sc = static_cast<cudaStream_t>(stream);
    const size_t bytes = (size_t)plan->mesh.n_nodes * plan->ncomp * sizeof(double);
    cudaEvent_t *ev = plan->pipe_ev;   // [b*3 + 0] h2d done, [b*3 + 1] action done, [b*3 + 2] d2h done
    // the copy streams start after everything the caller queued on `stream`
    if (cudaEventRecord(ev[1], sc) != cudaSuccess || cudaEventRecord(ev[4], sc) != cudaSuccess ||
        cudaEventRecord(ev[2], sc) != cudaSuccess || cudaEventRecord(ev[5], sc) != cudaSuccess)
        return FE_ERR_CUDA;
    for (int i = 0; i < n_steps; ++i) {
        const int b = i & 1;
        cudaEvent_t h2d = ev[3 * b], act = ev[3 * b + 1], d2h = ev[3 * b + 2];
        // input copy: after the action that last read u_dev[b]
        if (cudaStreamWaitEvent(plan->pipe_h2d, act, 0) != cudaSuccess ||
            cudaMemcpyAsync(u_dev[b], u_host[i], bytes, cudaMemcpyHostToDevice, plan->pipe_h2d) != cudaSuccess ||
            cudaEventRecord(h2d, plan->pipe_h2d) != cudaSuccess)
            return FE_ERR_CUDA;
        // action: after its input arrived and after the copy that last read y_dev[b]
        if (cudaStreamWaitEvent(sc, h2d, 0) != cudaSuccess || cudaStreamWaitEvent(sc, d2h, 0) != cudaSuccess)
            return FE_ERR_CUDA;
        const int rc = fe_action(plan, u_dev[b], y_dev[b], stream);
        if (rc != FE_OK) return rc;
        if (cudaEventRecord(act, sc) != cudaSuccess) return FE_ERR_CUDA;
        // result copy
        if (cudaStreamWaitEvent(plan->pipe_d2h, act, 0) != cudaSuccess ||
            cudaMemcpyAsync(y_host[i], y_dev[b], bytes, cudaMemcpyDeviceToHost, plan->pipe_d2h) != cudaSuccess ||
            cudaEventRecord(d2h, plan->pipe_d2h) != cudaSuccess)
            return FE_ERR_CUDA;
    }
    // the caller's stream ends after the last result copy
    if (cudaStreamWaitEvent(sc, ev[3 * ((n_steps - 1) & 1) + 2], 0) != cudaSuccess) return FE_ERR_CUDA;
    if (cudaStreamSynchronize(sc) != cudaSuccess) return FE_ERR_CUDA;
    return FE_OK;
}

extern "C" int fe_plan_status(fe_plan *plan, int *device_status)
{
    if (!plan || !device_status) return FE_ERR_INVALID_ARG;
    int32_t words[8] = {0};
    if (cudaDeviceSynchronize() != cudaSuccess) return FE_ERR_CUDA;
    if (cudaMemcpy(words, plan->d_status, sizeof(words), cudaMemcpyDeviceToHost) != cudaSuccess)
        return FE_ERR_CUDA;
    int32_t st = words[0];
    // With the device idle, every launch has left the work queue and its last
    // warp reset the counters; anything else means a launch did not complete.
    if (words[4] || words[5] || words[6] || words[7]) {
        if (st == FE_OK) st = FE_ERR_CUDA;
    }
    if (cudaMemset(plan->d_status, 0, sizeof(words)) != cudaSuccess) return FE_ERR_CUDA;
    *device_status = st;
    return FE_OK;
}

extern "C" int fe_plan_get_info(const fe_plan *plan, fe_plan_info *info)
{
    if (!plan || !info) return FE_ERR_INVALID_ARG;
    info->nq = plan->nq;
    info->n_loc = plan->n_loc;
    info->ncomp = plan->ncomp;
    info->kernel = plan->var.kernel_id;
    info->threads_per_block = plan->var.block;
    info->grid_blocks = plan->grid_blocks;
    info->n_dofs = (int64_t)plan->mesh.n_nodes * plan->ncomp;
    info->flops_per_cell = plan->flops_per_cell;
    info->flops_per_cell_dense = plan->flops_per_cell_dense;
    info->bytes_min = plan->bytes_min;
    return FE_OK;
}

extern "C" int fe_measure_fp64_peak(double *scratch, size_t scratch_doubles, double *gflops)
{
    if (!scratch || !gflops) return FE_ERR_INVALID_ARG;
    const int block = 256;
    const int grid = num_sms() * 8;
    if (scratch_doubles < (size_t)grid * block) return FE_ERR_INVALID_ARG;
    const int iters = 2048;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return FE_ERR_CUDA;
    k_dfma<<<grid, block>>>(scratch, iters / 8, 0.9999999, 1e-7);  // warm-up
    cudaEventRecord(e0);
    k_dfma<<<grid, block>>>(scratch, iters, 0.9999999, 1e-7);
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess) return FE_ERR_CUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const double flops = 2.0 * 8.0 * 4.0 * iters * (double)grid * block;
    *gflops = flops / (ms * 1e-3) / 1e9;
    return FE_OK;
}

namespace fe {
namespace {
// Self-test of the bit-pattern conversions against the hardware conversions,
// inputs below binary32's normal range expected as signed zero: count[0] +=
// binary64->binary32 mismatches, count[1] += binary32->binary64 mismatches (NaN
// results compare equal to NaN).
__global__ void k_selftest_conversions(const double *x, long long n, unsigned long long *count)
{
    unsigned long long bad32 = 0, bad64 = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double v = x[i];
        const float a = f64_to_f32_rn(v);
        const float b = fabs(v) < 0x1p-126 ? copysignf(0.f, (float)v) : __double2float_rn(v);
        if (__float_as_uint(a) != __float_as_uint(b) && !(isnan(a) && isnan(b))) ++bad32;
        const float h = __double2float_rn(v);   // binary32 inputs for the widening, subnormals included
        const double c = f32_to_f64(h), d = fabsf(h) < 0x1p-126f ? copysign(0.0, (double)h) : (double)h;
        if (__double_as_longlong(c) != __double_as_longlong(d) && !(isnan(c) && isnan(d))) ++bad64;
    }
    if (bad32) atomicAdd(count, bad32);
    if (bad64) atomicAdd(count + 1, bad64);
}

// Self-test of the kernels' bounded mbarrier wait: one CTA waits on an mbarrier
// that nothing ever completes (no arrival, no copy); the wait must give up after
// `polls` polls, record FE_ERR_TIMEOUT in the status word and return, leaving
// the context usable.
__global__ void k_selftest_bounded_wait(int32_t *status, int polls)
{
    __shared__ __align__(8) uint64_t bar;
    const uint32_t sbar = (uint32_t)__cvta_generic_to_shared(&bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sbar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int done = bounded_wait(sbar, 0, polls);
    if (!__syncthreads_or(done) && threadIdx.x == 0) set_status(status, FE_ERR_TIMEOUT);
}

// Self-test of the binary64 -> bfloat16 / binary16 / TF32 conversions of the
// tensor-core kernel.  The exact integer conversions against CUDA's: count[0] +=
// bfloat16 mismatches, count[1] += binary16 mismatches (NaN compares equal to
// NaN).  The rounding-to-odd conversions of the rounding pass against the exact
// integer ones, bit for bit, at scales 2^0, 2^5, 2^-9 and 2^-20: count[2] +=
// mismatches (bfloat16, binary16 and TF32).
__global__ void k_selftest_conversions16(const double *x, long long n, unsigned long long *count)
{
    unsigned long long bad_b = 0, bad_h = 0, bad_odd = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double v = x[i];
        const __nv_bfloat16 hb = __double2bfloat16(v);
        const __half hh = __double2half(v);
        const uint16_t rb = *reinterpret_cast<const uint16_t *>(&hb), rh = *reinterpret_cast<const uint16_t *>(&hh);
        const uint16_t mb = to16_bits<__nv_bfloat16>(v), mh = to16_bits<__half>(v);
        const bool nan_b = (rb & 0x7F80) == 0x7F80 && (rb & 0x7F), nan_mb = (mb & 0x7F80) == 0x7F80 && (mb & 0x7F);
        const bool nan_h = (rh & 0x7C00) == 0x7C00 && (rh & 0x3FF), nan_mh = (mh & 0x7C00) == 0x7C00 && (mh & 0x3FF);
        if (rb != mb && !(nan_b && nan_mb)) ++bad_b;
        if (rh != mh && !(nan_h && nan_mh)) ++bad_h;
        const int ks[4] = {0, -5, 9, 20};
        for (int t = 0; t < 4; ++t) {
            const int k = ks[t];
            const uint32_t eb = to16_bits<__nv_bfloat16>(v, k), eh = to16_bits<__half>(v, k);
            const uint32_t pb = pack2_from_f64<__nv_bfloat16>(v, -v, k), ph = pack2_from_f64<__half>(v, -v, k);
            const uint32_t nb = to16_bits<__nv_bfloat16>(-v, k), nh = to16_bits<__half>(-v, k);
            if (pb != (eb | (nb << 16)) || ph != (eh | (nh << 16))) ++bad_odd;
            if (tf32_from_f64(v, k) != to_tf32_bits(v, k)) ++bad_odd;
        }
    }
    if (bad_b) atomicAdd(count, bad_b);
    if (bad_h) atomicAdd(count + 1, bad_h);
    if (bad_odd) atomicAdd(count + 2, bad_odd);
}

}  // namespace
}  // namespace fe

extern "C" int fe_selftest_conversions16(const double *x, long long n, unsigned long long *count, void *stream)
{
    if (!x || !count || n < 0) return FE_ERR_INVALID_ARG;
    if (n == 0) return FE_OK;
    long long g = (n + 255) / 256;
    if (g > 4096) g = 4096;
    k_selftest_conversions16<<<(int)g, 256, 0, static_cast<cudaStream_t>(stream)>>>(x, n, count);
    return cudaGetLastError() == cudaSuccess ? FE_OK : FE_ERR_CUDA;
}

extern "C" int fe_selftest_bounded_wait(int32_t *status, int polls, void *stream)
{
    if (!status || polls < 1 || polls > (1 << 24)) return FE_ERR_INVALID_ARG;
    k_selftest_bounded_wait<<<1, 64, 0, static_cast<cudaStream_t>(stream)>>>(status, polls);
    return cudaGetLastError() == cudaSuccess ? FE_OK : FE_ERR_CUDA;
}

namespace fe {
namespace {
__global__ void k_selftest_log_rcp(const double *x, long long n, const double *tab, double *log_out, double *rcp_out)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double v = x[i];
        log_out[i] = fe_log(v, tab);
        rcp_out[i] = fe_rcp(v);
    }
}
}  // namespace
}  // namespace fe

extern "C" int fe_selftest_log_rcp(const double *x, long long n, double *table, double *log_out, double *rcp_out,
                                   void *stream)
{
    if (n < 0 || !table || (n > 0 && (!x || !log_out || !rcp_out))) return FE_ERR_INVALID_ARG;
    std::vector<double> t(kLogTabDoubles);
    fill_log_table(t.data());
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(table, t.data(), t.size() * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return FE_ERR_CUDA;
    if (n == 0) return FE_OK;
    long long g = (n + 255) / 256;
    if (g > 4096) g = 4096;
    k_selftest_log_rcp<<<(int)g, 256, 0, s>>>(x, n, table, log_out, rcp_out);
    return cudaGetLastError() == cudaSuccess ? FE_OK : FE_ERR_CUDA;
}

extern "C" int fe_round16(const double *x, size_t n, int precision, uint16_t *bits)
{
    if ((n > 0 && (!x || !bits))) return FE_ERR_INVALID_ARG;
    if (precision != FE_PREC_BF16 && precision != FE_PREC_FP16) return FE_ERR_UNSUPPORTED;
    for (size_t i = 0; i < n; ++i)
        bits[i] = precision == FE_PREC_BF16 ? to16_bits<__nv_bfloat16>(x[i]) : to16_bits<__half>(x[i]);
    return FE_OK;
}

extern "C" int fe_round_tf32(const double *x, size_t n, int from_binary32, uint32_t *bits)
{
    if ((n > 0 && (!x || !bits))) return FE_ERR_INVALID_ARG;
    for (size_t i = 0; i < n; ++i) {
        if (from_binary32) {
            const float v = (float)x[i];   // IEEE round to nearest even
            uint32_t b;
            std::memcpy(&b, &v, 4);
            bits[i] = f32_bits_to_tf32(b);
        } else {
            bits[i] = to_tf32_bits(x[i]);
        }
    }
    return FE_OK;
}

extern "C" int fe_selftest_conversions(const double *x, long long n, unsigned long long *count, void *stream)
{
    if (!x || !count || n < 0) return FE_ERR_INVALID_ARG;
    if (n == 0) return FE_OK;
    long long g = (n + 255) / 256;
    if (g > 4096) g = 4096;
    k_selftest_conversions<<<(int)g, 256, 0, static_cast<cudaStream_t>(stream)>>>(x, n, count);
    return cudaGetLastError() == cudaSuccess ? FE_OK : FE_ERR_CUDA;
}
