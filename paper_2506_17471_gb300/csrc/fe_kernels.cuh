// Thread-per-cell FP64 action kernels for sm_103a.
//
// One thread owns one cell and runs the paper's Algorithm 2 for it: gather the
// cell's vertex coordinates and DoFs, compute the affine Jacobian, its
// determinant and inverse once (affine geometry, Sec. "Towards
// Discretization"), then for every quadrature point evaluate the trial field's
// values/reference derivatives against the tabulation, apply the pointwise form
// and the geometry mapping, and accumulate the test-side contraction; finally
// scatter-add with FP64 atomics (the scatter's cross-cell dependence, Sec.
// "Towards Discretization", resolved as in the single-cell-per-work-item
// scheme, Algorithm 3).
//
// GB300 design points:
//  * The tabulation block (all quadrature points, basis values and reference
//    derivatives, then the weights) is staged once per CTA into shared memory
//    with a 1-D bulk async copy (cp.async.bulk + mbarrier, bounded wait); every
//    read of it inside the hot loops is warp-uniform (a broadcast).
//  * DoFs, outputs and geometry live in registers; every contraction is an
//    unrolled chain of DFMA (FP64 throughput, not HBM bandwidth, bounds these
//    kernels on this part).
//  * The launch is persistent (grid = resident CTAs of all 152 SMs) and warps
//    pull 32-cell chunks from a work queue, which keeps the FP64 pipe of every
//    SM busy until the last chunk.
//  * Index maps are range-checked (cheap integer work); a bad index, a
//    degenerate cell or det F <= 0 set the plan's status word; nothing traps.
#pragma once

#include <cstdint>
#include <type_traits>

#include "fe_internal.h"

namespace fe {

constexpr int kTpcBlock = 128;
constexpr int kWaitLimit = 1 << 21;   // bounded mbarrier polls (~0.1-0.3 s with backoff)

// *p += v as a global reduction that returns nothing (the scatter-add never
// reads the old value, so no register waits on the reply).
__device__ __forceinline__ void red_add(double *p, double v)
{
    asm volatile("red.global.add.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}

__device__ __forceinline__ void set_status(int32_t *status, int32_t code)
{
    if (status) atomicCAS(status, 0, code);
}

// Natural logarithm for the hyperelastic laws, by Tang's table-driven method
// (P. T. P. Tang, "Table-driven implementation of the logarithm function in IEEE
// floating-point arithmetic", ACM TOMS 16(4), 1990).  x = 2^e m with m in
// [1/sqrt2, sqrt2); c = i/128 is the table point nearest to m (i in 91..181), so
// log x = e ln2 + log c + log1p(u), u = (m - c)/c, |u| <= 2^-7.4.  m - c is exact
// (Sterbenz), u is carried as u + ur with ur = (m - c - u c)/c from one fused
// multiply-add, and log1p(u) is its Taylor polynomial to degree 8 (truncation
// below 2^-58 relative).  The table (built on the host, see fill_log_table)
// holds per i: c, 1/c rounded, and log c split into a head that is a multiple
// of 2^-42 and a tail; its last two entries split ln 2 the same way, so
// e ln2_head + logc_head is exact and only the final addition rounds.  Zero,
// negative, subnormal, infinite and NaN arguments take CUDA's log.
constexpr int kLogTabFirst = 90, kLogTabLast = 181;
constexpr int kLogTabDoubles = 4 * (kLogTabLast - kLogTabFirst + 1) + 2;

__device__ __forceinline__ double fe_log(double x, const double *__restrict__ t)
{
    const long long b = __double_as_longlong(x);
    if (!(x >= 0x1p-1022) || b >= 0x7ff0000000000000LL) return log(x);
    const long long mant = b & 0x000fffffffffffffLL;
    int e = (int)(b >> 52) - 1023;
    long long mb;
    int i;
    if (mant >= 0x6a09e667f3bcdLL) {   // m >= sqrt 2: take m / 2 and e + 1
        ++e;
        mb = mant | 0x3fe0000000000000LL;
        i = (int)(((1LL << 52) + mant + (1LL << 45)) >> 46);
    } else {
        mb = mant | 0x3ff0000000000000LL;
        i = (int)(((1LL << 52) + mant + (1LL << 44)) >> 45);
    }
    const double m = __longlong_as_double(mb);
    const double *ti = t + 4 * (i - kLogTabFirst);
    const double c = __ldg(ti), inv = __ldg(ti + 1);
    const double f = m - c;
    const double u = f * inv;
    const double ur = fma(-u, c, f) * inv;
    double q = -0.125;
    q = fma(q, u, 1.0 / 7.0);
    q = fma(q, u, -1.0 / 6.0);
    q = fma(q, u, 0.2);
    q = fma(q, u, -0.25);
    q = fma(q, u, 1.0 / 3.0);
    q = fma(q, u, -0.5);
    const double ed = (double)e;
    const double head = fma(ed, __ldg(t + kLogTabDoubles - 2), __ldg(ti + 2));   // exact
    const double tail = fma(ed, __ldg(t + kLogTabDoubles - 1), __ldg(ti + 3)) + ur;
    return head + (fma(u * u, q, u) + tail);
}

// 1/x for the hyperelastic laws: the hardware's approximate reciprocal
// (rcp.approx.ftz.f64) refined by two Newton-Raphson steps r <- r + r (1 - x r),
// each of which squares the relative error.  Zero, subnormal, infinite and NaN
// arguments take the IEEE division.
__device__ __forceinline__ double fe_rcp(double x)
{
    const double ax = fabs(x);
    if (!(ax >= 0x1p-1022) || !(ax < 0x1p1020)) return 1.0 / x;
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    double e = fma(-x, r, 1.0);
    r = fma(r, e, r);
    e = fma(-x, r, 1.0);
    return fma(r, e, r);
}

// log(x) through the table when the plan provides one, else CUDA's log.
__device__ __forceinline__ double law_log(double x, const double *t)
{
    return t ? fe_log(x, t) : log(x);
}

// Bounded wait on phase `parity` of the shared-memory mbarrier at sbar: at most
// `limit` polls with a short sleep between them.  Returns 1 if the phase
// completed, 0 if the wait gave up (the caller records FE_ERR_TIMEOUT).
__device__ __forceinline__ int bounded_wait(uint32_t sbar, uint32_t parity, int limit)
{
    for (int it = 0; it < limit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(sbar), "r"(parity)
            : "memory");
        if (ok) return 1;
        __nanosleep(64);
    }
    return 0;
}

// Stage the table block into shared memory with one bulk async copy.  Returns
// false (and records FE_ERR_TIMEOUT) if the copy did not complete within the
// bounded wait; the caller must then return.
__device__ __forceinline__ bool stage_table(double *sm_tab, const double *g_tab, int ndoubles,
                                            uint64_t *bar, int32_t *status)
{
    const uint32_t bytes = (uint32_t)ndoubles * 8u;   // multiple of 16 by construction
    const uint32_t sbar = (uint32_t)__cvta_generic_to_shared(bar);
    const uint32_t sdst = (uint32_t)__cvta_generic_to_shared(sm_tab);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sbar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint64_t gsrc = (uint64_t)__cvta_generic_to_global(g_tab);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sbar), "r"(bytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                sdst),
            "l"(gsrc), "r"(bytes), "r"(sbar)
            : "memory");
    }
    const int done = bounded_wait(sbar, 0, kWaitLimit);
    if (__syncthreads_and(done)) return true;
    // The copy did not land in time: record it, give the in-flight copy a second
    // bounded chance to finish before this CTA's shared memory is released.
    if (threadIdx.x == 0) set_status(status, FE_ERR_TIMEOUT);
    bounded_wait(sbar, 0, kWaitLimit);
    __syncthreads();
    return false;
}

// Affine geometry of one cell: J[i][k] = x_k[i] - x_0[i]; returns det J and J^{-1}.
template <int D>
__device__ __forceinline__ double cell_geometry(const double (&X)[D + 1][D], double (&Jinv)[D][D])
{
    double J[D][D];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int k = 0; k < D; ++k) J[i][k] = X[k + 1][i] - X[0][i];
    double det;
    if constexpr (D == 2) {
        det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        const double r = 1.0 / det;
        Jinv[0][0] = J[1][1] * r;
        Jinv[0][1] = -J[0][1] * r;
        Jinv[1][0] = -J[1][0] * r;
        Jinv[1][1] = J[0][0] * r;
    } else {
        const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
        const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
        const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
        det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
        const double r = 1.0 / det;
        Jinv[0][0] = c00 * r;
        Jinv[1][0] = c01 * r;
        Jinv[2][0] = c02 * r;
        Jinv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * r;
        Jinv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * r;
        Jinv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * r;
        Jinv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * r;
        Jinv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * r;
        Jinv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * r;
    }
    return det;
}

// det and cofactor matrix (cof = det * A^{-T}) of a small matrix.
template <int D>
__device__ __forceinline__ double det_cof(const double (&A)[D][D], double (&C)[D][D])
{
    if constexpr (D == 2) {
        C[0][0] = A[1][1];
        C[0][1] = -A[1][0];
        C[1][0] = -A[0][1];
        C[1][1] = A[0][0];
        return A[0][0] * A[1][1] - A[0][1] * A[1][0];
    } else {
        C[0][0] = A[1][1] * A[2][2] - A[1][2] * A[2][1];
        C[0][1] = A[1][2] * A[2][0] - A[1][0] * A[2][2];
        C[0][2] = A[1][0] * A[2][1] - A[1][1] * A[2][0];
        C[1][0] = A[0][2] * A[2][1] - A[0][1] * A[2][2];
        C[1][1] = A[0][0] * A[2][2] - A[0][2] * A[2][0];
        C[1][2] = A[0][1] * A[2][0] - A[0][0] * A[2][1];
        C[2][0] = A[0][1] * A[1][2] - A[0][2] * A[1][1];
        C[2][1] = A[0][2] * A[1][0] - A[0][0] * A[1][2];
        C[2][2] = A[0][0] * A[1][1] - A[0][1] * A[1][0];
        return A[0][0] * C[0][0] + A[0][1] * C[0][1] + A[0][2] * C[0][2];
    }
}

// IEEE 754 binary64 -> binary32 with round-to-nearest-even, computed with
// integer operations on the bit patterns and without branches.  On this part
// the hardware conversion issues on the FP64 pipe (about 1/64 of the FP32
// rate), and a hardware fallback for rare inputs would be predicated into every
// call, so the mixed-precision kernels convert DoFs, outputs and geometry this
// way.  Inputs below binary32's normal range (|x| < 2^-126) give signed zero;
// overflow gives infinity; NaN stays a quiet NaN.
__device__ __forceinline__ float f64_to_f32_rn(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x);
    const unsigned lo = (unsigned)__double2loint(x);
    const unsigned sign = hi & 0x80000000u;
    const int fexp = (int)((hi >> 20) & 0x7FFu) - 896;   // binary32 biased exponent
    unsigned bits = sign | ((unsigned)fexp << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    const unsigned rest = lo & 0x1FFFFFFFu;               // the 29 discarded mantissa bits
    bits += (rest > 0x10000000u) || (rest == 0x10000000u && (bits & 1u));   // a carry may reach infinity
    const bool nan = fexp == 0x7FF - 896 && ((hi & 0xFFFFFu) | lo);
    bits = fexp < 1 ? sign : bits;
    bits = fexp > 254 ? (sign | 0x7F800000u | (nan ? 0x400000u : 0u)) : bits;
    return __uint_as_float(bits);
}

// IEEE 754 binary32 -> binary64 by re-biasing the exponent and widening the
// mantissa, without branches: exact for normal inputs; zero and subnormal inputs
// give signed zero; infinity stays infinity, NaN a quiet NaN.
__device__ __forceinline__ double f32_to_f64(float f)
{
    const unsigned b = __float_as_uint(f);
    const unsigned e = (b >> 23) & 0xFFu, sign = b & 0x80000000u, m = b & 0x7FFFFFu;
    unsigned hi = sign | ((e + 896u) << 20) | (m >> 3), lo = m << 29;
    hi = e == 0u ? sign : hi;
    lo = e == 0u ? 0u : lo;
    hi = e == 255u ? (sign | 0x7FF00000u | (m >> 3) | (m ? 0x80000u : 0u)) : hi;
    return __hiloint2double((int)hi, (int)lo);
}

template <typename U, typename T>
__device__ __forceinline__ U cvt(T x)
{
    if constexpr (std::is_same<U, T>::value)
        return x;
    else if constexpr (std::is_same<U, float>::value)
        return f64_to_f32_rn(x);
    else
        return f32_to_f64(x);
}

// Structural zeros of the reference gradient tables.  The basis is the product
// phi_alpha = prod_m L_{alpha_m}(lam_m) over the barycentric coordinates, and
// d/dxhat_k reaches it only through lam_{k+1} and lam_0 = 1 - sum xhat; the term
// through lam_m carries L'_{alpha_m}, which vanishes for alpha_m = 0 (L_0 = 1).
// So d phi_alpha / dxhat_k is identically zero when alpha_0 = alpha_{k+1} = 0,
// and the tabulation holds exactly 0.0 there at every quadrature point.  Bit j of
// grad_zero_mask(D, N, k) flags such a local node j (node order of the
// tabulation: alpha_1 outermost, then alpha_2, alpha_3).  The thread-per-cell
// contractions skip those terms; for finite operands the result is unchanged,
// since a fused multiply-add with a zero factor returns its addend (up to the
// sign of a zero sum).
__host__ __device__ constexpr int lagrange_degree(int D, int N)
{
    for (int p = 0; p <= 20; ++p) {
        const int n = D == 2 ? (p + 1) * (p + 2) / 2 : (p + 1) * (p + 2) * (p + 3) / 6;
        if (n == N) return p;
    }
    return -1;
}

__host__ __device__ constexpr uint64_t grad_zero_mask(int D, int N, int k)
{
    const int p = lagrange_degree(D, N);
    if ((D != 2 && D != 3) || p < 0 || N > 64 || k < 0 || k >= D) return 0;
    uint64_t mask = 0;
    int j = 0;
    for (int a = 0; a <= p; ++a)
        for (int b = 0; b <= p - a; ++b)
            for (int c = 0; c <= (D == 3 ? p - a - b : 0); ++c) {
                const int alpha[4] = {p - a - b - c, a, b, c};
                if (alpha[0] == 0 && alpha[k + 1] == 0) mask |= uint64_t(1) << j;
                ++j;
            }
    return mask;
}

static_assert(grad_zero_mask(3, 4, 0) == 0x6 && grad_zero_mask(3, 4, 1) == 0xA &&
                  grad_zero_mask(3, 4, 2) == 0xC,
              "P1 tetrahedron: node 1 = (0,0,1), 2 = (0,1,0), 3 = (1,0,0)");
static_assert(grad_zero_mask(2, 6, 0) == 0x4 && grad_zero_mask(2, 6, 1) == 0x20,
              "P2 triangle: nodes 2 = (0,2) and 5 = (2,0) in (alpha_1, alpha_2)");

// Whether T_{k+1}[j] is a structural zero (k, j compile-time after unrolling).
template <int D, int N>
__device__ __forceinline__ bool grad_zero(int k, int j)
{
    constexpr uint64_t z0 = grad_zero_mask(D, N, 0), z1 = grad_zero_mask(D, N, 1),
                       z2 = grad_zero_mask(D, N, 2);
    const uint64_t z = k == 0 ? z0 : (k == 1 ? z1 : z2);
    return (z >> j) & 1u;
}

// Evaluation phase: reference gradient gh[c][k] = sum_j T_{k+1}[j] l[j][c], in
// the contraction type R (double, or float for the mixed-precision variant).
template <int D, int N, int NC, typename R>
__device__ __forceinline__ void eval_grad(const R *__restrict__ T, const R (&l)[N][NC], R (&gh)[NC][D])
{
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int k = 0; k < D; ++k) gh[c][k] = R(0);
#pragma unroll
    for (int j = 0; j < N; ++j) {
#pragma unroll
        for (int k = 0; k < D; ++k) {
            if (grad_zero<D, N>(k, j)) continue;
            const R t = T[(k + 1) * N + j];
#pragma unroll
            for (int c = 0; c < NC; ++c) gh[c][k] = fma(t, l[j][c], gh[c][k]);
        }
    }
}

// Quadrature phase: out[j][c] += sum_k T_{k+1}[j] e[c][k].
template <int D, int N, int NC, typename R>
__device__ __forceinline__ void quad_grad(const R *__restrict__ T, const R (&e)[NC][D], R (&out)[N][NC])
{
#pragma unroll
    for (int j = 0; j < N; ++j) {
#pragma unroll
        for (int k = 0; k < D; ++k) {
            if (grad_zero<D, N>(k, j)) continue;
            const R t = T[(k + 1) * N + j];
#pragma unroll
            for (int c = 0; c < NC; ++c) out[j][c] = fma(t, e[c][k], out[j][c]);
        }
    }
}

// A[c][i] = sum_k B[c][k] Jinv[k][i]  (reference -> physical gradient)
template <int D, typename R>
__device__ __forceinline__ void map_grad(const R (&B)[D][D], const R (&Jinv)[D][D], R (&A)[D][D])
{
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
        for (int i = 0; i < D; ++i) {
            R s = B[c][0] * Jinv[0][i];
#pragma unroll
            for (int k = 1; k < D; ++k) s = fma(B[c][k], Jinv[k][i], s);
            A[c][i] = s;
        }
}

// e[c][k] = sum_i S[c][i] Jinv[k][i]  (physical stress -> reference test weights)
template <int D, typename R>
__device__ __forceinline__ void pull_back(const R (&S)[D][D], const R (&Jinv)[D][D], R (&e)[D][D])
{
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
        for (int k = 0; k < D; ++k) {
            R s = S[c][0] * Jinv[k][0];
#pragma unroll
            for (int i = 1; i < D; ++i) s = fma(S[c][i], Jinv[k][i], s);
            e[c][k] = s;
        }
}

template <int A, int B, typename T, typename U>
__device__ __forceinline__ void convert(const T (&x)[A][B], U (&y)[A][B])
{
#pragma unroll
    for (int i = 0; i < A; ++i)
#pragma unroll
        for (int k = 0; k < B; ++k) y[i][k] = cvt<U>(x[i][k]);
}

// Internal operation ids (forms of the public API plus the Neo-Hookean adjoint).
enum Op {
    OP_MASS = 0,
    OP_ELASTICITY = 1,
    OP_NH_RESIDUAL = 2,
    OP_NH_JACOBIAN = 3,
    OP_NH_ADJOINT = 4,
    OP_LAPLACE = 5,
    OP_HELMHOLTZ = 6,
    OP_SVK_RESIDUAL = 7,
    OP_SVK_JACOBIAN = 8
};

// Public form kind (enum fe_form_kind) of an operation; the adjoint belongs to
// the Neo-Hookean residual.
__host__ __device__ constexpr int form_of(int op)
{
    return op == OP_NH_ADJOINT     ? FE_FORM_NH_RESIDUAL
           : op == OP_LAPLACE      ? FE_FORM_LAPLACE
           : op == OP_HELMHOLTZ    ? FE_FORM_HELMHOLTZ
           : op == OP_SVK_RESIDUAL ? FE_FORM_SVK_RESIDUAL
           : op == OP_SVK_JACOBIAN ? FE_FORM_SVK_JACOBIAN
                                   : op;
}

template <int OP, int D>
struct OpTraits {
    static constexpr bool kScalar = (OP == OP_MASS || OP == OP_LAPLACE || OP == OP_HELMHOLTZ);
    static constexpr int NC = kScalar ? 1 : D;
    static constexpr bool kTwoFields = (OP == OP_NH_JACOBIAN || OP == OP_NH_ADJOINT || OP == OP_SVK_JACOBIAN);
    static constexpr bool kCellCoeff = (OP == OP_NH_RESIDUAL || OP == OP_NH_JACOBIAN || OP == OP_NH_ADJOINT ||
                                        OP == OP_SVK_RESIDUAL || OP == OP_SVK_JACOBIAN);
    // the law needs FP64 pointwise evaluation (hyperelastic forms)
    static constexpr bool kNonlinear = kCellCoeff;
};

// St. Venant-Kirchhoff law (Appendix A, Hyperelasticity) at one point, FP64:
// F = I + G, E = (F^T F - I)/2, S = lambda tr(E) I + 2 mu E.  For the Jacobian
// action, with H = grad du: dE = (H^T F + F^T H)/2, dS = lambda tr(dE) I +
// 2 mu dE and dP = H S + F dS; for the residual P = F S.  Writes P (or dP),
// already multiplied by scale.
template <int D, bool kTangent>
__device__ __forceinline__ void svk_stress(const double (&G)[D][D], const double (&H)[D][D], double mu,
                                           double lam, double scale, double (&P)[D][D])
{
    double F[D][D], E[D][D], S[D][D];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int k = 0; k < D; ++k) F[i][k] = G[i][k] + (i == k ? 1.0 : 0.0);
    double trE = 0.0;
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int k = i; k < D; ++k) {
            double c = F[0][i] * F[0][k];
#pragma unroll
            for (int m = 1; m < D; ++m) c = fma(F[m][i], F[m][k], c);
            E[i][k] = 0.5 * (c - (i == k ? 1.0 : 0.0));
            E[k][i] = E[i][k];
        }
#pragma unroll
    for (int i = 0; i < D; ++i) trE += E[i][i];
    const double m2 = 2.0 * mu * scale, lt = lam * trE * scale;
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int k = 0; k < D; ++k) S[i][k] = fma(m2, E[i][k], i == k ? lt : 0.0);
    if constexpr (!kTangent) {
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int k = 0; k < D; ++k) {
                double p = F[i][0] * S[0][k];
#pragma unroll
                for (int m = 1; m < D; ++m) p = fma(F[i][m], S[m][k], p);
                P[i][k] = p;
            }
    } else {
        double dE[D][D], dS[D][D];
        double trdE = 0.0;
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int k = i; k < D; ++k) {
                double c = fma(H[0][i], F[0][k], F[0][i] * H[0][k]);
#pragma unroll
                for (int m = 1; m < D; ++m) c = fma(H[m][i], F[m][k], fma(F[m][i], H[m][k], c));
                dE[i][k] = 0.5 * c;
                dE[k][i] = dE[i][k];
            }
#pragma unroll
        for (int i = 0; i < D; ++i) trdE += dE[i][i];
        const double ldt = lam * trdE * scale;
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int k = 0; k < D; ++k) dS[i][k] = fma(m2, dE[i][k], i == k ? ldt : 0.0);
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int k = 0; k < D; ++k) {
                double p = fma(H[i][0], S[0][k], F[i][0] * dS[0][k]);
#pragma unroll
                for (int m = 1; m < D; ++m) p = fma(H[i][m], S[m][k], fma(F[i][m], dS[m][k], p));
                P[i][k] = p;
            }
    }
}

template <int D, int N, int NC>
__device__ __forceinline__ bool gather_nodes(const int32_t *__restrict__ c2n, int cell, int n_nodes,
                                             int (&nodes)[N])
{
    bool ok = true;
    const int32_t *row = c2n + (size_t)cell * N;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const int v = __ldg(row + j);
        ok &= (unsigned)v < (unsigned)n_nodes;
        nodes[j] = v;
    }
    return ok;
}

// Gather DoFs (double in memory) into the contraction type R.
template <int N, int NC, typename R, bool kRel = false>
__device__ __forceinline__ void gather_dofs(const double *__restrict__ u, const int (&nodes)[N],
                                            R (&l)[N][NC])
{
    // kRel: the DoFs relative to the cell's first node, differenced in FP64 before
    // the conversion to R.  The basis gradients sum to zero, so the gradients are
    // unchanged and node 0's term vanishes exactly (its difference is 0); the R
    // operands carry only the cell-local variation, which a smooth field would
    // otherwise lose to cancellation when its values are rounded to FP32.
    double base[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) base[c] = 0.0;
    if constexpr (kRel) {
#pragma unroll
        for (int c = 0; c < NC; ++c) base[c] = __ldg(u + (size_t)nodes[0] * NC + c);
    }
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const double *p = u + (size_t)nodes[j] * NC;
        if constexpr (NC == 2) {
            const double2 v = __ldg(reinterpret_cast<const double2 *>(p));
            l[j][0] = cvt<R>(kRel ? v.x - base[0] : v.x);
            l[j][1] = cvt<R>(kRel ? v.y - base[1] : v.y);
        } else {
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const double v = __ldg(p + c);
                l[j][c] = cvt<R>(kRel ? v - base[c] : v);
            }
        }
    }
}

// Table block layout in shared memory: tab [nq][1+D][N] in R, padded to a
// multiple of 8 bytes, then the weights [nq] in double, then the weights [nq]
// again in R (used by forms whose pointwise work runs in R).
template <typename R>
__host__ __device__ constexpr size_t table_weights_offset_bytes(int nq, int d, int n)
{
    return ((size_t)nq * (d + 1) * n * sizeof(R) + 7) & ~(size_t)7;
}

// Node-gather scatter: a skipped cell's outputs are zeros, so that the gather
// does not sum values of an earlier call.
template <int N, int NC, typename R>
__device__ __forceinline__ void store_zero_cell(const ActionArgs &a, int cell)
{
    if (!a.cell_out) return;
    R *o = static_cast<R *>(a.cell_out) + (size_t)cell * N * NC;
#pragma unroll
    for (int i = 0; i < N * NC; ++i) o[i] = R(0);
}

// One cell of Algorithm 2 for operation OP, contractions in R.  Geometry, the
// quadrature weights, the Neo-Hookean kinematics/stress and the scatter are
// always FP64.
// Shared-memory aggregation of the scatter (FP32 thread-per-cell mass kernels):
// the 128 cells of a CTA's tile share many nodes on a mesh numbered for
// locality (a 128-cell run of the structured P3 triangle mesh touches ~400
// distinct nodes through 1,280 cell-node incidences), so their updates are
// first summed per node in an open-addressing hash table in shared memory and
// then added to y with one global reduction per distinct node.  For large y
// the scatter's reductions dominate this gather/scatter-bound kernel, and
// cutting them by the sharing factor pays (mass P3 on 3.6M triangles: 0.48 ->
// 0.29 ms, y larger than L2; 0.103 -> 0.092 ms on 0.9M triangles).  Measured on
// the vector forms (elasticity P1/P2 tetrahedra, structured or random
// numbering), on Helmholtz and the Laplacian with y in L2, the table's atomics
// cost more than they save, so plans enable it only for mass, with y of at
// least 16 MB and a numbering whose tiles share nodes.
// agg_slots_for(N) >= 128 N slots: a tile has at most 128 N distinct nodes, so
// an insertion always finds a slot; on the meshes plans enable it for (tiles
// that share nodes) the table is at most ~60 % full.  (Twice the slots made the
// per-tile flush and the shared memory per CTA larger and the kernel slower:
// 0.29 -> 0.38 ms at 16M DoFs.)
__host__ __device__ constexpr int agg_slots_for(int n_loc)
{
    int s = 1;
    while (s < kTpcBlock * n_loc) s <<= 1;
    return s;
}

template <int NC>
struct AggTable {
    int *keys;     // [slots] node id, or -1
    float *vals;   // [slots][NC] partial sums
    int slots;     // power of two
};

// Slot of `node` in the table, inserting it if absent (linear probing from a
// multiplicative hash).  Returns -1 only if the table is full.
template <int NC>
__device__ __forceinline__ int agg_slot(const AggTable<NC> &t, int node)
{
    const int shift = 32 - (31 - __clz(t.slots));
    unsigned h = ((unsigned)node * 0x9E3779B1u) >> shift;
    for (int probe = 0; probe < t.slots; ++probe) {
        const int prev = atomicCAS(t.keys + h, -1, node);
        if (prev == -1 || prev == node) return (int)h;
        h = (h + 1) & (unsigned)(t.slots - 1);
    }
    return -1;
}

// WF: the table's rows of point q are scaled by sqrt(w_q) (FP64 plans of the
// linear forms; see the plan's table construction).  The evaluation then
// yields sqrt(w_q) times the values / reference gradients, the pointwise form is
// linear in them and the quadrature contraction supplies the other sqrt(w_q), so
// w_q |det J| becomes the per-cell |det J| and its per-point products drop out.
template <int OP, int D, int P, typename R, int AGG_NC = 0, bool WF = false>
__device__ __forceinline__ void action_cell(const ActionArgs &a, const R *__restrict__ tab,
                                            const double *__restrict__ wts, const R *__restrict__ wts_r,
                                            int cell, const AggTable<(AGG_NC > 0 ? AGG_NC : 1)> *agg = nullptr)
{
    constexpr int N = nloc(D, P);
    constexpr int NC = OpTraits<OP, D>::NC;
    constexpr bool kMixed = !std::is_same<R, double>::value;

    // gather coordinates (Algorithm 2: gather of coords through iota_P1)
    int vtx[D + 1];
    bool ok = true;
#pragma unroll
    for (int m = 0; m <= D; ++m) {
        vtx[m] = __ldg(a.c2v + (size_t)cell * (D + 1) + m);
        ok &= (unsigned)vtx[m] < (unsigned)a.n_vertices;
    }
    int nodes[N];
    ok &= gather_nodes<D, N, NC>(a.c2n, cell, a.n_nodes, nodes);
    if (!ok) {
        set_status(a.status, FE_ERR_INDEX);
        store_zero_cell<N, NC, R>(a, cell);
        return;
    }
    double X[D + 1][D];
#pragma unroll
    for (int m = 0; m <= D; ++m) {
        if constexpr (D == 2) {
            const double2 v = __ldg(reinterpret_cast<const double2 *>(a.coords + (size_t)vtx[m] * 2));
            X[m][0] = v.x;
            X[m][1] = v.y;
        } else {
#pragma unroll
            for (int i = 0; i < D; ++i) X[m][i] = __ldg(a.coords + (size_t)vtx[m] * D + i);
        }
    }
    // geometry: J, det J, J^{-1}, once per cell (affine), in FP64
    double Jinv[D][D];
    const double det = cell_geometry<D>(X, Jinv);
    if (!(det != 0.0) || !isfinite(det)) {
        set_status(a.status, FE_ERR_BAD_MESH);
        store_zero_cell<N, NC, R>(a, cell);
        return;
    }
    const double absdet = fabs(det);
    const R absdet_r = cvt<R>(absdet);
    [[maybe_unused]] R Jinv_r[D][D];
    if constexpr (kMixed) convert<D, D>(Jinv, Jinv_r);

    // gather DoFs
    R l[N][NC];
    // hyperelastic forms in reduced precision use only gradients: gather relative
    // to node 0 (see gather_dofs)
    constexpr bool kRel = kMixed && OpTraits<OP, D>::kNonlinear;
    gather_dofs<N, NC, R, kRel>(a.u, nodes, l);
    [[maybe_unused]] R l0[OpTraits<OP, D>::kTwoFields ? N : 1][NC];
    if constexpr (OpTraits<OP, D>::kTwoFields) gather_dofs<N, NC, R, kRel>(a.u_lin, nodes, l0);
    double mu = a.mu, lam = a.lam;
    if constexpr (OpTraits<OP, D>::kCellCoeff) {
        if (a.mu_cell) mu = __ldg(a.mu_cell + cell);
        if (a.lam_cell) lam = __ldg(a.lam_cell + cell);
    }

    R out[N][NC];
#pragma unroll
    for (int j = 0; j < N; ++j)
#pragma unroll
        for (int c = 0; c < NC; ++c) out[j][c] = R(0);
    [[maybe_unused]] double acc_mu = 0.0, acc_lam = 0.0;
    bool nh_ok = true;

    [[maybe_unused]] const R mu_r = cvt<R>(mu), lam_r = cvt<R>(lam);
    // weight-folded elasticity: mu |det J|, 2 mu |det J| and lambda |det J| per cell
    [[maybe_unused]] const R c_smu = WF ? mu_r * absdet_r : R(0), c_smu2 = R(2) * c_smu,
                             c_slam = WF ? lam_r * absdet_r : R(0);
    // weight-folded Laplacian / Helmholtz: M = |det J| J^{-1} J^{-T} per cell, so that
    // the gradient term at a point is M times the reference gradient
    constexpr bool kFoldM = WF && (OP == OP_LAPLACE || OP == OP_HELMHOLTZ);
    [[maybe_unused]] R Mw[kFoldM ? D : 1][D];
    if constexpr (kFoldM) {
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
            for (int k = 0; k < D; ++k) {
                double mk = Jinv[i][0] * Jinv[k][0];
#pragma unroll
                for (int r = 1; r < D; ++r) mk = fma(Jinv[i][r], Jinv[k][r], mk);
                Mw[i][k] = absdet * mk;
            }
    }
    for (int q = 0; q < a.nq; ++q) {
        const R *__restrict__ T = tab + (size_t)q * (D + 1) * N;
        // w_q |det J| in R for the forms evaluated in R, in FP64 for Neo-Hookean
        [[maybe_unused]] const R wdet_r = WF ? absdet_r : wts_r[q] * absdet_r;
        if constexpr (OP == OP_MASS) {
            R uq = R(0);
#pragma unroll
            for (int j = 0; j < N; ++j) uq = fma(T[j], l[j][0], uq);
            const R e = uq * wdet_r;
#pragma unroll
            for (int j = 0; j < N; ++j) out[j][0] = fma(T[j], e, out[j][0]);
        } else if constexpr (OP == OP_LAPLACE || OP == OP_HELMHOLTZ) {
            // grad u . grad v (+ u v): scalar gradient mapped with J^{-1}, pulled back
            R gs[D];
#pragma unroll
            for (int k = 0; k < D; ++k) gs[k] = R(0);
#pragma unroll
            for (int j = 0; j < N; ++j)
#pragma unroll
                for (int k = 0; k < D; ++k)
                    if (!grad_zero<D, N>(k, j)) gs[k] = fma(T[(k + 1) * N + j], l[j][0], gs[k]);
            R e[D];
            if constexpr (kFoldM) {
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    R s = Mw[k][0] * gs[0];
#pragma unroll
                    for (int i = 1; i < D; ++i) s = fma(Mw[k][i], gs[i], s);
                    e[k] = s;
                }
            } else {
                R g[D];
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    R s = R(0);
#pragma unroll
                    for (int k = 0; k < D; ++k) s = fma(gs[k], kMixed ? Jinv_r[k][i] : R(Jinv[k][i]), s);
                    g[i] = s * wdet_r;
                }
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    R s = R(0);
#pragma unroll
                    for (int i = 0; i < D; ++i) s = fma(g[i], kMixed ? Jinv_r[k][i] : R(Jinv[k][i]), s);
                    e[k] = s;
                }
            }
            [[maybe_unused]] R ev = R(0);
            if constexpr (OP == OP_HELMHOLTZ) {
                R uq = R(0);
#pragma unroll
                for (int j = 0; j < N; ++j) uq = fma(T[j], l[j][0], uq);
                ev = uq * wdet_r;
            }
#pragma unroll
            for (int j = 0; j < N; ++j) {
                R o = out[j][0];
                if constexpr (OP == OP_HELMHOLTZ) o = fma(T[j], ev, o);
#pragma unroll
                for (int k = 0; k < D; ++k)
                    if (!grad_zero<D, N>(k, j)) o = fma(T[(k + 1) * N + j], e[k], o);
                out[j][0] = o;
            }
        } else if constexpr (OP == OP_SVK_RESIDUAL || OP == OP_SVK_JACOBIAN) {
            // St. Venant-Kirchhoff law in FP64 (contractions in R)
            const double wdet = wts[q] * absdet;
            R ghr[D][D], er[D][D];
            double gh[D][D], G[D][D], H[D][D], Pk[D][D], e[D][D];
            if constexpr (OP == OP_SVK_JACOBIAN) {
                eval_grad<D, N, D, R>(T, l0, ghr);   // linearisation point
                convert<D, D>(ghr, gh);
                map_grad<D, double>(gh, Jinv, G);
                eval_grad<D, N, D, R>(T, l, ghr);    // direction du
                convert<D, D>(ghr, gh);
                map_grad<D, double>(gh, Jinv, H);
            } else {
                eval_grad<D, N, D, R>(T, l, ghr);
                convert<D, D>(ghr, gh);
                map_grad<D, double>(gh, Jinv, G);
            }
            svk_stress<D, OP == OP_SVK_JACOBIAN>(G, H, mu, lam, wdet, Pk);
            pull_back<D, double>(Pk, Jinv, e);
            convert<D, D>(e, er);
            quad_grad<D, N, D, R>(T, er, out);
        } else if constexpr (OP == OP_ELASTICITY) {
            // linear stress: evaluated in the contraction type
            R gh[D][D], G[D][D], S[D][D], e[D][D];
            eval_grad<D, N, D, R>(T, l, gh);
            if constexpr (kMixed)
                map_grad<D, R>(gh, Jinv_r, G);
            else
                map_grad<D, R>(gh, Jinv, G);
            R tr = G[0][0];
#pragma unroll
            for (int i = 1; i < D; ++i) tr += G[i][i];
            const R smu = WF ? c_smu : wdet_r * mu_r;
            const R smu2 = WF ? c_smu2 : R(2) * smu;
            const R slt = WF ? c_slam * tr : wdet_r * lam_r * tr;
#pragma unroll
            for (int i = 0; i < D; ++i) {
                S[i][i] = fma(smu2, G[i][i], slt);
#pragma unroll
                for (int k = i + 1; k < D; ++k) {
                    const R s = smu * (G[i][k] + G[k][i]);
                    S[i][k] = s;
                    S[k][i] = s;
                }
            }
            if constexpr (kMixed)
                pull_back<D, R>(S, Jinv_r, e);
            else
                pull_back<D, R>(S, Jinv, e);
            quad_grad<D, N, D, R>(T, e, out);
        } else if constexpr (OP == OP_NH_RESIDUAL) {
            const double wdet = wts[q] * absdet;
            R ghr[D][D], er[D][D];
            double gh[D][D], F[D][D], C[D][D], S[D][D], e[D][D];
            eval_grad<D, N, D, R>(T, l, ghr);
            convert<D, D>(ghr, gh);
            map_grad<D, double>(gh, Jinv, F);
#pragma unroll
            for (int i = 0; i < D; ++i) F[i][i] += 1.0;
            const double Jd = det_cof<D>(F, C);  // F^{-T} = C / Jd
            nh_ok &= (Jd > 0.0);
            const double lnJ = law_log(Jd, a.log_tab);
            // P = mu F + (lam lnJ - mu) F^{-T}, scaled by w_q |det J|
            const double smu = wdet * mu;
            const double scf = wdet * fma(lam, lnJ, -mu) * (a.log_tab ? fe_rcp(Jd) : 1.0 / Jd);
#pragma unroll
            for (int i = 0; i < D; ++i)
#pragma unroll
                for (int k = 0; k < D; ++k) S[i][k] = fma(smu, F[i][k], scf * C[i][k]);
            pull_back<D, double>(S, Jinv, e);
            convert<D, D>(e, er);
            quad_grad<D, N, D, R>(T, er, out);
        } else {  // OP_NH_JACOBIAN / OP_NH_ADJOINT: tangent applied to H = grad(du) (or grad w)
            const double wdet = wts[q] * absdet;
            R ghr[D][D], er[D][D];
            double gh[D][D], F[D][D], H[D][D], C[D][D], Fit[D][D], A[D][D], S[D][D], e[D][D];
            eval_grad<D, N, D, R>(T, l0, ghr);
            convert<D, D>(ghr, gh);
            map_grad<D, double>(gh, Jinv, F);
#pragma unroll
            for (int i = 0; i < D; ++i) F[i][i] += 1.0;
            eval_grad<D, N, D, R>(T, l, ghr);
            convert<D, D>(ghr, gh);
            map_grad<D, double>(gh, Jinv, H);
            const double Jd = det_cof<D>(F, C);
            nh_ok &= (Jd > 0.0);
            const double rJ = a.log_tab ? fe_rcp(Jd) : 1.0 / Jd;
            const double lnJ = law_log(Jd, a.log_tab);
            double tr = 0.0;  // tr(F^{-1} H) = F^{-T} : H
#pragma unroll
            for (int i = 0; i < D; ++i)
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    Fit[i][k] = C[i][k] * rJ;
                    tr = fma(Fit[i][k], H[i][k], tr);
                }
            // A = F^{-T} H^T ; M = A F^{-T}
#pragma unroll
            for (int i = 0; i < D; ++i)
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    double s = Fit[i][0] * H[k][0];
#pragma unroll
                    for (int m = 1; m < D; ++m) s = fma(Fit[i][m], H[k][m], s);
                    A[i][k] = s;
                }
            const double smu = wdet * mu;
            const double sm2 = wdet * fma(-lam, lnJ, mu);  // (mu - lam lnJ)
            const double str = wdet * lam * tr;
#pragma unroll
            for (int i = 0; i < D; ++i)
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    double m = A[i][0] * Fit[0][k];
#pragma unroll
                    for (int mm = 1; mm < D; ++mm) m = fma(A[i][mm], Fit[mm][k], m);
                    S[i][k] = fma(smu, H[i][k], fma(sm2, m, str * Fit[i][k]));
                }
            if constexpr (OP == OP_NH_ADJOINT) {
                // dr/dmu . w = (F - F^{-T}) : grad w ; dr/dlam . w = lnJ F^{-T} : grad w
#pragma unroll
                for (int i = 0; i < D; ++i)
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        acc_mu = fma(wdet * (F[i][k] - Fit[i][k]), H[i][k], acc_mu);
                        acc_lam = fma(wdet * lnJ * Fit[i][k], H[i][k], acc_lam);
                    }
            }
            pull_back<D, double>(S, Jinv, e);
            convert<D, D>(e, er);
            quad_grad<D, N, D, R>(T, er, out);
        }
    }
    if (!nh_ok) set_status(a.status, FE_ERR_NONFINITE);

    // scatter (Algorithm 2): FP64 atomics into y, or the cell's outputs stored for
    // the node-gather scatter (the adjoint always adds into its output)
    if (OP != OP_NH_ADJOINT && a.cell_out) {
        R *o = static_cast<R *>(a.cell_out) + (size_t)cell * N * NC;
#pragma unroll
        for (int j = 0; j < N; ++j)
#pragma unroll
            for (int c = 0; c < NC; ++c) o[j * NC + c] = out[j][c];
    } else if constexpr (AGG_NC > 0) {
        static_assert(AGG_NC == NC && std::is_same<R, float>::value, "aggregation: FP32, one slot per node");
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const int slot = agg_slot<NC>(*agg, nodes[j]);
            if (slot >= 0) {
#pragma unroll
                for (int c = 0; c < NC; ++c) atomicAdd(agg->vals + slot * NC + c, out[j][c]);
            } else {
#pragma unroll
                for (int c = 0; c < NC; ++c) red_add(a.y + (size_t)nodes[j] * NC + c, cvt<double>(out[j][c]));
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < N; ++j)
#pragma unroll
            for (int c = 0; c < NC; ++c) red_add(a.y + (size_t)nodes[j] * NC + c, cvt<double>(out[j][c]));
    }
    if constexpr (OP == OP_NH_ADJOINT) {
        a.dmu[cell] = acc_mu;   // one thread per cell: plain stores, no reduction
        a.dlam[cell] = acc_lam;
    }
}

// Warp-level work queue: each warp takes chunks of 32 consecutive cells (one per
// lane) from a global counter until the cells run out, so SMs that finish early
// take more work and the tail is at most one chunk.  The last warp to leave
// resets both counters, so every launch starts from zero without a memset.
// No fence is needed: every fetch from the first counter is an atomic whose
// returned value the fetching thread used before its warp (or, for the CTA-level
// queues, its CTA after a barrier) reached this point, so all fetches are
// performed before the leave count reaches the last warp; and the next launch
// sees the reset through the kernel boundary.  (A fence here would make each
// warp wait for its scatter reductions before it leaves.)
__device__ __forceinline__ void leave_queue(int32_t *sched)
{
    if ((threadIdx.x & 31) == 0) {
        const int total_warps = (int)(gridDim.x * (blockDim.x >> 5));
        if (atomicAdd(sched + 1, 1) == total_warps - 1) {
            sched[0] = 0;
            sched[1] = 0;
        }
    }
}

// Resident CTAs per SM the compiler must allow (register cap 65536 / (128 x this)).
// Measured with FP32 contractions: the Neo-Hookean residual P4 triangles runs
// 287 -> 262 us with five (at most 102 registers, no more spills than it can
// hide); elasticity P2 tets gets slower with any cap (52.9 -> 57.0 us at five,
// 66.2 us at eight: the spills cost more than the extra warps return), so every
// other variant (the tetrahedral Neo-Hookean ones included) keeps the compiler's
// choice.
template <int OP, int D, typename R>
__host__ __device__ constexpr int tpc_min_blocks()
{
    return (OP == OP_NH_RESIDUAL && D == 2 && sizeof(R) == 4) ? 5 : 1;
}

template <int OP, int D, int P, typename R, bool WF = false>
__global__ void __launch_bounds__(kTpcBlock, tpc_min_blocks<OP, D, R>()) k_action_tpc(const ActionArgs a)
{
    extern __shared__ __align__(128) double smem[];
    __shared__ __align__(8) uint64_t bar;
    if (!stage_table(smem, a.tab, a.tab_doubles, &bar, a.status)) {
        leave_queue(a.sched);
        return;
    }
    constexpr int N = nloc(D, P);
    const R *tab = reinterpret_cast<const R *>(smem);
    const double *wts = reinterpret_cast<const double *>(
        reinterpret_cast<const char *>(smem) + table_weights_offset_bytes<R>(a.nq, D, N));
    const R *wts_r = reinterpret_cast<const R *>(wts + a.nq);
    const int lane = threadIdx.x & 31;
    const int n_chunks = (a.n_cells + 31) >> 5;
    for (;;) {
        int chunk = 0;
        if (lane == 0) chunk = atomicAdd(a.sched, 1);
        chunk = __shfl_sync(0xffffffffu, chunk, 0);
        if (chunk >= n_chunks) break;
        const int cell = (chunk << 5) + lane;
        if (cell < a.n_cells) action_cell<OP, D, P, R, 0, WF>(a, tab, wts, wts_r, cell);
    }
    leave_queue(a.sched);
}

// Thread-per-cell kernel with the scatter aggregated per CTA tile in shared
// memory (see agg_slots_for).  The CTA takes tiles of blockDim.x consecutive
// cells from a CTA-level queue; after each tile its threads flush the table:
// one reduction per distinct node and component, slots reset for the next tile.
// Shared memory: the staged table block, then keys [slots] and vals [slots][NC].
template <int OP, int D, int P, typename R>
__global__ void __launch_bounds__(kTpcBlock) k_action_tpc_agg(const ActionArgs a)
{
    extern __shared__ __align__(128) double smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_tile;
    constexpr int N = nloc(D, P);
    constexpr int NC = OpTraits<OP, D>::NC;
    if (!stage_table(smem, a.tab, a.tab_doubles, &bar, a.status)) {
        leave_queue(a.sched);
        return;
    }
    const R *tab = reinterpret_cast<const R *>(smem);
    const double *wts = reinterpret_cast<const double *>(
        reinterpret_cast<const char *>(smem) + table_weights_offset_bytes<R>(a.nq, D, N));
    const R *wts_r = reinterpret_cast<const R *>(wts + a.nq);
    AggTable<NC> t;
    t.slots = a.agg_slots;
    t.keys = reinterpret_cast<int *>(smem + a.tab_doubles);
    t.vals = reinterpret_cast<float *>(t.keys + t.slots);
    for (int i = threadIdx.x; i < t.slots; i += blockDim.x) {
        t.keys[i] = -1;
#pragma unroll
        for (int c = 0; c < NC; ++c) t.vals[i * NC + c] = 0.0f;
    }
    const int n_tiles = (a.n_cells + (int)blockDim.x - 1) / (int)blockDim.x;
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(a.sched, 1);
        __syncthreads();   // also orders the table reset before the first insertions
        const int tile = s_tile;
        if (tile >= n_tiles) break;
        const int cell = tile * (int)blockDim.x + (int)threadIdx.x;
        if (cell < a.n_cells) action_cell<OP, D, P, R, NC>(a, tab, wts, wts_r, cell, &t);
        __syncthreads();
        for (int i = threadIdx.x; i < t.slots; i += blockDim.x) {
            const int node = t.keys[i];
            if (node >= 0) {
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    red_add(a.y + (size_t)node * NC + c, cvt<double>(t.vals[i * NC + c]));
                    t.vals[i * NC + c] = 0.0f;
                }
                t.keys[i] = -1;
            }
        }
        // the next tile's insertions start after the barrier at the top of the loop
    }
    leave_queue(a.sched);
}

template <int OP, int D, int P, typename R, bool WF = false>
cudaError_t launch_tpc(const ActionArgs &a, int grid, int block, size_t smem, cudaStream_t s)
{
    if constexpr (std::is_same<R, float>::value && OP == OP_MASS) {
        if (a.agg_slots > 0) {
            k_action_tpc_agg<OP, D, P, R><<<grid, block, smem, s>>>(a);
            return cudaGetLastError();
        }
    }
    k_action_tpc<OP, D, P, R, WF><<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
}

// WF: the variant takes weight-folded tables (action_cell)
template <int OP, int D, int P, typename R = double, bool WF = false>
Variant make_tpc_variant()
{
    Variant v;
    v.form = form_of(OP);
    v.dim = D;
    v.degree = P;
    v.op = OP == OP_NH_ADJOINT ? 1 : 0;
    v.precision = std::is_same<R, double>::value ? FE_PREC_FP64 : FE_PREC_FP32;
    v.kernel_id = 0;
    v.block = kTpcBlock;
    static_assert(!WF || (std::is_same<R, double>::value && (OP == OP_MASS || OP == OP_ELASTICITY ||
                                                             OP == OP_LAPLACE || OP == OP_HELMHOLTZ)),
                  "weight-folded tables: the FP64 linear forms");
    v.wfold = WF;
    v.launch = &launch_tpc<OP, D, P, R, WF>;
    v.func = reinterpret_cast<const void *>(&k_action_tpc<OP, D, P, R, WF>);
    if constexpr (std::is_same<R, float>::value && OP == OP_MASS)
        v.func_agg = reinterpret_cast<const void *>(&k_action_tpc_agg<OP, D, P, R>);
    return v;
}

}  // namespace fe
