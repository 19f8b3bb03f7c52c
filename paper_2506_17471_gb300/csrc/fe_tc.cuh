// Tensor-core (tcgen05) action with 16-bit contractions for high-degree cells.
//
// A tile of 128 cells runs the two contractions of Algorithm 2 as GEMMs with
// the cells on the M dimension:
//   evaluation:  E_m[c, (q,k)] = sum_j  U_m[c, j] Phi_k[q][j]          (per component m)
//   quadrature:  Y_m[c, j]     = sum_{(q,k)} E'_m[c, (q,k)] Phi_k[q][j]
// U_m holds the tile's gathered DoFs, E'_m the weighted pointwise stress pulled
// back to the reference cell (Sec. "Towards Discretization": evaluation,
// pointwise and quadrature phases).  Row c of every GEMM is cell c, which is
// TMEM lane c and thread c of the tile (or its tpc threads, each taking every
// tpc-th node batch, column block and output group, the cell's geometry computed
// by the first and shared where shared memory allows): the cell's thread gathers
// its cell, reads its own accumulator row with tcgen05.ld, evaluates the
// pointwise form for its cell at every point and scatter-adds its own result,
// like the thread-per-cell kernel, while the contractions run on the
// tensor cores (tcgen05.mma kind::f16, BF16 or FP16 operands, FP32 accumulators
// in TMEM, issued by one thread, completion through tcgen05.commit and an
// mbarrier with a bounded wait).
//
// The tabulation operands (Phi as the evaluation GEMM's B, Phi^T as the
// quadrature GEMM's B) are laid out by the plan in the tensor cores' K-major
// core-matrix layout and staged once per CTA by one bulk copy.  Quadrature
// points are processed in chunks of qc points so the evaluation accumulators of
// a chunk and the quadrature accumulators of the whole tile fit in TMEM; the
// quadrature GEMM accumulates over the chunks.  A CTA runs one to four
// independent 128-cell pipelines (128 threads each) that share the staged
// tables, split the SM's 512 TMEM columns and synchronise with named barriers:
// a CTA that uses tensor memory is resident alone on its SM, so the pipelines
// are what hides one another's gather, MMA and scatter latency.
//
// Precision: for the gradient-only forms (elasticity, Neo-Hookean) each
// cell's DoFs are first shifted by a per-cell constant c (the midrange of each
// component, FP64): the basis gradients sum to zero, so grad u = grad (u - c)
// exactly, and the 16-bit operands carry only the cell-local variation of the
// field (a smooth field no longer loses its gradient to cancellation).  The
// shifted DoFs (mass: the DoFs) are scaled per cell by a power of two
// s_u > max |u - c| and rounded to 16 bits; J^{-1} is scaled by a power of two
// s_J > max |J^{-1}_ik|.  The pointwise values then stay O(1) whatever the
// mesh size and field magnitude (FP16 neither overflows nor goes subnormal).
// The output factor |det J| s_u s_J^2 is applied as an FP32 multiply by the
// significand of |det J| (relative error 2^-24, far below the 16-bit
// rounding) and an exponent add on the widened FP64 value.  All power-of-two
// scalings are exponent arithmetic on the bit patterns: on this part FP64
// instructions issue at about 1/64 of the FP32 rate, and the only ones left are
// the FP64 geometry (det J, J^{-1}), the offset subtraction u - c and the FP64
// scatter-add.  The rounding of u - c to 16 bits narrows it to binary32 by
// rounding to odd with integer operations and leaves the last rounding to the
// hardware's binary32 conversion (pack2_from_f64).
//
// Operand layout (K-major, no swizzle): 8x8 core matrices of 16-bit elements
// (128 bytes), ordered [row group][K group][row][col]; LBO = 128 B between
// K-adjacent core matrices, SBO = (Kp/8) * 128 B between row groups.
#pragma once

#include <climits>
#include <cstring>
#include <type_traits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fe_kernels.cuh"

namespace fe {

constexpr int kTcRows = 128;   // cells (threads, TMEM lanes) per pipeline
constexpr int kTcMaxPipes = 4; // pipelines per CTA (a CTA that uses TMEM has an SM to itself)

__host__ __device__ inline int tc_round_up(int x, int m) { return (x + m - 1) / m * m; }
__host__ __device__ inline size_t tc_round_up_sz(size_t x, size_t m) { return (x + m - 1) / m * m; }

// Tile geometry, computed identically by the plan and the kernel.
struct TcLayout {
    int n, nq, NC, KD, KDP, F;   // KD derivative terms per point (KDP: padded to 1, 2 or 4); F fields
    int qc, nch;                 // points per chunk, chunks
    int N1p, K1p;                // evaluation GEMM: N (chunk columns), K (n padded to 16)
    int N2p, K2;                 // quadrature GEMM: N (n padded to 16), K (nch * N1p)
    int pipes;
    int terms;                   // terms per operand: 1, or 2 (hi + lo binary16 pairs)
    int esz;                     // operand element bytes: 2 (BF16, FP16) or 4 (TF32)
    size_t b1_off, b2_off, wd_off, wf_off, staged_bytes;   // staged block
    size_t a1_off, a2_off, nodes_off, pipe_bytes;          // per-pipeline scratch (from its base)
    size_t total;                                          // dynamic shared memory
    int acc1_cols, acc2_cols, pipe_cols, tmem_cols;
};

__host__ __device__ inline int tc_kdp(int kd) { return kd == 1 ? 1 : (kd == 2 ? 2 : 4); }

__host__ __device__ inline TcLayout tc_layout(int n, int nq, int NC, int KD, int F, int qc, int pipes,
                                              int terms = 1, int esz = 2)
{
    TcLayout L;
    L.n = n;
    L.nq = nq;
    L.NC = NC;
    L.KD = KD;
    L.KDP = tc_kdp(KD);
    L.F = F;
    L.qc = qc < 1 ? 1 : qc;
    L.nch = (nq + L.qc - 1) / L.qc;
    L.N1p = tc_round_up(L.qc * L.KDP, 16);
    L.K1p = tc_round_up(n, 16);
    L.N2p = tc_round_up(n, 16);
    L.K2 = L.nch * L.N1p;
    L.pipes = pipes;
    L.terms = terms;
    L.esz = esz;
    // every operand region is repeated per term (term 0 = hi, term 1 = lo)
    L.b1_off = 0;
    L.b2_off = (size_t)terms * L.nch * L.N1p * L.K1p * esz;
    L.wd_off = L.b2_off + (size_t)terms * L.N2p * L.K2 * esz;
    L.wf_off = L.wd_off + (size_t)nq * 8;
    L.staged_bytes = tc_round_up_sz(L.wf_off + (size_t)nq * 4, 128);
    L.a1_off = 0;
    L.a2_off = L.a1_off + (size_t)terms * F * NC * kTcRows * L.K1p * esz;
    L.nodes_off = L.a2_off + (size_t)terms * NC * kTcRows * L.N1p * esz;
    L.pipe_bytes = tc_round_up_sz(L.nodes_off + (size_t)(n | 1) * kTcRows * 4, 128);   // nodes [128][n | 1]
    L.total = L.staged_bytes + (size_t)pipes * L.pipe_bytes;
    L.acc1_cols = F * NC * L.N1p;
    L.acc2_cols = NC * L.N2p;
    L.pipe_cols = L.acc1_cols + L.acc2_cols;
    // each pipeline owns tmem_cols / pipes columns (a power of two >= 32 in total)
    int t = 32;
    while (t / pipes < L.pipe_cols) t <<= 1;
    L.tmem_cols = t;
    return L;
}

// Element offset of (row r, k) in a K-major no-swizzle operand with Kp columns
// of esz-byte elements: core matrices of 8 rows x 16 bytes (ce = 16 / esz
// elements), ordered [row group][K group][row][element].
__host__ __device__ inline size_t tc_off(int r, int k, int Kp, int esz = 2)
{
    const int ce = 16 / esz;
    return (size_t)(r >> 3) * (Kp / ce) * (8 * ce) + (size_t)(k / ce) * (8 * ce) + (r & 7) * ce + (k % ce);
}

// Round-to-nearest-even conversion of x * 2^-k (x an IEEE binary64 value) to
// a small format with EB exponent and MB fraction bits (binary16: 5, 10;
// bfloat16: 8, 7; TF32: 8, 10), done on the integer bit pattern (no FP64-pipe
// operation; the power-of-two scaling is an exponent offset).  Returns the
// 1 + EB + MB bit pattern.  NaN maps to a quiet NaN, overflow to infinity,
// results below half the smallest subnormal to signed zero.
template <int EB, int MB>
__host__ __device__ __forceinline__ uint32_t f64_to_small_rn(double x, int k = 0)
{
    uint64_t b;
#ifdef __CUDA_ARCH__
    b = (uint64_t)__double_as_longlong(x);
#else
    std::memcpy(&b, &x, 8);
#endif
    constexpr int kBias = (1 << (EB - 1)) - 1;
    constexpr uint32_t kInf = ((1u << EB) - 1u) << MB;
    const uint32_t sign = (uint32_t)(b >> 63) << (EB + MB);
    const uint64_t frac = b & 0xFFFFFFFFFFFFFull;
    const int e = (int)((b >> 52) & 0x7FF);
    if (e == 0x7FF) return sign | kInf | (frac ? (1u << (MB - 1)) : 0u);
    const int te = (e ? e : 1) - 1023 + kBias - k;   // biased exponent in the target format
    uint64_t m;
    int shift;
    if (te >= 1) {
        m = ((uint64_t)te << 52) | frac;   // exponent and fraction: a carry rounds into the exponent
        shift = 52 - MB;
    } else {
        m = frac | (e ? (1ull << 52) : 0ull);
        shift = 52 - MB + 1 - te;
        if (shift > 62) return sign;
    }
    if (te > 2 * kBias + 1) {
        return sign | kInf;   // far above the largest finite value
    }
    uint64_t r = m >> shift;
    const uint64_t rem = m & ((1ull << shift) - 1ull), halfway = 1ull << (shift - 1);
    if (rem > halfway || (rem == halfway && (r & 1ull))) ++r;
    if (r >= kInf) return sign | kInf;
    return sign | (uint32_t)r;
}

template <typename TE>
__host__ __device__ __forceinline__ uint16_t to16_bits(double x, int k = 0);
template <>
__host__ __device__ __forceinline__ uint16_t to16_bits<__nv_bfloat16>(double x, int k)
{
    return (uint16_t)f64_to_small_rn<8, 7>(x, k);
}
template <>
__host__ __device__ __forceinline__ uint16_t to16_bits<__half>(double x, int k)
{
    return (uint16_t)f64_to_small_rn<5, 10>(x, k);
}

// TF32 operand: a binary32 container whose 13 low fraction bits are zero (the
// tensor cores read sign, 8 exponent and 10 fraction bits).
struct tf32_t {
    uint32_t bits;
};

// x * 2^-k rounded to nearest even TF32, as its binary32 container bits.
__host__ __device__ __forceinline__ uint32_t to_tf32_bits(double x, int k = 0)
{
    return f64_to_small_rn<8, 10>(x, k) << 13;
}

// binary32 v rounded to nearest even TF32 (integer arithmetic: a carry out of
// the kept fraction rounds into the exponent, up to infinity); inf stays inf,
// NaN stays a quiet NaN.
__host__ __device__ __forceinline__ uint32_t f32_bits_to_tf32(uint32_t b)
{
    if ((b & 0x7F800000u) == 0x7F800000u) return (b & 0xFFFFE000u) | ((b & 0x7FFFFFu) ? 0x400000u : 0u);
    return (b + 0xFFFu + ((b >> 13) & 1u)) & 0xFFFFE000u;
}

// Operand element traits: bytes, the instruction descriptor's A/B format
// (kind::f16: 0 = F16, 1 = BF16; kind::tf32: 2) and the MMA K per instruction
// (32 bytes of K: 16 elements of 2 bytes, 8 of 4).
template <typename T>
struct TcElem;
template <>
struct TcElem<__half> {
    static constexpr int kBytes = 2, kFmt = 0, kK = 16;
};
template <>
struct TcElem<__nv_bfloat16> {
    static constexpr int kBytes = 2, kFmt = 1, kK = 16;
};
template <>
struct TcElem<tf32_t> {
    static constexpr int kBytes = 4, kFmt = 2, kK = 8;
};

// 2^e as a binary32 value for e <= 127; 0 below the normal range (the terms it
// scales are then negligible against the other term of the sum).
__device__ __forceinline__ float exp2_float(int e)
{
    return e < -126 ? 0.f : __uint_as_float((unsigned)min(e + 127, 254) << 23);
}

// Monotone map of binary64 values to signed integers (integer order = value
// order, -0 just below +0) and its inverse: min/max without FP64 compares.
__device__ __forceinline__ long long ordered_key(double x)
{
    const long long b = __double_as_longlong(x);
    return b >= 0 ? b : (b ^ 0x7FFFFFFFFFFFFFFFll);
}
__device__ __forceinline__ double from_ordered_key(long long k)
{
    return __longlong_as_double(k >= 0 ? k : (k ^ 0x7FFFFFFFFFFFFFFFll));
}

// Biased binary64 exponent field of x (0: zero or subnormal, 2047: inf or NaN).
__device__ __forceinline__ int exp_field(double x) { return (int)(((unsigned)__double2hiint(x) >> 20) & 0x7FFu); }

// Exponent k of a power of two 2^k > max(|x|, |y|) (0 if both are zero or
// either is not finite), from the exponent fields alone.
__device__ __forceinline__ int mat_shift(double x, double y)
{
    const int e = max(exp_field(x), exp_field(y));
    return (e == 0 || e == 0x7FF) ? 0 : e - 1022;
}

// binary32 v times 2^k, widened to binary64 exactly, with integer operations
// only (no FP64-pipe instruction on any path).  Zero and binary32 subnormals
// give signed zero (they are below 2^-126 of an O(1) accumulator), inf and NaN
// stay inf and NaN, a result outside binary64's normal range gives zero or inf.
__device__ __forceinline__ double widen_pow2(float v, int k)
{
    const unsigned b = __float_as_uint(v);
    const unsigned sign = b & 0x80000000u, mant = b & 0x7FFFFFu;
    const int e = (int)((b >> 23) & 0xFFu);
    const int E = e - 127 + 1023 + k;
    unsigned hi, lo;
    if (e == 0 || E < 1) {
        hi = sign;
        lo = 0u;
    } else if (e == 255 || E > 2046) {
        hi = sign | 0x7FF00000u | (e == 255 ? (mant >> 3) | (mant ? 0x80000u : 0u) : 0u);
        lo = 0u;
    } else {
        hi = sign | ((unsigned)E << 20) | (mant >> 3);
        lo = mant << 29;
    }
    return __hiloint2double((int)hi, (int)lo);
}

// binary64 x times 2^-k rounded to binary32 (nearest even) with integer
// operations only; results below 2^-126 flush to signed zero, overflow gives
// inf, NaN stays NaN.
__device__ __forceinline__ float narrow_pow2_ftz(double x, int k)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7FFu);
    if (e == 0x7FF) return __uint_as_float(sign | 0x7F800000u | ((hi & 0xFFFFFu) | lo ? 0x400000u : 0u));
    const int fe = e - 1023 + 127 - k;   // binary32 biased exponent
    if (e == 0 || fe < 1) return __uint_as_float(sign);
    if (fe > 254) return __uint_as_float(sign | 0x7F800000u);
    const unsigned bits = sign | ((unsigned)fe << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    const unsigned rest = lo & 0x1FFFFFFFu;
    const unsigned up = (rest > 0x10000000u) || (rest == 0x10000000u && (bits & 1u));
    return __uint_as_float(bits + up);   // a carry may round up to the next binade or inf
}

// Two FP32 values to a packed pair of 16-bit values (round to nearest even);
// the first value lands at the lower address.
template <typename TE>
__device__ __forceinline__ uint32_t pack2(float lo, float hi);
template <>
__device__ __forceinline__ uint32_t pack2<__nv_bfloat16>(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}
template <>
__device__ __forceinline__ uint32_t pack2<__half>(float lo, float hi)
{
    const __half2 v = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// binary64 x times 2^-k narrowed to binary32 with rounding to odd: the 29 dropped
// fraction bits are truncated and the last kept bit is set if any of them was
// nonzero (integer operations only).  Returns false, leaving f = 0, where the
// result is not a binary32 normal number or zero (x subnormal, inf or NaN, or
// x 2^-k outside [2^-126, 2^128)).
__device__ __forceinline__ bool f64_to_f32_odd(double x, int k, float &f)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7FFu);
    f = 0.f;
    if (((hi & 0x7FFFFFFFu) | lo) == 0u) {
        f = __uint_as_float(sign);
        return true;
    }
    const int fe = e - 1023 + 127 - k;   // binary32 biased exponent
    if (e == 0 || e == 0x7FF || fe < 1 || fe > 254) return false;
    const unsigned bits = sign | ((unsigned)fe << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29) |
                          ((lo & 0x1FFFFFFFu) != 0u ? 1u : 0u);
    f = __uint_as_float(bits);
    return true;
}

// Two binary64 values times 2^-k rounded to nearest even 16-bit values (TE),
// packed, the first at the lower address; equal to to16_bits on each.  Each is
// narrowed to binary32 by rounding to odd, then rounded by the hardware's
// binary32 -> 16-bit conversion: rounding to odd at 24 bits followed by rounding
// to nearest at p <= 22 bits equals rounding to nearest directly (Boldo and
// Melquiond, "Emulation of FMA and correctly rounded sums: proved algorithms
// using rounding to odd", IEEE Trans. Computers 57(4), 2008).  Values outside
// binary32's normal range take the exact integer path.
template <typename TE>
__device__ __forceinline__ uint32_t pack2_from_f64(double x0, double x1, int k)
{
    float f0, f1;
    const bool ok0 = f64_to_f32_odd(x0, k, f0), ok1 = f64_to_f32_odd(x1, k, f1);
    if (ok0 && ok1) return pack2<TE>(f0, f1);
    return (uint32_t)to16_bits<TE>(x0, k) | ((uint32_t)to16_bits<TE>(x1, k) << 16);
}

// x times 2^-k rounded to nearest even TF32 (container bits); equal to
// to_tf32_bits, by the same rounding-to-odd argument (TF32 keeps 11 bits).
__device__ __forceinline__ uint32_t tf32_from_f64(double x, int k)
{
    float f;
    if (f64_to_f32_odd(x, k, f)) return f32_bits_to_tf32(__float_as_uint(f));
    return to_tf32_bits(x, k);
}

// The two 16-bit values of a packed pair back in binary32.
template <typename TE>
__device__ __forceinline__ float2 unpack2(uint32_t w);
template <>
__device__ __forceinline__ float2 unpack2<__nv_bfloat16>(uint32_t w)
{
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w));
}
template <>
__device__ __forceinline__ float2 unpack2<__half>(uint32_t w)
{
    return __half22float2(*reinterpret_cast<const __half2 *>(&w));
}

// Stores 8 consecutive K entries of one operand row, p at the first: for the
// 16-bit types one 16-byte core-matrix row, for TF32 the 4-element rows of two
// K-adjacent core matrices (32 elements apart).  Term 0 is the rounding of v;
// with TERMS == 2 term 1, region_elems further on, holds the rounding of the
// remainder v - term0 (a binary16 hi + lo pair, ~2 x the significand bits).
template <typename TE, int TERMS>
__device__ __forceinline__ void store8(TE *p, size_t region_elems, const float (&v)[8])
{
    if constexpr (TcElem<TE>::kBytes == 4) {
        static_assert(TERMS == 1, "TF32 operands are single-term");
        uint32_t w[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) w[i] = f32_bits_to_tf32(__float_as_uint(v[i]));
        *reinterpret_cast<uint4 *>(p) = make_uint4(w[0], w[1], w[2], w[3]);
        *reinterpret_cast<uint4 *>(p + 32) = make_uint4(w[4], w[5], w[6], w[7]);
        return;
    } else {
    uint32_t w[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) w[h] = pack2<TE>(v[2 * h], v[2 * h + 1]);
    *reinterpret_cast<uint4 *>(p) = make_uint4(w[0], w[1], w[2], w[3]);
    if constexpr (TERMS == 2) {
        uint32_t r[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const float2 hi = unpack2<TE>(w[h]);
            r[h] = pack2<TE>(v[2 * h] - hi.x, v[2 * h + 1] - hi.y);
        }
        *reinterpret_cast<uint4 *>(p + region_elems) = make_uint4(r[0], r[1], r[2], r[3]);
    }
    }
}

__device__ __forceinline__ uint64_t tc_smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((lbo & 0x3FFFF) >> 4) << 16) |
           ((uint64_t)((sbo & 0x3FFFF) >> 4) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of tcgen05.mma kind::f16 / kind::tf32: FP32
// accumulator, A and B of the same type (fmt 0 = F16, 1 = BF16, 2 = TF32),
// both K-major.
__host__ __device__ constexpr uint32_t tc_idesc(int fmt, int M, int N)
{
    return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

template <bool kTf32>
__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc)
{
    if constexpr (kTf32)
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(da), "l"(db), "r"(idesc), "r"(acc)
            : "memory");
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
            "l"(da), "l"(db), "r"(idesc), "r"(acc)
            : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t sbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(sbar)
                 : "memory");
}

// 16 consecutive accumulator columns of this warp's 32 lanes (no wait).
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

// 16 consecutive columns of this warp's 32 lanes from registers (no wait).
__device__ __forceinline__ void tc_st16(uint32_t taddr, const uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
        ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
          "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}
__device__ __forceinline__ void tc_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// 8 consecutive accumulator columns of this warp's 32 lanes (no wait).
__device__ __forceinline__ void tc_ld8(uint32_t taddr, uint32_t (&r)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}

__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Barrier over the 128 x tpc threads of one pipeline (named barrier 1 + pipe;
// pipes x tpc <= 4).  Ids and counts are immediates, so the kernel reserves
// only the barriers it uses.
#define FE_TC_BAR(ID, CNT) asm volatile("bar.sync " #ID ", " #CNT ";" ::: "memory")
__device__ __forceinline__ void pipe_sync(int pipe, int tpc)
{
    if (tpc == 1) {
        switch (pipe) {
        case 0: FE_TC_BAR(1, 128); break;
        case 1: FE_TC_BAR(2, 128); break;
        case 2: FE_TC_BAR(3, 128); break;
        default: FE_TC_BAR(4, 128); break;
        }
    } else if (tpc == 2) {
        if (pipe == 0)
            FE_TC_BAR(1, 256);
        else
            FE_TC_BAR(2, 256);
    } else {
        FE_TC_BAR(1, 512);
    }
}
#undef FE_TC_BAR

#define FE_TC_BAR_RED_AND(ID, CNT)                                                         \
    asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"                      \
                 "bar.red.and.pred q, " #ID ", " #CNT ", p;\n\tselp.u32 %0, 1, 0, q;\n\t}"    \
                 : "=r"(r)                                                                  \
                 : "r"((uint32_t)pred)                                                      \
                 : "memory")

// Barrier over one pipeline that also returns whether pred held on all its threads.
__device__ __forceinline__ bool pipe_all(int pipe, int tpc, bool pred)
{
    uint32_t r;
    if (tpc == 1) {
        switch (pipe) {
        case 0: FE_TC_BAR_RED_AND(1, 128); break;
        case 1: FE_TC_BAR_RED_AND(2, 128); break;
        case 2: FE_TC_BAR_RED_AND(3, 128); break;
        default: FE_TC_BAR_RED_AND(4, 128); break;
        }
    } else if (tpc == 2) {
        if (pipe == 0)
            FE_TC_BAR_RED_AND(1, 256);
        else
            FE_TC_BAR_RED_AND(2, 256);
    } else {
        FE_TC_BAR_RED_AND(1, 512);
    }
    return r != 0;
}
#undef FE_TC_BAR_RED_AND

// Bounded wait on an mbarrier phase; true if it completed.
__device__ __forceinline__ bool tc_wait(uint32_t sbar, uint32_t parity)
{
    for (int it = 0; it < kWaitLimit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(sbar), "r"(parity)
            : "memory");
        if (ok) return true;
        __nanosleep(32);
    }
    return false;
}

// Hyperelastic Jacobian pointwise phase (Neo-Hookean or St. Venant-Kirchhoff)
// for one chunk, for this thread's cell at the chunk's points.  The du and
// u_lin reference gradients come from the evaluation accumulators (8 columns at
// a time).  The kinematic contractions with J^{-1} (F = I + grad u_lin,
// u_lin's per-cell scaling undone exactly by a power of two; H = grad du with
// J^{-1} 2^-kj) and the pull-back run in FP32, far below the 16-bit rounding of
// their inputs and output; the law itself is FP64 (Neo-Hookean: det F, F^{-T},
// log det F and the tangent applied to H; St. Venant-Kirchhoff: E, S, dE, dS,
// dP = H S + F dS — the same algebra as the FP64 kernels).  E' = w_q e is
// rounded to 16 bits.  Returns false if det F <= 0 at a live Neo-Hookean point.
template <int OP, int D, typename TE, int TERMS>
__device__ __forceinline__ bool tc_pointwise_hyper_jacobian(const TcLayout &L, uint32_t tlane, unsigned char *hb,
                                                            const double *wd, int t, int h, int tpc, int ch, int nq, bool good,
                                                            int ku_lin, const float (&Jf)[D][D],
                                                            const float (&Jh)[D][D], double mu, double lam,
                                                            const double *log_tab)
{
    constexpr int NC = D, KDP = (D == 2) ? 2 : 4, PPB = 8 / KDP;
    // 2^ku_lin as a binary32 value (the u_lin gradient is O(h) in reference
    // coordinates, so the product stays in range)
    const float s_lin = __uint_as_float((unsigned)min(max(ku_lin + 127, 1), 254) << 23);
    bool ok = true;
    for (int blk = h; blk < L.N1p / 8; blk += tpc) {   // the cell's tpc threads split the columns
        uint32_t r[2 * NC][8];
#pragma unroll
        for (int fm = 0; fm < 2 * NC; ++fm) tc_ld8(tlane + (uint32_t)(fm * L.N1p + blk * 8), r[fm]);
        tc_wait_ld();
        float out[NC][8];
#pragma unroll
        for (int p = 0; p < PPB; ++p) {
            const int ql = blk * PPB + p, q = ch * L.qc + ql;
            const bool live = good && ql < L.qc && q < nq;
            float gd[D][D], gl[D][D], Ff[D][D], Hf[D][D], Sf[D][D], ef[D][D];
#pragma unroll
            for (int m = 0; m < D; ++m)
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    gd[m][k] = __uint_as_float(r[m][p * KDP + k]);
                    gl[m][k] = __uint_as_float(r[NC + m][p * KDP + k]) * s_lin;
                }
            map_grad<D, float>(gl, Jf, Ff);   // grad u_lin (physical), F = I + Ff
            map_grad<D, float>(gd, Jh, Hf);   // grad du with J^{-1} 2^-kj
            const double w = live ? wd[q] : 0.0;
            if constexpr (OP == OP_SVK_JACOBIAN) {
                // St. Venant-Kirchhoff tangent dP = H S + F dS in FP64 (no det F condition)
                double G[D][D], H[D][D], Pd[D][D];
#pragma unroll
                for (int i = 0; i < D; ++i)
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        G[i][k] = widen_pow2(Ff[i][k], 0);
                        H[i][k] = widen_pow2(Hf[i][k], 0);
                    }
                svk_stress<D, true>(G, H, mu, lam, w, Pd);
#pragma unroll
                for (int i = 0; i < D; ++i)
#pragma unroll
                    for (int k = 0; k < D; ++k) Sf[i][k] = narrow_pow2_ftz(Pd[i][k], 0);
            } else {
                double F[D][D], H[D][D], C[D][D], Fit[D][D], A[D][D];
#pragma unroll
                for (int i = 0; i < D; ++i)
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        F[i][k] = widen_pow2(Ff[i][k], 0) + (i == k ? 1.0 : 0.0);
                        H[i][k] = widen_pow2(Hf[i][k], 0);
                    }
                const double Jd = det_cof<D>(F, C);
                ok &= !live || (Jd > 0.0);
                const double Jd_safe = live && Jd > 0.0 ? Jd : 1.0;
                const double rJ = log_tab ? fe_rcp(Jd_safe) : 1.0 / Jd_safe;
                const double lnJ = law_log(Jd_safe, log_tab);
                double tr = 0.0;   // F^{-T} : H
#pragma unroll
                for (int i = 0; i < D; ++i)
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        Fit[i][k] = C[i][k] * rJ;
                        tr = fma(Fit[i][k], H[i][k], tr);
                    }
#pragma unroll
                for (int i = 0; i < D; ++i)
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        double s = Fit[i][0] * H[k][0];
#pragma unroll
                        for (int mm = 1; mm < D; ++mm) s = fma(Fit[i][mm], H[k][mm], s);
                        A[i][k] = s;
                    }
                const double smu = w * mu, sm2 = w * fma(-lam, lnJ, mu), str = w * lam * tr;
#pragma unroll
                for (int i = 0; i < D; ++i)
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        double mk = A[i][0] * Fit[0][k];
#pragma unroll
                        for (int mm = 1; mm < D; ++mm) mk = fma(A[i][mm], Fit[mm][k], mk);
                        Sf[i][k] = narrow_pow2_ftz(fma(smu, H[i][k], fma(sm2, mk, str * Fit[i][k])), 0);
                    }
            }
            pull_back<D, float>(Sf, Jh, ef);
#pragma unroll
            for (int m = 0; m < NC; ++m)
#pragma unroll
                for (int k = 0; k < KDP; ++k) out[m][p * KDP + k] = (k < D && live) ? ef[m][k] : 0.f;
        }
#pragma unroll
        for (int m = 0; m < NC; ++m) {
            const size_t region = (size_t)kTcRows * L.N1p;
            TE *A2 = reinterpret_cast<TE *>(hb + L.a2_off) + (size_t)m * TERMS * region;
            store8<TE, TERMS>(A2 + tc_off(t, blk * 8, L.N1p, TcElem<TE>::kBytes), region, out[m]);
        }
    }
    return ok;
}

template <int OP, int D, typename TE, int TERMS>
__global__ void __launch_bounds__(kTcMaxPipes * kTcRows, 1) k_action_tc(const ActionArgs a)
{
    constexpr int NC = OpTraits<OP, D>::NC;
    // derivative terms per point: value (mass), value + gradient (Helmholtz), gradient
    constexpr int KD = (OP == OP_MASS) ? 1 : (OP == OP_HELMHOLTZ ? 1 + D : D);
    constexpr int KDP = (KD == 1) ? 1 : (KD == 2 ? 2 : 4);
    // hyperelastic Jacobian actions gather two fields: du, then the linearisation point
    constexpr bool kHyperJac = (OP == OP_NH_JACOBIAN || OP == OP_SVK_JACOBIAN);
    constexpr int F = kHyperJac ? 2 : 1;
    // gradient-only forms round u - c (c a per-cell constant): the basis
    // gradients sum to zero, so the constant drops out of every gradient
    constexpr bool kOffset = OP != OP_MASS && OP != OP_HELMHOLTZ;
    constexpr int PPB = 16 / KDP;   // quadrature points per 16 accumulator columns
    constexpr int FMT = TcElem<TE>::kFmt, ESZ = TcElem<TE>::kBytes, KK = TcElem<TE>::kK;
    constexpr bool kTf32 = ESZ == 4;
    extern __shared__ __align__(128) unsigned char tc_smem[];
    __shared__ __align__(8) uint64_t bars[1 + kTcMaxPipes];   // table copy; one MMA barrier per pipeline
    __shared__ uint32_t s_tmem;
    __shared__ int s_tile[kTcMaxPipes];

    const TcLayout L = tc_layout(a.coop_n, a.nq, NC, KD, F, a.tc_qc, a.tc_pipes, TERMS, ESZ);
    // tpc threads per cell (tile row): thread (h, t) of a pipeline works on row t
    // and takes every tpc-th node batch, column block and output group
    const int tpc = (int)blockDim.x / (kTcRows * L.pipes);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int pipe = tid / (kTcRows * tpc), pt = tid % (kTcRows * tpc), t = pt & (kTcRows - 1), h = pt >> 7;
    const int n = L.n;
    const uint32_t bar0 = (uint32_t)__cvta_generic_to_shared(&bars[0]);
    const uint32_t barp = (uint32_t)__cvta_generic_to_shared(&bars[1 + pipe]);

    if (tid == 0) {
        for (int i = 0; i <= L.pipes; ++i) {
            const uint32_t b = (uint32_t)__cvta_generic_to_shared(&bars[i]);
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&s_tmem);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst),
                     "r"((uint32_t)L.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = s_tmem;
    if (tid == 0) {
        const uint32_t bytes = (uint32_t)L.staged_bytes;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar0), "r"(bytes) : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                (uint32_t)__cvta_generic_to_shared(tc_smem)),
            "l"((uint64_t)__cvta_generic_to_global(a.tab)), "r"(bytes), "r"(bar0)
            : "memory");
    }
    bool ok = __syncthreads_and(tc_wait(bar0, 0));
    if (!ok) tc_wait(bar0, 0);   // let a late copy land before the CTA exits

    const unsigned char *staged = tc_smem;
    unsigned char *hb = tc_smem + L.staged_bytes + (size_t)pipe * L.pipe_bytes;
    const float *wf = reinterpret_cast<const float *>(staged + L.wf_off);
    int *snodes = reinterpret_cast<int *>(hb + L.nodes_off);   // [128][P]
    const int P = n | 1;
    const uint32_t b1s = (uint32_t)__cvta_generic_to_shared(staged + L.b1_off);
    const uint32_t b2s = (uint32_t)__cvta_generic_to_shared(staged + L.b2_off);
    const uint32_t a1s = (uint32_t)__cvta_generic_to_shared(hb + L.a1_off);
    const uint32_t a2s = (uint32_t)__cvta_generic_to_shared(hb + L.a2_off);
    const uint32_t tpipe = tbase + (uint32_t)(pipe * (L.tmem_cols / L.pipes));
    const uint32_t tlane = tpipe + ((uint32_t)((warp & 3) * 32) << 16);   // this warp's TMEM lanes
    // the DoFs staged in TMEM between the two gather passes: 2 columns per binary64
    // value, nodes padded to a multiple of 8 (one 16-column store per 8 nodes).
    // Only with one pipeline per CTA: there the second gather's latency is exposed
    // and staging saves 4-5 % (elasticity P4 tets, split FP16 and TF32); with two or
    // four pipelines the others hide it and the TMEM round trip costs up to 5 %
    // (mass P3 triangles, four pipelines).
    const int n8 = (n + 7) & ~7;
    const bool stage_tm = L.pipes == 1 && 2 * F * NC * n8 <= L.tmem_cols;
    // With tpc > 1 the cell's threads combine their DoF ranges through kXS 64-bit
    // words each; where the region also holds kGeoWords 32-bit words per cell, the
    // geometry (16 loads and ~60 FP64-pipe instructions) is computed once per cell
    // and shared instead of by each of its threads.
    constexpr int kXS = kOffset ? 2 * F * NC + 1 : F + 1;
    constexpr int kGeoWords = 3 + (OP == OP_HELMHOLTZ ? 2 : 0) + (OP != OP_MASS ? D * D : 0) + (kHyperJac ? D * D : 0);
    const bool share_geo = tpc > 1 && (size_t)kTcRows * tpc * kXS * 8 + (size_t)kTcRows * kGeoWords * 4 <=
                                          L.nodes_off - L.a2_off;
    const bool do_geo = !share_geo || h == 0;
    const int n_tiles = (a.n_cells + kTcRows - 1) / kTcRows;
    // elasticity: lambda, mu scaled by a power of two 2^km > max(|lambda|, |mu|)
    // (E' stays O(1) for any material); the factor returns in the output exponent
    [[maybe_unused]] const int km_el = mat_shift(a.lam, a.mu);
    [[maybe_unused]] const float lam_f = narrow_pow2_ftz(a.lam, km_el), mu_f = narrow_pow2_ftz(a.mu, km_el);
    uint32_t phase = 0;
    bool timed_out = false;
    bool nh_ok = true;
    const double *wd = reinterpret_cast<const double *>(staged + L.wd_off);

    while (ok) {
        if (pt == 0) s_tile[pipe] = atomicAdd(a.sched, 1);
        pipe_sync(pipe, tpc);
        const int tile = s_tile[pipe];
        if (tile >= n_tiles) break;

        // ---- gather (Algorithm 2).  The tile's cell2node rows are contiguous:
        // copy them with coalesced 16-byte loads into snodes (odd row pitch P, so
        // the per-thread row reads below are free of bank conflicts).
        const int nb = min(kTcRows, a.n_cells - tile * kTcRows);
        {
            const int total = nb * n;
            const int32_t *src = a.c2n + (size_t)tile * kTcRows * n;
            const int n4 = total >> 2;
            for (int i4 = pt; i4 < n4; i4 += kTcRows * tpc) {
                const int4 v = __ldg(reinterpret_cast<const int4 *>(src) + i4);
                const int vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    const int e = 4 * i4 + s, c = e / n, j = e - c * n;
                    snodes[c * P + j] = (unsigned)vv[s] < (unsigned)a.n_nodes ? vv[s] : -1;
                }
            }
            for (int e = 4 * n4 + pt; e < total; e += kTcRows * tpc) {
                const int v = __ldg(src + e), c = e / n, j = e - c * n;
                snodes[c * P + j] = (unsigned)v < (unsigned)a.n_nodes ? v : -1;
            }
        }
        pipe_sync(pipe, tpc);
        tc_fence_after();   // the previous tile's TMEM reads come before this tile's stores

        // geometry in FP64 (this thread's cell), then the DoFs' largest exponent
        int K = 0;              // output factor 2^K (with mdet below)
        float mdet = 0.f;       // |det J| / 2^(its exponent), in [1, 2)
        int ku[F] = {};         // field f is rounded as (u_f - off_f) * 2^-ku[f]
        double off[F][NC] = {}; // per-cell offsets (gradient forms; zero for mass)
        [[maybe_unused]] float Jh[D][D];
        [[maybe_unused]] float s_val = 1.f, s_grad = 1.f;   // Helmholtz: value / gradient term factors
        [[maybe_unused]] float Jf[D][D];   // Neo-Hookean: J^{-1} in binary32
        [[maybe_unused]] double mu_c = a.mu, lam_c = a.lam;
        bool good = t < nb;
        // mass: largest exponent of |u|; gradient forms: range [min, max] of each
        // component (ordered integer keys, no FP64 compare)
        int emax[F] = {};
        [[maybe_unused]] long long kmin[F][NC], kmax[F][NC];
#pragma unroll
        for (int f = 0; f < F; ++f)
#pragma unroll
            for (int m = 0; m < NC; ++m) {
                kmin[f][m] = LLONG_MAX;
                kmax[f][m] = LLONG_MIN;
            }
        bool nodes_ok = true;
        // The cell's geometry and what derives from it alone: geo bit 0 = vertex
        // indices in range, bit 1 = det J nonzero and finite; Kg = the exponent of
        // the output factor without the DoF scale.  With shared geometry only the
        // cell's first thread computes them, the others read them after the
        // exchange below.
        int geo = 0, Kg = 0;
        double Jinv[D][D], det = 0.0;
        bool in_all = true;
        if (good && do_geo) {
            const int cell = tile * kTcRows + t;
            double X[D + 1][D];
#pragma unroll
            for (int m = 0; m <= D; ++m) {
                const int v = __ldg(a.c2v + (size_t)cell * (D + 1) + m);
                const bool in = (unsigned)v < (unsigned)a.n_vertices;
                in_all &= in;
#pragma unroll
                for (int i = 0; i < D; ++i) X[m][i] = in ? __ldg(a.coords + (size_t)v * D + i) : 0.0;
            }
            det = cell_geometry<D>(X, Jinv);
            good &= in_all;
        }
        if constexpr (kHyperJac) {
            if (good) {
                const int cell = tile * kTcRows + t;
                if (a.mu_cell) mu_c = __ldg(a.mu_cell + cell);
                if (a.lam_cell) lam_c = __ldg(a.lam_cell + cell);
            }
        }
        // the DoF range pass (every thread of the warp together: the TMEM stores
        // below are warp-collective).  Where the pipeline's TMEM columns can hold
        // the cell's DoFs (free until the evaluation GEMM), the binary64 values are
        // kept there, two 32-bit columns each, and the rounding pass below reads
        // them back instead of gathering them from global memory a second time.
        for (int j0 = 8 * h; j0 < n; j0 += 8 * tpc) {
            int nd[8];
#pragma unroll
            for (int s = 0; s < 8; ++s) nd[s] = (good && j0 + s < n) ? snodes[t * P + j0 + s] : -2;
#pragma unroll
            for (int f = 0; f < F; ++f) {
                const double *uf = f == 0 ? a.u : a.u_lin;
                double v[8][NC];
#pragma unroll
                for (int s = 0; s < 8; ++s)
#pragma unroll
                    for (int m = 0; m < NC; ++m) v[s][m] = nd[s] >= 0 ? __ldg(uf + (size_t)nd[s] * NC + m) : 0.0;
#pragma unroll
                for (int s = 0; s < 8; ++s)
#pragma unroll
                    for (int m = 0; m < NC; ++m) {
                        if constexpr (kOffset) {
                            if (nd[s] >= 0) {
                                const long long key = ordered_key(v[s][m]);
                                kmin[f][m] = min(kmin[f][m], key);
                                kmax[f][m] = max(kmax[f][m], key);
                            }
                        } else {
                            emax[f] = max(emax[f], exp_field(v[s][m]));
                        }
                    }
                if (stage_tm) {
#pragma unroll
                    for (int m = 0; m < NC; ++m) {
                        uint32_t w[16];
#pragma unroll
                        for (int s = 0; s < 8; ++s) {
                            w[2 * s] = (uint32_t)__double2loint(v[s][m]);
                            w[2 * s + 1] = (uint32_t)__double2hiint(v[s][m]);
                        }
                        tc_st16(tlane + (uint32_t)(2 * ((f * NC + m) * n8 + j0)), w);
                    }
                }
            }
#pragma unroll
            for (int s = 0; s < 8; ++s) nodes_ok &= nd[s] != -1;
        }
        if (stage_tm) tc_wait_st();
        // the geometry-derived values (of a cell with geo == 3): with shared geometry
        // the cell's first thread derives them here, before the exchange; otherwise
        // every thread does below, after its status checks
        auto derive = [&]() {
            const int ed = exp_field(det) - 1023;
            const double m64 = __hiloint2double((__double2hiint(det) & 0x000FFFFF) | (1023 << 20),
                                                __double2loint(det));
            mdet = narrow_pow2_ftz(m64, 0);
            Kg = ed - a.tc_wshift;
            if constexpr (OP == OP_ELASTICITY) Kg += km_el;
            if constexpr (OP != OP_MASS) {
                int ej = 0;
#pragma unroll
                for (int i = 0; i < D; ++i)
#pragma unroll
                    for (int k = 0; k < D; ++k) ej = max(ej, exp_field(Jinv[i][k]));
                const int kj = ej - 1022;   // s_J = 2^kj > max |J^{-1}_ik|
                if constexpr (OP == OP_HELMHOLTZ) {
                    // value term ~ |det J| u, gradient term ~ |det J| 2^2kj (O(1) each
                    // before these factors): the common scale follows the larger one
                    const int sig = max(2 * kj, 0);
                    Kg += sig;
                    s_val = exp2_float(-sig);
                    s_grad = exp2_float(2 * kj - sig);
                } else {
                    Kg += 2 * kj;
                }
#pragma unroll
                for (int i = 0; i < D; ++i)
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        Jh[i][k] = narrow_pow2_ftz(Jinv[i][k], kj);
                        if constexpr (kHyperJac) Jf[i][k] = narrow_pow2_ftz(Jinv[i][k], 0);
                    }
            }
        };
        if (good && do_geo) geo = (in_all ? 1 : 0) | ((det != 0.0) && isfinite(det) ? 2 : 0);
        if (share_geo && h == 0 && geo == 3) derive();
        if (tpc > 1) {
            // combine the partial ranges of the cell's tpc threads through the
            // quadrature A-operand region (free until this tile's pointwise phase);
            // with shared geometry the cell's first thread also leaves its
            // geometry words there, behind the range slots
            long long *xch = reinterpret_cast<long long *>(hb + L.a2_off);
            long long *mine = xch + (size_t)(h * kTcRows + t) * kXS;
            int q = 0;
#pragma unroll
            for (int f = 0; f < F; ++f) {
                if constexpr (kOffset) {
#pragma unroll
                    for (int m = 0; m < NC; ++m) {
                        mine[q++] = kmin[f][m];
                        mine[q++] = kmax[f][m];
                    }
                } else {
                    mine[q++] = emax[f];
                }
            }
            mine[q] = nodes_ok ? 1 : 0;
            uint32_t *gx = reinterpret_cast<uint32_t *>(xch + (size_t)tpc * kTcRows * kXS) + (size_t)t * kGeoWords;
            if (share_geo && h == 0) {
                int w = 0;
                gx[w++] = (uint32_t)geo;
                gx[w++] = (uint32_t)Kg;
                gx[w++] = __float_as_uint(mdet);
                if constexpr (OP == OP_HELMHOLTZ) {
                    gx[w++] = __float_as_uint(s_val);
                    gx[w++] = __float_as_uint(s_grad);
                }
                if constexpr (OP != OP_MASS) {
#pragma unroll
                    for (int i = 0; i < D; ++i)
#pragma unroll
                        for (int k = 0; k < D; ++k) gx[w++] = __float_as_uint(Jh[i][k]);
                }
                if constexpr (kHyperJac) {
#pragma unroll
                    for (int i = 0; i < D; ++i)
#pragma unroll
                        for (int k = 0; k < D; ++k) gx[w++] = __float_as_uint(Jf[i][k]);
                }
            }
            pipe_sync(pipe, tpc);
            for (int hh = 0; hh < tpc; ++hh) {
                if (hh == h) continue;
                const long long *other = xch + (size_t)(hh * kTcRows + t) * kXS;
                int r = 0;
#pragma unroll
                for (int f = 0; f < F; ++f) {
                    if constexpr (kOffset) {
#pragma unroll
                        for (int m = 0; m < NC; ++m) {
                            kmin[f][m] = min(kmin[f][m], other[r++]);
                            kmax[f][m] = max(kmax[f][m], other[r++]);
                        }
                    } else {
                        emax[f] = max(emax[f], (int)other[r++]);
                    }
                }
                nodes_ok &= other[r] != 0;
            }
            if (share_geo && h != 0) {
                int w = 0;
                geo = (int)gx[w++];
                Kg = (int)gx[w++];
                mdet = __uint_as_float(gx[w++]);
                if constexpr (OP == OP_HELMHOLTZ) {
                    s_val = __uint_as_float(gx[w++]);
                    s_grad = __uint_as_float(gx[w++]);
                }
                if constexpr (OP != OP_MASS) {
#pragma unroll
                    for (int i = 0; i < D; ++i)
#pragma unroll
                        for (int k = 0; k < D; ++k) Jh[i][k] = __uint_as_float(gx[w++]);
                }
                if constexpr (kHyperJac) {
#pragma unroll
                    for (int i = 0; i < D; ++i)
#pragma unroll
                        for (int k = 0; k < D; ++k) Jf[i][k] = __uint_as_float(gx[w++]);
                }
            }
        }
        if (t < nb) {
            if (!good || !nodes_ok || !(geo & 1)) {
                set_status(a.status, FE_ERR_INDEX);
                good = false;
            } else if (!(geo & 2)) {
                set_status(a.status, FE_ERR_BAD_MESH);
                good = false;
            }
            if (good) {
                if constexpr (kOffset) {
                    // offset c = midrange of each component; the half-range bounds |u - c|
#pragma unroll
                    for (int f = 0; f < F; ++f)
#pragma unroll
                        for (int m = 0; m < NC; ++m) {
                            const double lo = from_ordered_key(kmin[f][m]), hi = from_ordered_key(kmax[f][m]);
                            off[f][m] = 0.5 * (lo + hi);
                            emax[f] = max(emax[f], exp_field(hi - off[f][m]));
                        }
                }
                // s_u = 2^ku > max |u - c| >= 2^(ku-1) (no scaling for zero or non-finite ranges)
#pragma unroll
                for (int f = 0; f < F; ++f) ku[f] = (emax[f] == 0 || emax[f] == 0x7FF) ? 0 : emax[f] - 1022;
                if (!share_geo) derive();
                K = Kg + ku[0];
                if constexpr (kHyperJac) {
                    const int km = mat_shift(lam_c, mu_c);
                    K += km;
                    mu_c = ldexp(mu_c, -km);
                    lam_c = ldexp(lam_c, -km);
                }
            }
        }
        // A operands of the evaluation GEMM (one per field and component): row t =
        // this cell, K = local node j
        for (int j0 = 8 * h; j0 < L.K1p; j0 += 8 * tpc) {
            int nd[8];
#pragma unroll
            for (int s = 0; s < 8; ++s) nd[s] = (good && j0 + s < n) ? snodes[t * P + j0 + s] : -1;
#pragma unroll
            for (int f = 0; f < F; ++f) {
                const double *uf = f == 0 ? a.u : a.u_lin;
                double v[8][NC];
                if (stage_tm) {
                    if (j0 < n) {
                        uint32_t w[NC][16];
#pragma unroll
                        for (int m = 0; m < NC; ++m) tc_ld16(tlane + (uint32_t)(2 * ((f * NC + m) * n8 + j0)), w[m]);
                        tc_wait_ld();
#pragma unroll
                        for (int s = 0; s < 8; ++s)
#pragma unroll
                            for (int m = 0; m < NC; ++m)
                                v[s][m] = nd[s] >= 0 ? __hiloint2double((int)w[m][2 * s + 1], (int)w[m][2 * s]) : 0.0;
                    } else {
#pragma unroll
                        for (int s = 0; s < 8; ++s)
#pragma unroll
                            for (int m = 0; m < NC; ++m) v[s][m] = 0.0;
                    }
                } else {
#pragma unroll
                    for (int s = 0; s < 8; ++s)
#pragma unroll
                        for (int m = 0; m < NC; ++m) v[s][m] = nd[s] >= 0 ? __ldg(uf + (size_t)nd[s] * NC + m) : 0.0;
                }
#pragma unroll
                for (int m = 0; m < NC; ++m) {
                    const size_t region = (size_t)kTcRows * L.K1p;
                    TE *A1 = reinterpret_cast<TE *>(hb + L.a1_off) + (size_t)(f * NC + m) * TERMS * region;
                    if constexpr (kTf32) {
                        // binary64 rounded to TF32 directly (two K-adjacent core matrices)
                        uint32_t w[8];
#pragma unroll
                        for (int s = 0; s < 8; ++s)
                            w[s] = tf32_from_f64(nd[s] >= 0 ? v[s][m] - off[f][m] : 0.0, ku[f]);
                        TE *q = A1 + tc_off(t, j0, L.K1p, ESZ);
                        *reinterpret_cast<uint4 *>(q) = make_uint4(w[0], w[1], w[2], w[3]);
                        *reinterpret_cast<uint4 *>(q + 32) = make_uint4(w[4], w[5], w[6], w[7]);
                    } else if constexpr (TERMS == 1) {
                        // one term: binary64 rounded to 16 bits directly
                        uint32_t w[4];
#pragma unroll
                        for (int h = 0; h < 4; ++h)
                            w[h] = pack2_from_f64<TE>(nd[2 * h] >= 0 ? v[2 * h][m] - off[f][m] : 0.0,
                                                      nd[2 * h + 1] >= 0 ? v[2 * h + 1][m] - off[f][m] : 0.0, ku[f]);
                        *reinterpret_cast<uint4 *>(A1 + tc_off(t, j0, L.K1p, ESZ)) = make_uint4(w[0], w[1], w[2], w[3]);
                    } else {
                        // hi + lo pair from the scaled value in binary32
                        float xs[8];
#pragma unroll
                        for (int s = 0; s < 8; ++s)
                            xs[s] = nd[s] >= 0 ? narrow_pow2_ftz(v[s][m] - off[f][m], ku[f]) : 0.f;
                        store8<TE, TERMS>(A1 + tc_off(t, j0, L.K1p, ESZ), region, xs);
                    }
                }
            }
        }
        fence_async_smem();
        tc_fence_before();
        pipe_sync(pipe, tpc);
        tc_fence_after();

        const uint32_t id1 = tc_idesc(FMT, kTcRows, L.N1p), id2 = tc_idesc(FMT, kTcRows, L.N2p);
        for (int ch = 0; ch < L.nch; ++ch) {
            // ---- evaluation GEMM of chunk ch (its commit also covers the previous chunk's quadrature GEMM)
            if (pt == 0) {
                // K steps of KK elements (32 bytes: two core matrices) at 256 B each
                const uint32_t sbo = (uint32_t)L.K1p * 8u * ESZ;
                const uint32_t a_region = (uint32_t)(kTcRows * L.K1p * ESZ),
                               b_region = (uint32_t)(L.nch * L.N1p * L.K1p * ESZ);
                for (int m = 0; m < F * NC; ++m)
                    for (int s = 0; s < L.K1p / KK; ++s)
                        // one product, or hi*hi + hi*lo + lo*hi for split operands
                        for (int pr = 0; pr < (TERMS == 2 ? 3 : 1); ++pr) {
                            const uint32_t ta = pr == 2 ? 1u : 0u, tb = pr == 1 ? 1u : 0u;
                            const uint64_t da = tc_smem_desc(
                                a1s + ((uint32_t)m * TERMS + ta) * a_region + (uint32_t)s * 256u, 128u, sbo);
                            const uint64_t db = tc_smem_desc(
                                b1s + tb * b_region + (uint32_t)(ch * L.N1p * L.K1p * ESZ) + (uint32_t)s * 256u, 128u, sbo);
                            tc_mma<kTf32>(tpipe + (uint32_t)(m * L.N1p), da, db, id1, (s > 0 || pr > 0) ? 1u : 0u);
                        }
                tc_commit(barp);
            }
            if (!pipe_all(pipe, tpc, tc_wait(barp, phase))) {
                tc_wait(barp, phase);
                timed_out = true;
                break;
            }
            phase ^= 1u;
            tc_fence_after();

            // ---- pointwise: this thread's cell at the chunk's points, E' into the quadrature A operand
            if constexpr (kHyperJac) {
                nh_ok &= tc_pointwise_hyper_jacobian<OP, D, TE, TERMS>(L, tlane, hb, wd, t, h, tpc, ch, a.nq, good, ku[1],
                                                                        Jf, Jh, mu_c, lam_c, a.log_tab);
            } else
            for (int blk = h; blk < L.N1p / 16; blk += tpc) {   // the cell's tpc threads split the columns
                uint32_t r[NC][16];
#pragma unroll
                for (int m = 0; m < NC; ++m) tc_ld16(tlane + (uint32_t)(m * L.N1p + blk * 16), r[m]);
                tc_wait_ld();
                float v[NC][16];
#pragma unroll
                for (int m = 0; m < NC; ++m)
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[m][i] = __uint_as_float(r[m][i]);
#pragma unroll
                for (int p = 0; p < PPB; ++p) {
                    const int ql = blk * PPB + p, q = ch * L.qc + ql;
                    const bool live = good && ql < L.qc && q < a.nq;
                    const float w = live ? wf[q] : 0.f;
                    if constexpr (OP == OP_MASS) {
                        v[0][p] = w * v[0][p];
                    } else if constexpr (OP == OP_LAPLACE || OP == OP_HELMHOLTZ) {
                        // e = w J^{-1} J^{-T} grad_ref u (scaled by 2^-2kj), value term w u / 2^2kj
                        constexpr int kV = (OP == OP_HELMHOLTZ) ? 1 : 0;
                        float g[D];
#pragma unroll
                        for (int i = 0; i < D; ++i) {
                            float sg = 0.f;
#pragma unroll
                            for (int k = 0; k < D; ++k) sg = fmaf(v[0][p * KDP + kV + k], Jh[k][i], sg);
                            g[i] = sg * w;
                        }
                        float ek[D];
#pragma unroll
                        for (int k = 0; k < D; ++k) {
                            float sk = 0.f;
#pragma unroll
                            for (int i = 0; i < D; ++i) sk = fmaf(g[i], Jh[k][i], sk);
                            ek[k] = OP == OP_HELMHOLTZ ? sk * s_grad : sk;
                        }
                        if constexpr (OP == OP_HELMHOLTZ) v[0][p * KDP] = live ? w * s_val * v[0][p * KDP] : 0.f;
#pragma unroll
                        for (int k = 0; k < KDP - kV; ++k) v[0][p * KDP + kV + k] = (k < D && live) ? ek[k] : 0.f;
                    } else {
                        float gh[D][D], G[D][D], S[D][D], e[D][D];
#pragma unroll
                        for (int m = 0; m < D; ++m)
#pragma unroll
                            for (int k = 0; k < D; ++k) gh[m][k] = v[m][p * KDP + k];
                        map_grad<D, float>(gh, Jh, G);
                        float tr = G[0][0];
#pragma unroll
                        for (int i = 1; i < D; ++i) tr += G[i][i];
                        const float smu = w * mu_f, slt = w * lam_f * tr;
#pragma unroll
                        for (int i = 0; i < D; ++i) {
                            S[i][i] = fmaf(2.f * smu, G[i][i], slt);
#pragma unroll
                            for (int k = i + 1; k < D; ++k) {
                                const float s = smu * (G[i][k] + G[k][i]);
                                S[i][k] = s;
                                S[k][i] = s;
                            }
                        }
                        pull_back<D, float>(S, Jh, e);
#pragma unroll
                        for (int m = 0; m < D; ++m)
#pragma unroll
                            for (int k = 0; k < KDP; ++k) v[m][p * KDP + k] = (k < D && live) ? e[m][k] : 0.f;
                    }
                }
#pragma unroll
                for (int m = 0; m < NC; ++m) {
                    const size_t region = (size_t)kTcRows * L.N1p;
                    TE *A2 = reinterpret_cast<TE *>(hb + L.a2_off) + (size_t)m * TERMS * region;
                    float first[8], second[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        first[i] = v[m][i];
                        second[i] = v[m][8 + i];
                    }
                    store8<TE, TERMS>(A2 + tc_off(t, blk * 16, L.N1p, ESZ), region, first);
                    store8<TE, TERMS>(A2 + tc_off(t, blk * 16 + 8, L.N1p, ESZ), region, second);
                }
            }
            fence_async_smem();
            tc_fence_before();
            pipe_sync(pipe, tpc);
            tc_fence_after();

            // ---- quadrature GEMM of chunk ch, accumulated over the chunks
            if (pt == 0) {
                const uint32_t sboa = (uint32_t)L.N1p * 8u * ESZ, sbob = (uint32_t)L.K2 * 8u * ESZ;
                const uint32_t a_region = (uint32_t)(kTcRows * L.N1p * ESZ), b_region = (uint32_t)(L.N2p * L.K2 * ESZ);
                for (int m = 0; m < NC; ++m)
                    for (int s = 0; s < L.N1p / KK; ++s)
                        for (int pr = 0; pr < (TERMS == 2 ? 3 : 1); ++pr) {
                            const uint32_t ta = pr == 2 ? 1u : 0u, tb = pr == 1 ? 1u : 0u;
                            const uint64_t da = tc_smem_desc(
                                a2s + ((uint32_t)m * TERMS + ta) * a_region + (uint32_t)s * 256u, 128u, sboa);
                            const uint64_t db = tc_smem_desc(
                                b2s + tb * b_region + (uint32_t)((ch * L.N1p / KK + s) * 256), 128u, sbob);
                            tc_mma<kTf32>(tpipe + (uint32_t)(L.acc1_cols + m * L.N2p), da, db, id2,
                                   (ch > 0 || s > 0 || pr > 0) ? 1u : 0u);
                        }
            }
        }
        if (timed_out) break;
        if (pt == 0) tc_commit(barp);
        if (!pipe_all(pipe, tpc, tc_wait(barp, phase))) {
            tc_wait(barp, phase);
            timed_out = true;
            break;
        }
        phase ^= 1u;
        tc_fence_after();

        // ---- scatter-add (FP64): row t of Y_m holds this cell's node contributions;
        // the cell's tpc threads take every tpc-th group of W nodes (W = 16 for one
        // thread per cell, 8 otherwise, so that the groups split evenly)
        auto scatter = [&](auto width) {
            constexpr int W = decltype(width)::value;
            for (int blk = h; blk < L.N2p / W; blk += tpc) {
                uint32_t r[NC][W];
#pragma unroll
                for (int m = 0; m < NC; ++m) {
                    const uint32_t col = tlane + (uint32_t)(L.acc1_cols + m * L.N2p + blk * W);
                    if constexpr (W == 16)
                        tc_ld16(col, r[m]);
                    else
                        tc_ld8(col, r[m]);
                }
                tc_wait_ld();
                if (a.cell_out && t < nb) {
                    // node-gather scatter: store this cell's outputs (zeros for a skipped cell)
                    double *o = static_cast<double *>(a.cell_out) + (size_t)(tile * kTcRows + t) * n * NC;
#pragma unroll
                    for (int i = 0; i < W; ++i) {
                        const int j = blk * W + i;
                        if (j < n) {
#pragma unroll
                            for (int m = 0; m < NC; ++m)
                                o[j * NC + m] = good ? widen_pow2(__uint_as_float(r[m][i]) * mdet, K) : 0.0;
                        }
                    }
                } else if (good && !a.cell_out) {
#pragma unroll
                    for (int i = 0; i < W; ++i) {
                        const int j = blk * W + i;
                        if (j < n) {
                            const int node = snodes[t * P + j];
#pragma unroll
                            for (int m = 0; m < NC; ++m) {
                                // y += acc |det J| 2^K: FP32 multiply by the mantissa of |det J|,
                                // exact widening, exponent add
                                red_add(a.y + (size_t)node * NC + m, widen_pow2(__uint_as_float(r[m][i]) * mdet, K));
                            }
                        }
                    }
                }
            }
        };
        if (tpc == 1)
            scatter(std::integral_constant<int, 16>{});
        else
            scatter(std::integral_constant<int, 8>{});
        tc_fence_before();
        pipe_sync(pipe, tpc);
    }
    if (timed_out && pt == 0) set_status(a.status, FE_ERR_TIMEOUT);
    if (!nh_ok) set_status(a.status, FE_ERR_NONFINITE);
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"((uint32_t)L.tmem_cols)
                     : "memory");
    leave_queue(a.sched);
}

template <int OP, int D, typename TE, int TERMS>
cudaError_t launch_tc(const ActionArgs &a, int grid, int block, size_t smem, cudaStream_t s)
{
    k_action_tc<OP, D, TE, TERMS><<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
}

// TERMS == 2 (binary16 hi + lo pairs) is the FE_PREC_FP16X2 precision; tf32_t
// operands are FE_PREC_TF32.
template <int OP, int D, typename TE, int TERMS = 1>
Variant make_tc_variant()
{
    Variant v;
    v.form = form_of(OP);
    v.dim = D;
    v.degree = 0;   // any degree with at most 256 local nodes
    v.op = 0;
    v.precision = TERMS == 2                                      ? FE_PREC_FP16X2
                  : std::is_same<TE, tf32_t>::value              ? FE_PREC_TF32
                  : std::is_same<TE, __nv_bfloat16>::value       ? FE_PREC_BF16
                                                                  : FE_PREC_FP16;
    v.kernel_id = 2;   // 128-cell tensor-core tiles
    v.block = kTcRows;
    v.launch = &launch_tc<OP, D, TE, TERMS>;
    v.func = reinterpret_cast<const void *>(&k_action_tc<OP, D, TE, TERMS>);
    return v;
}

}  // namespace fe
