// Krylov building blocks for conjugate gradients with FP64 iterative refinement.
//
// The action is the operator; these kernels supply the vector work of one CG
// iteration with every scalar kept on the device (no host round trip per
// iteration, so a run of iterations can be captured in a CUDA graph):
//   start:        r = M (b - A x), p = r, rr = r.r
//   direction:    q <- M q (Dirichlet rows), pq = p.q, alpha = rr / pq
//   update:       x += alpha p, r -= alpha q, beta = r.r / rr, rr = r.r
//   new direction p = r + beta p
// M is the diagonal 0/1 mask of free DoFs (NULL: all free).  Reductions are
// deterministic: a fixed grid, a fixed per-block summation order, and the last
// block to finish adds the per-block partials in index order.
#include <cstdint>

#include "fe_internal.h"

namespace fe {
namespace {

constexpr int kVecBlock = 256;
constexpr int kVecGrid = FE_CG_PARTIALS;   // partial sums (one per block)

// workspace layout (doubles): [0, kVecGrid) partials, then scalars
enum Scalar { S_RR = 0, S_PQ = 1, S_ALPHA = 2, S_BETA = 3, S_RRNEW = 4, S_DOT = 5, S_COUNTER = 15 };

__device__ __forceinline__ double *scalars(double *ws) { return ws + kVecGrid; }

__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double warp_sums[kVecBlock / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kVecBlock / 32; ++w) s += warp_sums[w];
    return s;  // valid in thread 0
}

// Writes this block's partial; returns true in thread 0 of the last block to
// finish, after which all partials are visible.
__device__ __forceinline__ bool publish_partial(double *ws, double partial)
{
    __shared__ int last;
    if (threadIdx.x == 0) {
        ws[blockIdx.x] = partial;
        __threadfence();
        unsigned int *counter = reinterpret_cast<unsigned int *>(scalars(ws) + S_COUNTER);
        last = (atomicAdd(counter, 1u) == gridDim.x - 1);
        if (last) *counter = 0u;  // self-reset for the next reduction
    }
    __syncthreads();
    return threadIdx.x == 0 && last;
}

__device__ __forceinline__ double sum_partials(const double *ws)
{
    __threadfence();
    double s = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) s += ((volatile const double *)ws)[b];
    return s;
}

__device__ __forceinline__ double free_of(const uint8_t *mask, long long i)
{
    return mask ? (double)mask[i] : 1.0;
}

__global__ void __launch_bounds__(kVecBlock) k_cg_start(long long n, const double *__restrict__ b,
                                                        const double *__restrict__ Ax,
                                                        const uint8_t *__restrict__ mask, double *r,
                                                        double *p, double *ws)
{
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double ri = free_of(mask, i) * (b[i] - Ax[i]);
        r[i] = ri;
        p[i] = ri;
        acc = fma(ri, ri, acc);
    }
    const double part = block_sum(acc);
    if (publish_partial(ws, part)) scalars(ws)[S_RR] = sum_partials(ws);
}

__global__ void __launch_bounds__(kVecBlock) k_cg_direction(long long n, const double *__restrict__ p,
                                                            double *q, const uint8_t *__restrict__ mask,
                                                            double *ws)
{
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double qi = q[i];
        if (mask && !mask[i]) {
            qi = 0.0;
            q[i] = 0.0;
        }
        acc = fma(p[i], qi, acc);
    }
    const double part = block_sum(acc);
    if (publish_partial(ws, part)) {
        double *sc = scalars(ws);
        const double pq = sum_partials(ws);
        sc[S_PQ] = pq;
        sc[S_ALPHA] = (pq != 0.0) ? sc[S_RR] / pq : 0.0;
    }
}

__global__ void __launch_bounds__(kVecBlock) k_cg_update(long long n, double *x, double *r,
                                                         const double *__restrict__ p,
                                                         const double *__restrict__ q, double *ws)
{
    const double alpha = scalars(ws)[S_ALPHA];
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        x[i] = fma(alpha, p[i], x[i]);
        const double ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        acc = fma(ri, ri, acc);
    }
    const double part = block_sum(acc);
    if (publish_partial(ws, part)) {
        double *sc = scalars(ws);
        const double rr_new = sum_partials(ws);
        sc[S_BETA] = (sc[S_RR] != 0.0) ? rr_new / sc[S_RR] : 0.0;
        sc[S_RRNEW] = rr_new;
        sc[S_RR] = rr_new;
    }
}

__global__ void __launch_bounds__(kVecBlock) k_cg_new_direction(long long n, const double *__restrict__ r,
                                                                double *p, const double *ws)
{
    const double beta = scalars(const_cast<double *>(ws))[S_BETA];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = fma(beta, p[i], r[i]);
}

__global__ void __launch_bounds__(kVecBlock) k_axpy(long long n, double a, const double *__restrict__ x, double *y)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = fma(a, x[i], y[i]);
}

__global__ void __launch_bounds__(kVecBlock) k_dot(long long n, const double *__restrict__ x,
                                                   const double *__restrict__ y, const uint8_t *__restrict__ mask,
                                                   double *ws, int slot)
{
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        acc = fma(free_of(mask, i) * x[i], y[i], acc);
    const double part = block_sum(acc);
    if (publish_partial(ws, part)) scalars(ws)[slot] = sum_partials(ws);
}

int vec_grid(long long n)
{
    long long g = (n + kVecBlock - 1) / kVecBlock;
    if (g > kVecGrid) g = kVecGrid;
    return (int)(g < 1 ? 1 : g);
}

int finish() { return cudaGetLastError() == cudaSuccess ? FE_OK : FE_ERR_CUDA; }

}  // namespace
}  // namespace fe

using namespace fe;

extern "C" int fe_cg_start(long long n, const double *b, const double *Ax, const uint8_t *mask, double *r,
                           double *p, double *ws, void *stream)
{
    if (n < 1 || !b || !Ax || !r || !p || !ws) return FE_ERR_INVALID_ARG;
    k_cg_start<<<vec_grid(n), kVecBlock, 0, static_cast<cudaStream_t>(stream)>>>(n, b, Ax, mask, r, p, ws);
    return finish();
}

extern "C" int fe_cg_direction(long long n, const double *p, double *q, const uint8_t *mask, double *ws,
                               void *stream)
{
    if (n < 1 || !p || !q || !ws) return FE_ERR_INVALID_ARG;
    k_cg_direction<<<vec_grid(n), kVecBlock, 0, static_cast<cudaStream_t>(stream)>>>(n, p, q, mask, ws);
    return finish();
}

extern "C" int fe_cg_update(long long n, double *x, double *r, const double *p, const double *q, double *ws,
                            void *stream)
{
    if (n < 1 || !x || !r || !p || !q || !ws) return FE_ERR_INVALID_ARG;
    k_cg_update<<<vec_grid(n), kVecBlock, 0, static_cast<cudaStream_t>(stream)>>>(n, x, r, p, q, ws);
    return finish();
}

extern "C" int fe_cg_new_direction(long long n, const double *r, double *p, const double *ws, void *stream)
{
    if (n < 1 || !r || !p || !ws) return FE_ERR_INVALID_ARG;
    k_cg_new_direction<<<vec_grid(n), kVecBlock, 0, static_cast<cudaStream_t>(stream)>>>(n, r, p, ws);
    return finish();
}

extern "C" int fe_vec_axpy(long long n, double a, const double *x, double *y, void *stream)
{
    if (n < 1 || !x || !y) return FE_ERR_INVALID_ARG;
    k_axpy<<<vec_grid(n), kVecBlock, 0, static_cast<cudaStream_t>(stream)>>>(n, a, x, y);
    return finish();
}

extern "C" int fe_vec_dot(long long n, const double *x, const double *y, const uint8_t *mask, double *ws,
                          int slot, void *stream)
{
    if (n < 1 || !x || !y || !ws || slot < 0 || slot >= 15) return FE_ERR_INVALID_ARG;
    k_dot<<<vec_grid(n), kVecBlock, 0, static_cast<cudaStream_t>(stream)>>>(n, x, y, mask, ws, slot);
    return finish();
}
