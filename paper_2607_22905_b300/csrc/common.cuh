// Shared device definitions of the AlgMortar CUDA path.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "tile.h"

namespace am {

// Load a stored factor entry as the accumulation type.
template <typename TA, typename TS>
__device__ __forceinline__ TA ldf(const TS* p) { return (TA)(*p); }
template <>
__device__ __forceinline__ float ldf<float, __nv_bfloat16>(const __nv_bfloat16* p) {
    return __bfloat162float(*p);
}
template <>
__device__ __forceinline__ double ldf<double, __nv_bfloat16>(const __nv_bfloat16* p) {
    return (double)__bfloat162float(*p);
}

template <typename TS>
__device__ __forceinline__ TS stf(double x) { return (TS)x; }
template <>
__device__ __forceinline__ __nv_bfloat16 stf<__nv_bfloat16>(double x) {
    return __float2bfloat16_rn((float)x);
}

// Storage of a 32x32 tile in the sweep streams: row-major, 16-byte chunks of row r
// XOR-swizzled by a per-row key so that 32 lanes reading their own rows with 128-bit
// shared loads hit distinct banks within each quarter-warp.
template <typename TS>
__host__ __device__ __forceinline__ int swz_row_key(int r) {
    return sizeof(TS) == 2 ? ((r >> 1) & 3) : (r & 7);
}
template <typename TS>
__host__ __device__ __forceinline__ int swz_index(int r, int c) {
    constexpr int E = 16 / sizeof(TS);          // elements per 16-byte chunk
    return r * TILE + (((c / E) ^ swz_row_key<TS>(r)) * E) + (c % E);
}

// Tile-profile descriptor set of a batch of lower-triangular factors (one per subdomain,
// or the single interface matrix).  Tile (I, J), lo[I] <= J <= I, of item s lives at
// tile index base[s] + fwd[row0[s] + I] + (J - lo[row0[s] + I]) of the forward stream,
// column-major inside the tile.  The backward stream holds, for I = T-1 .. 0, the tiles
// (L_JI)^T for J = I+1 .. hi[I] followed by the diagonal slot, from bwd[row0 + I].
struct Profile {
    const int32_t* rows;      // rows of item s
    const int32_t* ntiles;    // tile rows T of item s
    const int64_t* row0;      // first tile-row descriptor of item s
    const int64_t* base;      // first tile of item s
    const int32_t* lo;
    const int32_t* hi;
    const int64_t* fwd;
    const int64_t* bwd;
};

// Device-side PCG scalars (FP64 throughout, Sec. 7).
struct PcgScalars {
    double rz;        // rho_k = r_k . z_k of the current search direction
    double rz_next;   // r . z of the latest preconditioned residual
    double pq;        // p_k . A p_k
    double alpha, beta;
    double rr;        // ||r_k||^2 (checked)
    double rr_new;    // ||r||^2 after the latest update
    double bb;        // ||b||^2
    double tol2;      // tol^2 ||b||^2
    double res2;      // ||b - A x||^2 (true residual, on request)
    double rz_mix;    // r_{k+1} . z_k (flexible beta only)
    int32_t iter;     // products with A so far
    int32_t done;     // 1: stop (converged or failed)
    int32_t status;   // 0 converged, 5 max_it, 6 breakdown
    int32_t max_it;
    int32_t flexible; // 1: Polak-Ribiere beta
    int32_t restart;  // 1: the residual was just replaced by b - A x; next beta = 0
    int32_t step_ok;  // p . A p > 0 and alpha finite (set with alpha)
    int32_t pad_;
};

// Column layout of a batch of right-hand sides processed by one launch (gridDim.y =
// columns): N-vectors of column j start j * v doubles after column 0, interface vectors
// j * l after, and column j's stop flag is done[j * done_stride] (null: never stop).
struct ColStrides {
    int64_t v;
    int64_t l;
    const int32_t* done;
    int done_stride;
    int sc_stride;        // doubles between consecutive columns' PCG states
};

// Deterministic grid-wide sum: every CTA writes its block sum to part[blockIdx.x]; the
// CTA that finishes last (atomic ticket) adds the partials in a fixed order, stores the
// total and re-arms the ticket.  Same inputs -> bit-identical result.
struct GridSum {
    double* part;          // >= gridDim.x doubles
    unsigned int* ticket;  // 0 between launches
};

// Deterministic fixed-order sum of `n` partials by one warp; result in all lanes.
__device__ __forceinline__ double warp_sum_partials(const double* part, int n) {
    int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int i = lane; i < n; i += 32) s += part[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// Same as warp_sum_partials, reading with L1 bypass (partials written by other CTAs).
__device__ __forceinline__ double warp_sum_partials_cg(const double* part, int n) {
    int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int i = lane; i < n; i += 32) s += __ldcg(part + i);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// Block-wide sum (blockDim.x a multiple of 32); result valid in thread 0.  `sh` holds
// blockDim.x doubles: every thread stores its value and warp 0 alone adds them (a
// fixed strided assignment, then a shuffle tree).  One warp doing the additions costs
// blockDim.x / 32 + 5 warp-wide FP64 adds, against 5 per warp plus 5 for a shuffle tree
// in every warp; B300 runs FP64 at 1/64 of its FP32 rate, so at several CTAs per SM
// the shorter form is visible in the dot-product kernels.
__device__ __forceinline__ double block_sum(double v, double* sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    sh[threadIdx.x] = v;
    __syncthreads();
    double s = 0.0;
    if (w == 0) {
        for (int i = lane; i < (int)blockDim.x; i += 32) s += sh[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    __syncthreads();
    return s;
}

// Two grid-wide sums at once (partials interleaved, 2 per CTA); same contract as grid_sum.
__device__ __forceinline__ bool grid_sum2(double v0, double v1, double* sh, GridSum g, double* r0, double* r1) {
    __shared__ int last2;
    const double s0 = block_sum(v0, sh);
    const double s1 = block_sum(v1, sh);
    if (threadIdx.x == 0) {
        g.part[2 * blockIdx.x] = s0;
        g.part[2 * blockIdx.x + 1] = s1;
        __threadfence();
        last2 = atomicAdd(g.ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last2) {
        __threadfence();
        double t0 = 0.0, t1 = 0.0;
        for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
            t0 += __ldcg(g.part + 2 * i);
            t1 += __ldcg(g.part + 2 * i + 1);
        }
        t0 = block_sum(t0, sh);
        t1 = block_sum(t1, sh);
        if (threadIdx.x == 0) {
            *r0 = t0;
            *r1 = t1;
            *g.ticket = 0;
        }
    }
    return last2 != 0;
}

// Grid-wide deterministic sum of v into *result (see GridSum); returns true in the CTA
// that wrote the result (its threads may then use *result after a __syncthreads).  The
// last CTA adds the partials with all its threads (fixed strided assignment, then a
// fixed-order block reduction), so the tail stays short.
__device__ __forceinline__ bool grid_sum(double v, double* sh, GridSum g, double* result) {
    __shared__ int last;
    double s = block_sum(v, sh);
    if (threadIdx.x == 0) {
        g.part[blockIdx.x] = s;
        __threadfence();
        last = atomicAdd(g.ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
        __threadfence();
        double t = 0.0;
        for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) t += __ldcg(g.part + i);
        t = block_sum(t, sh);
        if (threadIdx.x == 0) {
            *result = t;
            *g.ticket = 0;
        }
    }
    return last != 0;
}

}  // namespace am
