// Dense 32x32 tile factorization shared by the local and the interface Cholesky kernels.
#pragma once
#include "common.cuh"

namespace am {

// Cholesky factor and its inverse of the 32x32 tile X (X(r, c) at c * ldx + r, lower
// triangle used) by one warp: lane r keeps row r of the factor and of the inverse in
// registers.  L goes to Lout (if not null), L^{-1} to Dout (both column-major, zero above
// the diagonal).  A non-positive or non-finite pivot sets *bad and is replaced by 1.
template <typename TW>
__device__ __forceinline__ void warp_chol_inv(const TW* X, int ldx, TW* __restrict__ Lout, TW* __restrict__ Dout,
                                           int lane, int* bad) {
    TW a[TILE];
#pragma unroll
    for (int c = 0; c < TILE; ++c) a[c] = X[c * ldx + lane];
    TW rd_own = (TW)1;   // 1 / L(lane, lane)
#pragma unroll
    for (int k = 0; k < TILE; ++k) {
        TW d = __shfl_sync(0xffffffffu, a[k], k);
        if (!(d > (TW)0) || !isfinite(d)) {   // warp-uniform
            if (lane == 0) *bad = 1;
            d = (TW)1;
        }
        d = sqrt(d);
        const TW rd = (TW)1 / d;
        if (lane > k) a[k] *= rd;
        if (lane == k) {
            a[k] = d;
            rd_own = rd;
        }
        // constant trip counts (a predicate instead of j = k + 1 ..): with a bound that
        // depends on k the compiler left the row in local memory
#pragma unroll
        for (int j = 0; j < TILE; ++j) {
            if (j > k) {
                const TW ljk = __shfl_sync(0xffffffffu, a[k], j);
                if (lane >= j) a[j] -= a[k] * ljk;
            }
        }
    }
    // W = L^{-1}: row t of W is complete (up to its scaling) once rows < t have been
    // subtracted from it; lane r > t then subtracts L(r, t) W(t, :)
    TW w[TILE];
#pragma unroll
    for (int c = 0; c < TILE; ++c) w[c] = c == lane ? (TW)1 : (TW)0;
#pragma unroll
    for (int t = 0; t < TILE; ++t) {
        if (lane == t) {
#pragma unroll
            for (int c = 0; c < TILE; ++c)
                if (c <= t) w[c] *= rd_own;
        }
#pragma unroll
        for (int c = 0; c < TILE; ++c) {
            if (c <= t) {
                const TW wtc = __shfl_sync(0xffffffffu, w[c], t);
                if (lane > t) w[c] -= a[t] * wtc;
            }
        }
    }
#pragma unroll
    for (int c = 0; c < TILE; ++c) {
        if (Lout) Lout[c * TILE + lane] = lane >= c ? a[c] : (TW)0;
        Dout[c * TILE + lane] = w[c];
    }
}

}  // namespace am
