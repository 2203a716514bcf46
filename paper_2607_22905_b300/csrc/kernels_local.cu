// Local (subdomain) kernels of AlgMortar on sm_103a: assembly of the diagonally
// modified blocks A_i (Eq. A_i), their tile-profile Cholesky factorisation (Algorithm 1,
// "compute the Cholesky factorization A_i = L_i L_i^T"), the sweep streams, and the
// batched forward/backward triangular solves used for the particular solutions
// (Eq. def-pbar-local), the MBFs (Eq. def-phat-local) and the explicit interface inverse.
#include "async.cuh"
#include "common.cuh"
#include "kernels.h"
#include "tile_chol.cuh"

namespace am {

// ---------------------------------------------------------------------------------
// Diagonal of A_i = A_ii - sum_j D_ij (Eqs. Dij-def, A_i): a_kk minus the row's couplings
// to other subdomains (which are <= 0, so the diagonal grows).  sc = 1/sqrt(diag) when
// symmetric diagonal scaling is on, else 1.
// ---------------------------------------------------------------------------------
__global__ void k_local_diag(int64_t n, const int32_t* __restrict__ rowptr,
                             const int32_t* __restrict__ col, const double* __restrict__ val,
                             const int32_t* __restrict__ row_sub, int diag_scale, int modified,
                             double* __restrict__ dloc, double* __restrict__ sc, float* __restrict__ sc32) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        int32_t s = row_sub[k];
        double d = 0.0, cross = 0.0;
        for (int32_t e = rowptr[k]; e < rowptr[k + 1]; ++e) {
            int32_t c = col[e];
            if (c == k) d = val[e];
            else if (row_sub[c] != s) cross += val[e];
        }
        // A_i = A_ii - sum_j D_ij (Eq. A_i); the block-Jacobi smoother factors A_ii itself
        double dl = modified ? d - cross : d;
        dloc[k] = dl;
        const double f = diag_scale ? 1.0 / sqrt(dl) : 1.0;
        sc[k] = f;
        sc32[k] = (float)f;
    }
}

// Scatter the (scaled) lower triangle of every A_i into its tile-profile work storage.
template <typename TW>
__global__ void k_scatter_local(int64_t n, const int32_t* __restrict__ rowptr,
                                const int32_t* __restrict__ col, const double* __restrict__ val,
                                const int32_t* __restrict__ row_sub,
                                const int64_t* __restrict__ sub_off, Profile pf,
                                const double* __restrict__ dloc, const double* __restrict__ sc,
                                TW* __restrict__ work) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        int32_t s = row_sub[k];
        int64_t a = sub_off[s];
        int32_t r = (int32_t)(k - a);
        int64_t rd = pf.row0[s] + (r >> 5);
        int32_t lo = pf.lo[rd];
        int64_t trow = pf.base[s] + pf.fwd[rd];
        double sk = sc[k];
        for (int32_t e = rowptr[k]; e < rowptr[k + 1]; ++e) {
            int32_t c = col[e];
            if (row_sub[c] != s) continue;
            int32_t lc = (int32_t)(c - a);
            if (lc > r) continue;
            double v = (c == k) ? dloc[k] : val[e];
            v *= sk * sc[c];
            int64_t t = trow + ((lc >> 5) - lo);
            work[t * TILE2 + (lc & 31) * TILE + (r & 31)] = (TW)v;
        }
    }
}

// Unit diagonal on the padding rows of each item's last tile.
template <typename TW>
__global__ void k_pad_diag(int nitems, Profile pf, TW* __restrict__ work) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nitems) return;
    int32_t T = pf.ntiles[s], n = pf.rows[s];
    int64_t rd = pf.row0[s] + T - 1;
    int64_t t = pf.base[s] + pf.fwd[rd] + (T - 1 - pf.lo[rd]);
    for (int r = n; r < T * TILE; ++r) work[t * TILE2 + (r & 31) * (TILE + 1)] = (TW)1;
}

// Dense Cholesky of the 32x32 tile X (lower triangle used) in shared memory by a CTA of
// 256 threads, followed by the inverse of the lower-triangular factor into Ainv (one
// column per thread).  A non-positive or non-finite pivot sets *bad and is replaced by 1.
template <typename TW>
__device__ void chol_inv_tile(TW (*X)[TILE + 1], TW (*Ainv)[TILE + 1], int tid, int* bad) {
    for (int k = 0; k < TILE; ++k) {
        if (tid == 0) {
            TW d = X[k][k];
            if (!(d > (TW)0) || !isfinite((double)d)) {
                *bad = 1;
                d = (TW)1;
            }
            X[k][k] = sqrt(d);
        }
        __syncthreads();
        if (tid > k && tid < TILE) X[tid][k] /= X[k][k];
        __syncthreads();
        for (int e = tid; e < TILE2; e += blockDim.x) {
            int r = e >> 5, cc = e & 31;
            if (cc > k && r >= cc) X[r][cc] -= X[r][k] * X[cc][k];
        }
        __syncthreads();
    }
    if (tid < TILE) {
        const int cc = tid;
        for (int r = 0; r < TILE; ++r) {
            TW v;
            if (r < cc) {
                v = 0;
            } else {
                v = (r == cc) ? (TW)1 : (TW)0;
                for (int t = cc; t < r; ++t) v -= X[r][t] * Ainv[t][cc];
                v /= X[r][r];
            }
            Ainv[r][cc] = v;
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------------
// Tile-profile Cholesky, one CTA (256 threads) per item, up-looking by tile rows:
//   L_IJ = (A_IJ - sum_K L_IK L_JK^T) L_JJ^{-T},   J = lo(I) .. I-1
//   L_II = chol(A_II - sum_K L_IK L_IK^T)
// Fill stays inside the envelope of A (Cholesky of a profile matrix), hence inside the
// tile profile.  The inverse of every diagonal tile is kept in dinv (one tile per tile
// row): it turns the panel update into a product and becomes the diagonal block of the
// sweep streams.  A non-positive pivot sets err = {1, item} and continues with pivot 1.
// ---------------------------------------------------------------------------------
template <typename TW>
__global__ void __launch_bounds__(256) k_tile_chol(Profile pf, const int32_t* __restrict__ order,
                                                   TW* __restrict__ work, TW* __restrict__ dinv,
                                                   int* __restrict__ err) {
    const int s = order ? order[blockIdx.x] : blockIdx.x;
    const int T = pf.ntiles[s];
    const int64_t r0 = pf.row0[s];
    const int32_t* lo = pf.lo + r0;
    const int64_t* fwd = pf.fwd + r0;
    TW* Wb = work + pf.base[s] * TILE2;
    TW* Db = dinv + r0 * TILE2;
    __shared__ TW X[TILE][TILE + 1];
    __shared__ TW Ab[2][TILE][TILE + 1];   // the K loop's tiles, double-buffered
    __shared__ TW Bb[2][TILE][TILE + 1];
    __shared__ int bad;
    TW(*As)[TILE + 1] = Ab[0];
    TW(*Bs)[TILE + 1] = Bb[0];
    const int tid = threadIdx.x, c = tid & 31, rb = (tid >> 5) * 4;
    if (tid == 0) bad = 0;
    auto tile = [&](int I, int J) { return Wb + (fwd[I] + (J - lo[I])) * TILE2; };
    auto load = [&](TW(*dst)[TILE + 1], const TW* g) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int e = tid + 256 * q;
            dst[e & 31][e >> 5] = g[e];
        }
    };
    // asynchronous element copies into the same transposed, padded layout: the tiles of
    // step K + 1 load while step K multiplies (the chain of a large subdomain otherwise
    // waits one global round trip per step)
    auto load_async = [&](TW(*dst)[TILE + 1], const TW* g) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int e = tid + 256 * q;
            if constexpr (sizeof(TW) == 8)
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(&dst[e & 31][e >> 5])),
                             "l"(g + e) : "memory");
            else
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(&dst[e & 31][e >> 5])),
                             "l"(g + e) : "memory");
        }
    };
    for (int I = 0; I < T; ++I) {
        const int li = lo[I];
        for (int J = li; J <= I; ++J) {
            const TW* Aij = tile(I, J);
            TW acc[4];
            const int k0 = max(li, lo[J]);
            if (k0 < J) {
                load_async(Ab[0], tile(I, k0));
                load_async(Bb[0], tile(J, k0));
                asm volatile("cp.async.commit_group;" ::: "memory");
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = Aij[c * TILE + rb + q];
            int kb = 0;
            for (int K = k0; K < J; ++K) {
                if (K + 1 < J) {
                    load_async(Ab[kb ^ 1], tile(I, K + 1));
                    load_async(Bb[kb ^ 1], tile(J, K + 1));
                    asm volatile("cp.async.commit_group;" ::: "memory");
                    asm volatile("cp.async.wait_group 1;" ::: "memory");
                } else {
                    asm volatile("cp.async.wait_group 0;" ::: "memory");
                }
                __syncthreads();
#pragma unroll 8
                for (int t = 0; t < TILE; ++t) {
                    TW b = Bb[kb][c][t];
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[q] -= Ab[kb][rb + q][t] * b;
                }
                __syncthreads();   // before buffer kb is refilled
                kb ^= 1;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) X[rb + q][c] = acc[q];
            if (J < I) {
                load(Bs, Db + (int64_t)J * TILE2);          // L_JJ^{-1}
                __syncthreads();
                TW* Lij = Wb + (fwd[I] + (J - li)) * TILE2;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    TW v = 0;
#pragma unroll 8
                    for (int t = 0; t < TILE; ++t) v += X[rb + q][t] * Bs[c][t];
                    Lij[c * TILE + rb + q] = v;
                }
                __syncthreads();
            } else {
                __syncthreads();
                chol_inv_tile<TW>(X, As, tid, &bad);
                TW* Lii = Wb + (fwd[I] + (I - li)) * TILE2;
                TW* Dii = Db + (int64_t)I * TILE2;
                for (int e = tid; e < TILE2; e += 256) {
                    int r = e & 31, cc = e >> 5;
                    Lii[e] = r >= cc ? X[r][cc] : (TW)0;
                    Dii[e] = As[r][cc];
                }
                __syncthreads();
            }
        }
    }
    if (tid == 0 && bad) {
        if (atomicCAS(err + 1, -1, s) == -1) atomicExch(err, 1);
    }
}


// ---------------------------------------------------------------------------------
// The same factorization with the current tile row resident in shared memory: one CTA
// (4 warps) per item; thread (lane c, warp w) owns the 8 entries (8w .. 8w+7, c) of every
// tile it computes.  For tile (I, J) the CTA
//   1. copies row J's tiles L_J,k0 .. L_J,J-1 (one contiguous block of the work array)
//      and L_JJ^{-1} into shared memory with 16-byte asynchronous copies (J < I), while
//      each thread loads its 8 entries of A_IJ;
//   2. subtracts sum_K L_IK L_JK^T, the L_IK from the resident row (no reloads);
//   3. J < I: L_IJ = X L_JJ^{-T} (X staged in shared memory), stored to the work array
//      and to the resident row; J = I: one warp factors X (row `lane` in registers,
//      pivots by shuffles) and inverts the factor by forward substitution on all 32
//      right-hand sides at once, then writes L_II and L_II^{-1}.
// Every tile therefore costs one global round trip, where the per-step version pays one
// per K step and two more for A_IJ and L_JJ^{-1}; the diagonal tile needs no barriers.
// Shared memory: wm resident tiles + wm staged tiles + X, wm = widest tile row.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ void ld8(const float* p, float (&v)[8]) {
    const float4 x = reinterpret_cast<const float4*>(p)[0], y = reinterpret_cast<const float4*>(p)[1];
    v[0] = x.x, v[1] = x.y, v[2] = x.z, v[3] = x.w, v[4] = y.x, v[5] = y.y, v[6] = y.z, v[7] = y.w;
}
__device__ __forceinline__ void ld8(const double* p, double (&v)[8]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const double2 x = reinterpret_cast<const double2*>(p)[i];
        v[2 * i] = x.x, v[2 * i + 1] = x.y;
    }
}
__device__ __forceinline__ void st8(float* p, const float (&v)[8]) {
    reinterpret_cast<float4*>(p)[0] = make_float4(v[0], v[1], v[2], v[3]);
    reinterpret_cast<float4*>(p)[1] = make_float4(v[4], v[5], v[6], v[7]);
}
__device__ __forceinline__ void st8(double* p, const double (&v)[8]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) reinterpret_cast<double2*>(p)[i] = make_double2(v[2 * i], v[2 * i + 1]);
}

template <typename TW>
__global__ void __launch_bounds__(128) k_tile_chol_row(Profile pf, const int32_t* __restrict__ order,
                                                       TW* __restrict__ work, TW* __restrict__ dinv,
                                                       int* __restrict__ err, int wm) {
    constexpr int VE = 16 / sizeof(TW);
    constexpr int LDR = TILE + VE;   // padded column stride of the resident row and X
    const int s = order ? order[blockIdx.x] : blockIdx.x;
    const int T = pf.ntiles[s];
    const int64_t r0 = pf.row0[s];
    const int32_t* lo = pf.lo + r0;
    const int64_t* fwd = pf.fwd + r0;
    TW* Wb = work + pf.base[s] * TILE2;
    TW* Db = dinv + r0 * TILE2;
    extern __shared__ __align__(16) unsigned char tc_raw[];
    TW* rowt = reinterpret_cast<TW*>(tc_raw);           // [wm][TILE * LDR]: L_I,lo .. L_I,I-1
    TW* stg = rowt + (size_t)wm * TILE * LDR;            // [wm - 1][TILE2] L_J,K + [TILE2] L_JJ^{-1}
    TW* dstg = stg + (size_t)(wm - 1) * TILE2;
    TW* X = dstg + TILE2;                                // [TILE * LDR]
    int* bad = reinterpret_cast<int*>(X + TILE * LDR);
    const int tid = threadIdx.x, c = tid & 31, w = tid >> 5, rb = w * 8;
    if (tid == 0) *bad = 0;
    auto tile = [&](int I, int J) { return Wb + (fwd[I] + (J - lo[I])) * TILE2; };
    for (int I = 0; I < T; ++I) {
        const int li = lo[I];
        for (int J = li; J <= I; ++J) {
            const int k0 = max(li, lo[J]);
            const int nK = J - k0;
            if (J < I) {
                const char* gsrc = reinterpret_cast<const char*>(tile(J, k0));
                const int nch = nK * (int)(TILE2 * sizeof(TW) / 16);
                for (int i = tid; i < nch; i += blockDim.x)
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(stg) + 16u * i),
                                 "l"(gsrc + 16 * (int64_t)i) : "memory");
                const char* dsrc = reinterpret_cast<const char*>(Db + (int64_t)J * TILE2);
                for (int i = tid; i < (int)(TILE2 * sizeof(TW) / 16); i += blockDim.x)
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dstg) + 16u * i),
                                 "l"(dsrc + 16 * (int64_t)i) : "memory");
                asm volatile("cp.async.commit_group;" ::: "memory");
            }
            TW acc[8];
            const TW* Aij = tile(I, J);
            ld8(Aij + c * TILE + rb, acc);
            if (J < I) asm volatile("cp.async.wait_group 0;" ::: "memory");
            __syncthreads();
            // X = A_IJ - sum_K L_IK L_JK^T
            for (int K = k0; K < J; ++K) {
                const TW* Ak = rowt + (size_t)(K - li) * TILE * LDR;
                const TW* Bk = J < I ? stg + (size_t)(K - k0) * TILE2 : rowt + (size_t)(K - li) * TILE * LDR;
                const int ldb = J < I ? TILE : LDR;
#pragma unroll 4
                for (int t = 0; t < TILE; ++t) {
                    const TW b = Bk[t * ldb + c];
                    TW av[8];
                    ld8(Ak + t * LDR + rb, av);
#pragma unroll
                    for (int q = 0; q < 8; ++q) acc[q] -= av[q] * b;
                }
            }
            st8(X + c * LDR + rb, acc);
            __syncthreads();
            if (J < I) {
                // L_IJ(r, c) = sum_t X(r, t) L_JJ^{-1}(c, t)
                TW v[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) v[q] = (TW)0;
#pragma unroll 4
                for (int t = 0; t < TILE; ++t) {
                    const TW d = dstg[t * TILE + c];
                    TW xv[8];
                    ld8(X + t * LDR + rb, xv);
#pragma unroll
                    for (int q = 0; q < 8; ++q) v[q] += xv[q] * d;
                }
                st8(tile(I, J) + c * TILE + rb, v);
                st8(rowt + (size_t)(J - li) * TILE * LDR + c * LDR + rb, v);
            } else if (w == 0) {
                warp_chol_inv<TW>(X, LDR, tile(I, I), Db + (int64_t)I * TILE2, c, bad);
            }
            __syncthreads();   // X, the staged tiles and the resident row are reused
        }
    }
    if (tid == 0 && *bad) {
        if (atomicCAS(err + 1, -1, s) == -1) atomicExch(err, 1);
    }
}

size_t tile_chol_row_smem(int wm, size_t elem) {
    const size_t ve = 16 / elem, ldr = TILE + ve;
    return ((size_t)wm * TILE * ldr + (size_t)wm * TILE2 + TILE * ldr) * elem + 16;
}

// ---------------------------------------------------------------------------------
// Sweep streams from the factor: forward rows [L_I,lo .. L_I,I-1 | L_II^{-1}], backward
// rows [(L_I+1,I)^T .. (L_hi,I)^T | L_II^{-T}], in precision TS.  Every 32x32 tile M is
// stored row-major with its 16-byte chunks XOR-swizzled (swz_index), so that the solve
// reads row `lane` of a tile with conflict-free 128-bit shared loads.
//
// FP32 arithmetic (FP32 and BF16 streams) solves tile rows in pairs (a, b) = (2P, 2P+1):
// with the 64x64 diagonal block [[L_aa, 0], [L_ba, L_bb]] its inverse is
// [[D_a, 0], [C, D_b]], D = L^{-1} of the diagonal tiles and C = -D_b L_ba D_a, so
//   forward   x_a = D_a t_a,      x_b = D_b t_b + C t_a
//   backward  x_b = D_b^T t_b,    x_a = D_a^T t_a + C^T t_b
// (t_I: row I's right-hand side minus its terms outside the pair).  The tile L_ba is
// stored as C in the forward row b and as C^T in the backward row a -- same tiles, same
// bytes -- and both come from one FP32 product, so the backward stream stays the exact
// transpose of the forward one and L^{-T} L^{-1} stays symmetric after rounding.  FP64
// streams keep the plain factor.
// ---------------------------------------------------------------------------------
// factor entry (FP32 or FP64 work precision) -> stream precision, directly: a conversion
// through double would run twice on B300's FP64 pipe per entry (float -> double -> float)
template <typename TS, typename TW>
__device__ __forceinline__ TS to_stream(TW x) {
    if constexpr (std::is_same<TS, __nv_bfloat16>::value) {
        if constexpr (std::is_same<TW, float>::value) return __float2bfloat16_rn(x);
        else return stf<TS>((double)x);
    } else {
        return (TS)x;
    }
}

template <typename TW, typename TS>
__global__ void __launch_bounds__(256) k_finalize(Profile pf, const TW* __restrict__ work,
                                                  const TW* __restrict__ dinv,
                                                  TS* __restrict__ fwdS, TS* __restrict__ bwdS) {
    constexpr bool kPair = sizeof(TW) == 4;
    __shared__ TW As[kPair ? TILE : 1][TILE + 1];
    __shared__ TW Bs[kPair ? TILE : 1][TILE + 1];
    __shared__ TW Ms[TILE][TILE + 1];   // a forward tile, read coalesced
    const int s = blockIdx.x;
    const int T = pf.ntiles[s];
    const int64_t r0 = pf.row0[s];
    const int32_t* lo = pf.lo + r0;
    const int32_t* hi = pf.hi + r0;
    const int64_t* fwd = pf.fwd + r0;
    const int64_t* bwd = pf.bwd + r0;
    const int64_t base = pf.base[s];
    const TW* Wb = work + base * TILE2;
    const TW* Db = dinv + r0 * TILE2;
    const int tid = threadIdx.x, cc = tid & 31, rb = (tid >> 5) * 4;
    for (int I = blockIdx.y; I < T; I += gridDim.y) {
        const int nt = I - lo[I];
        const int64_t fo = (base + fwd[I]) * TILE2;
        // the pair's coupling tile: forward row I = b (odd) at t = nt - 1 (J = I - 1)
        const bool cfw = kPair && (I & 1) && nt > 0;
        // forward: M = L_IJ (column-major source: M[r][c] at c*32 + r), then L_II^{-1}
        for (int t = 0; t <= nt; ++t) {
            if (cfw && t == nt - 1) continue;
            const TW* src = t < nt ? Wb + (fwd[I] + t) * TILE2 : Db + (int64_t)I * TILE2;
            for (int e = tid; e < TILE2; e += blockDim.x) Ms[e >> 5][e & 31] = src[e];   // Ms[c][r] = M[r][c]
            __syncthreads();
            for (int e = tid; e < TILE2; e += blockDim.x) {
                const int r = e >> 5, c = e & 31;
                fwdS[fo + (int64_t)t * TILE2 + swz_index<TS>(r, c)] = to_stream<TS>(Ms[c][r]);
            }
            __syncthreads();
        }
        if constexpr (kPair) {
            if (cfw) {   // C = -D_b (L_ba D_a), b = I, a = I - 1
                const TW* Lba = Wb + (fwd[I] + nt - 1) * TILE2;
                const TW* Da = Db + (int64_t)(I - 1) * TILE2;
                const TW* Dbb = Db + (int64_t)I * TILE2;
                for (int e = tid; e < TILE2; e += blockDim.x) {   // column-major sources
                    As[e & 31][e >> 5] = Lba[e];
                    Bs[e & 31][e >> 5] = Da[e];
                }
                __syncthreads();
                TW acc[4] = {0, 0, 0, 0};
#pragma unroll 8
                for (int u = 0; u < TILE; ++u) {
                    const TW bv = Bs[u][cc];
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[q] += As[rb + q][u] * bv;
                }
                __syncthreads();
#pragma unroll
                for (int q = 0; q < 4; ++q) As[rb + q][cc] = acc[q];   // L_ba D_a
                for (int e = tid; e < TILE2; e += blockDim.x) Bs[e & 31][e >> 5] = Dbb[e];
                __syncthreads();
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[q] = 0;
#pragma unroll 8
                for (int u = 0; u < TILE; ++u) {
                    const TW av = As[u][cc];
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[q] -= Bs[rb + q][u] * av;
                }
                // C[r][c]: forward row b at t = nt - 1, backward row a at t = 0 as C^T
                TS* cf = fwdS + fo + (int64_t)(nt - 1) * TILE2;
                TS* cb = bwdS + (base + bwd[I - 1]) * TILE2;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const TS cv = to_stream<TS>(acc[q]);
                    cf[swz_index<TS>(rb + q, cc)] = cv;
                    cb[swz_index<TS>(cc, rb + q)] = cv;
                }
                __syncthreads();
            }
        }
        // backward: M = (L_JI)^T (M[r][c] = L_JI[c][r] at r*32 + c), then L_II^{-T}
        const int nb = hi[I] - I;
        const int64_t bo = (base + bwd[I]) * TILE2;
        // the pair's coupling tile: backward row I = a (even) at t = 0 (J = I + 1), written
        // with the forward row b above
        const bool cbw = kPair && !(I & 1) && nb > 0;
        for (int t = 0; t <= nb; ++t) {
            if (cbw && t == 0) continue;
            const TW* src = t < nb ? Wb + (fwd[I + 1 + t] + (I - lo[I + 1 + t])) * TILE2 : Db + (int64_t)I * TILE2;
            for (int e = tid; e < TILE2; e += blockDim.x) {
                const int r = e >> 5, c = e & 31;
                bwdS[bo + (int64_t)t * TILE2 + swz_index<TS>(r, c)] = to_stream<TS>(src[r * TILE + c]);
            }
        }
    }
}

// ---------------------------------------------------------------------------------
// Batched triangular solves  out = S L^{-T} L^{-1} S in  for a list of jobs
// (item, input offset, output offset); S = diag(sc) is the symmetric scaling (or 1).
//
// One CTA per job walks the tile rows in order (forward stream, then backward stream).
// The item's tiles are consumed strictly in storage order, so a producer warp streams
// them through an R-slot shared-memory ring by bulk async copies (one 32x32 tile per
// copy, completion on full[slot]) and reloads a slot as soon as the consumer warp that
// read its tile releases it (empty[slot]).  NW consumer warps form, per tile row I, the
// partial sums sum_J T_IJ v_J (lane = tile row, 128-bit shared loads of the swizzled row
// and of v_J), meet at one named barrier, and warp 0 applies the stored inverse diagonal
// tile.  Measured on B300 (clock64 probes): with every warp issuing its own refills and
// every warp repeating the diagonal product, a step took ~2300-3600 cycles, a quarter
// of it in the refill path.  This single-row form serves FP64 factors (FP64-pipe bound);
// FP32 arithmetic uses the pair-stepped k_chain_solve_pairs below.
// ---------------------------------------------------------------------------------
template <typename TS, typename TA>
__device__ __forceinline__ TA row_dot(const TS* tile, int lane, const TA* v);

// FP64 tiles: 16 chunks of 2 doubles per row
template <>
__device__ __forceinline__ double row_dot<double, double>(const double* tile, int lane, const double* v) {
    const double2* row = reinterpret_cast<const double2*>(tile + lane * TILE);
    const double2* vv = reinterpret_cast<const double2*>(v);
    double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    const int sw = lane & 7;
#pragma unroll
    for (int j = 0; j < 16; j += 2) {
        const double2 t0 = row[j ^ sw], t1 = row[(j + 1) ^ sw];
        const double2 x0 = vv[j], x1 = vv[j + 1];
        a0 = fma(t0.x, x0.x, a0);
        a1 = fma(t0.y, x0.y, a1);
        a2 = fma(t1.x, x1.x, a2);
        a3 = fma(t1.y, x1.y, a3);
    }
    return (a0 + a1) + (a2 + a3);
}

// FP32 tiles: 8 chunks of 4 floats per row
template <>
__device__ __forceinline__ float row_dot<float, float>(const float* tile, int lane, const float* v) {
    const float4* row = reinterpret_cast<const float4*>(tile + lane * TILE);
    const float4* vv = reinterpret_cast<const float4*>(v);
    float a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    const int sw = lane & 7;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float4 t = row[j ^ sw];
        const float4 x = vv[j];
        a0 = fmaf(t.x, x.x, a0);
        a1 = fmaf(t.y, x.y, a1);
        a2 = fmaf(t.z, x.z, a2);
        a3 = fmaf(t.w, x.w, a3);
    }
    return (a0 + a1) + (a2 + a3);
}

// BF16 tiles: 4 chunks of 8 bf16 per row, FP32 accumulation
template <>
__device__ __forceinline__ float row_dot<__nv_bfloat16, float>(const __nv_bfloat16* tile, int lane, const float* v) {
    const uint4* row = reinterpret_cast<const uint4*>(tile + lane * TILE);
    const float4* vv = reinterpret_cast<const float4*>(v);
    float a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    const int sw = (lane >> 1) & 3;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint4 t = row[j ^ sw];
        const float4 x0 = vv[2 * j], x1 = vv[2 * j + 1];
        const float2 p0 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&t.x));
        const float2 p1 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&t.y));
        const float2 p2 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&t.z));
        const float2 p3 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&t.w));
        a0 = fmaf(p0.x, x0.x, a0);
        a1 = fmaf(p0.y, x0.y, a1);
        a2 = fmaf(p1.x, x0.z, a2);
        a3 = fmaf(p1.y, x0.w, a3);
        a0 = fmaf(p2.x, x1.x, a0);
        a1 = fmaf(p2.y, x1.y, a1);
        a2 = fmaf(p3.x, x1.z, a2);
        a3 = fmaf(p3.y, x1.w, a3);
    }
    return (a0 + a1) + (a2 + a3);
}

__device__ __forceinline__ void named_barrier(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Row `lane` of two tiles times one vector, sharing the vector's shared-memory loads;
// each result is accumulated exactly as row_dot does (bitwise the same values).
template <typename TS, typename TA>
__device__ __forceinline__ void row_dot2(const TS* A, const TS* B, int lane, const TA* v, TA& oa, TA& ob);

template <>
__device__ __forceinline__ void row_dot2<float, float>(const float* A, const float* B, int lane, const float* v,
                                                       float& oa, float& ob) {
    const float4* ra = reinterpret_cast<const float4*>(A + lane * TILE);
    const float4* rb = reinterpret_cast<const float4*>(B + lane * TILE);
    const float4* vv = reinterpret_cast<const float4*>(v);
    float a0 = 0, a1 = 0, a2 = 0, a3 = 0, b0 = 0, b1 = 0, b2 = 0, b3 = 0;
    const int sw = lane & 7;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float4 x = vv[j];
        const float4 ta = ra[j ^ sw], tb = rb[j ^ sw];
        a0 = fmaf(ta.x, x.x, a0);
        a1 = fmaf(ta.y, x.y, a1);
        a2 = fmaf(ta.z, x.z, a2);
        a3 = fmaf(ta.w, x.w, a3);
        b0 = fmaf(tb.x, x.x, b0);
        b1 = fmaf(tb.y, x.y, b1);
        b2 = fmaf(tb.z, x.z, b2);
        b3 = fmaf(tb.w, x.w, b3);
    }
    oa = (a0 + a1) + (a2 + a3);
    ob = (b0 + b1) + (b2 + b3);
}

template <>
__device__ __forceinline__ void row_dot2<__nv_bfloat16, float>(const __nv_bfloat16* A, const __nv_bfloat16* B,
                                                               int lane, const float* v, float& oa, float& ob) {
    const uint4* ra = reinterpret_cast<const uint4*>(A + lane * TILE);
    const uint4* rb = reinterpret_cast<const uint4*>(B + lane * TILE);
    const float4* vv = reinterpret_cast<const float4*>(v);
    float a0 = 0, a1 = 0, a2 = 0, a3 = 0, b0 = 0, b1 = 0, b2 = 0, b3 = 0;
    const int sw = (lane >> 1) & 3;
    auto f2 = [](uint32_t w) { return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w)); };
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float4 x0 = vv[2 * j], x1 = vv[2 * j + 1];
        const uint4 ta = ra[j ^ sw], tb = rb[j ^ sw];
        const float2 p0 = f2(ta.x), p1 = f2(ta.y), p2 = f2(ta.z), p3 = f2(ta.w);
        const float2 q0 = f2(tb.x), q1 = f2(tb.y), q2 = f2(tb.z), q3 = f2(tb.w);
        a0 = fmaf(p0.x, x0.x, a0);
        a1 = fmaf(p0.y, x0.y, a1);
        a2 = fmaf(p1.x, x0.z, a2);
        a3 = fmaf(p1.y, x0.w, a3);
        a0 = fmaf(p2.x, x1.x, a0);
        a1 = fmaf(p2.y, x1.y, a1);
        a2 = fmaf(p3.x, x1.z, a2);
        a3 = fmaf(p3.y, x1.w, a3);
        b0 = fmaf(q0.x, x0.x, b0);
        b1 = fmaf(q0.y, x0.y, b1);
        b2 = fmaf(q1.x, x0.z, b2);
        b3 = fmaf(q1.y, x0.w, b3);
        b0 = fmaf(q2.x, x1.x, b0);
        b1 = fmaf(q2.y, x1.y, b1);
        b2 = fmaf(q3.x, x1.z, b2);
        b3 = fmaf(q3.y, x1.w, b3);
    }
    oa = (a0 + a1) + (a2 + a3);
    ob = (b0 + b1) + (b2 + b3);
}

template <typename TS, typename TA, int G, int RG, int CR, int NW>
__global__ void __launch_bounds__((NW + 2) * 32) k_chain_solve(SolveArgs a) {
    // Two rings.  The critical ring holds, per step (tile row), the two tiles on the
    // chain's critical path -- the off-diagonal tile next to the diagonal and the inverse
    // diagonal tile -- CR steps ahead; the main ring holds the remaining ("far")
    // off-diagonal tiles, R = RG * G slots filled by bulk copies of G far tiles.
    constexpr int R = RG * G;
    // 8-byte words of barriers, flags and slot tags, padded so that what follows stays
    // 16-byte aligned (128-bit shared loads)
    constexpr int HDR = 3 * RG + 2 * CR + 3, HDRP = HDR + (HDR & 1);
    // batched solves put the column in blockIdx.x, so the CTAs of one subdomain's columns
    // run side by side and share its factor stream through L2
    const int col = a.col_fast ? blockIdx.x : 0;
    const int job = a.col_fast ? blockIdx.y : blockIdx.x;
    if (a.done && a.done[col * a.done_stride]) return;
    const int s = a.job_sub[job];
    const Profile pf = a.pf;
    const int n = pf.rows[s], T = pf.ntiles[s];
    const int64_t r0 = pf.row0[s];
    const int64_t nts = pf.fwd[r0 + T - 1] + (T - 1 - pf.lo[r0 + T - 1]) + 1;   // tiles per stream
    // Optional start row t0 (identity right-hand side e_j, j in tile row t0): rows above
    // t0 stay zero in the forward sweep, and only rows >= t0 of the result are wanted, so
    // the forward sweep starts and the backward sweep stops at t0.  The consumed tiles are
    // then stream positions [q0, qend), still contiguous.
    const int t0 = a.job_t0 ? a.job_t0[job] : 0;
    const int64_t q0 = pf.fwd[r0 + t0];
    const int nsteps = 2 * (T - t0);
    const TS* F = (const TS*)a.fwdS + pf.base[s] * TILE2;
    const TS* Bk = (const TS*)a.bwdS + pf.base[s] * TILE2;
    const double* sc = a.scale ? a.scale + a.scale_off[s] : nullptr;
    const float* sc32 = a.scale32 ? a.scale32 + a.scale_off[s] : nullptr;
    const double* in = a.in + a.job_in[job] + col * a.ldin;
    double* out = a.out + a.job_out[job] + col * a.ldout;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    constexpr int NT = (NW + 2) * 32;
    constexpr uint32_t TB = TILE2 * sizeof(TS);

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TS* ring = reinterpret_cast<TS*>(smem_raw);
    TS* cring = ring + (int64_t)R * TILE2;                                   // [CR][2 tiles]
    uint64_t* full = reinterpret_cast<uint64_t*>(cring + (int64_t)2 * CR * TILE2);   // [RG]
    uint64_t* empty = full + RG;                                             // [RG]
    uint64_t* cfull = empty + RG;                                            // [CR]
    uint64_t* cempty = cfull + CR;                                           // [CR]
    volatile int* abort_flag = reinterpret_cast<volatile int*>(cempty + CR);
    int64_t* issued = reinterpret_cast<int64_t*>(cempty + CR + 1);   // [0] far groups, [1] steps
    // index of the far group last issued into each group slot: tiles are released out of
    // order (by different warps), and a parity wait alone cannot tell "use u + 1 landed"
    // from "use u not landed yet", so a consumer first waits for its own group here
    volatile int64_t* slot_g = reinterpret_cast<volatile int64_t*>(cempty + CR + 3);   // [RG]
    TA* part = reinterpret_cast<TA*>(full + HDRP);            // [2][NW][32]
    TA* tbuf = part + 2 * NW * TILE;                          // [32] (warp 0)
    int32_t* lo_s = reinterpret_cast<int32_t*>(tbuf + TILE);
    int32_t* hi_s = lo_s + T;
    TA* v = reinterpret_cast<TA*>(hi_s + T + ((2 * T) & 3));   // 16-byte aligned
    auto src = [&](int64_t q) -> const TS* { return q < nts ? F + q * TILE2 : Bk + (q - nts) * TILE2; };
    // step k: tile row, number of off-diagonal tiles, first stream position
    auto row_of = [&](int k) { return k < T - t0 ? t0 + k : T - 1 - (k - (T - t0)); };
    auto nt_of = [&](int k) {
        const int I = row_of(k);
        return k < T - t0 ? I - lo_s[I] : hi_s[I] - I;
    };
    if (tid == 0) {
        for (int i = 0; i < RG; ++i) {
            mbar_init(smem_u32(&full[i]), 1);
            mbar_init(smem_u32(&empty[i]), G);   // one release per tile of the group
            slot_g[i] = -1;
        }
        for (int i = 0; i < CR; ++i) {
            mbar_init(smem_u32(&cfull[i]), 1);
            mbar_init(smem_u32(&cempty[i]), 1);  // warp 0 releases the pair once
        }
        *abort_flag = 0;
        issued[0] = 0;
        issued[1] = 0;
        fence_async_smem();
    }
    for (int i = tid; i < T; i += NT) {
        lo_s[i] = pf.lo[r0 + i];
        hi_s[i] = pf.hi[r0 + i];
    }
    // scaling in the solve's arithmetic: FP32 solves scale in FP32 (B300's FP64 pipe is
    // ~1/64 of FP32, so FP64 work per row is kept off the chain's prologue/epilogue)
    if constexpr (sizeof(TA) == 4) {
        for (int i = tid; i < T * TILE; i += NT) v[i] = i < n ? (float)in[i] * (sc32 ? sc32[i] : 1.0f) : 0.0f;
    } else {
        for (int i = tid; i < T * TILE; i += NT) v[i] = i < n ? in[i] * (sc ? sc[i] : 1.0) : 0.0;
    }
    __syncthreads();

    if (w == NW + 1) {
        // Critical producer: per step, the nearest off-diagonal tile and the diagonal tile
        // into slot k % CR once warp 0 has released step k - CR.
        if (lane == 0) {
            int64_t q = q0;
            int k = 0;
            for (; k < nsteps; ++k) {
                const int nt = nt_of(k);
                const int cs = k % CR, u = k / CR;
                if (u > 0 && (*abort_flag || !mbar_poll(smem_u32(&cempty[cs]), (uint32_t)((u - 1) & 1)))) {
                    *abort_flag = 1;
                    break;
                }
                const uint32_t bar = smem_u32(&cfull[cs]);
                TS* dst = cring + (int64_t)(2 * cs) * TILE2;
                mbar_expect_tx(bar, (uint32_t)(nt > 0 ? 2 : 1) * TB);
                if (nt == 0) {
                    bulk_copy(smem_u32(dst + TILE2), src(q), TB, bar);
                } else if (k < T - t0) {   // forward: nearest and diagonal are adjacent
                    bulk_copy(smem_u32(dst), src(q + nt - 1), 2 * TB, bar);
                } else {                   // backward: nearest first in the row
                    bulk_copy(smem_u32(dst), src(q), TB, bar);
                    bulk_copy(smem_u32(dst + TILE2), src(q + nt), TB, bar);
                }
                q += nt + 1;
            }
            issued[1] = k;
        }
    } else if (w == NW) {
        // Far producer: the far tiles of the steps in order, G per group (a group may span
        // several rows: one copy per contiguous run); a group slot is reloaded once every
        // tile of its previous group has been released.
        if (lane == 0) {
            int k = 0, off = 0;
            int64_t q = q0;
            int nt = nsteps > 0 ? nt_of(0) : 0;
            int64_t gi = 0;
            auto nf_of = [&](int nt_) { return nt_ > 1 ? nt_ - 1 : 0; };
            while (true) {
                while (k < nsteps && off >= nf_of(nt)) {   // next step with far tiles left
                    q += nt + 1;
                    ++k;
                    off = 0;
                    if (k < nsteps) nt = nt_of(k);
                }
                if (k >= nsteps) break;
                const int gs = (int)(gi % RG);
                const int64_t u = gi / RG;
                if (u > 0 && (*abort_flag || !mbar_poll(smem_u32(&empty[gs]), (uint32_t)((u - 1) & 1)))) {
                    *abort_flag = 1;
                    break;
                }
                // gather the group: up to G far tiles, as contiguous runs
                int64_t seg_p[G];
                int seg_n[G];
                int nseg = 0, cnt = 0;
                int k2 = k, off2 = off, nt2 = nt;
                int64_t q2 = q;
                while (cnt < G && k2 < nsteps) {
                    const int nf2 = nf_of(nt2);
                    if (off2 < nf2) {
                        const int m = min(G - cnt, nf2 - off2);
                        // far tiles of a forward row: t = 0 .. nt-2; backward: t = 1 .. nt-1
                        const int64_t p = q2 + (k2 < T - t0 ? 0 : 1) + off2;
                        seg_p[nseg] = p;
                        seg_n[nseg] = m;
                        ++nseg;
                        cnt += m;
                        off2 += m;
                    }
                    if (off2 >= nf2) {
                        q2 += nt2 + 1;
                        ++k2;
                        off2 = 0;
                        if (k2 < nsteps) nt2 = nt_of(k2);
                    }
                }
                k = k2;
                off = off2;
                nt = nt2;
                q = q2;
                slot_g[gs] = gi;
                const uint32_t bar = smem_u32(&full[gs]);
                mbar_expect_tx(bar, (uint32_t)cnt * TB);
                TS* dst = ring + (int64_t)(gs * G) * TILE2;
                for (int e = 0; e < nseg; ++e) {
                    bulk_copy(smem_u32(dst), src(seg_p[e]), (uint32_t)seg_n[e] * TB, bar);
                    dst += (int64_t)seg_n[e] * TILE2;
                }
                ++gi;
            }
            issued[0] = gi;
        }
    } else {
        // Consumer warps.  Step for tile row I: warp 0 takes the off-diagonal tile nearest
        // the diagonal (it needs the row solved in the previous step, which warp 0 itself
        // produced), warps 1..NW-1 share the far tiles (they need only rows solved at least
        // two steps back, ordered by the previous step's barrier), one named barrier, then
        // warp 0 alone reduces the partial sums and applies the stored inverse diagonal
        // tile.  Every tile is read by exactly one warp, which releases it at once.
        auto wait_far = [&](int64_t f) -> const TS* {
            const int64_t gi = f / G;
            const int gs = (int)(gi % RG);
            if (!__any_sync(0xffffffffu, *abort_flag != 0)) {
                bool r = false;
                for (long long i = 0; i < kWaitLimit; ++i)
                    if (slot_g[gs] == gi) {
                        r = true;
                        break;
                    }
                r = r && mbar_poll(smem_u32(&full[gs]), (uint32_t)((gi / RG) & 1));
                r = __all_sync(0xffffffffu, r);
                if (!r && lane == 0) *abort_flag = 1;
            }
            return ring + (f % R) * TILE2;
        };
        auto release_far = [&](int64_t f) {
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&empty[(f / G) % RG]));
        };
        auto wait_crit = [&](int k) -> const TS* {
            const int cs = k % CR;
            if (!__any_sync(0xffffffffu, *abort_flag != 0)) {
                const bool r = __all_sync(0xffffffffu, mbar_poll(smem_u32(&cfull[cs]), (uint32_t)((k / CR) & 1)));
                if (!r && lane == 0) *abort_flag = 1;
            }
            return cring + (int64_t)(2 * cs) * TILE2;
        };
        int64_t fb = 0;   // far-tile index of the step's first far tile
        int par = 0;
        for (int k = 0; k < nsteps; ++k) {
            const bool fwd = k < T - t0;
            const int I = row_of(k);
            const int j0 = fwd ? lo_s[I] : I + 1;
            const int nt = fwd ? I - lo_s[I] : hi_s[I] - I;
            const int nf = nt > 1 ? nt - 1 : 0;
            TA acc = 0;
            const TS* cp = nullptr;
            if (w == 0) {
                cp = wait_crit(k);
                if (nt > 0) acc = row_dot<TS, TA>(cp, lane, v + (fwd ? I - 1 : I + 1) * TILE);
            } else {
                for (int e = w - 1; e < nf; e += NW - 1) {
                    const TS* tl = wait_far(fb + e);
                    acc += row_dot<TS, TA>(tl, lane, v + (j0 + (fwd ? e : e + 1)) * TILE);
                    release_far(fb + e);
                }
            }
            part[(par * NW + w) * TILE + lane] = acc;
            named_barrier(1, NW * 32);
            if (w == 0) {
                TA* vi = v + I * TILE;
                TA sum = 0;
#pragma unroll
                for (int u = 0; u < NW; ++u) sum += part[(par * NW + u) * TILE + lane];
                // y = D t: t goes through shared memory so that row `lane` of D and t
                // are both read with 128-bit loads (row_dot)
                tbuf[lane] = vi[lane] - sum;
                __syncwarp();
                const TA y = row_dot<TS, TA>(cp + TILE2, lane, tbuf);
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&cempty[k % CR]));
                vi[lane] = y;
                __syncwarp();
            }
            fb += nf;
            par ^= 1;
        }
    }
    __syncthreads();
    if (*abort_flag) {
        if (tid == 0) {
            atomicExch(a.err, 1);
            // only the last use of a slot can still be in flight (a reload waits for the
            // release of the previous use, which follows its arrival): drain those
            for (int sl = 0; sl < RG; ++sl)
                if (issued[0] > sl) mbar_wait(smem_u32(&full[sl]), (uint32_t)(((issued[0] - 1 - sl) / RG) & 1));
            for (int sl = 0; sl < CR; ++sl)
                if (issued[1] > sl) mbar_wait(smem_u32(&cfull[sl]), (uint32_t)(((issued[1] - 1 - sl) / CR) & 1));
        }
        __syncthreads();
        return;
    }
    if constexpr (sizeof(TA) == 4) {
        if (a.accumulate)
            for (int i = tid; i < n; i += NT) out[i] += (double)(v[i] * (sc32 ? sc32[i] : 1.0f));
        else
            for (int i = tid; i < n; i += NT) out[i] = (double)(v[i] * (sc32 ? sc32[i] : 1.0f));
    } else {
        if (a.accumulate)
            for (int i = tid; i < n; i += NT) out[i] += v[i] * (sc ? sc[i] : 1.0);
        else
            for (int i = tid; i < n; i += NT) out[i] = v[i] * (sc ? sc[i] : 1.0);
    }
}

// ---------------------------------------------------------------------------------
// Pair-stepped chain for FP32 arithmetic (FP32 / BF16 streams from k_finalize): one step
// solves the two tile rows of a pair, halving the number of dependent steps of a chain.
//
// A step's tiles, by role:
//   near  tiles of the pair's rows that multiply the previous step's pair (forward
//         J = a-2, a-1; backward J = a+2, a+3): on the critical path;
//   far   tiles that multiply pairs solved two or more steps earlier;
//   diag  D of both rows and the coupling tile C (C^T backward).
// Within a step the first row f (forward a, backward b) is solved before the second s:
//   x_f = D_f t_f,  x_s = D_s t_s + K t_f   (K = C forward, C^T backward).
// Stream positions of a step follow from lo/hi of its rows and the stream position q of
// its first tile; pair_step() is the single definition used by both producers and the
// consumers.
// ---------------------------------------------------------------------------------
struct PairStep {
    int f, s;               // rows solved first / second (s < 0: a single row, T odd)
    int nfn, nsn;           // near tiles of f / s
    int hasC;               // coupling tile present (b's profile reaches a)
    int ff, fs;             // far tiles of f / s
    int Jnear0;             // J of near slot 0 (both rows)
    int Jf0, Js0;           // J of the first far tile of f / s
    int64_t q_ff, q_sf;     // stream positions of the far runs
    int64_t q_fc, q_sc;     // critical runs: forward f [near, D], s [near, C, D];
                            //                backward f [near], s [C^T, near]
    int64_t q_fd, q_sd;     // backward: D_f, D_s
    int64_t q_next;         // first position of the next step
};

__device__ __forceinline__ PairStep pair_step(int k, int NP, int T, const int32_t* lo, const int32_t* hi,
                                              int64_t q) {
    PairStep p;
    const bool fwd = k < NP;
    const int P = fwd ? k : 2 * NP - 1 - k;
    const int a = 2 * P, b = a + 1;
    const bool hb = b < T;
    if (fwd) {
        const int la = lo[a];
        p.f = a;
        p.nfn = a - max(la, a - 2);
        p.ff = max(0, a - 2 - la);
        p.q_ff = q;
        p.q_fc = q + p.ff;
        p.Jnear0 = a - 2;
        p.Jf0 = la;
        int64_t qn = q + (a - la + 1);
        if (hb) {
            const int lb = lo[b];
            p.s = b;
            p.hasC = lb <= a;
            p.nsn = p.hasC ? a - max(lb, a - 2) : 0;
            p.fs = max(0, a - 2 - lb);
            p.q_sf = qn;
            p.q_sc = qn + p.fs;
            p.Js0 = lb;
            qn += b - lb + 1;
        } else {
            p.s = -1;
            p.hasC = 0;
            p.nsn = 0;
            p.fs = 0;
            p.q_sf = p.q_sc = qn;
            p.Js0 = 0;
        }
        p.q_fd = p.q_sd = 0;
        p.q_next = qn;
    } else {
        p.Jnear0 = a + 2;
        p.Jf0 = p.Js0 = a + 4;
        int64_t qn = q;
        if (hb) {
            const int hbv = hi[b], ha = hi[a];
            p.f = b;
            p.s = a;
            p.nfn = min(hbv - b, 2);
            p.ff = max(0, hbv - b - 2);
            p.q_fc = qn;
            p.q_ff = qn + p.nfn;
            p.q_fd = p.q_ff + p.ff;
            qn += hbv - b + 1;
            p.hasC = ha >= b;
            p.nsn = max(0, min(ha, a + 3) - (a + 1));
            p.fs = max(0, ha - a - 3);
            p.q_sc = qn;
            p.q_sf = qn + p.hasC + p.nsn;
            p.q_sd = p.q_sf + p.fs;
            qn += ha - a + 1;
        } else {   // a = T - 1: nothing right of its diagonal tile
            p.f = a;
            p.s = -1;
            p.nfn = p.ff = 0;
            p.q_fc = p.q_ff = p.q_fd = qn;
            qn += 1;
            p.hasC = p.nsn = p.fs = 0;
            p.q_sc = p.q_sf = p.q_sd = qn;
        }
        p.q_next = qn;
    }
    return p;
}

template <typename TS, typename TA, int G, int RG, int CR, int NW>
// BF16 with 4 consumer warps, or with a 3-group far ring: 3 CTAs per SM (their shared
// memory fits 3 as well).  FP32 tiles fill shared memory at 2 CTAs per SM.
__global__ void __launch_bounds__((NW + 2) * 32, (sizeof(TS) == 2 && (NW == 4 || RG <= 3)) ? 3 : 2)
    k_chain_solve_pairs(SolveArgs a) {
    // Critical slot of a step (7 tiles): forward [nf0 nf1 D_f | ns0 ns1 C D_s], backward
    // [nf0 nf1 D_f | C^T ns0 ns1 D_s]; near slot i multiplies row Jnear0 + i.
    constexpr int R = RG * G, CT = 7;
    static_assert(CR >= 2, "a critical slot is refilled while the next one is in use");
    static_assert(NW >= 3, "warps 0 and 1 take the critical path, the others the far tiles");
    constexpr int HDR = 3 * RG + 2 * CR + 3, HDRP = HDR + (HDR & 1);
    const int col = a.col_fast ? blockIdx.x : 0;
    const int job = a.col_fast ? blockIdx.y : blockIdx.x;
    if (a.done && a.done[col * a.done_stride]) return;
    const int s = a.job_sub[job];
    const Profile pf = a.pf;
    const int n = pf.rows[s], T = pf.ntiles[s];
    const int64_t r0 = pf.row0[s];
    const int64_t nts = pf.fwd[r0 + T - 1] + (T - 1 - pf.lo[r0 + T - 1]) + 1;   // tiles per stream
    const int NP = (T + 1) / 2, nsteps = 2 * NP;
    const TS* F = (const TS*)a.fwdS + pf.base[s] * TILE2;
    const TS* Bk = (const TS*)a.bwdS + pf.base[s] * TILE2;
    const float* sc32 = a.scale32 ? a.scale32 + a.scale_off[s] : nullptr;
    const double* in = a.in + a.job_in[job] + col * a.ldin;
    double* out = a.out + a.job_out[job] + col * a.ldout;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    constexpr int NT = (NW + 2) * 32;
    constexpr uint32_t TB = TILE2 * sizeof(TS);

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TS* ring = reinterpret_cast<TS*>(smem_raw);
    TS* cring = ring + (int64_t)R * TILE2;                                   // [CR][CT tiles]
    uint64_t* full = reinterpret_cast<uint64_t*>(cring + (int64_t)CT * CR * TILE2);   // [RG]
    uint64_t* empty = full + RG;                                             // [RG]
    uint64_t* cfull = empty + RG;                                            // [CR]
    uint64_t* cempty = cfull + CR;                                           // [CR]
    volatile int* abort_flag = reinterpret_cast<volatile int*>(cempty + CR);
    int64_t* issued = reinterpret_cast<int64_t*>(cempty + CR + 1);   // [0] far groups, [1] steps
    volatile int64_t* slot_g = reinterpret_cast<volatile int64_t*>(cempty + CR + 3);   // [RG]
    TA* part = reinterpret_cast<TA*>(full + HDRP);            // [2][NW][2 rows][32]
    TA* tbuf = part + 4 * NW * TILE;                          // [3][32]: t_f (warp 0), t_s (warp 1), u
    uint4* stab = reinterpret_cast<uint4*>(tbuf + 3 * TILE + TILE);   // [nsteps] packed step counts
    int32_t* lo_s = reinterpret_cast<int32_t*>(stab + nsteps);
    int32_t* hi_s = lo_s + T;
    TA* v = reinterpret_cast<TA*>(hi_s + T + ((2 * T) & 3));   // 16-byte aligned
    auto src = [&](int64_t q) -> const TS* { return q < nts ? F + q * TILE2 : Bk + (q - nts) * TILE2; };
    if (tid == 0) {
        for (int i = 0; i < RG; ++i) {
            mbar_init(smem_u32(&full[i]), 1);
            mbar_init(smem_u32(&empty[i]), G);   // one release per tile of the group
            slot_g[i] = -1;
        }
        for (int i = 0; i < CR; ++i) {
            mbar_init(smem_u32(&cfull[i]), 1);
            mbar_init(smem_u32(&cempty[i]), 2);  // warps 0 and 1 release the slot
        }
        *abort_flag = 0;
        issued[0] = 0;
        issued[1] = 0;
        fence_async_smem();
    }
    for (int i = tid; i < T; i += NT) {
        lo_s[i] = pf.lo[r0 + i];
        hi_s[i] = pf.hi[r0 + i];
    }
    for (int i = tid; i < T * TILE; i += NT) v[i] = i < n ? (float)in[i] * (sc32 ? sc32[i] : 1.0f) : 0.0f;
    __syncthreads();
    // the consumers' per-step counts, packed (positions are the producers' business)
    for (int k = tid; k < nsteps; k += NT) {
        const PairStep p = pair_step(k, NP, T, lo_s, hi_s, 0);
        stab[k] = make_uint4((uint32_t)p.f | ((uint32_t)(p.s + 1) << 16),
                             (uint32_t)p.nfn | ((uint32_t)p.nsn << 2) | ((uint32_t)p.hasC << 4) |
                                 ((uint32_t)p.ff << 8) | ((uint32_t)p.fs << 20),
                             (uint32_t)(p.Jnear0 + 2) | ((uint32_t)p.Jf0 << 16), (uint32_t)p.Js0);
    }
    __syncthreads();

    if (w == NW + 1) {
        // Critical producer: a step's near, diagonal and coupling tiles into slot k % CR
        // once warp 0 has released step k - CR.
        if (lane == 0) {
            int64_t q = 0;
            int k = 0;
            for (; k < nsteps; ++k) {
                const PairStep p = pair_step(k, NP, T, lo_s, hi_s, q);
                const int cs = k % CR, u = k / CR;
                if (u > 0 && (*abort_flag || !mbar_poll(smem_u32(&cempty[cs]), (uint32_t)((u - 1) & 1)))) {
                    *abort_flag = 1;
                    break;
                }
                const uint32_t bar = smem_u32(&cfull[cs]);
                TS* dst = cring + (int64_t)(CT * cs) * TILE2;
                const int ntl = p.nfn + 1 + (p.s >= 0 ? p.nsn + p.hasC + 1 : 0);
                mbar_expect_tx(bar, (uint32_t)ntl * TB);
                if (k < NP) {
                    bulk_copy(smem_u32(dst + (int64_t)(2 - p.nfn) * TILE2), src(p.q_fc), (uint32_t)(p.nfn + 1) * TB, bar);
                    if (p.s >= 0) {
                        const int c = p.nsn + p.hasC + 1;
                        bulk_copy(smem_u32(dst + (int64_t)(7 - c) * TILE2), src(p.q_sc), (uint32_t)c * TB, bar);
                    }
                } else {
                    if (p.nfn > 0) bulk_copy(smem_u32(dst), src(p.q_fc), (uint32_t)p.nfn * TB, bar);
                    bulk_copy(smem_u32(dst + 2 * TILE2), src(p.q_fd), TB, bar);
                    if (p.s >= 0) {
                        const int c = p.hasC + p.nsn;
                        if (c > 0) bulk_copy(smem_u32(dst + 3 * TILE2), src(p.q_sc), (uint32_t)c * TB, bar);
                        bulk_copy(smem_u32(dst + 6 * TILE2), src(p.q_sd), TB, bar);
                    }
                }
                q = p.q_next;
            }
            issued[1] = k;
        }
    } else if (w == NW) {
        // Far producer: the far runs of the steps in order (f's run, then s's), G tiles
        // per group (one copy per contiguous piece); a group slot is reloaded once every
        // tile of its previous group has been released.
        if (lane == 0) {
            int k = 0, rs = 0, off = 0;
            int64_t q = 0;
            PairStep p = pair_step(0, NP, T, lo_s, hi_s, 0);
            auto advance = [&]() {
                off = 0;
                if (rs == 0) {
                    rs = 1;
                } else {
                    rs = 0;
                    q = p.q_next;
                    if (++k < nsteps) p = pair_step(k, NP, T, lo_s, hi_s, q);
                }
            };
            int64_t gi = 0;
            while (true) {
                while (k < nsteps && off >= (rs ? p.fs : p.ff)) advance();
                if (k >= nsteps) break;
                const int gs = (int)(gi % RG);
                const int64_t u = gi / RG;
                if (u > 0 && (*abort_flag || !mbar_poll(smem_u32(&empty[gs]), (uint32_t)((u - 1) & 1)))) {
                    *abort_flag = 1;
                    break;
                }
                int64_t seg_p[G];
                int seg_n[G];
                int nseg = 0, cnt = 0;
                while (cnt < G && k < nsteps) {
                    const int rc = rs ? p.fs : p.ff;
                    if (off < rc) {
                        const int m = min(G - cnt, rc - off);
                        seg_p[nseg] = (rs ? p.q_sf : p.q_ff) + off;
                        seg_n[nseg] = m;
                        ++nseg;
                        cnt += m;
                        off += m;
                    }
                    if (off >= rc) advance();
                }
                slot_g[gs] = gi;
                const uint32_t bar = smem_u32(&full[gs]);
                mbar_expect_tx(bar, (uint32_t)cnt * TB);
                TS* dst = ring + (int64_t)(gs * G) * TILE2;
                for (int e = 0; e < nseg; ++e) {
                    bulk_copy(smem_u32(dst), src(seg_p[e]), (uint32_t)seg_n[e] * TB, bar);
                    dst += (int64_t)seg_n[e] * TILE2;
                }
                ++gi;
            }
            issued[0] = gi;
        }
    } else {
        // Consumer warps.  Warps 0 and 1 take a step's critical path: warp i applies near
        // slot i of both rows (one vector, two tiles), so both need the pair solved in the
        // previous step, exchanged at named barrier 2.  After the step's named barrier 1,
        // warp 0 forms t_f and, in one pass over t_f, x_f = D_f t_f and u = K t_f; warp 1
        // forms t_s and D_s t_s, and after named barrier 3 (u ready) x_s = D_s t_s + u.
        // Warps 2..NW-1 take the far tiles, dealt round-robin, each read by one warp and
        // released at once.
        auto wait_far = [&](int64_t f) -> const TS* {
            const int64_t gi = f / G;
            const int gs = (int)(gi % RG);
            if (!__any_sync(0xffffffffu, *abort_flag != 0)) {
                bool r = false;
                for (long long i = 0; i < kWaitLimit; ++i)
                    if (slot_g[gs] == gi) {
                        r = true;
                        break;
                    }
                r = r && mbar_poll(smem_u32(&full[gs]), (uint32_t)((gi / RG) & 1));
                r = __all_sync(0xffffffffu, r);
                if (!r && lane == 0) *abort_flag = 1;
            }
            return ring + (f % R) * TILE2;
        };
        auto release_far = [&](int64_t f) {
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&empty[(f / G) % RG]));
        };
        auto wait_crit = [&](int k) -> const TS* {
            const int cs = k % CR;
            const uint32_t bar = smem_u32(&cfull[cs]), par = (uint32_t)((k / CR) & 1);
            if (!__all_sync(0xffffffffu, mbar_test_wait(bar, par)) && !__any_sync(0xffffffffu, *abort_flag != 0)) {
                const bool r = __all_sync(0xffffffffu, mbar_poll(bar, par));
                if (!r && lane == 0) *abort_flag = 1;
            }
            return cring + (int64_t)(CT * cs) * TILE2;
        };
        int64_t fb = 0;   // far-tile index of the step's first far tile
        int par = 0;
        for (int k = 0; k < nsteps; ++k) {
            const bool fwd = k < NP;
            const uint4 st = stab[k];
            const int f = (int)(st.x & 0xffffu), sr = (int)(st.x >> 16) - 1;
            const int nfn = (int)(st.y & 3u), nsn = (int)((st.y >> 2) & 3u), hasC = (int)((st.y >> 4) & 1u);
            const int ff = (int)((st.y >> 8) & 0xfffu), fs = (int)(st.y >> 20);
            const int Jn0 = (int)(st.z & 0xffffu) - 2, Jf0 = (int)(st.z >> 16), Js0 = (int)st.w;
            TA acc_f = 0, acc_s = 0;
            const TS* cp = nullptr;
            if (w < 2) {
                cp = wait_crit(k);
                const int i = w;                              // near slot of this warp
                const bool okf = fwd ? i >= 2 - nfn : i < nfn;
                const bool oks = fwd ? i >= 2 - nsn : i < nsn;
                const TS* tf = cp + (int64_t)i * TILE2;
                const TS* ts = cp + (int64_t)((fwd ? 3 : 4) + i) * TILE2;
                if (okf || oks) {
                    const TA* xv = v + (Jn0 + i) * TILE;
                    if (okf && oks) row_dot2<TS, TA>(tf, ts, lane, xv, acc_f, acc_s);
                    else if (okf) acc_f = row_dot<TS, TA>(tf, lane, xv);
                    else acc_s = row_dot<TS, TA>(ts, lane, xv);
                }
            } else {
                const int nfar = ff + fs;
                for (int e = w - 2; e < nfar; e += NW - 2) {
                    const TS* tl = wait_far(fb + e);
                    if (e < ff) acc_f += row_dot<TS, TA>(tl, lane, v + (Jf0 + e) * TILE);
                    else acc_s += row_dot<TS, TA>(tl, lane, v + (Js0 + e - ff) * TILE);
                    release_far(fb + e);
                }
            }
            TA* pw = part + (int64_t)((par * NW + w) * 2) * TILE;
            pw[lane] = acc_f;
            pw[TILE + lane] = acc_s;
            named_barrier(1, NW * 32);
            if (w < 2) {
                TA* ub = tbuf + 2 * TILE;   // u = K t_f, warp 0 -> warp 1
                TA ys = 0;
                if (w == 0) {
                    TA sf = 0;
#pragma unroll
                    for (int u = 0; u < NW; ++u) sf += part[((par * NW + u) * 2) * TILE + lane];
                    tbuf[lane] = v[f * TILE + lane] - sf;
                    __syncwarp();
                    TA yf, uk = 0;
                    if (sr >= 0 && hasC)
                        row_dot2<TS, TA>(cp + 2 * TILE2, cp + (int64_t)(fwd ? 5 : 3) * TILE2, lane, tbuf, yf, uk);
                    else
                        yf = row_dot<TS, TA>(cp + 2 * TILE2, lane, tbuf);
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&cempty[k % CR]));
                    v[f * TILE + lane] = yf;
                    ub[lane] = uk;
                } else {
                    if (sr >= 0) {
                        TA ss = 0;
#pragma unroll
                        for (int u = 0; u < NW; ++u) ss += part[((par * NW + u) * 2 + 1) * TILE + lane];
                        TA* tb = tbuf + TILE;
                        tb[lane] = v[sr * TILE + lane] - ss;
                        __syncwarp();
                        ys = row_dot<TS, TA>(cp + 6 * TILE2, lane, tb);
                        __syncwarp();
                    }
                    if (lane == 0) mbar_arrive(smem_u32(&cempty[k % CR]));
                }
                named_barrier(3, 64);   // u ready
                if (w == 1 && sr >= 0) v[sr * TILE + lane] = ys + ub[lane];
                named_barrier(2, 64);   // the pair's solution, for both warps' next near tiles
            }
            fb += ff + fs;
            par ^= 1;
        }
    }
    __syncthreads();
    if (*abort_flag) {
        if (tid == 0) {
            atomicExch(a.err, 1);
            // only the last use of a slot can still be in flight (a reload waits for the
            // release of the previous use, which follows its arrival): drain those
            for (int sl = 0; sl < RG; ++sl)
                if (issued[0] > sl) mbar_wait(smem_u32(&full[sl]), (uint32_t)(((issued[0] - 1 - sl) / RG) & 1));
            for (int sl = 0; sl < CR; ++sl)
                if (issued[1] > sl) mbar_wait(smem_u32(&cfull[sl]), (uint32_t)(((issued[1] - 1 - sl) / CR) & 1));
        }
        __syncthreads();
        return;
    }
    if (a.accumulate)
        for (int i = tid; i < n; i += NT) out[i] += (double)(v[i] * (sc32 ? sc32[i] : 1.0f));
    else
        for (int i = tid; i < n; i += NT) out[i] = (double)(v[i] * (sc32 ? sc32[i] : 1.0f));
}

// ---------------------------------------------------------------------------------
// Column-block variant for many right-hand sides of one item (the MBF panels, the
// identity columns of the interface inverses, batched PCG columns): consumer warp w
// solves column w of the job on its own (lane = tile row, as above, its own solution
// vector in shared memory), all NW warps walking the same tile stream, so each factor
// tile is copied from memory once per NW columns.  Every warp reads every tile and
// releases it (NW arrivals per tile on empty[group]); no named barriers.
// ---------------------------------------------------------------------------------
template <typename TS, typename TA, int G, int RG, int NW>
__global__ void __launch_bounds__((NW + 1) * 32) k_chain_solve_cols(SolveArgs a) {
    static_assert(RG % 2 == 0, "the barrier block keeps 16-byte alignment for even RG");
    constexpr int R = RG * G;
    const int job = blockIdx.x;
    const int nc = a.job_nc ? a.job_nc[job] : NW;
    const int c0 = a.job_col0 ? a.job_col0[job] : 0;
    {
        bool any = false;   // the job's columns that still run (PCG stop flags)
        for (int c = 0; c < nc; ++c) any = any || !(a.done && a.done[(c0 + c) * a.done_stride]);
        if (!any) return;
    }
    const int s = a.job_sub[job];
    const Profile pf = a.pf;
    const int n = pf.rows[s], T = pf.ntiles[s];
    const int64_t r0 = pf.row0[s];
    const int64_t nts = pf.fwd[r0 + T - 1] + (T - 1 - pf.lo[r0 + T - 1]) + 1;
    const int t0 = a.job_t0 ? a.job_t0[job] : 0;   // smallest start row of the job's columns
    const int64_t q0 = pf.fwd[r0 + t0];
    const int64_t qend = nts + pf.bwd[r0 + t0] + (pf.hi[r0 + t0] - t0) + 1;
    const TS* F = (const TS*)a.fwdS + pf.base[s] * TILE2;
    const TS* Bk = (const TS*)a.bwdS + pf.base[s] * TILE2;
    const double* sc = a.scale ? a.scale + a.scale_off[s] : nullptr;
    const float* sc32 = a.scale32 ? a.scale32 + a.scale_off[s] : nullptr;
    const int64_t ld = a.job_ld ? a.job_ld[job] : a.ldin;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const bool act = w < nc && !(a.done && a.done[(c0 + w) * a.done_stride]);
    constexpr uint32_t TB = TILE2 * sizeof(TS);

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TS* ring = reinterpret_cast<TS*>(smem_raw);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + R * TB);
    uint64_t* empty = full + RG;
    volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + RG);
    int64_t* issued = reinterpret_cast<int64_t*>(empty + RG + 1);
    volatile int64_t* slot_q = reinterpret_cast<volatile int64_t*>(empty + RG + 2);
    TA* tbuf = reinterpret_cast<TA*>(empty + 2 * RG + 2);   // [NW][2][32]
    int32_t* lo_s = reinterpret_cast<int32_t*>(tbuf + 2 * NW * TILE);
    int32_t* hi_s = lo_s + T;
    TA* v = reinterpret_cast<TA*>(hi_s + T + ((2 * T) & 3));   // [NW][T * 32], 16-byte aligned
    auto src = [&](int64_t q) -> const TS* { return q < nts ? F + q * TILE2 : Bk + (q - nts) * TILE2; };
    if (tid == 0) {
        for (int i = 0; i < RG; ++i) {
            mbar_init(smem_u32(&full[i]), 1);
            mbar_init(smem_u32(&empty[i]), G * NW);
            slot_q[i] = -1;
        }
        *abort_flag = 0;
        *issued = q0;
        fence_async_smem();
    }
    for (int i = tid; i < T; i += (NW + 1) * 32) {
        lo_s[i] = pf.lo[r0 + i];
        hi_s[i] = pf.hi[r0 + i];
    }
    if (w < NW) {
        TA* vw = v + (int64_t)w * T * TILE;
        const double* in = a.in + a.job_in[job] + (int64_t)w * ld;
        for (int i = lane; i < T * TILE; i += 32) {
            TA x = 0;
            if (act && i < n) {
                if constexpr (sizeof(TA) == 4) x = (float)in[i] * (sc32 ? sc32[i] : 1.0f);
                else x = in[i] * (sc ? sc[i] : 1.0);
            }
            vw[i] = x;
        }
    }
    __syncthreads();

    if (w == NW) {
        if (lane == 0) {   // producer, as in k_chain_solve
            int64_t g0 = q0;
            for (; g0 < qend; g0 += G) {
                const int64_t gi = (g0 - q0) / G;
                const int gs = (int)(gi % RG);
                const int64_t u = gi / RG;
                if (u > 0 && (*abort_flag || !mbar_poll(smem_u32(&empty[gs]), (uint32_t)((u - 1) & 1)))) {
                    *abort_flag = 1;
                    break;
                }
                const int cnt = (int)min((int64_t)G, qend - g0);
                slot_q[gs] = g0;
                const uint32_t bar = smem_u32(&full[gs]);
                mbar_expect_tx(bar, (uint32_t)cnt * TB);
                TS* dst = ring + (int64_t)(gs * G) * TILE2;
                const int c1 = g0 < nts ? (int)min((int64_t)cnt, nts - g0) : 0;
                if (c1 > 0) bulk_copy(smem_u32(dst), src(g0), (uint32_t)c1 * TB, bar);
                if (cnt > c1) bulk_copy(smem_u32(dst + (int64_t)c1 * TILE2), src(g0 + c1), (uint32_t)(cnt - c1) * TB, bar);
            }
            *issued = g0;
        }
    } else {
        TA* vw = v + (int64_t)w * T * TILE;
        TA* tw = tbuf + w * 2 * TILE;   // t of the last two rows solved (alternating)
        auto wait_full = [&](int64_t qq) -> const TS* {
            const int64_t gi = (qq - q0) / G;
            const int gs = (int)(gi % RG);
            if (!__any_sync(0xffffffffu, *abort_flag != 0)) {
                const int64_t gq = q0 + gi * G;
                bool r = false;
                for (long long i = 0; i < kWaitLimit; ++i)
                    if (slot_q[gs] == gq) {
                        r = true;
                        break;
                    }
                r = r && mbar_poll(smem_u32(&full[gs]), (uint32_t)((gi / RG) & 1));
                r = __all_sync(0xffffffffu, r);
                if (!r && lane == 0) *abort_flag = 1;
            }
            return ring + ((qq - q0) % R) * TILE2;
        };
        auto release = [&](int64_t qq) {
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&empty[((qq - q0) / G) % RG]));
        };
        // FP32 arithmetic: rows are paired as in k_chain_solve_pairs; the pair's coupling
        // tile (forward row b: its last off-diagonal tile, C; backward row a: its first,
        // C^T) multiplies t of the pair's other row, solved just before in stream order.
        constexpr bool kPair = sizeof(TA) == 4;
        tw[lane] = 0;
        tw[TILE + lane] = 0;
        __syncwarp();
        int cur = 0;
        int64_t q = q0;
        for (int pass = 0; pass < 2; ++pass) {
            for (int step = t0; step < T; ++step) {
                const int I = pass == 0 ? step : T - 1 - (step - t0);
                const int j0 = pass == 0 ? lo_s[I] : I + 1;
                const int nt = pass == 0 ? I - lo_s[I] : hi_s[I] - I;
                const int tc = !kPair || nt == 0 ? -1 : (pass == 0 ? ((I & 1) ? nt - 1 : -1) : ((I & 1) ? -1 : 0));
                const TA* tp = tw + cur * TILE;
                TA acc = 0, cpl = 0;
                for (int t = 0; t < nt; ++t) {
                    const TS* tl = wait_full(q + t);
                    if (act) {
                        if (t == tc) cpl = row_dot<TS, TA>(tl, lane, tp);
                        else acc += row_dot<TS, TA>(tl, lane, vw + (j0 + t) * TILE);
                    }
                    release(q + t);
                }
                TA* vi = vw + I * TILE;
                TA* tn = tw + (cur ^ 1) * TILE;
                tn[lane] = vi[lane] - acc;
                __syncwarp();
                const TS* D = wait_full(q + nt);
                const TA y = act ? row_dot<TS, TA>(D, lane, tn) + cpl : (TA)0;
                release(q + nt);
                vi[lane] = y;
                __syncwarp();
                cur ^= 1;
                q += nt + 1;
            }
        }
    }
    __syncthreads();
    if (*abort_flag) {
        if (tid == 0) {
            atomicExch(a.err, 1);
            const int64_t ng = (*issued - q0 + G - 1) / G;
            for (int sl = 0; sl < RG; ++sl) {
                if (ng <= sl) continue;
                const int64_t u = (ng - 1 - sl) / RG;
                mbar_wait(smem_u32(&full[sl]), (uint32_t)(u & 1));
            }
        }
        __syncthreads();
        return;
    }
    if (w < NW && act) {
        const TA* vw = v + (int64_t)w * T * TILE;
        double* out = a.out + a.job_out[job] + (int64_t)w * ld;
        for (int i = lane; i < n; i += 32) {
            double x;
            if constexpr (sizeof(TA) == 4) x = (double)(vw[i] * (sc32 ? sc32[i] : 1.0f));
            else x = vw[i] * (sc ? sc[i] : 1.0);
            if (a.accumulate) out[i] += x;
            else out[i] = x;
        }
    }
}

template <typename TS, typename TA, int G, int RG>
static cudaError_t launch_cols_ring(const SolveArgs& a, int njobs, int max_tiles, cudaStream_t st) {
    constexpr int NW = COLS_PER_JOB;
    constexpr int R = RG * G;
    size_t smem = (size_t)R * TILE2 * sizeof(TS) + (3 * RG + 2) * sizeof(uint64_t) + 2 * NW * TILE * sizeof(TA) +
                  (size_t)(2 * max_tiles + 4) * sizeof(int32_t) + (size_t)NW * max_tiles * TILE * sizeof(TA) + 16;
    cudaError_t e = cudaFuncSetAttribute(k_chain_solve_cols<TS, TA, G, RG, NW>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (njobs > 0) {
        count_launch();
        k_chain_solve_cols<TS, TA, G, RG, NW><<<njobs, (NW + 1) * 32, smem, st>>>(a);
    }
    return cudaGetLastError();
}

template <typename TS, typename TA>
cudaError_t launch_tile_solve_cols(const SolveArgs& a, int njobs, int max_tiles, cudaStream_t st) {
    // 8 KB bulk copies, 32 KB ring (the per-warp solution vectors take the rest)
    return launch_cols_ring<TS, TA, 8192 / (TILE2 * sizeof(TS)) < 1 ? 1 : 8192 / (TILE2 * sizeof(TS)), 4>(
        a, njobs, max_tiles, st);
}

// ---------------------------------------------------------------------------------
// MBF right-hand sides  -B_i psi_m = -G[Omega_i, m]  scattered into the (zeroed) panel
// buffer, column-major per subdomain (Eq. def-phat-local).
// ---------------------------------------------------------------------------------
__global__ void k_mbf_rhs(int m, const int64_t* __restrict__ g_off, const int32_t* __restrict__ g_row,
                          const int32_t* __restrict__ g_col, const double* __restrict__ g_val,
                          const int32_t* __restrict__ rows, const int64_t* __restrict__ phi_off,
                          double* __restrict__ rhs) {
    int s = blockIdx.x;
    if (s >= m) return;
    int64_t ns = rows[s];
    for (int64_t t = g_off[s] + threadIdx.x; t < g_off[s + 1]; t += blockDim.x)
        rhs[phi_off[s] + g_col[t] * ns + g_row[t]] = -g_val[t];
}

template <typename TS>
__global__ void k_convert(int64_t n, const double* __restrict__ src, TS* __restrict__ dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = stf<TS>(src[i]);
}

// Identity right-hand sides for the explicit interface inverse (column q = e_q).
__global__ void k_eye(int L, double* __restrict__ E) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < L) E[(int64_t)q * L + q] = 1.0;
}

// ---------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------
static inline int grid_for(int64_t n, int bs) {
    int64_t g = (n + bs - 1) / bs;
    return (int)(g < 1 ? 1 : (g > 65535 * 4 ? 65535 * 4 : g));
}

void launch_local_diag(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                       const int32_t* row_sub, int diag_scale, int modified, double* dloc, double* sc, float* sc32,
                       cudaStream_t st) {
    count_launch();
    k_local_diag<<<grid_for(n, 256), 256, 0, st>>>(n, rowptr, col, val, row_sub, diag_scale, modified, dloc, sc,
                                                    sc32);
}

template <typename TW>
void launch_scatter_local(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                          const int32_t* row_sub, const int64_t* sub_off, const Profile& pf,
                          const double* dloc, const double* sc, TW* work, int nitems, cudaStream_t st) {
    count_launch();
    k_scatter_local<TW><<<grid_for(n, 256), 256, 0, st>>>(n, rowptr, col, val, row_sub, sub_off, pf,
                                                          dloc, sc, work);
    count_launch();
    k_pad_diag<TW><<<(nitems + 127) / 128, 128, 0, st>>>(nitems, pf, work);
}

template <typename TW>
void launch_pad_diag(int nitems, const Profile& pf, TW* work, cudaStream_t st) {
    count_launch();
    k_pad_diag<TW><<<(nitems + 127) / 128, 128, 0, st>>>(nitems, pf, work);
}

// wm = widest tile row of all items (tiles I - lo(I) + 1).  FP32: the resident-row kernel
// when its shared memory fits an SM, else the per-step kernel.  FP64 keeps the per-step
// kernel: measured at config 3 on B300, the resident-row version (178 KB of shared memory,
// one CTA per SM) took 40.9 ms against 35.5 ms, both bound by the FP64 pipe.
template <typename TW>
void launch_tile_chol(int nitems, const Profile& pf, const int32_t* order, TW* work, TW* dinv, int* err, int wm,
                      cudaStream_t st) {
    if (nitems <= 0) return;
    count_launch();
    const size_t smem = tile_chol_row_smem(wm, sizeof(TW));
    if (sizeof(TW) == 4 && wm >= 1 && smem <= 227 * 1024 &&
        cudaFuncSetAttribute(k_tile_chol_row<TW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
            cudaSuccess) {
        k_tile_chol_row<TW><<<nitems, 128, smem, st>>>(pf, order, work, dinv, err, wm);
    } else {
        (void)cudaGetLastError();
        k_tile_chol<TW><<<nitems, 256, 0, st>>>(pf, order, work, dinv, err);
    }
}

template <typename TW, typename TS>
void launch_finalize(int nitems, const Profile& pf, const TW* work, const TW* dinv, TS* fwdS, TS* bwdS,
                     cudaStream_t st) {
    count_launch();
    k_finalize<TW, TS><<<dim3(nitems, 32), 256, 0, st>>>(pf, work, dinv, fwdS, bwdS);
}

// Tiles per bulk copy of the far-tile ring, chosen by measurement at config 3 on B300:
// FP32 16 KB and BF16 8 KB copies, FP64 one 8 KB tile per copy (FP64 solves are bound by
// the FP64 pipe, not by the copies).
template <typename TS>
constexpr int group_tiles() {
    return sizeof(TS) == 8 ? 1 : 4;
}

template <typename TS, typename TA, int G, int RG, int CR>
static cudaError_t launch_ring(const SolveArgs& a, int njobs, int max_tiles, cudaStream_t st, int ncols) {
    constexpr int NW = 4;   // consumer warps (+ 2 producer warps)
    constexpr int R = RG * G;
    constexpr int HDR = 3 * RG + 2 * CR + 3, HDRP = HDR + (HDR & 1);
    size_t smem = (size_t)(R + 2 * CR) * TILE2 * sizeof(TS) + HDRP * sizeof(uint64_t) +
                  (2 * NW + 1) * TILE * sizeof(TA) + (size_t)(2 * max_tiles + 4) * sizeof(int32_t) +
                  (size_t)max_tiles * TILE * sizeof(TA) + 16;
    cudaError_t e = cudaFuncSetAttribute(k_chain_solve<TS, TA, G, RG, CR, NW>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (njobs > 0) {
        count_launch();
        SolveArgs b = a;
        b.col_fast = ncols > 1;
        const dim3 grid = ncols > 1 ? dim3(ncols, njobs) : dim3(njobs);
        k_chain_solve<TS, TA, G, RG, CR, NW><<<grid, (NW + 2) * 32, smem, st>>>(b);
    }
    return cudaGetLastError();
}

template <typename TS, typename TA, int G, int RG, int CR, int NW>
static cudaError_t launch_pairs(const SolveArgs& a, int njobs, int max_tiles, cudaStream_t st, int ncols) {
    constexpr int R = RG * G, CT = 7;
    constexpr int HDR = 3 * RG + 2 * CR + 3, HDRP = HDR + (HDR & 1);
    if (a.job_t0) return cudaErrorInvalidValue;   // identity right-hand sides: FP64 only
    const int max_steps = 2 * ((max_tiles + 1) / 2);
    size_t smem = (size_t)(R + CT * CR) * TILE2 * sizeof(TS) + HDRP * sizeof(uint64_t) +
                  (4 * NW + 4) * TILE * sizeof(TA) + (size_t)max_steps * sizeof(uint4) +
                  (size_t)(2 * max_tiles + 4) * sizeof(int32_t) + (size_t)max_tiles * TILE * sizeof(TA) + 16;
    cudaError_t e = cudaFuncSetAttribute(k_chain_solve_pairs<TS, TA, G, RG, CR, NW>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (njobs > 0) {
        count_launch();
        SolveArgs b = a;
        b.col_fast = ncols > 1;
        const dim3 grid = ncols > 1 ? dim3(ncols, njobs) : dim3(njobs);
        k_chain_solve_pairs<TS, TA, G, RG, CR, NW><<<grid, (NW + 2) * 32, smem, st>>>(b);
    }
    return cudaGetLastError();
}

template <typename TS, typename TA>
cudaError_t launch_tile_solve(const SolveArgs& a, int njobs, int max_tiles, cudaStream_t st, int ncols) {
    constexpr int G = group_tiles<TS>();
    if constexpr (sizeof(TA) == 4) {   // pair-stepped chains (FP32 / BF16 streams)
        // Far-ring groups (G tiles each) and consumer warps, chosen by measurement at config
        // 3 on B300 (local solve per application): BF16 4 groups (32 KB ring), 6 consumer
        // warps, 0.134 ms; FP32 2 groups (32 KB), 6 warps, 0.174 ms.  The alternatives are
        // kept selectable for measurement.
        constexpr int RG = sizeof(TS) == 2 ? 4 : 2;
        switch (a.deep_ring) {
            case 1: return launch_pairs<TS, TA, G, RG, 2, 4>(a, njobs, max_tiles, st, ncols);      // 4 consumer warps
            case 2: return launch_pairs<TS, TA, G, RG, 3, 6>(a, njobs, max_tiles, st, ncols);      // 3 critical slots
            case 3: return launch_pairs<TS, TA, G, RG + 1, 2, 6>(a, njobs, max_tiles, st, ncols);  // deeper far ring
            // BF16: a 3-group far ring, so that 3 CTAs fit an SM's shared memory
            case 4: return launch_pairs<TS, TA, G, (sizeof(TS) == 2 ? 3 : RG), 2, 6>(a, njobs, max_tiles, st, ncols);
            default: return launch_pairs<TS, TA, G, RG, 2, 6>(a, njobs, max_tiles, st, ncols);
        }
    } else {
        constexpr int CR = 2;   // critical pairs in flight
        switch (a.deep_ring) {
            case 1: return launch_ring<TS, TA, G, 2, CR>(a, njobs, max_tiles, st, ncols);       // half far ring
            case 2: return launch_ring<TS, TA, G, 4, 2 * CR>(a, njobs, max_tiles, st, ncols);   // 2x critical
            case 3: return launch_ring<TS, TA, G, 2, 2 * CR>(a, njobs, max_tiles, st, ncols);
            default: return launch_ring<TS, TA, G, 4, CR>(a, njobs, max_tiles, st, ncols);
        }
    }
}

void launch_mbf_rhs(int m, const int64_t* g_off, const int32_t* g_row, const int32_t* g_col,
                    const double* g_val, const int32_t* rows, const int64_t* phi_off, double* rhs,
                    cudaStream_t st) {
    if (m > 0) {
        count_launch();
        k_mbf_rhs<<<m, 128, 0, st>>>(m, g_off, g_row, g_col, g_val, rows, phi_off, rhs);
    }
}

template <typename TS>
void launch_convert(int64_t n, const double* src, TS* dst, cudaStream_t st) {
    if (n > 0) {
        count_launch();
        k_convert<TS><<<grid_for(n, 256), 256, 0, st>>>(n, src, dst);
    }
}

void launch_eye(int L, double* E, cudaStream_t st) {
    if (L > 0) {
        count_launch();
        k_eye<<<(L + 127) / 128, 128, 0, st>>>(L, E);
    }
}

template void launch_scatter_local<double>(int64_t, const int32_t*, const int32_t*, const double*,
                                           const int32_t*, const int64_t*, const Profile&, const double*,
                                           const double*, double*, int, cudaStream_t);
template void launch_scatter_local<float>(int64_t, const int32_t*, const int32_t*, const double*,
                                          const int32_t*, const int64_t*, const Profile&, const double*,
                                          const double*, float*, int, cudaStream_t);
template void launch_pad_diag<double>(int, const Profile&, double*, cudaStream_t);
template void launch_tile_chol<double>(int, const Profile&, const int32_t*, double*, double*, int*, int,
                                        cudaStream_t);
template void launch_tile_chol<float>(int, const Profile&, const int32_t*, float*, float*, int*, int,
                                       cudaStream_t);
template void launch_finalize<double, double>(int, const Profile&, const double*, const double*, double*,
                                              double*, cudaStream_t);
template void launch_finalize<float, float>(int, const Profile&, const float*, const float*, float*, float*,
                                            cudaStream_t);
template void launch_finalize<float, __nv_bfloat16>(int, const Profile&, const float*, const float*,
                                                    __nv_bfloat16*, __nv_bfloat16*, cudaStream_t);
template cudaError_t launch_tile_solve<double, double>(const SolveArgs&, int, int, cudaStream_t, int);
template cudaError_t launch_tile_solve_cols<double, double>(const SolveArgs&, int, int, cudaStream_t);
template cudaError_t launch_tile_solve_cols<float, float>(const SolveArgs&, int, int, cudaStream_t);
template cudaError_t launch_tile_solve_cols<__nv_bfloat16, float>(const SolveArgs&, int, int, cudaStream_t);
template cudaError_t launch_tile_solve<float, float>(const SolveArgs&, int, int, cudaStream_t, int);
template cudaError_t launch_tile_solve<__nv_bfloat16, float>(const SolveArgs&, int, int, cudaStream_t, int);
template void launch_convert<float>(int64_t, const double*, float*, cudaStream_t);
template void launch_convert<__nv_bfloat16>(int64_t, const double*, __nv_bfloat16*, cudaStream_t);

}  // namespace am
