// Supernodal local factors on sm_103a: the numeric Cholesky factorisation of every A_i
// (Algorithm 1, "compute the Cholesky factorization A_i = L_i L_i^T") in the nested-
// dissection supernodal layout of snode_plan.cpp, and the batched forward/backward
// solves that apply A_i^{-1} for the particular solutions (Eq. def-pbar-local), the MBFs
// (Eq. def-phat-local) and the block-Jacobi smoother (Sec. 5.4).
//
// The solves read the factor as per-warp record streams (snode_stream.h): every entry of
// L_J (its panel and the inverse D_J of its diagonal block) appears once in the forward
// records and once in the backward ones, both rounded from the same FP32/FP64 value, so
// the backward sweep applies exactly the transpose of what the forward sweep applies and
// the local solve stays symmetric after rounding.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "snode_stream.h"
#include "tma.cuh"

namespace am {

namespace {

// Column-major packed lower triangle of a w x w matrix: entry (r, c), r >= c.
__host__ __device__ __forceinline__ int64_t cpack(int r, int c, int w) {
    return (int64_t)c * w - (int64_t)c * (c - 1) / 2 + (r - c);
}
// Row-major packed lower triangle: entry (r, c), r >= c.
__host__ __device__ __forceinline__ int64_t rpack(int r, int c) { return (int64_t)r * (r + 1) / 2 + c; }

// Dense Cholesky of the 32x32 tile X (lower triangle used) by a CTA of 256 threads,
// followed by the inverse of the factor into Xi (one column per thread).  A non-positive
// or non-finite pivot sets *bad and is replaced by 1.
template <typename TW>
__device__ void tile_chol_inv(TW (*X)[TILE + 1], TW (*Xi)[TILE + 1], int tid, int* bad) {
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
            const int r = e >> 5, cc = e & 31;
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
                for (int t = cc; t < r; ++t) v -= X[r][t] * Xi[t][cc];
                v /= X[r][r];
            }
            Xi[r][cc] = v;
        }
    }
    __syncthreads();
}

}  // namespace

// ---------------------------------------------------------------------------------
// Numeric factorisation, one CTA (256 threads) per subdomain, supernodes in postorder
// (left-looking): the front F_J = (J u R_J) x J (column-major, ld = w + nr, in `work`)
// receives the entries of the scaled A_i, the updates -L_{.,K} L_{J,K}^T of every
// descendant K whose structure reaches J, then a blocked dense Cholesky (32-column
// panels: factor the diagonal tile, solve the rows below, update the columns to the
// right).  D_J = L_JJ^{-1} follows by block forward substitution from the inverted
// diagonal tiles, into `dwork` (row-major packed).  A non-positive pivot sets
// err = {1, subdomain} and continues with pivot 1.
// ---------------------------------------------------------------------------------
template <typename TW>
__global__ void __launch_bounds__(256) k_sn_factor(SnTables t, const int32_t* __restrict__ order,
                                                   const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                                   const double* __restrict__ val, const double* __restrict__ dloc,
                                                   const double* __restrict__ sc, TW* __restrict__ work,
                                                   TW* __restrict__ dwork, int* __restrict__ err) {
    const int s = order ? order[blockIdx.x] : blockIdx.x;
    const int64_t g0 = t.sub_off[s];
    const int ns = (int)(t.sub_off[s + 1] - g0);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint16_t* relpos = reinterpret_cast<uint16_t*>(smem_raw);   // [ns]
    __shared__ TW X[TILE][TILE + 1];
    __shared__ TW Xi[TILE][TILE + 1];
    __shared__ TW As[TILE][TILE + 1];
    __shared__ TW Bs[TILE][TILE + 1];
    __shared__ int bad;
    const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5, cc = tid & 31, rb = (tid >> 5) * 4;
    if (tid == 0) bad = 0;
    for (int J = t.sn_off[s]; J < t.sn_off[s + 1]; ++J) {
        const int c0 = t.c0[J], w = t.w[J], nr = t.nr[J], h = w + nr;
        const uint16_t* R = t.rows + t.roff[J];
        TW* F = work + t.foff[J];
        TW* D = dwork + t.doff[J];
        for (int i = tid; i < w; i += 256) relpos[c0 + i] = (uint16_t)i;
        for (int i = tid; i < nr; i += 256) relpos[R[i]] = (uint16_t)(w + i);
        for (int64_t e = tid; e < (int64_t)h * w; e += 256) F[e] = (TW)0;
        __syncthreads();
        // entries of the scaled A_i in columns J, rows >= the column (A's row k of the
        // column by symmetry); the symbolic structure puts every such row in J u R_J
        for (int c = wp; c < w; c += 8) {
            const int64_t k = g0 + c0 + c;
            const double sk = sc[k];
            for (int e = rowptr[k] + lane; e < rowptr[k + 1]; e += 32) {
                const int64_t gc = col[e];
                const int lc = (int)(gc - g0);
                if (lc < c0 + c || lc >= ns) continue;
                const double v = (gc == k ? dloc[k] : val[e]) * sk * sc[gc];
                F[relpos[lc] + (int64_t)c * h] = (TW)v;
            }
        }
        __syncthreads();
        // updates from the descendants K: F[relpos(R_K[i]), R_K[j] - c0] -= L_K,i . L_K,j
        for (int64_t u = t.upd_ptr[J]; u < t.upd_ptr[J + 1]; ++u) {
            const int K = t.upd[3 * u], a = t.upd[3 * u + 1], b = t.upd[3 * u + 2];
            const int wK = t.w[K], nrK = t.nr[K], hK = wK + nrK;
            const TW* LK = work + t.foff[K];
            const uint16_t* RK = t.rows + t.roff[K];
            const int M = nrK - a, N = b - a;
            for (int ti = 0; ti * TILE < M; ++ti)
                for (int tj = 0; tj * TILE < N && tj <= ti; ++tj) {
                    TW acc[4] = {0, 0, 0, 0};
                    for (int k0 = 0; k0 < wK; k0 += TILE) {
                        for (int e = tid; e < TILE2; e += 256) {
                            const int r = e & 31, kk = e >> 5;
                            const int ia = a + ti * TILE + r, ib = a + tj * TILE + r, kc = k0 + kk;
                            As[r][kk] = (ia < nrK && kc < wK) ? LK[(wK + ia) + (int64_t)kc * hK] : (TW)0;
                            Bs[r][kk] = (ib < b && kc < wK) ? LK[(wK + ib) + (int64_t)kc * hK] : (TW)0;
                        }
                        __syncthreads();
#pragma unroll 8
                        for (int kk = 0; kk < TILE; ++kk) {
                            const TW bv = Bs[cc][kk];
#pragma unroll
                            for (int q = 0; q < 4; ++q) acc[q] += As[rb + q][kk] * bv;
                        }
                        __syncthreads();
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int i = a + ti * TILE + rb + q, j = a + tj * TILE + cc;
                        if (i < nrK && j < b && i >= j) F[relpos[RK[i]] + (int64_t)(RK[j] - c0) * h] -= acc[q];
                    }
                }
        }
        __syncthreads();
        // blocked dense Cholesky of the front
        const int nb = (w + TILE - 1) / TILE;
        for (int p = 0; p < nb; ++p) {
            const int pw = min(TILE, w - p * TILE);
            for (int e = tid; e < TILE2; e += 256) {
                const int r = e >> 5, c = e & 31;
                X[r][c] = (r < pw && c < pw) ? F[(p * TILE + r) + (int64_t)(p * TILE + c) * h] : (TW)(r == c ? 1 : 0);
            }
            __syncthreads();
            tile_chol_inv<TW>(X, Xi, tid, &bad);
            for (int e = tid; e < TILE2; e += 256) {
                const int r = e >> 5, c = e & 31;
                if (r < pw && c <= r) {
                    F[(p * TILE + r) + (int64_t)(p * TILE + c) * h] = X[r][c];
                    D[rpack(p * TILE + r, p * TILE + c)] = Xi[r][c];
                }
            }
            // rows below the diagonal tile: L_ip = A_ip L_pp^{-T}
            for (int r0 = p * TILE + pw; r0 < h; r0 += TILE) {
                __syncthreads();
                for (int e = tid; e < TILE2; e += 256) {
                    const int r = e & 31, k = e >> 5;
                    As[r][k] = (r0 + r < h && k < pw) ? F[(r0 + r) + (int64_t)(p * TILE + k) * h] : (TW)0;
                }
                __syncthreads();
                TW acc[4] = {0, 0, 0, 0};
#pragma unroll 8
                for (int k = 0; k < TILE; ++k) {
                    const TW bv = Xi[cc][k];
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[q] += As[rb + q][k] * bv;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (r0 + rb + q < h && cc < pw) F[(r0 + rb + q) + (int64_t)(p * TILE + cc) * h] = acc[q];
            }
            __syncthreads();
            // columns to the right: F[rows >= q0, q-block] -= L[rows, p] L[q-block, p]^T
            for (int qb = p + 1; qb < nb; ++qb) {
                const int q0 = qb * TILE, qw = min(TILE, w - q0);
                for (int e = tid; e < TILE2; e += 256) {
                    const int r = e & 31, k = e >> 5;
                    Bs[r][k] = (r < qw && k < pw) ? F[(q0 + r) + (int64_t)(p * TILE + k) * h] : (TW)0;
                }
                for (int r0 = q0; r0 < h; r0 += TILE) {
                    __syncthreads();
                    for (int e = tid; e < TILE2; e += 256) {
                        const int r = e & 31, k = e >> 5;
                        As[r][k] = (r0 + r < h && k < pw) ? F[(r0 + r) + (int64_t)(p * TILE + k) * h] : (TW)0;
                    }
                    __syncthreads();
                    TW acc[4] = {0, 0, 0, 0};
#pragma unroll 8
                    for (int k = 0; k < TILE; ++k) {
                        const TW bv = Bs[cc][k];
#pragma unroll
                        for (int q = 0; q < 4; ++q) acc[q] += As[rb + q][k] * bv;
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (r0 + rb + q < h && cc < qw) F[(r0 + rb + q) + (int64_t)(q0 + cc) * h] -= acc[q];
                }
                __syncthreads();
            }
        }
        __syncthreads();
        // D_J: D_II = Xi_I (stored above); D_IJ = -D_II sum_{K=J}^{I-1} L_IK D_KJ
        for (int I = 1; I < nb; ++I) {
            const int iw = min(TILE, w - I * TILE);
            __syncthreads();   // the previous row's last reads of Xi and X are done
            for (int e = tid; e < TILE2; e += 256) {
                const int r = e >> 5, c = e & 31;
                Xi[r][c] = (r < iw && c <= r) ? D[rpack(I * TILE + r, I * TILE + c)] : (TW)0;
            }
            for (int Jt = 0; Jt < I; ++Jt) {
                TW acc[4] = {0, 0, 0, 0};
                for (int K = Jt; K < I; ++K) {
                    __syncthreads();
                    for (int e = tid; e < TILE2; e += 256) {
                        const int r = e & 31, k = e >> 5;
                        // As[r][k] = L(I r, K k); Bs[k][c] = D(K k, Jt c)
                        As[r][k] = (r < iw) ? F[(I * TILE + r) + (int64_t)(K * TILE + k) * h] : (TW)0;
                        const int dr = K * TILE + (e >> 5), dc = Jt * TILE + (e & 31);
                        Bs[e >> 5][e & 31] = (dr < w && dc <= dr) ? D[rpack(dr, dc)] : (TW)0;
                    }
                    __syncthreads();
#pragma unroll 8
                    for (int k = 0; k < TILE; ++k) {
                        const TW bv = Bs[k][cc];
#pragma unroll
                        for (int q = 0; q < 4; ++q) acc[q] += As[rb + q][k] * bv;
                    }
                }
                __syncthreads();
#pragma unroll
                for (int q = 0; q < 4; ++q) X[rb + q][cc] = acc[q];   // Y = sum L D
                __syncthreads();
                TW out[4] = {0, 0, 0, 0};
#pragma unroll 8
                for (int k = 0; k < TILE; ++k) {
                    const TW yv = X[k][cc];
#pragma unroll
                    for (int q = 0; q < 4; ++q) out[q] -= Xi[rb + q][k] * yv;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int r = I * TILE + rb + q, c = Jt * TILE + cc;
                    if (rb + q < iw) D[rpack(r, c)] = out[q];
                }
            }
        }
        __syncthreads();
    }
    if (tid == 0 && bad) {
        if (atomicCAS(err + 1, -1, s) == -1) atomicExch(err, 1);
    }
}

// ---------------------------------------------------------------------------------
// Entries of the solve streams from the factor (one warp per record, grid-stride): the
// fronts in `work` (column-major (w + nr) x w per supernode) and D_J in `dwork` (row-
// major packed), rounded to TS, at the positions snode_stream.h defines.
// ---------------------------------------------------------------------------------
template <typename TW, typename TS>
__global__ void __launch_bounds__(256) k_sn_fill(SnTables t, const SnFill* __restrict__ fill, int64_t nfill,
                                                 const TW* __restrict__ work, const TW* __restrict__ dwork,
                                                 uint8_t* __restrict__ stream) {
    constexpr int V = 8 / (int)sizeof(TS);
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t k = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); k < nfill; k += nwarps) {
        const SnFill f = fill[k];
        TS* dst = reinterpret_cast<TS*>(stream + f.off);
        const int J = f.sn, w = t.w[J], h = w + t.nr[J], L = f.lanes;
        const TW* F = work + t.foff[J];
        const TW* D = dwork + t.doff[J];
        if (f.kind == SN_FCONTRIB) {
            for (int e = lane; e < f.n * f.rows; e += 32) {
                const int c = e / f.rows, i = e - c * f.rows;
                dst[(int64_t)(c / V) * f.rows * V + i * V + c % V] =
                    stf<TS>((double)F[(w + f.p0 + i) + (int64_t)(f.p1 + c) * h]);
            }
        } else if (f.kind == SN_FDIAG) {
            const int rel0 = f.p1 - f.p0;
            for (int j = 0; j < f.n; ++j) {
                const int c = f.p1 + j, gi = j / V, st = max(0, rel0 + gi * V);
                const int64_t o = sn_fdiag_off(gi, rel0, L, V) + j % V;
                for (int l = max(st, c - f.p0) + lane; l < L; l += 32)
                    dst[o + (int64_t)(l - st) * V] = stf<TS>((double)D[rpack(f.p0 + l, c)]);
            }
        } else if (f.kind == SN_BPANEL) {
            for (int e = lane; e < f.rows * L; e += 32) {
                const int i = e / L, c = e - i * L;
                dst[(int64_t)(i / V) * L * V + c * V + i % V] =
                    stf<TS>((double)F[(w + f.p0 + i) + (int64_t)(f.p1 + c) * h]);
            }
        } else if (f.kind == SN_BDIAG) {
            const int rel0 = f.p1 - f.p0;
            for (int j = 0; j < f.n; ++j) {
                const int r = f.p1 + j, gj = j / V, len = min(r - f.p0 + 1, L);
                const int64_t o = sn_bdiag_off(gj, rel0, L, V) + j % V;
                for (int c = lane; c < len; c += 32) dst[o + (int64_t)c * V] = stf<TS>((double)D[rpack(r, f.p0 + c)]);
            }
        }
    }
}

// ---------------------------------------------------------------------------------
// Batched local solves  out = S L^{-T} L^{-1} S in  (S = diag(scale)), one CTA of NW
// warps per job (subdomain, input offset, output offset) and column.  Shared memory: v
// and y over the subdomain's rows, and per warp a RING-byte ring with its mbarriers.
//
// Each warp interprets its own record stream (snode_stream.h): lane 0 keeps up to RING
// bytes of it in flight as bulk async copies of kChunk bytes (chunk k lands in slot
// k % NSLOT once the bytes of chunk k - NSLOT have been consumed), the warp waits for a
// record's chunks, applies it from shared memory and moves on; across record and level
// boundaries the copies stay ahead.  Forward records (levels from the leaves up):
// descendants' panel rows times their solved values subtracted from the unit's rows, then
// D_J applied (y); backward records (levels from the top down): the panel's transpose
// times the ancestors' final values subtracted, then D_J^T applied (v).  Barrier records
// separate the levels (and the two phases of levels holding a supernode wider than 32).
// Every wait is bounded: on timeout the warp sets the error word, still passes the
// barriers its stream has left (so no warp of the CTA waits forever), waits (bounded)
// for its own copies in flight and skips the output.
// ---------------------------------------------------------------------------------
constexpr int kRing = 4096;     // bytes of stream in shared memory per warp
constexpr int kChunk = 1024;    // bytes per bulk copy
constexpr int kSlots = kRing / kChunk;

// Narrow units use groups of lanes: lanes = (item, group) with RB = next power of two of
// the unit's items (rows or columns) and G = 32 / RB groups that split the loop; the
// groups' partial sums are added by xor shuffles at the end.
__device__ __forceinline__ int pow2_ceil(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}
template <typename TA>
__device__ __forceinline__ TA group_sum(TA x, int rb) {
    for (int o = rb; o < 32; o <<= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}
template <typename TS, typename TA>
struct G8;
template <>
struct G8<__nv_bfloat16, float> {
    __device__ static void get(uint2 u, float (&e)[4]) {
        const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
        const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
        e[0] = a.x;
        e[1] = a.y;
        e[2] = b.x;
        e[3] = b.y;
    }
};
template <>
struct G8<float, float> {
    __device__ static void get(uint2 u, float (&e)[2]) {
        e[0] = __uint_as_float(u.x);
        e[1] = __uint_as_float(u.y);
    }
};
template <>
struct G8<double, double> {
    __device__ static void get(uint2 u, double (&e)[1]) { e[0] = __hiloint2double((int)u.y, (int)u.x); }
};
// Operand x[x0 + k] for a group position k, zero past the record's columns (padding).
template <typename TA>
__device__ __forceinline__ TA xval(const TA* x, int x0, int k, int n) {
    return k < n ? x[x0 + k] : (TA)0;
}

template <typename TS, typename TA, int NW>
__global__ void __launch_bounds__(NW * 32) k_sn_stream(SnSolveArgs a) {
    constexpr int V = 8 / (int)sizeof(TS);
    const int col = a.col_fast ? blockIdx.x : 0;
    const int job = a.col_fast ? blockIdx.y : blockIdx.x;
    if (a.done && a.done[col * a.done_stride]) return;
    const SnTables& t = a.t;
    const int s = a.job_sub[job];
    const int64_t g0 = t.sub_off[s];
    const int n = (int)(t.sub_off[s + 1] - g0);
    const int npad = (n + 3) & ~3;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint8_t* rings = smem_raw;                                            // [NW][kRing]
    uint64_t* bars = reinterpret_cast<uint64_t*>(rings + NW * kRing);     // [NW][kSlots]
    TA* tmp = reinterpret_cast<TA*>(bars + NW * kSlots);                  // [NW][32]
    int* flag = reinterpret_cast<int*>(tmp + NW * 32);                    // [4]
    TA* v = reinterpret_cast<TA*>(flag + 4);
    TA* y = v + npad;
    const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
    constexpr int NT = NW * 32;
    constexpr bool f32 = sizeof(TA) == 4;
    constexpr unsigned FULL = 0xffffffffu;
    uint8_t* ring = rings + wp * kRing;
    uint64_t* bar = bars + wp * kSlots;
    TA* tw = tmp + wp * 32;
    const uint8_t* gs = a.stream + a.woff[(int64_t)s * NW + wp];
    const int64_t len = a.woff[(int64_t)s * NW + wp + 1] - a.woff[(int64_t)s * NW + wp];
    const int nbar = a.nbar[s];
    if (lane == 0) {
        for (int i = 0; i < kSlots; ++i) mbar_init(smem_u32(&bar[i]), 1);
        fence_async_smem();
    }
    if (tid == 0) flag[0] = 0;
    const double* in = a.in + a.job_in[job] + col * a.ldin;
    double* out = a.out + a.job_out[job] + col * a.ldout;
    for (int i = tid; i < n; i += NT) {
        if (f32) v[i] = (TA)((float)in[i] * (a.scale32 ? a.scale32[g0 + i] : 1.0f));
        else v[i] = (TA)(in[i] * (a.scale ? a.scale[g0 + i] : 1.0));
    }
    __syncthreads();
    int64_t issued = 0, landed = 0, consumed = 0;   // chunks issued / landed, bytes consumed
    const int64_t nchunks = (len + kChunk - 1) / kChunk;
    auto refill = [&]() {
        if (lane == 0) {
            while (issued < nchunks && (issued + 1) * kChunk <= consumed + kRing) {
                const int sl = (int)(issued % kSlots);
                const uint32_t b = (uint32_t)min((int64_t)kChunk, len - issued * kChunk);
                mbar_expect_tx(smem_u32(&bar[sl]), b);
                bulk_copy(smem_u32(ring + sl * kChunk), gs + issued * kChunk, b, smem_u32(&bar[sl]));
                ++issued;
            }
        }
        issued = __shfl_sync(FULL, issued, 0);
    };
    // waits until bytes [.., upto) of the stream have landed; false on timeout
    auto land = [&](int64_t upto) -> bool {
        while (landed * kChunk < upto) {
            if (landed >= issued) refill();
            if (landed >= issued) return false;   // nothing in flight covers it (malformed)
            const bool ok = mbar_wait(smem_u32(&bar[landed % kSlots]), (uint32_t)((landed / kSlots) & 1));
            if (!__all_sync(FULL, ok)) return false;
            ++landed;
        }
        return true;
    };
    int bars_done = 0;
    bool ok = true;
    TA acc = 0, dacc = 0;
    for (;;) {
        refill();
        if (!(ok = land(consumed + 16))) break;
        SnRec rc;
        {
            const uint4 hv = *reinterpret_cast<const uint4*>(ring + (consumed & (kRing - 1)));
            rc = *reinterpret_cast<const SnRec*>(&hv);
        }
        if (!(ok = land(consumed + rc.bytes))) break;
        if (rc.kind == SN_END) break;
        if (rc.kind == SN_BARRIER) {
            __syncthreads();
            ++bars_done;
            consumed += rc.bytes;
            continue;
        }
        const int64_t ip = consumed + 16, dp = ip + rc.hdr;
        // 8-byte entry group q of the record (a group never straddles the ring's end)
        auto grp = [&](int64_t q, TA(&e)[V]) {
            G8<TS, TA>::get(*reinterpret_cast<const uint2*>(ring + ((dp + 8 * q) & (kRing - 1))), e);
        };
        auto idx8 = [&](int k) -> int { return ring[(ip + k) & (kRing - 1)]; };
        auto idx16 = [&](int k) -> int {
            return *reinterpret_cast<const uint16_t*>(ring + ((ip + 2 * k) & (kRing - 1)));
        };
        const int L = rc.lanes;
        if (rc.kind == SN_FCONTRIB) {
            const int R = rc.rows, RB = pow2_ceil(R), G = 32 / RB;
            const int i = lane & (RB - 1), g = lane / RB;
            const int ng = (rc.ncols + V - 1) / V;
            if (rc.flags & SN_FIRST) acc = lane < L ? v[rc.t0 + lane] : (TA)0;
            tw[lane] = 0;
            TA s0 = 0, s1 = 0;
            if (i < R) {
                int q = g;
                for (; q + G < ng; q += 2 * G) {
                    TA e0[V], e1[V];
                    grp((int64_t)q * R + i, e0);
                    grp((int64_t)(q + G) * R + i, e1);
#pragma unroll
                    for (int u = 0; u < V; ++u) {
                        s0 += e0[u] * xval(y, rc.x0, q * V + u, rc.ncols);
                        s1 += e1[u] * xval(y, rc.x0, (q + G) * V + u, rc.ncols);
                    }
                }
                if (q < ng) {
                    TA e0[V];
                    grp((int64_t)q * R + i, e0);
#pragma unroll
                    for (int u = 0; u < V; ++u) s0 += e0[u] * xval(y, rc.x0, q * V + u, rc.ncols);
                }
            }
            const TA sdot = group_sum<TA>(s0 + s1, RB);
            __syncwarp();
            if (g == 0 && i < R) tw[idx8(i)] = sdot;
            __syncwarp();
            acc -= tw[lane];
            if ((rc.flags & SN_LAST) && lane < L) v[rc.t0 + lane] = acc;
        } else if (rc.kind == SN_FDIAG) {
            const int RB = pow2_ceil(L), G = 32 / RB;
            const int l = lane & (RB - 1), g = lane / RB;
            const int ng = (rc.ncols + V - 1) / V, rel0 = (int)rc.x0 - (int)rc.t0;
            if (rc.flags & SN_FIRST) dacc = 0;
            if (l < L) {
                for (int q = g; q < ng; q += G) {
                    const int st = max(0, rel0 + q * V);
                    if (l >= st) {
                        TA e0[V];
                        grp((sn_fdiag_off(q, rel0, L, V) + (int64_t)(l - st) * V) / V, e0);
#pragma unroll
                        for (int u = 0; u < V; ++u) dacc += e0[u] * xval(v, rc.x0, q * V + u, rc.ncols);
                    }
                }
            }
            if (rc.flags & SN_LAST) {
                const TA sum = group_sum<TA>(dacc, RB);
                if (g == 0 && l < L) y[rc.t0 + l] = sum;
            }
        } else if (rc.kind == SN_BPANEL) {
            const int RB = pow2_ceil(L), G = 32 / RB;
            const int c = lane & (RB - 1), g = lane / RB;
            const int ng = (rc.rows + V - 1) / V;
            if (rc.flags & SN_FIRST) acc = (g == 0 && c < L) ? y[rc.t0 + c] : (TA)0;
            if (c < L) {
                TA s0 = 0, s1 = 0;
                int q = g;
                for (; q + G < ng; q += 2 * G) {
                    TA e0[V], e1[V];
                    grp((int64_t)q * L + c, e0);
                    grp((int64_t)(q + G) * L + c, e1);
#pragma unroll
                    for (int u = 0; u < V; ++u) {
                        s0 += e0[u] * v[idx16(q * V + u)];
                        s1 += e1[u] * v[idx16((q + G) * V + u)];
                    }
                }
                if (q < ng) {
                    TA e0[V];
                    grp((int64_t)q * L + c, e0);
#pragma unroll
                    for (int u = 0; u < V; ++u) s0 += e0[u] * v[idx16(q * V + u)];
                }
                acc -= s0 + s1;
            }
            if (rc.flags & SN_LAST) {
                const TA sum = group_sum<TA>(acc, RB);
                if (g == 0 && c < L) y[rc.t0 + c] = sum;
            }
        } else if (rc.kind == SN_BDIAG) {
            const int RB = pow2_ceil(L), G = 32 / RB;
            const int c = lane & (RB - 1), g = lane / RB;
            const int ng = (rc.ncols + V - 1) / V, rel0 = (int)rc.x0 - (int)rc.t0;
            if (rc.flags & SN_FIRST) dacc = 0;
            if (c < L) {
                for (int q = g; q < ng; q += G) {
                    const int cnt = min(L, rel0 + q * V + V);
                    if (c < cnt) {
                        TA e0[V];
                        grp((sn_bdiag_off(q, rel0, L, V) + (int64_t)c * V) / V, e0);
#pragma unroll
                        for (int u = 0; u < V; ++u) dacc += e0[u] * xval(y, rc.x0, q * V + u, rc.ncols);
                    }
                }
            }
            if (rc.flags & SN_LAST) {
                const TA sum = group_sum<TA>(dacc, RB);
                if (g == 0 && c < L) v[rc.t0 + c] = sum;
            }
        }
        __syncwarp();
        consumed += rc.bytes;
    }
    if (!ok) {
        if (lane == 0) {
            atomicExch(a.err, 1);
            flag[0] = 1;
        }
        for (; bars_done < nbar; ++bars_done) __syncthreads();
        // copies still in flight land in this warp's ring: wait for them (bounded)
        for (; landed < issued; ++landed) mbar_wait(smem_u32(&bar[landed % kSlots]), (uint32_t)((landed / kSlots) & 1));
    }
    __syncthreads();
    if (flag[0]) return;
    for (int i = tid; i < n; i += NT) {
        double x;
        if (f32) x = (double)((float)v[i] * (a.scale32 ? a.scale32[g0 + i] : 1.0f));
        else x = (double)v[i] * (a.scale ? a.scale[g0 + i] : 1.0);
        if (a.accumulate) out[i] += x;
        else out[i] = x;
    }
}

// ---------------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------------
template <typename TW>
cudaError_t launch_sn_factor(const SnTables& t, int m, int max_part, const int32_t* order, const int32_t* rowptr,
                             const int32_t* col, const double* val, const double* dloc, const double* sc, TW* work,
                             TW* dwork, int* err, cudaStream_t st) {
    const size_t smem = ((size_t)max_part * sizeof(uint16_t) + 15) & ~(size_t)15;
    cudaError_t e = cudaFuncSetAttribute(k_sn_factor<TW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_sn_factor<TW><<<m, 256, smem, st>>>(t, order, rowptr, col, val, dloc, sc, work, dwork, err);
    count_launch();
    return cudaGetLastError();
}

template <typename TW, typename TS>
cudaError_t launch_sn_fill(const SnTables& t, const SnFill* fill, int64_t nfill, const TW* work, const TW* dwork,
                           uint8_t* stream, cudaStream_t st) {
    if (nfill == 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((nfill + 7) / 8, 148 * 32);
    k_sn_fill<TW, TS><<<(int)blocks, 256, 0, st>>>(t, fill, nfill, work, dwork, stream);
    count_launch();
    return cudaGetLastError();
}

constexpr int kSolveWarps = 8;
int sn_solve_warps() { return kSolveWarps; }
// a record must land while the next chunk is still free to be issued
int sn_max_record() { return kRing - kChunk; }

size_t sn_solve_smem(int max_part, size_t ta_bytes) {
    return (size_t)kSolveWarps * kRing + (size_t)kSolveWarps * kSlots * 8 + (size_t)kSolveWarps * 32 * ta_bytes +
           16 + 2 * (size_t)((max_part + 3) & ~3) * ta_bytes;
}

template <typename TS, typename TA>
cudaError_t launch_sn_solve(const SnSolveArgs& a, int njobs, int ncols, int max_part, cudaStream_t st) {
    if (njobs == 0 || ncols == 0) return cudaSuccess;
    constexpr int NW = kSolveWarps;
    const size_t smem = sn_solve_smem(max_part, sizeof(TA));
    cudaError_t e = cudaFuncSetAttribute(k_sn_stream<TS, TA, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    SnSolveArgs b = a;
    dim3 grid;
    if (ncols > 1 || a.col_fast) {
        b.col_fast = 1;
        grid = dim3(ncols, njobs);
    } else {
        b.col_fast = 0;
        grid = dim3(njobs);
    }
    k_sn_stream<TS, TA, NW><<<grid, NW * 32, smem, st>>>(b);
    count_launch();
    return cudaGetLastError();
}

template cudaError_t launch_sn_factor<float>(const SnTables&, int, int, const int32_t*, const int32_t*, const int32_t*,
                                             const double*, const double*, const double*, float*, float*, int*,
                                             cudaStream_t);
template cudaError_t launch_sn_factor<double>(const SnTables&, int, int, const int32_t*, const int32_t*, const int32_t*,
                                              const double*, const double*, const double*, double*, double*, int*,
                                              cudaStream_t);
template cudaError_t launch_sn_fill<double, double>(const SnTables&, const SnFill*, int64_t, const double*,
                                                    const double*, uint8_t*, cudaStream_t);
template cudaError_t launch_sn_fill<float, float>(const SnTables&, const SnFill*, int64_t, const float*, const float*,
                                                  uint8_t*, cudaStream_t);
template cudaError_t launch_sn_fill<float, __nv_bfloat16>(const SnTables&, const SnFill*, int64_t, const float*,
                                                          const float*, uint8_t*, cudaStream_t);
template cudaError_t launch_sn_solve<double, double>(const SnSolveArgs&, int, int, int, cudaStream_t);
template cudaError_t launch_sn_solve<float, float>(const SnSolveArgs&, int, int, int, cudaStream_t);
template cudaError_t launch_sn_solve<__nv_bfloat16, float>(const SnSolveArgs&, int, int, int, cudaStream_t);

}  // namespace am
