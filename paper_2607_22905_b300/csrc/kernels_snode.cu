// Supernodal local factors on sm_103a: the numeric Cholesky factorisation of every A_i
// (Algorithm 1, "compute the Cholesky factorization A_i = L_i L_i^T") in the nested-
// dissection supernodal layout of snode_plan.cpp, and the batched forward/backward
// solves that apply A_i^{-1} for the particular solutions (Eq. def-pbar-local), the MBFs
// (Eq. def-phat-local) and the block-Jacobi smoother (Sec. 5.4).
//
// Storage per supernode J (w columns, row structure R_J of nr rows):
//   D_J = L_JJ^{-1}, packed lower triangle, twice: column-major (forward sweep: lane =
//       row, so a column is read with consecutive lanes) and row-major (backward sweep:
//       lane = column);
//   P_J = L_{R_J, J}, nr x w, twice: column-major (forward: lane = row of R_J) and
//       row-major (backward: lane = column of J).
// Both copies of an entry are rounded from the same FP32/FP64 value, so the backward
// sweep applies exactly the transpose of what the forward sweep applies and the local
// solve stays symmetric after rounding.
#include "common.cuh"
#include "kernels.h"

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
// Solve streams from the factor: per supernode (one CTA), the panel L_{R_J,J} in column-
// and row-major order and D_J in column- and row-major packed order, in precision TS.
// ---------------------------------------------------------------------------------
template <typename TW, typename TS>
__global__ void __launch_bounds__(256) k_sn_finalize(SnTables t, int nsn, const TW* __restrict__ work,
                                                     const TW* __restrict__ dwork, TS* __restrict__ Pf,
                                                     TS* __restrict__ Pb, TS* __restrict__ Df, TS* __restrict__ Db) {
    for (int J = blockIdx.x; J < nsn; J += gridDim.x) {
        const int w = t.w[J], nr = t.nr[J], h = w + nr;
        const TW* F = work + t.foff[J];
        const TW* D = dwork + t.doff[J];
        const int64_t po = t.poff[J], dof = t.doff[J];
        for (int64_t e = threadIdx.x; e < (int64_t)nr * w; e += blockDim.x) {
            const int i = (int)(e / w), c = (int)(e % w);
            const TS v = stf<TS>((double)F[(w + i) + (int64_t)c * h]);
            Pb[po + (int64_t)i * w + c] = v;
            Pf[po + (int64_t)c * nr + i] = v;
        }
        for (int64_t e = threadIdx.x; e < (int64_t)w * (w + 1) / 2; e += blockDim.x) {
            int r = (int)((sqrt(8.0 * (double)e + 1.0) - 1.0) * 0.5);
            while (rpack(r + 1, 0) <= e) ++r;
            while (rpack(r, 0) > e) --r;
            const int c = (int)(e - rpack(r, 0));
            const TS v = stf<TS>((double)D[e]);
            Db[dof + e] = v;
            Df[dof + cpack(r, c, w)] = v;
        }
    }
}

// ---------------------------------------------------------------------------------
// Batched local solves  out = S L^{-T} L^{-1} S in  (S = diag(scale)), one CTA of NW
// warps per job (subdomain, input offset, output offset) and column.  Shared memory: v
// and y (one entry per row of the subdomain) and U (the pushed updates, sum_J |R_J|).
//
// Forward sweep, levels from the leaves up; at a level, with a CTA barrier after each
// phase:  pull    v_r -= sum of U entries targeting row r (fixed order)   [rows of J]
//         diag    y_J = D_J v_J                                           [rows of J]
//         push    U_J = L_{R_J,J} y_J                                     [rows of R_J]
// Backward sweep, levels from the top down:
//         panel   y_J = y_J - L_{R_J,J}^T v_{R_J}   (ancestors' final values in v)
//         diag    v_J = D_J^T y_J
// Work units are (supernode, 32-row chunk), dealt round-robin to the warps; lane = row
// for column-major streams, lane = column for row-major ones, so every stream read is a
// run of consecutive addresses across the lanes.
// ---------------------------------------------------------------------------------
template <typename TS, typename TA, int NW>
__global__ void __launch_bounds__(NW * 32) k_sn_solve(SnSolveArgs a) {
    const int col = a.col_fast ? blockIdx.x : 0;
    const int job = a.col_fast ? blockIdx.y : blockIdx.x;
    if (a.done && a.done[col * a.done_stride]) return;
    const SnTables& t = a.t;
    const int s = a.job_sub[job];
    const int64_t g0 = t.sub_off[s];
    const int n = (int)(t.sub_off[s + 1] - g0);
    const int npad = (n + 3) & ~3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TA* v = reinterpret_cast<TA*>(smem_raw);
    TA* y = v + npad;
    TA* U = y + npad;
    const TS* Pf = (const TS*)a.Pf;
    const TS* Pb = (const TS*)a.Pb;
    const TS* Df = (const TS*)a.Df;
    const TS* Db = (const TS*)a.Db;
    const double* in = a.in + a.job_in[job] + col * a.ldin;
    double* out = a.out + a.job_out[job] + col * a.ldout;
    const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
    constexpr int NT = NW * 32;
    const bool f32 = sizeof(TA) == 4;
    for (int i = tid; i < n; i += NT) {
        if (f32) v[i] = (TA)((float)in[i] * (a.scale32 ? a.scale32[g0 + i] : 1.0f));
        else v[i] = (TA)(in[i] * (a.scale ? a.scale[g0 + i] : 1.0));
    }
    __syncthreads();
    const int sn0 = t.sn_off[s], nlev = t.nlev[s], l0 = t.lev0[s];
    // ----- forward: L y = v -----
    for (int lv = 0; lv < nlev; ++lv) {
        const int gl = l0 + lv;
        const int du0 = t.lev_du[gl], du1 = t.lev_du[gl + 1];
        for (int u = du0 + wp; u < du1; u += NW) {
            const uint32_t pk = t.du[u];
            const int J = sn0 + (int)(pk >> 10), q = (int)(pk & 1023);
            const int rr = q * TILE + lane;
            if (rr < t.w[J]) {
                const int r = t.c0[J] + rr;
                TA acc = v[r];
                const int k1 = t.inv_ptr[g0 + r + 1];
                for (int k = t.inv_ptr[g0 + r]; k < k1; ++k) acc -= U[t.inv_idx[k]];
                v[r] = acc;
            }
        }
        __syncthreads();
        for (int u = du0 + wp; u < du1; u += NW) {
            const uint32_t pk = t.du[u];
            const int J = sn0 + (int)(pk >> 10), q = (int)(pk & 1023);
            const int w = t.w[J], c0 = t.c0[J];
            const int rr = q * TILE + lane;
            const TS* Dj = Df + t.doff[J];
            const int cend = min(w, q * TILE + TILE);
            TA a0 = 0, a1 = 0;
            int c = 0;
            if (rr < w) {
                for (; c + 1 < cend && c + 1 <= rr; c += 2) {
                    a0 += ldf<TA, TS>(Dj + cpack(rr, c, w)) * v[c0 + c];
                    a1 += ldf<TA, TS>(Dj + cpack(rr, c + 1, w)) * v[c0 + c + 1];
                }
                for (; c <= rr; ++c) a0 += ldf<TA, TS>(Dj + cpack(rr, c, w)) * v[c0 + c];
                y[c0 + rr] = a0 + a1;
            }
        }
        __syncthreads();
        const int pu0 = t.lev_pu[gl], pu1 = t.lev_pu[gl + 1];
        for (int u = pu0 + wp; u < pu1; u += NW) {
            const uint32_t pk = t.pu[u];
            const int J = sn0 + (int)(pk >> 10), q = (int)(pk & 1023);
            const int w = t.w[J], nr = t.nr[J], c0 = t.c0[J];
            const int i = q * TILE + lane;
            if (i < nr) {
                const TS* Pj = Pf + t.poff[J] + i;
                TA a0 = 0, a1 = 0, a2 = 0, a3 = 0;
                int c = 0;
                for (; c + 3 < w; c += 4) {
                    a0 += ldf<TA, TS>(Pj + (int64_t)c * nr) * y[c0 + c];
                    a1 += ldf<TA, TS>(Pj + (int64_t)(c + 1) * nr) * y[c0 + c + 1];
                    a2 += ldf<TA, TS>(Pj + (int64_t)(c + 2) * nr) * y[c0 + c + 2];
                    a3 += ldf<TA, TS>(Pj + (int64_t)(c + 3) * nr) * y[c0 + c + 3];
                }
                for (; c < w; ++c) a0 += ldf<TA, TS>(Pj + (int64_t)c * nr) * y[c0 + c];
                U[t.uoff[J] + i] = (a0 + a1) + (a2 + a3);
            }
        }
        __syncthreads();
    }
    // ----- backward: L^T x = y -----
    for (int lv = nlev - 1; lv >= 0; --lv) {
        const int gl = l0 + lv;
        const int du0 = t.lev_du[gl], du1 = t.lev_du[gl + 1];
        for (int u = du0 + wp; u < du1; u += NW) {
            const uint32_t pk = t.du[u];
            const int J = sn0 + (int)(pk >> 10), q = (int)(pk & 1023);
            const int w = t.w[J], nr = t.nr[J], c0 = t.c0[J];
            const int c = q * TILE + lane;
            if (c < w) {
                const TS* Pj = Pb + t.poff[J] + c;
                const uint16_t* R = t.rows + t.roff[J];
                TA a0 = y[c0 + c], a1 = 0, a2 = 0, a3 = 0;
                int i = 0;
                for (; i + 3 < nr; i += 4) {
                    a0 -= ldf<TA, TS>(Pj + (int64_t)i * w) * v[R[i]];
                    a1 -= ldf<TA, TS>(Pj + (int64_t)(i + 1) * w) * v[R[i + 1]];
                    a2 -= ldf<TA, TS>(Pj + (int64_t)(i + 2) * w) * v[R[i + 2]];
                    a3 -= ldf<TA, TS>(Pj + (int64_t)(i + 3) * w) * v[R[i + 3]];
                }
                for (; i < nr; ++i) a0 -= ldf<TA, TS>(Pj + (int64_t)i * w) * v[R[i]];
                y[c0 + c] = (a0 + a1) + (a2 + a3);
            }
        }
        __syncthreads();
        for (int u = du0 + wp; u < du1; u += NW) {
            const uint32_t pk = t.du[u];
            const int J = sn0 + (int)(pk >> 10), q = (int)(pk & 1023);
            const int w = t.w[J], c0 = t.c0[J];
            const int c = q * TILE + lane;
            if (c < w) {
                const TS* Dj = Db + t.doff[J];
                TA a0 = 0, a1 = 0;
                int r = c;
                for (; r + 1 < w; r += 2) {
                    a0 += ldf<TA, TS>(Dj + rpack(r, c)) * y[c0 + r];
                    a1 += ldf<TA, TS>(Dj + rpack(r + 1, c)) * y[c0 + r + 1];
                }
                for (; r < w; ++r) a0 += ldf<TA, TS>(Dj + rpack(r, c)) * y[c0 + r];
                v[c0 + c] = a0 + a1;
            }
        }
        __syncthreads();
    }
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
cudaError_t launch_sn_finalize(const SnTables& t, int nsn, const TW* work, const TW* dwork, TS* Pf, TS* Pb, TS* Df,
                               TS* Db, cudaStream_t st) {
    if (nsn == 0) return cudaSuccess;
    k_sn_finalize<TW, TS><<<min(nsn, 148 * 16), 256, 0, st>>>(t, nsn, work, dwork, Pf, Pb, Df, Db);
    count_launch();
    return cudaGetLastError();
}

size_t sn_solve_smem(int max_part, int max_usum, size_t ta_bytes) {
    return (2 * (size_t)((max_part + 3) & ~3) + (size_t)max_usum) * ta_bytes;
}

template <typename TS, typename TA>
cudaError_t launch_sn_solve(const SnSolveArgs& a, int njobs, int ncols, int max_part, int max_usum, cudaStream_t st) {
    if (njobs == 0 || ncols == 0) return cudaSuccess;
    constexpr int NW = 8;
    const size_t smem = sn_solve_smem(max_part, max_usum, sizeof(TA));
    cudaError_t e = cudaFuncSetAttribute(k_sn_solve<TS, TA, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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
    k_sn_solve<TS, TA, NW><<<grid, NW * 32, smem, st>>>(b);
    count_launch();
    return cudaGetLastError();
}

template cudaError_t launch_sn_factor<float>(const SnTables&, int, int, const int32_t*, const int32_t*, const int32_t*,
                                             const double*, const double*, const double*, float*, float*, int*,
                                             cudaStream_t);
template cudaError_t launch_sn_factor<double>(const SnTables&, int, int, const int32_t*, const int32_t*, const int32_t*,
                                              const double*, const double*, const double*, double*, double*, int*,
                                              cudaStream_t);
template cudaError_t launch_sn_finalize<double, double>(const SnTables&, int, const double*, const double*, double*,
                                                        double*, double*, double*, cudaStream_t);
template cudaError_t launch_sn_finalize<float, float>(const SnTables&, int, const float*, const float*, float*, float*,
                                                      float*, float*, cudaStream_t);
template cudaError_t launch_sn_finalize<float, __nv_bfloat16>(const SnTables&, int, const float*, const float*,
                                                              __nv_bfloat16*, __nv_bfloat16*, __nv_bfloat16*,
                                                              __nv_bfloat16*, cudaStream_t);
template cudaError_t launch_sn_solve<double, double>(const SnSolveArgs&, int, int, int, int, cudaStream_t);
template cudaError_t launch_sn_solve<float, float>(const SnSolveArgs&, int, int, int, int, cudaStream_t);
template cudaError_t launch_sn_solve<__nv_bfloat16, float>(const SnSolveArgs&, int, int, int, int, cudaStream_t);

}  // namespace am
