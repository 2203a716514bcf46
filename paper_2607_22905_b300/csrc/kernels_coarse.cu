// Interface (coarse) system of AlgMortar on sm_103a: assembly of
//   S_eta = diag(T) + 1/4 G^T Phi     (Eq. interface-problem-alg with W M = B^T / 4,
//                                       Prop. proposition-BWM; SPD by Cor. cor-schur-eta)
// and its exact FP64 solve  eta = S_eta^{-1} b_eta  (Algorithm 2, "solve the interface
// system") by one level of nested dissection:
//
//   S = [ S_11 ..      S_1G  ]      interior blocks S_gg: interfaces whose two subdomains
//       [       S_GG   S_GG' ]      lie in group g; separator: all other interfaces.
//       [ S_G'1 ...    S_G'G']
//
//   y_g  = S_gg^{-1} b_g,   P_g = W_g^T b_g  with  W_g = S_gg^{-1} S_{g,A_g}
//   eta_sep = C^{-1} (b_sep - sum_g P_g),   C = S_sep,sep - sum_g S_{A_g,g} W_g
//   eta_g = y_g - W_g eta_{A_g}
//
// (A_g: separator unknowns coupled to group g.)  Every per-iteration product runs as a
// wide warp-per-row GEMV over all SMs (FP64 ALU-bound on B300), with no sequential
// triangular sweep on the critical path.
#include <algorithm>
#include <type_traits>
#include <vector>

#include "async.cuh"
#include "common.cuh"
#include "kernels.h"
#include "tile_chol.cuh"

namespace am {

// ---------------------------------------------------------------------------------
// Value-dependent interface tables, recomputed for every numeric setup:
//   c_k^(I) = sum of row k's couplings a_kl to the other subdomain of interface I
//   r_coef  = -1/2 c_k^(I)          (restriction, b_eta = -1/4 G^T pbar)
//   G[k, I] = 2 c_k^(I) = -4 r_coef (coupling B psi_I, Eq. Bij-contrib)
//   T_I     = sum_{(k,l) in E_I} |a_kl| = sum over both sides of -1/2 c_k^(I)
// ---------------------------------------------------------------------------------
__global__ void k_iface_coef(int64_t nr, const int64_t* __restrict__ rp_ptr, const int32_t* __restrict__ rp_pos,
                             const double* __restrict__ val, double* __restrict__ rcoef) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nr; t += (int64_t)gridDim.x * blockDim.x) {
        double c = 0.0;
        for (int64_t e = rp_ptr[t]; e < rp_ptr[t + 1]; ++e) c += val[rp_pos[e]];
        rcoef[t] = -0.5 * c;
    }
}

__global__ void k_iface_T_g(int L, const int64_t* __restrict__ r_ptr, const double* __restrict__ rcoef,
                            double* __restrict__ T, int64_t ng, const int32_t* __restrict__ g_from_r,
                            double* __restrict__ gval) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < L) {
        double s = 0.0;
        for (int64_t t = r_ptr[i]; t < r_ptr[i + 1]; ++t) s += rcoef[t];
        T[i] = s;
    }
    for (int64_t u = i; u < ng; u += (int64_t)gridDim.x * blockDim.x) gval[u] = -4.0 * rcoef[g_from_r[u]];
}

// ---------------------------------------------------------------------------------
// Assembly into a dense, ND-ordered, symmetric n_lambda x n_lambda matrix Sd (row-major).
// One CTA per subdomain; one warp per pair (a <= b) of its interfaces; off-diagonal
// entries come from the single subdomain the two interfaces share (symmetrised there),
// diagonal contributions of both sides are summed in a fixed order by k_nd_diag.
// ---------------------------------------------------------------------------------
__global__ void k_nd_assemble(NdAssembleArgs a) {
    const int s = blockIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t i0 = a.if_off[s];
    const int k = (int)(a.if_off[s + 1] - i0);
    const int64_t ns = a.rows[s];
    const double* phi = a.phi + a.phi_off[s];
    const int64_t* cp = a.g_cptr + i0 + s;
    const int64_t L = a.L;
    for (int pr = w; pr < k * k; pr += nw) {
        const int ai = pr / k, bi = pr % k;
        if (bi < ai) continue;
        double cab = 0.0, cba = 0.0;
        for (int64_t t = cp[ai] + lane; t < cp[ai + 1]; t += 32)
            cab += a.g_val[t] * phi[bi * ns + a.g_row[t]];
        for (int64_t t = cp[bi] + lane; t < cp[bi + 1]; t += 32)
            cba += a.g_val[t] * phi[ai * ns + a.g_row[t]];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            cab += __shfl_xor_sync(0xffffffffu, cab, o);
            cba += __shfl_xor_sync(0xffffffffu, cba, o);
        }
        if (lane == 0) {
            const int I = a.if_list[i0 + ai], J = a.if_list[i0 + bi];
            if (ai == bi) {
                const int side = (a.pairs[2 * I] == s) ? 0 : 1;
                a.diagc[2 * I + side] = 0.25 * cab;
            } else if (!a.Sd) {
                const double v = 0.125 * (cab + cba);
                a.pv[a.pv_off[s] + (int64_t)ai * k + bi] = v;
                a.pv[a.pv_off[s] + (int64_t)bi * k + ai] = v;
            } else {
                const int64_t p = a.nd_pos[I], q = a.nd_pos[J];
                const double v = 0.125 * (cab + cba);
                a.Sd[p * L + q] = v;
                a.Sd[q * L + p] = v;
            }
        }
    }
}

__global__ void k_nd_diag(int L, const double* __restrict__ T, const double* __restrict__ diagc,
                          const int32_t* __restrict__ nd_pos, double* __restrict__ Sd) {
    int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= L) return;
    int64_t p = nd_pos[I];
    Sd[p * L + p] = T[I] + diagc[2 * I] + diagc[2 * I + 1];
}

// Dense lower tile storage of an n x n block (tile (I, J), J <= I, at I(I+1)/2 + J,
// column-major inside the tile) from a row-major source with leading dimension ld;
// padding rows get a unit diagonal.  One CTA per tile, items laid out by `base`.
template <typename T>
__global__ void k_dense_to_tiles(const double* __restrict__ src, int64_t ld, const int64_t* __restrict__ src_off,
                                 const int32_t* __restrict__ rows, const int64_t* __restrict__ base,
                                 const int32_t* __restrict__ tile_item, const int32_t* __restrict__ tile_I,
                                 const int32_t* __restrict__ tile_J, T* __restrict__ work) {
    const int64_t t = blockIdx.x;
    const int g = tile_item[t], I = tile_I[t], J = tile_J[t];
    const int n = rows[g];
    const double* S = src + src_off[g];
    T* dst = work + (base[g] + (int64_t)I * (I + 1) / 2 + J) * TILE2;
    for (int e = threadIdx.x; e < TILE2; e += blockDim.x) {
        const int r = I * TILE + (e & 31), c = J * TILE + (e >> 5);
        double v;
        if (r < n && c < n) v = S[(int64_t)r * ld + c];
        else v = (r == c) ? 1.0 : 0.0;
        dst[e] = (T)v;
    }
}

// Column-major square blocks whose lower triangle holds a symmetric matrix: copy it to
// the upper triangle (M[j][i] = M[i][j] for i > j).
__global__ void k_mirror_lower(const int32_t* __restrict__ rows, const int64_t* __restrict__ off, int nitems,
                               double* __restrict__ M) {
    const int g = blockIdx.y;
    if (g >= nitems) return;
    const int64_t n = rows[g];
    double* A = M + off[g];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / n, r = e % n;     // column c, row r (column-major element e)
        if (r < c) A[e] = A[r * n + c];          // (r, c) above the diagonal <- (c, r) below it
    }
}

// Row-major copy of the column-major n_g x a_g blocks W_g.
__global__ void k_transpose_blocks(const int64_t* __restrict__ goff, const int64_t* __restrict__ aoff,
                                   const int64_t* __restrict__ woff, int G, const double* __restrict__ Wcm,
                                   double* __restrict__ Wrm) {
    const int g = blockIdx.y;
    if (g >= G) return;
    const int64_t ng = goff[g + 1] - goff[g], ag = aoff[g + 1] - aoff[g];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ng * ag;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / ag, j = e % ag;
        Wrm[woff[g] + e] = Wcm[woff[g] + j * ng + i];
    }
}

// W_g = S_gg^{-1} S_{g,A_g} from the explicit symmetric inverse and the sparse coupling
// block: S_{g,A_g} has a nonzero (i, a) only where interior interface i and separator
// interface a share a subdomain, so column a of W_g is a short combination of columns
// of S_gg^{-1} (n_g * nnz FMAs instead of the n_g^2 * |A_g| of triangular solves).
// One CTA per column r (group prow_g[r], local column r - aoff[g]); the coupling rows
// wc_row[wc_ptr[r] .. wc_ptr[r+1]) are local interior indices, values read from Sd.
__global__ void k_nd_w_sparse(int64_t L, const double* __restrict__ Sd, const int64_t* __restrict__ goff,
                              const int64_t* __restrict__ aoff, const int32_t* __restrict__ alist, int64_t sep0,
                              const int32_t* __restrict__ prow_g, const int64_t* __restrict__ wc_ptr,
                              const int32_t* __restrict__ wc_row, const int64_t* __restrict__ gioff,
                              const double* __restrict__ Ginv, const int64_t* __restrict__ woff,
                              double* __restrict__ Wcm) {
    constexpr int MAXNZ = 256;
    __shared__ double sv[MAXNZ];
    __shared__ int32_t si[MAXNZ];
    const int64_t r = blockIdx.x;
    const int g = prow_g[r];
    const int64_t g0 = goff[g], ng = goff[g + 1] - g0, j = r - aoff[g];
    const int64_t q = sep0 + alist[aoff[g] + j];
    const double* Gi = Ginv + gioff[g];
    double* out = Wcm + woff[g] + j * ng;
    for (int64_t t0 = wc_ptr[r]; t0 < wc_ptr[r + 1]; t0 += MAXNZ) {
        const int cnt = (int)min((int64_t)MAXNZ, wc_ptr[r + 1] - t0);
        __syncthreads();
        for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
            const int32_t i = wc_row[t0 + t];
            si[t] = i;
            sv[t] = Sd[(g0 + i) * L + q];
        }
        __syncthreads();
        for (int64_t k = threadIdx.x; k < ng; k += blockDim.x) {
            double a0 = 0.0, a1 = 0.0;
            int t = 0;
            for (; t + 1 < cnt; t += 2) {
                a0 += Gi[(int64_t)si[t] * ng + k] * sv[t];
                a1 += Gi[(int64_t)si[t + 1] * ng + k] * sv[t + 1];
            }
            if (t < cnt) a0 += Gi[(int64_t)si[t] * ng + k] * sv[t];
            if (t0 == wc_ptr[r]) out[k] = a0 + a1;
            else out[k] += a0 + a1;
        }
    }
    if (wc_ptr[r] == wc_ptr[r + 1])
        for (int64_t k = threadIdx.x; k < ng; k += blockDim.x) out[k] = 0.0;
}

// D_g = S_{A_g,g} W_g with the same sparse pattern: row j of D_g is sum over the coupling
// rows i of S(i, a_j) W_g[i, :] (row-major copy of W_g).  One warp per (g, j).
__global__ void k_nd_schur_sparse(int64_t L, int64_t np, const double* __restrict__ Sd,
                                  const int64_t* __restrict__ goff, const int64_t* __restrict__ aoff,
                                  const int32_t* __restrict__ alist, int64_t sep0, const int32_t* __restrict__ prow_g,
                                  const int64_t* __restrict__ wc_ptr, const int32_t* __restrict__ wc_row,
                                  const int64_t* __restrict__ woff, const double* __restrict__ Wrm,
                                  const int64_t* __restrict__ doff, double* __restrict__ D) {
    const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= np) return;
    const int g = prow_g[r];
    const int64_t g0 = goff[g], ag = aoff[g + 1] - aoff[g], j = r - aoff[g];
    const int64_t q = sep0 + alist[aoff[g] + j];
    const double* Wg = Wrm + woff[g];
    double* out = D + doff[g] + j * ag;
    for (int64_t k = lane; k < ag; k += 32) {
        double acc = 0.0;
        for (int64_t t = wc_ptr[r]; t < wc_ptr[r + 1]; ++t) {
            const int32_t i = wc_row[t];
            acc += Sd[(g0 + i) * L + q] * Wg[(int64_t)i * ag + k];
        }
        out[k] = acc;
    }
}

// Lower tiles of C = S_sep,sep - sum_g D_g (symmetrised), one CTA per tile.
template <typename T>
__global__ void k_nd_schur_tiles(int64_t L, int nsep, int64_t sep0, const double* __restrict__ Sd,
                                 const int32_t* __restrict__ sg, const int32_t* __restrict__ sidx,
                                 const int64_t* __restrict__ aoff, const int64_t* __restrict__ doff,
                                 const double* __restrict__ D, T* __restrict__ work) {
    const int64_t t = blockIdx.x;
    int I = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((int64_t)(I + 1) * (I + 2) / 2 <= t) ++I;
    while ((int64_t)I * (I + 1) / 2 > t) --I;
    const int J = (int)(t - (int64_t)I * (I + 1) / 2);
    T* dst = work + t * TILE2;
    for (int e = threadIdx.x; e < TILE2; e += blockDim.x) {
        const int s = I * TILE + (e & 31), u = J * TILE + (e >> 5);
        double v;
        if (s < nsep && u < nsep) {
            double cs = Sd[(sep0 + s) * L + sep0 + u], ct = Sd[(sep0 + u) * L + sep0 + s];
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b)
                    if (sg[2 * s + a] == sg[2 * u + b]) {
                        const int g = sg[2 * s + a];
                        const int64_t ag = aoff[g + 1] - aoff[g];
                        cs -= D[doff[g] + sidx[2 * s + a] * ag + sidx[2 * u + b]];
                        ct -= D[doff[g] + sidx[2 * u + b] * ag + sidx[2 * s + a]];
                    }
            v = 0.5 * (cs + ct);
        } else {
            v = (s == u) ? 1.0 : 0.0;
        }
        dst[e] = (T)v;
    }
}

// TF32 operand planes of a finished 32x32 factor tile for the tensor-core update (FP32
// interface factorization): plane 0 holds the tile itself (the tensor core reads the top
// 19 bits of each value, its TF32 rounding toward zero), plane 1 the remainder x - tf32(x);
// both in the K-major no-swizzle core-matrix layout with the tile's row r as the M/N index
// and its column c as K: float offset (r/8)*256 + (c/4)*32 + (r%8)*4 + c%4.  The product
// hi*hi + hi*lo + lo*hi (3xTF32) then carries ~FP32 accuracy.
__host__ __device__ __forceinline__ int plane_off(int r, int c) {
    return (r >> 3) * 256 + (c >> 2) * 32 + (r & 7) * 4 + (c & 3);
}
__device__ __forceinline__ void put_planes(float* planes, int r, int c, float x) {
    planes[plane_off(r, c)] = x;
    planes[TILE2 + plane_off(r, c)] = x - __int_as_float(__float_as_int(x) & 0xffffe000);
}
template <typename TW>
__device__ __forceinline__ void put_planes(TW*, int, int, TW) {}

__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }

// ---------------------------------------------------------------------------------
// Right-looking Cholesky of a batch of DENSE items (the interface blocks), all items
// advancing tile column k together: tile (I, J) of item g at base[g] + I(I+1)/2 + J,
// column-major inside the tile; inverse diagonal tiles at dinv + (row0[g] + I) tiles.
// ---------------------------------------------------------------------------------
// Four warps factor the 32x32 tile A_kk and invert the factor.  B300's FP64 rate is
// ~1.9 FMA per clock per SM, i.e. a single warp's FP64 instruction occupies its SM
// sub-partition for ~68 cycles, so the tile's FP64 work is spread over the four
// sub-partitions: warp w owns columns w, w + 4, ... (row `lane` of them in registers).
//   factor: at step kk every warp applies column kk to its columns right of kk; the
//     owner of column kk + 1 updates that column first, then scales it by 1/sqrt(pivot)
//     (one reciprocal square root, L_cc = pivot * rsqrt(pivot)) and publishes it, so the
//     pivot's dependent FP64 chain overlaps the other warps' updates (one-column
//     lookahead; one barrier per column);
//   inverse: with D = diag(L) and the unit lower N = D^{-1} L, L^{-1} = N^{-1} D^{-1};
//     the columns of N^{-1} are independent, so each warp forward-substitutes its own 8
//     columns (rows final in order, row r broadcast by shuffle) and scales them.
template <typename TW>
__global__ void __launch_bounds__(128) k_dpotrf_b(int nitems, const int32_t* __restrict__ T,
                                                  const int64_t* __restrict__ base,
                                                  const int64_t* __restrict__ row0, TW* __restrict__ work,
                                                  TW* __restrict__ dinv, int k, int* __restrict__ err,
                                                  TW* __restrict__ planes) {
    __shared__ TW Ls[TILE][TILE + 1];   // L (column c published at step c - 1)
    __shared__ TW rd_s[TILE];           // 1 / L[c][c]
    __shared__ int bad_s;
    const int g = blockIdx.x;
    if (g >= nitems || k >= T[g]) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    TW* t = work + (base[g] + (int64_t)k * (k + 1) / 2 + k) * TILE2;
    TW a[8];   // a[j]: row `lane` of column w + 4 j
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = t[(w + 4 * j) * TILE + lane];
    if (threadIdx.x == 0) bad_s = 0;
    __syncthreads();
    // owner warp of column c = w + 4 j: scale it by 1 / sqrt(pivot) and publish it
    auto pivot = [&](int c, TW& aj) {
        TW piv = __shfl_sync(0xffffffffu, aj, c);
        if (!(piv > 0.0) || !isfinite(piv)) {
            if (lane == 0) bad_s = 1;
            piv = TW(1);
        }
        const TW rs = rsq(piv);
        const TW lk = lane > c ? aj * rs : (lane == c ? piv * rs : TW(0));
        aj = lk;
        Ls[lane][c] = lk;
        if (lane == 0) rd_s[c] = rs;
    };
    if (w == 0) pivot(0, a[0]);
    for (int kk = 0; kk < TILE; ++kk) {
        __syncthreads();   // column kk published
        const TW lk = Ls[lane][kk];
        const int nx = kk + 1;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c = w + 4 * j;
            if (c == nx) {   // lookahead: column kk + 1 first, then its pivot
                if (lane >= c) a[j] -= lk * Ls[c][kk];
                pivot(c, a[j]);
            }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c = w + 4 * j;
            if (c > nx && lane >= c) a[j] -= lk * Ls[c][kk];
        }
    }
    // every column of L is in Ls now (published before the last step's barrier)
    TW x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = (w + 4 * j == lane) ? 1.0 : 0.0;
    const TW rdl = rd_s[lane];
    for (int r = 0; r < TILE; ++r) {
        const TW nr = lane > r ? Ls[lane][r] * rdl : TW(0);     // N[lane][r]
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (w + 4 * j > r) continue;                         // N^{-1} is lower triangular
            const TW yrc = __shfl_sync(0xffffffffu, x[j], r);
            x[j] -= nr * yrc;
        }
    }
    TW* D = dinv + (row0[g] + k) * TILE2;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int c = w + 4 * j;
        t[c * TILE + lane] = c <= lane ? Ls[lane][c] : TW(0);
        D[c * TILE + lane] = x[j] * rd_s[c];
        if (planes)
            put_planes(planes + (base[g] + (int64_t)k * (k + 1) / 2 + k) * 2 * TILE2, lane, c,
                       c <= lane ? Ls[lane][c] : TW(0));
    }
    if (threadIdx.x == 0 && bad_s) {
        if (atomicCAS(err + 1, -1, g) == -1) atomicExch(err, 1);
    }
}

// block -> (item, local index) over per-item counts cnt_g(k)
__device__ __forceinline__ int item_of_block(int nitems, const int32_t* T, int k, int64_t b, bool pairs,
                                             int64_t* local) {
    for (int g = 0; g < nitems; ++g) {
        const int64_t w = T[g] - 1 - k;
        const int64_t c = w <= 0 ? 0 : (pairs ? w * (w + 1) / 2 : w);
        if (b < c) {
            *local = b;
            return g;
        }
        b -= c;
    }
    return -1;
}

// L_Ik = A_Ik L_kk^{-T} for I = k+1 .. T_g-1 of every item
template <typename TW>
__global__ void __launch_bounds__(256) k_dtrsm_b(int nitems, const int32_t* __restrict__ T,
                                                 const int64_t* __restrict__ base,
                                                 const int64_t* __restrict__ row0, TW* __restrict__ work,
                                                 const TW* __restrict__ dinv, int k, TW* __restrict__ planes) {
    __shared__ TW X[TILE][TILE + 1];
    __shared__ TW Bs[TILE][TILE + 1];
    int64_t li;
    const int g = item_of_block(nitems, T, k, blockIdx.x, false, &li);
    if (g < 0) return;
    const int I = k + 1 + (int)li;
    const int tid = threadIdx.x, c = tid & 31, rb = (tid >> 5) * 4;
    TW* t = work + (base[g] + (int64_t)I * (I + 1) / 2 + k) * TILE2;
    const TW* D = dinv + (row0[g] + k) * TILE2;
    for (int e = tid; e < TILE2; e += 256) {
        X[e & 31][e >> 5] = t[e];
        Bs[e & 31][e >> 5] = D[e];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        TW v = 0;
#pragma unroll 8
        for (int u = 0; u < TILE; ++u) v += X[rb + q][u] * Bs[c][u];
        t[c * TILE + rb + q] = v;
        if (planes) put_planes(planes + (base[g] + (int64_t)I * (I + 1) / 2 + k) * 2 * TILE2, rb + q, c, v);
    }
}

// Tile column k of every item in one launch: CTA (g, 0) factors A_kk and stores
// L_kk^{-1}; CTA (g, i), i >= 1, factors the same A_kk itself (one warp, registers) and
// solves L_{k+i,k} = A_{k+i,k} L_kk^{-T} (8 outputs per thread), writing the 3xTF32
// planes for the tensor-core update.  Repeating the 32x32 factorization in every CTA
// costs less than a second launch and its serialisation.  FP32 only: one warp of FP64
// would hold one sub-partition's FP64 pipe for the whole tile (k_dpotrf_b spreads it
// over four).
// L_kk itself is not stored: later steps read only the tiles below the diagonal and the
// inverse diagonal tiles.
__device__ __forceinline__ int item_of_block_col(int nitems, const int32_t* T, int k, int64_t b, int64_t* local) {
    for (int g = 0; g < nitems; ++g) {
        const int64_t c = T[g] - k > 0 ? T[g] - k : 0;
        if (b < c) {
            *local = b;
            return g;
        }
        b -= c;
    }
    return -1;
}

template <typename TW>
__global__ void __launch_bounds__(128) k_dpotrf_trsm(int nitems, const int32_t* __restrict__ T,
                                                     const int64_t* __restrict__ base,
                                                     const int64_t* __restrict__ row0, TW* __restrict__ work,
                                                     TW* __restrict__ dinv, int k, int* __restrict__ err,
                                                     TW* __restrict__ planes) {
    __shared__ TW Xd[TILE * (TILE + 1)];   // A_kk, X(r, c) at c * 33 + r
    __shared__ TW Xo[TILE * (TILE + 1)];   // A_Ik
    __shared__ TW Dd[TILE2];               // L_kk^{-1}, column-major
    __shared__ int bad_s;
    int64_t li;
    const int g = item_of_block_col(nitems, T, k, blockIdx.x, &li);
    if (g < 0) return;
    const int I = k + (int)li;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const TW* tkk = work + (base[g] + (int64_t)k * (k + 1) / 2 + k) * TILE2;
    TW* tik = work + (base[g] + (int64_t)I * (I + 1) / 2 + k) * TILE2;
    if (tid == 0) bad_s = 0;
    {
        // all of a thread's loads issued before the first store (one round trip)
        TW xd[TILE2 / 128], xo[TILE2 / 128];
#pragma unroll
        for (int i = 0; i < TILE2 / 128; ++i) {
            xd[i] = tkk[tid + 128 * i];
            xo[i] = li > 0 ? tik[tid + 128 * i] : (TW)0;
        }
#pragma unroll
        for (int i = 0; i < TILE2 / 128; ++i) {
            const int e = tid + 128 * i;
            Xd[(e >> 5) * (TILE + 1) + (e & 31)] = xd[i];
            Xo[(e >> 5) * (TILE + 1) + (e & 31)] = xo[i];
        }
    }
    __syncthreads();
    if (w == 0) warp_chol_inv<TW>(Xd, TILE + 1, nullptr, Dd, lane, &bad_s);
    __syncthreads();
    if (li == 0) {
        TW* D = dinv + (row0[g] + k) * TILE2;
#pragma unroll
        for (int i = 0; i < TILE2 / 128; ++i) D[tid + 128 * i] = Dd[tid + 128 * i];
        if (tid == 0 && bad_s) {
            if (atomicCAS(err + 1, -1, g) == -1) atomicExch(err, 1);
        }
        return;
    }
    // L_Ik(r, c) = sum_u A_Ik(r, u) D(c, u), D(c, u) at u * 32 + c
    const int rb = w * 8;
    TW v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = (TW)0;
#pragma unroll 8
    for (int u = 0; u < TILE; ++u) {
        const TW d = Dd[u * TILE + lane];
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] += Xo[u * (TILE + 1) + rb + q] * d;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        tik[lane * TILE + rb + q] = v[q];
        if (planes) put_planes(planes + (base[g] + (int64_t)I * (I + 1) / 2 + k) * 2 * TILE2, rb + q, lane, v[q]);
    }
}

// A_IJ -= L_Ik L_Jk^T for k < J <= I < T_g of every item
template <typename TW>
__global__ void __launch_bounds__(256) k_dupdate_b(int nitems, const int32_t* __restrict__ T,
                                                   const int64_t* __restrict__ base, TW* __restrict__ work, int k) {
    __shared__ TW As[TILE][TILE + 1];
    __shared__ TW Bs[TILE][TILE + 1];
    int64_t p;
    const int g = item_of_block(nitems, T, k, blockIdx.x, true, &p);
    if (g < 0) return;
    int a = (int)((sqrt(8.0 * (double)p + 1.0) - 1.0) * 0.5);
    while ((int64_t)(a + 1) * (a + 2) / 2 <= p) ++a;
    while ((int64_t)a * (a + 1) / 2 > p) --a;
    const int b = (int)(p - (int64_t)a * (a + 1) / 2);
    const int I = k + 1 + a, J = k + 1 + b;
    const int tid = threadIdx.x, c = tid & 31, rb = (tid >> 5) * 4;
    const TW* LI = work + (base[g] + (int64_t)I * (I + 1) / 2 + k) * TILE2;
    const TW* LJ = work + (base[g] + (int64_t)J * (J + 1) / 2 + k) * TILE2;
    TW* t = work + (base[g] + (int64_t)I * (I + 1) / 2 + J) * TILE2;
    for (int e = tid; e < TILE2; e += 256) {
        As[e & 31][e >> 5] = LI[e];
        Bs[e & 31][e >> 5] = LJ[e];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        TW v = t[c * TILE + rb + q];
#pragma unroll 8
        for (int u = 0; u < TILE; ++u) v -= As[rb + q][u] * Bs[c][u];
        t[c * TILE + rb + q] = v;
    }
}

// ---------------------------------------------------------------------------------
// Left-looking tensor-core update of block column J of the FP32 dense factors:
//   A_IJ -= sum_{k < J} L_Ik L_Jk^T   for I >= J,
// for all items, before the column's diagonal tile is factored and its tiles below solved.
// One CTA per (item, 4 tile rows I0..I0+3): an M = 128, N = 32 product with K = 32 J on
// tcgen05 (kind::tf32, accumulator in tensor memory), 3xTF32 (hi*hi + hi*lo + lo*hi from
// the planes written with the finished tiles), so the update keeps FP32 accuracy.  Stage
// k accumulates into accumulator k % TC_ACC: the MMAs into one accumulator run in order,
// so one accumulator made the column's update a chain of 12 J dependent MMAs.
// Thread 0 streams the k-th planes of the four row tiles and of tile (J, k) into one of
// two shared-memory stages by bulk copies (16-byte aligned 4 KB planes, completion on
// full[s]); thread 32 issues the 12 MMAs of a stage and commits them to empty[s]; at the
// end four warps read the 128 x 32 product (one tile row each) and subtract it.  Every
// wait is bounded; a stuck wait sets *err (the bulk-copy error word) and skips the update.
// ---------------------------------------------------------------------------------
constexpr int TC_STAGES = 2;
constexpr int TC_ACC = 4;   // accumulators in tensor memory: stage k goes to k % TC_ACC
constexpr int TC_PLANE = TILE2 * 4;                          // bytes of one plane
constexpr int TC_STAGE = (4 * 2 + 2) * TC_PLANE;             // A hi, A lo (4 tiles), B hi, B lo
constexpr size_t TC_SMEM = (size_t)TC_STAGES * TC_STAGE + 128;

__global__ void __launch_bounds__(128) k_dupdate_tc(int nitems, const int32_t* __restrict__ T,
                                                    const int64_t* __restrict__ base, float* __restrict__ work,
                                                    const float* __restrict__ planes, int J, int nsplit,
                                                    float* __restrict__ part, unsigned int* __restrict__ ticket,
                                                    int* __restrict__ err) {
    // block -> (item, first tile row, K split)
    const int sp = (int)(blockIdx.x % (unsigned)nsplit);
    const int64_t bq = blockIdx.x / (unsigned)nsplit;   // row block, over all items
    int64_t b = bq;
    int g = -1;
    for (int q = 0; q < nitems; ++q) {
        const int64_t nb = T[q] > J ? (T[q] - J + 3) / 4 : 0;
        if (b < nb) {
            g = q;
            break;
        }
        b -= nb;
    }
    if (g < 0) return;
    const int I0 = J + 4 * (int)b, Tg = T[g];
    const int nA = min(4, Tg - I0);
    const int k0 = (int)((int64_t)J * sp / nsplit), k1 = (int)((int64_t)J * (sp + 1) / nsplit);
    const int nk = k1 - k0;
    extern __shared__ __align__(1024) unsigned char sm[];
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + TC_STAGES * TC_STAGE);
    uint64_t* empty = full + TC_STAGES;
    uint64_t* done = empty + TC_STAGES;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);     // [0] tensor memory, [2] verdict, [3] last
    volatile int* bad = reinterpret_cast<volatile int*>(tslot + 1);
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int64_t g0 = base[g];
    auto tile = [&](int I, int k) { return g0 + (int64_t)I * (I + 1) / 2 + k; };
    if (tid == 0) {
        for (int i = 0; i < TC_STAGES; ++i) {
            mbar_init(smem_u32(&full[i]), 1);
            mbar_init(smem_u32(&empty[i]), 1);
        }
        mbar_init(smem_u32(done), 1);
        *bad = 0;
        fence_async_smem();
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (w == 0) tc_alloc(smem_u32(tslot), 32 * TC_ACC);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;
    int issued = 0;
    if (tid == 0) {
        for (int i = 0; i < nk; ++i) {
            const int k = k0 + i, s = i % TC_STAGES;
            if (i >= TC_STAGES && !mbar_wait(smem_u32(&empty[s]), (uint32_t)((i / TC_STAGES - 1) & 1))) {
                *bad = 1;
                break;
            }
            unsigned char* st = sm + s * TC_STAGE;
            const uint32_t bar = smem_u32(&full[s]);
            mbar_expect_tx(bar, (uint32_t)((2 * nA + 2) * TC_PLANE));
            for (int r = 0; r < nA; ++r) {
                const float* src = planes + tile(I0 + r, k) * 2 * TILE2;
                bulk_copy(smem_u32(st + r * TC_PLANE), src, TC_PLANE, bar);
                bulk_copy(smem_u32(st + (4 + r) * TC_PLANE), src + TILE2, TC_PLANE, bar);
            }
            const float* srcB = planes + tile(J, k) * 2 * TILE2;
            bulk_copy(smem_u32(st + 8 * TC_PLANE), srcB, TC_PLANE, bar);
            bulk_copy(smem_u32(st + 9 * TC_PLANE), srcB + TILE2, TC_PLANE, bar);
            ++issued;
        }
    } else if (tid == 32) {
        constexpr uint32_t idesc = tc_idesc_tf32(128, 32);
        for (int i = 0; i < nk; ++i) {
            const int s = i % TC_STAGES;
            if (*bad || !mbar_wait(smem_u32(&full[s]), (uint32_t)((i / TC_STAGES) & 1))) {
                *bad = 1;
                break;
            }
            tc_fence_after();
            const uint32_t st = smem_u32(sm + s * TC_STAGE);
            const uint32_t d = tbase + 32u * (uint32_t)(i % TC_ACC);
            // A: 128 rows (4 tiles, 4 KB each = 4 groups of 8 rows at SBO 1024), K 8 per MMA
            for (int j = 0; j < 4; ++j) {
                const uint32_t o = j * 256;   // two core matrices along K
                const uint64_t aH = tc_smem_desc(st + o, 128, 1024), aL = tc_smem_desc(st + 4 * TC_PLANE + o, 128, 1024);
                const uint64_t bH = tc_smem_desc(st + 8 * TC_PLANE + o, 128, 1024);
                const uint64_t bL = tc_smem_desc(st + 9 * TC_PLANE + o, 128, 1024);
                tc_mma_tf32(d, aH, bH, idesc, (i >= TC_ACC || j > 0) ? 1u : 0u);
                tc_mma_tf32(d, aH, bL, idesc, 1u);
                tc_mma_tf32(d, aL, bH, idesc, 1u);
            }
            tc_commit(smem_u32(&empty[s]));
        }
        tc_commit(smem_u32(done));
    }
    // everyone: the product is complete (thread 0 decides for the CTA, so that the
    // warp-wide tensor-memory loads below run in whole warps or not at all)
    const bool done_ok = mbar_wait(smem_u32(done), 0u);
    __syncthreads();
    if (tid == 0) tslot[2] = (done_ok && !*bad) ? 1u : 0u;
    __syncthreads();
    const bool ok = tslot[2] != 0;
    tc_fence_after();
    float v[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) v[c] = 0.0f;
    if (ok && w < nA) {
        // the accumulators in use, summed in a fixed order
        float u[32];
        for (int a = 0; a < TC_ACC && a < nk; ++a) {
            tc_ld32(tbase + ((uint32_t)(32 * w) << 16) + 32u * a, u);
#pragma unroll
            for (int c = 0; c < 32; ++c) v[c] += u[c];
        }
    }
    if (!ok && tid == 0) atomicExch(err, 1);
    if (nsplit == 1) {
        if (ok && w < nA) {
            float* t = work + tile(I0 + w, J) * TILE2;   // column-major: (r, c) at c * 32 + r
#pragma unroll
            for (int c = 0; c < 32; ++c) t[c * TILE + lane] -= v[c];
        }
    } else {
        // K split: every CTA stores its partial product; the CTA that arrives last at the
        // row block's ticket adds the partials in split order and updates the tiles
        // (deterministic, as GridSum)
        float* mine = part + ((bq * nsplit + sp) * 4) * (int64_t)TILE2;
        if (w < nA) {
#pragma unroll
            for (int c = 0; c < 32; ++c) mine[w * TILE2 + c * TILE + lane] = v[c];
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) tslot[3] = atomicAdd(&ticket[bq], 1u) == (unsigned)(nsplit - 1) ? 1u : 0u;
        __syncthreads();
        if (tslot[3]) {
            __threadfence();
            if (w < nA) {
                float sum[32];
#pragma unroll
                for (int c = 0; c < 32; ++c) sum[c] = 0.0f;
                for (int q = 0; q < nsplit; ++q) {
                    const float* pq = part + ((bq * nsplit + q) * 4 + w) * (int64_t)TILE2;
#pragma unroll
                    for (int c = 0; c < 32; ++c) sum[c] += __ldcg(pq + c * TILE + lane);
                }
                float* t = work + tile(I0 + w, J) * TILE2;
#pragma unroll
                for (int c = 0; c < 32; ++c) t[c * TILE + lane] -= sum[c];
            }
            if (tid == 0) ticket[bq] = 0u;   // re-armed for the next launch
        }
    }
    // the producer's copies in flight land before the CTA leaves (bounded)
    if (tid == 0 && !ok)
        for (int k = max(0, issued - TC_STAGES); k < issued; ++k)
            mbar_wait(smem_u32(&full[k % TC_STAGES]), (uint32_t)((k / TC_STAGES) & 1));
    tc_fence_before();
    __syncthreads();
    if (w == 0) tc_dealloc(tbase, 32 * TC_ACC);
}

// ---------------------------------------------------------------------------------
// Explicit inverse of a dense FP32 item from its tile factor, S^{-1} = W^T W with
// W = L^{-1}, by batched 32x32 tile products (one CTA per output tile, 4 warps, thread
// (lane c, warp w) owns rows 8w .. 8w+7 of column c):
//   type 0: W_II = L_II^{-1} (copied from dinv);
//   type 1: P_IJ = sum_{k0 <= K < k1} L_IK W_KJ          (P = L21 W11 of a 2x2 split)
//   type 2: W_IJ = -sum_{k0 <= K < k1} W_IK P_KJ         (W21 = -W22 P)
//   type 3: (S^{-1})_IJ = sum_{k0 <= K < k1} W_KI^T W_KJ, I >= J, into the dense FP64
//           column-major output (rows and columns past the item's n dropped).
// A job is int4 {item, I << 16 | J, k0 << 16 | k1, type}.  Types 1 and 2 are issued level by
// level of a recursive halving of the tile range (both halves inverted first), so a level's
// products only read finished tiles.  Operand tiles are staged in shared memory through
// registers, the next pair loaded while the current one multiplies.
// ---------------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_tile_inv(const int4* __restrict__ jobs, const float* __restrict__ L,
                                                  const float* __restrict__ dinv, float* __restrict__ Wt,
                                                  float* __restrict__ Pt, double* __restrict__ out,
                                                  const int64_t* __restrict__ base, const int64_t* __restrict__ row0,
                                                  const int32_t* __restrict__ nrows,
                                                  const int64_t* __restrict__ out_off) {
    __shared__ __align__(16) float As[2][TILE * 36];   // A(r, t) at t * 36 + r
    __shared__ float Bs[2][TILE * 33];                 // B(t, c) at t * 33 + c
    const int4 jb = jobs[blockIdx.x];
    const int g = jb.x, I = jb.y >> 16, J = jb.y & 0xffff, k0 = jb.z >> 16, k1 = jb.z & 0xffff, type = jb.w;
    const int tid = threadIdx.x, c = tid & 31, rb = (tid >> 5) * 8;
    const int64_t b0 = base[g];
    auto tile = [&](int a, int b) { return (b0 + (int64_t)a * (a + 1) / 2 + b) * TILE2; };
    if (type == 0) {
        const float* D = dinv + (row0[g] + I) * TILE2;
        float* dst = Wt + tile(I, I);
#pragma unroll
        for (int u = 0; u < TILE2 / 128; ++u) dst[tid + 128 * u] = D[tid + 128 * u];
        return;
    }
    const float* Asrc = type == 1 ? L : Wt;
    const float* Bsrc = type == 1 ? Wt : (type == 2 ? Pt : Wt);
    float ra[TILE2 / 128], rbv[TILE2 / 128];
    auto gload = [&](int k) {
        const float* A = Asrc + (type == 3 ? tile(k, I) : tile(I, k));
        const float* B = Bsrc + tile(k, J);
#pragma unroll
        for (int u = 0; u < TILE2 / 128; ++u) {
            ra[u] = A[tid + 128 * u];
            rbv[u] = B[tid + 128 * u];
        }
    };
    auto sstore = [&](int buf) {
#pragma unroll
        for (int u = 0; u < TILE2 / 128; ++u) {
            const int e = tid + 128 * u, hi = e >> 5, lo = e & 31;   // element (lo, hi) of a column-major tile
            if (type == 3) As[buf][lo * 36 + hi] = ra[u];             // A = M^T: A(hi, lo) = M(lo, hi)
            else As[buf][hi * 36 + lo] = ra[u];                      // A(lo, hi)
            Bs[buf][lo * 33 + hi] = rbv[u];                           // B(lo, hi)
        }
    };
    float acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0.0f;
    if (k0 < k1) {
        gload(k0);
        sstore(0);
    }
    __syncthreads();
    for (int k = k0; k < k1; ++k) {
        const int buf = (k - k0) & 1;
        if (k + 1 < k1) gload(k + 1);
#pragma unroll 8
        for (int t = 0; t < TILE; ++t) {
            const float b = Bs[buf][t * 33 + c];
            const float4 x = *reinterpret_cast<const float4*>(&As[buf][t * 36 + rb]);
            const float4 y = *reinterpret_cast<const float4*>(&As[buf][t * 36 + rb + 4]);
            acc[0] += x.x * b, acc[1] += x.y * b, acc[2] += x.z * b, acc[3] += x.w * b;
            acc[4] += y.x * b, acc[5] += y.y * b, acc[6] += y.z * b, acc[7] += y.w * b;
        }
        if (k + 1 < k1) sstore(buf ^ 1);
        __syncthreads();
    }
    if (type == 3) {
        const int64_t n = nrows[g];
        const int64_t col = (int64_t)J * TILE + c;
        if (col < n) {
            double* o = out + out_off[g] + col * n;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int64_t row = (int64_t)I * TILE + rb + q;
                if (row < n) o[row] = (double)acc[q];
            }
        }
        return;
    }
    float* dst = (type == 1 ? Pt : Wt) + tile(I, J) + c * TILE + rb;
    const float sgn = type == 1 ? 1.0f : -1.0f;
    *reinterpret_cast<float4*>(dst) = make_float4(sgn * acc[0], sgn * acc[1], sgn * acc[2], sgn * acc[3]);
    *reinterpret_cast<float4*>(dst + 4) = make_float4(sgn * acc[4], sgn * acc[5], sgn * acc[6], sgn * acc[7]);
}

void launch_tile_inv(const int4* jobs, int njobs, const float* L, const float* dinv, float* Wt, float* Pt,
                     double* out, const int64_t* base, const int64_t* row0, const int32_t* nrows,
                     const int64_t* out_off, cudaStream_t st) {
    if (njobs <= 0) return;
    count_launch();
    k_tile_inv<<<(unsigned)njobs, 128, 0, st>>>(jobs, L, dinv, Wt, Pt, out, base, row0, nrows, out_off);
}

// Warp dot product of a contiguous row with x (len entries) in the row's arithmetic TM
// (FP64, or FP32 for the FP32 copies, x then FP32 too: a double -> float conversion runs
// on B300's FP64 pipe), eight independent accumulators per lane so that each lane has
// eight row loads in flight, lanes 0..31 strided.
template <typename TM>
__device__ __forceinline__ TM warp_row_dot(const TM* __restrict__ row, const TM* __restrict__ x, int64_t len,
                                           int lane) {
    TM s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int64_t j = lane;
    for (; j + 224 < len; j += 256) {
#pragma unroll
        for (int u = 0; u < 8; ++u) s[u] += row[j + 32 * u] * x[j + 32 * u];
    }
    for (int u = 0; j < len; j += 32, ++u) s[u & 7] += row[j] * x[j];
    TM t = ((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    return t;
}

template <typename TM>
struct NdMats {
    const TM *Ginv, *Wcm, *Wrm, *Cinv;
};
__device__ __forceinline__ NdMats<double> nd_mats(const NdSolveArgs& a, double) {
    return {a.Ginv, a.Wcm, a.Wrm, a.Cinv};
}
__device__ __forceinline__ NdMats<float> nd_mats(const NdSolveArgs& a, float) {
    return {a.Ginv32, a.Wcm32, a.Wrm32, a.Cinv32};
}

// Side vectors of one column in the solve's arithmetic TM: the right-hand side b, the
// separator right-hand side c = b_sep - sum_g S_{sep,g} S_gg^{-1} b_g (in the P buffer,
// nsep <= np entries) and the separator solution (FP64: b, P and eta themselves; FP32:
// float copies in `f32`, laid out [b: L | c: np | separator eta: nsep] per column).
template <typename TM>
struct NdVecs {
    const TM* b;
    TM* c;
    TM* es;
};
__device__ __forceinline__ NdVecs<double> nd_vecs(const NdSolveArgs& a, const double* b, double* eta, double* P,
                                                  float*, int64_t, double) {
    return {b, P, eta + a.goff[a.G]};
}
__device__ __forceinline__ NdVecs<float> nd_vecs(const NdSolveArgs& a, const double*, double*, double*, float* f32,
                                                 int64_t, float) {
    return {f32, f32 + a.L32, f32 + a.L32 + a.nsep4};
}

// 16-byte-load warp dot product of n4 float4 (FP32 rows and vectors of the padded layout)
__device__ __forceinline__ float warp_row_dot4(const float4* __restrict__ row, const float4* __restrict__ x,
                                               int64_t n4, int lane) {
    float s[4] = {0.f, 0.f, 0.f, 0.f};
    int64_t j = lane;
    for (; j + 96 < n4; j += 128) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float4 a = row[j + 32 * u], b = x[j + 32 * u];
            s[u] = fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, fmaf(a.w, b.w, s[u]))));
        }
    }
    for (int u = 0; j < n4; j += 32, ++u) {
        const float4 a = row[j], b = x[j];
        s[u & 3] = fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, fmaf(a.w, b.w, s[u & 3]))));
    }
    float t = (s[0] + s[1]) + (s[2] + s[3]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    return t;
}

// ---------------------------------------------------------------------------------
// Per-iteration solve (ND order in and out), in the arithmetic TM of the matrices used.
// Stage 1, one warp per row: eta_g = Ginv_g b_g for the interior rows, and for every
// separator unknown s (groups g1 < g2) c_s = b_s - (W_g1^T b_g1)_s - (W_g2^T b_g2)_s.
// ---------------------------------------------------------------------------------
template <typename TM>
__global__ void k_nd_stage1(NdSolveArgs a, const double* __restrict__ b, double* __restrict__ eta,
                            double* __restrict__ P, float* __restrict__ f32, int64_t fl, ColStrides cs) {
    const int col = blockIdx.y;
    if (cs.done && cs.done[col * cs.done_stride]) return;
    const NdMats<TM> M = nd_mats(a, TM(0));
    const NdVecs<TM> V = nd_vecs(a, b + col * cs.l, eta + col * cs.l, P + col * a.np, f32 ? f32 + col * fl : nullptr,
                                 a.nin + a.nsep, TM(0));
    eta += col * cs.l;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t nin = a.goff[a.G];
    if constexpr (std::is_same<TM, float>::value) {   // padded FP32 layout, 16-byte loads
        if (wid < nin) {
            const int g = a.row_g[wid];
            const int64_t g0 = a.goff[g], n4 = (a.goff[g + 1] - g0 + 3) >> 2, i = wid - g0;
            const float s = warp_row_dot4(reinterpret_cast<const float4*>(M.Ginv + a.gioff32[g] + i * 4 * n4),
                                          reinterpret_cast<const float4*>(V.b + a.gpo32[g]), n4, lane);
            if (lane == 0) eta[wid] = (double)s;
        } else if (wid < nin + a.nsep) {
            const int64_t sp = wid - nin;
            float c = V.b[a.spo32 + sp];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int g = a.sg[2 * sp + e];
                const int64_t n4 = (a.goff[g + 1] - a.goff[g] + 3) >> 2, j = a.sidx[2 * sp + e];
                c -= warp_row_dot4(reinterpret_cast<const float4*>(M.Wcm + a.woff32[g] + j * 4 * n4),
                                   reinterpret_cast<const float4*>(V.b + a.gpo32[g]), n4, lane);
            }
            if (lane == 0) V.c[sp] = c;
        }
    } else {
        if (wid < nin) {
            const int g = a.row_g[wid];
            const int64_t g0 = a.goff[g], ng = a.goff[g + 1] - g0, i = wid - g0;
            const TM s = warp_row_dot<TM>(M.Ginv + a.gioff[g] + i * ng, V.b + g0, ng, lane);
            if (lane == 0) eta[wid] = (double)s;
        } else if (wid < nin + a.nsep) {
            const int64_t sp = wid - nin;
            TM c = V.b[nin + sp];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int g = a.sg[2 * sp + e];
                const int64_t g0 = a.goff[g], ng = a.goff[g + 1] - g0, j = a.sidx[2 * sp + e];
                c -= warp_row_dot<TM>(M.Wcm + a.woff[g] + j * ng, V.b + g0, ng, lane);
            }
            if (lane == 0) V.c[sp] = c;
        }
    }
}

// Stage 2: eta_sep = Cinv c, c staged in shared memory by every CTA.
template <typename TM>
__global__ void k_nd_stage2(NdSolveArgs a, const double* __restrict__ b, double* __restrict__ eta,
                            double* __restrict__ P, float* __restrict__ f32, int64_t fl, ColStrides cs) {
    const int col = blockIdx.y;
    if (cs.done && cs.done[col * cs.done_stride]) return;
    const NdMats<TM> M = nd_mats(a, TM(0));
    const NdVecs<TM> V = nd_vecs(a, b + col * cs.l, eta + col * cs.l, P + col * a.np, f32 ? f32 + col * fl : nullptr,
                                 a.nin + a.nsep, TM(0));
    eta += col * cs.l;
    extern __shared__ __align__(16) unsigned char cvec_raw[];
    TM* cvec = reinterpret_cast<TM*>(cvec_raw);
    const int nsep = a.nsep;
    const int64_t sep0 = a.goff[a.G];
    const int nc = std::is_same<TM, float>::value ? a.nsep4 : nsep;   // FP32: zero-padded
    for (int s = threadIdx.x; s < nc; s += blockDim.x) cvec[s] = V.c[s];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (wid >= nsep) return;
    TM s;
    if constexpr (std::is_same<TM, float>::value)
        s = warp_row_dot4(reinterpret_cast<const float4*>(M.Cinv + wid * nc), reinterpret_cast<const float4*>(cvec),
                          nc >> 2, lane);
    else
        s = warp_row_dot<TM>(M.Cinv + wid * nsep, cvec, nsep, lane);
    if (lane == 0) {
        eta[sep0 + wid] = (double)s;
        if (!std::is_same<TM, double>::value) V.es[wid] = s;
    }
}

// Stage 3: eta_g -= W_g eta_{A_g}; the separator solution staged in shared memory.
template <typename TM>
__global__ void k_nd_stage3(NdSolveArgs a, double* __restrict__ eta, float* __restrict__ f32, int64_t fl,
                            ColStrides cs) {
    const int col = blockIdx.y;
    if (cs.done && cs.done[col * cs.done_stride]) return;
    const NdMats<TM> M = nd_mats(a, TM(0));
    const NdVecs<TM> V =
        nd_vecs(a, nullptr, eta + col * cs.l, nullptr, f32 ? f32 + col * fl : nullptr, a.nin + a.nsep, TM(0));
    eta += col * cs.l;
    extern __shared__ __align__(16) unsigned char es_raw[];
    TM* es = reinterpret_cast<TM*>(es_raw);
    for (int s = threadIdx.x; s < a.nsep; s += blockDim.x) es[s] = V.es[s];
    __syncthreads();
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t nin = a.goff[a.G];
    if (wid >= nin) return;
    const int g = a.row_g[wid];
    const int64_t g0 = a.goff[g], ag = a.aoff[g + 1] - a.aoff[g], i = wid - g0;
    const TM* row = M.Wrm + a.woff[g] + i * ag;
    const int32_t* al = a.alist + a.aoff[g];
    TM s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    int64_t j = lane;
    for (; j + 96 < ag; j += 128) {
        s0 += row[j] * es[al[j]];
        s1 += row[j + 32] * es[al[j + 32]];
        s2 += row[j + 64] * es[al[j + 64]];
        s3 += row[j + 96] * es[al[j + 96]];
    }
    for (; j < ag; j += 32) s0 += row[j] * es[al[j]];
    TM s = (s0 + s1) + (s2 + s3);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) eta[wid] -= (double)s;
}

// b -> its FP32 copy (callers whose right-hand side does not come from the restriction)
__global__ void k_nd_b32(int L, const double* __restrict__ b, float* __restrict__ b32, const int32_t* __restrict__ p32) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < L) b32[p32[i]] = (float)b[i];
}

__global__ void k_pad_convert(int64_t nlines, int64_t len, const double* __restrict__ src, int64_t ss,
                              float* __restrict__ dst, int64_t ds) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nlines * ds;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t l = e / ds, j = e - l * ds;
        dst[e] = j < len ? (float)src[l * ss + j] : 0.0f;
    }
}

// ------------------------------------------------------------------------ launchers
void launch_iface_tables(int L, int64_t nr, const int64_t* rp_ptr, const int32_t* rp_pos, const double* val,
                         const int64_t* r_ptr, double* rcoef, double* T, int64_t ng, const int32_t* g_from_r,
                         double* gval, cudaStream_t st) {
    if (nr > 0) {
        count_launch();
        k_iface_coef<<<(unsigned)std::min<int64_t>((nr + 255) / 256, 4096), 256, 0, st>>>(nr, rp_ptr, rp_pos, val,
                                                                                         rcoef);
        const int64_t work = std::max<int64_t>(L, 1);
        count_launch();
        k_iface_T_g<<<(unsigned)std::min<int64_t>((work + 255) / 256, 4096), 256, 0, st>>>(L, r_ptr, rcoef, T, ng,
                                                                                          g_from_r, gval);
    }
}
void launch_nd_assemble(int m, const NdAssembleArgs& a, cudaStream_t st) {
    if (m > 0) {
        count_launch();
        k_nd_assemble<<<m, 256, 0, st>>>(a);
    }
}
void launch_nd_diag(int L, const double* T, const double* diagc, const int32_t* nd_pos, double* Sd, cudaStream_t st) {
    if (L > 0) {
        count_launch();
        k_nd_diag<<<(L + 127) / 128, 128, 0, st>>>(L, T, diagc, nd_pos, Sd);
    }
}
template <typename TW>
void launch_dense_to_tiles(int64_t ntiles, const double* src, int64_t ld, const int64_t* src_off, const int32_t* rows,
                           const int64_t* base, const int32_t* tile_item, const int32_t* tile_I,
                           const int32_t* tile_J, TW* work, cudaStream_t st) {
    if (ntiles > 0) {
        count_launch();
        k_dense_to_tiles<TW><<<(unsigned)ntiles, 256, 0, st>>>(src, ld, src_off, rows, base, tile_item, tile_I, tile_J,
                                                               work);
    }
}
template <typename TW>
void launch_dense_cholesky(int nitems, const std::vector<int32_t>& T_host, const int32_t* T, const int64_t* base,
                           const int64_t* row0, TW* work, TW* dinv, int* err, cudaStream_t st, TW* planes,
                           int* kerr, TcSplit tcs) {
    int maxT = 0;
    for (int t : T_host) maxT = std::max(maxT, t);
    if (planes) {
        // FP32 (planes given): left-looking, column J updated by the tensor cores from the
        // planes of the finished columns, then its diagonal tile factored, then solved below
        cudaFuncSetAttribute(k_dupdate_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
        for (int J = 0; J < maxT; ++J) {
            int64_t nblk = 0, nt = 0, nd = 0;
            for (int t : T_host)
                if (t > J) {
                    nblk += (t - J + 3) / 4;
                    nt += t - 1 - J;
                    nd += 1;
                }
            if (J > 0 && nblk > 0) {
                // K split over CTAs: one CTA streams the 40 KB stage of every k through one SM
                // (~0.6 us a stage on B300), so the column's update is spread over up to two
                // CTAs per SM, at least two stages each
                int nsplit = 1;
                if (tcs.part) {
                    nsplit = (int)std::min<int64_t>(tcs.max_ctas / nblk, J / 2);
                    nsplit = std::max(1, nsplit);
                    if (nblk > tcs.max_blocks) nsplit = 1;
                }
                count_launch();
                k_dupdate_tc<<<(unsigned)(nblk * nsplit), 128, TC_SMEM, st>>>(
                    nitems, T, base, (float*)work, (const float*)planes, J, nsplit, tcs.part, tcs.ticket, kerr);
            }
            count_launch();
            k_dpotrf_trsm<TW><<<(unsigned)(nt + nd), 128, 0, st>>>(nitems, T, base, row0, work, dinv, J, err, planes);
        }
        return;
    }
    for (int k = 0; k < maxT; ++k) {
        int64_t nt = 0, np = 0;
        for (int t : T_host) {
            const int64_t w = t - 1 - k;
            if (w > 0) {
                nt += w;
                np += w * (w + 1) / 2;
            }
        }
        count_launch();
        k_dpotrf_b<TW><<<nitems, 128, 0, st>>>(nitems, T, base, row0, work, dinv, k, err, nullptr);
        if (nt > 0) {
            count_launch();
            k_dtrsm_b<TW><<<(unsigned)nt, 256, 0, st>>>(nitems, T, base, row0, work, dinv, k, nullptr);
            count_launch();
            k_dupdate_b<TW><<<(unsigned)np, 256, 0, st>>>(nitems, T, base, work, k);
        }
    }
}
void launch_mirror_lower(const int32_t* rows, const int64_t* off, int nitems, double* M, cudaStream_t st) {
    if (nitems > 0) {
        count_launch();
        k_mirror_lower<<<dim3(256, nitems), 256, 0, st>>>(rows, off, nitems, M);
    }
}
void launch_transpose_blocks(const int64_t* goff, const int64_t* aoff, const int64_t* woff, int G, const double* Wcm,
                             double* Wrm, cudaStream_t st) {
    if (G > 0) {
        count_launch();
        k_transpose_blocks<<<dim3(256, G), 256, 0, st>>>(goff, aoff, woff, G, Wcm, Wrm);
    }
}
void launch_nd_w_sparse(int64_t np, int64_t L, const double* Sd, const int64_t* goff, const int64_t* aoff,
                        const int32_t* alist, int64_t sep0, const int32_t* prow_g, const int64_t* wc_ptr,
                        const int32_t* wc_row, const int64_t* gioff, const double* Ginv, const int64_t* woff,
                        double* Wcm, cudaStream_t st) {
    if (np > 0) {
        count_launch();
        k_nd_w_sparse<<<(unsigned)np, 256, 0, st>>>(L, Sd, goff, aoff, alist, sep0, prow_g, wc_ptr, wc_row, gioff,
                                                    Ginv, woff, Wcm);
    }
}
void launch_nd_schur_sparse(int64_t np, int64_t L, const double* Sd, const int64_t* goff, const int64_t* aoff,
                            const int32_t* alist, int64_t sep0, const int32_t* prow_g, const int64_t* wc_ptr,
                            const int32_t* wc_row, const int64_t* woff, const double* Wrm, const int64_t* doff,
                            double* D, cudaStream_t st) {
    if (np > 0) {
        count_launch();
        k_nd_schur_sparse<<<(unsigned)((np + 7) / 8), 256, 0, st>>>(L, np, Sd, goff, aoff, alist, sep0, prow_g, wc_ptr,
                                                                    wc_row, woff, Wrm, doff, D);
    }
}
template <typename TW>
void launch_nd_schur_tiles(int64_t ntiles, int64_t L, int nsep, int64_t sep0, const double* Sd, const int32_t* sg,
                           const int32_t* sidx, const int64_t* aoff, const int64_t* doff, const double* D,
                           TW* work, cudaStream_t st) {
    if (ntiles > 0) {
        count_launch();
        k_nd_schur_tiles<TW><<<(unsigned)ntiles, 256, 0, st>>>(L, nsep, sep0, Sd, sg, sidx, aoff, doff, D, work);
    }
}
template <typename TM>
static void nd_solve_t(const NdSolveArgs& a, const double* b, double* eta, double* P, float* f32, int64_t fl,
                       ColStrides cs, int ncols, cudaStream_t st) {
    const int64_t nin = a.nin;
    if (nin + a.nsep > 0) {
        count_launch();
        k_nd_stage1<TM><<<dim3((unsigned)((nin + a.nsep + 7) / 8), ncols), 256, 0, st>>>(a, b, eta, P, f32, fl, cs);
    }
    if (a.nsep > 0) {
        const size_t smem = (size_t)(std::is_same<TM, float>::value ? a.nsep4 : a.nsep) * sizeof(TM);
        count_launch();
        k_nd_stage2<TM><<<dim3((unsigned)((a.nsep + 7) / 8), ncols), 256, smem, st>>>(a, b, eta, P, f32, fl, cs);
        if (nin > 0) {
            count_launch();
            k_nd_stage3<TM><<<dim3((unsigned)((nin + 7) / 8), ncols), 256, smem, st>>>(a, eta, f32, fl, cs);
        }
    }
}
void launch_nd_solve(const NdSolveArgs& a, const double* b, double* eta, double* P, float* f32, int64_t fl,
                     bool b32_ready, ColStrides cs, int ncols, cudaStream_t st) {
    if (a.Ginv32 || a.Cinv32) {
        if (!b32_ready) {
            const int L = (int)(a.nin + a.nsep);
            for (int c = 0; c < ncols; ++c) {
                count_launch();
                k_nd_b32<<<(L + 255) / 256, 256, 0, st>>>(L, b + c * cs.l, f32 + c * fl, a.p32);
            }
        }
        nd_solve_t<float>(a, b, eta, P, f32, fl, cs, ncols, st);
    } else {
        nd_solve_t<double>(a, b, eta, P, nullptr, 0, cs, ncols, st);
    }
}
void launch_pad_convert(int64_t nlines, int64_t len, const double* src, int64_t ss, float* dst, int64_t ds,
                        cudaStream_t st) {
    if (nlines > 0 && ds > 0) {
        count_launch();
        k_pad_convert<<<(unsigned)std::min<int64_t>((nlines * ds + 255) / 256, 4096), 256, 0, st>>>(nlines, len, src,
                                                                                                   ss, dst, ds);
    }
}
cudaError_t prepare_nd_solve(int nsep) {
    size_t smem = (size_t)(nsep + 3) * sizeof(double);
    if (smem > 48 * 1024) {
        const void* ks[] = {(const void*)k_nd_stage2<double>, (const void*)k_nd_stage2<float>,
                            (const void*)k_nd_stage3<double>, (const void*)k_nd_stage3<float>};
        for (const void* k : ks) {
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

#define INST_ND(TW)                                                                                           \
    template void launch_dense_to_tiles<TW>(int64_t, const double*, int64_t, const int64_t*, const int32_t*,       \
                                            const int64_t*, const int32_t*, const int32_t*, const int32_t*, TW*,     \
                                            cudaStream_t);                                                           \
    template void launch_dense_cholesky<TW>(int, const std::vector<int32_t>&, const int32_t*, const int64_t*,      \
                                            const int64_t*, TW*, TW*, int*, cudaStream_t, TW*, int*, TcSplit);                \
    template void launch_nd_schur_tiles<TW>(int64_t, int64_t, int, int64_t, const double*, const int32_t*,         \
                                            const int32_t*, const int64_t*, const int64_t*, const double*, TW*,      \
                                            cudaStream_t);
INST_ND(double)
INST_ND(float)

}  // namespace am
