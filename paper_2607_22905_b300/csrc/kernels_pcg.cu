// Global-vector kernels of AlgMortar-PCG on sm_103a: SpMV (sliced ELL), the fused FP64
// CG vector updates and dot products (Sec. 7: x0 = 0, Euclidean relative-residual stop),
// the interface restriction and prolongation of Algorithm 2, value refreshes, and the
// adjoint gradient of the TPFA transmissibilities.
//
// Vector kernels are grid-strided over rows.  Dot products are deterministic: each CTA
// writes its block sum, and the CTA that finishes last adds the partials in a fixed
// order (GridSum) and stores the scalar straight into the device-side PCG state, so
// repeated runs give bit-identical iterates and no partial arrays cross kernels.
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <initializer_list>
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace am {

static std::atomic<int64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void add_launches(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

// CTAs of the grid-strided vector kernels over n rows (= size of their GridSum partials):
// at most 8 resident CTAs of 256 threads on each of the device's SMs
static int g_max_vec_blocks = 8 * 148;
static int g_sms = 148;
void set_vec_sms(int sms) {
    g_sms = sms > 0 ? sms : 148;
    g_max_vec_blocks = 8 * g_sms;
}
int vec_blocks(int64_t n) {
    int64_t g = (n + VEC_BS - 1) / VEC_BS;
    return (int)(g < 1 ? 1 : (g > g_max_vec_blocks ? g_max_vec_blocks : g));
}
// CTAs of the per-iteration PCG kernels (SpMV, CG updates) over `work` thread items: at
// most `hot_ctas_per_sm` CTAs on each SM (<= 8, so the GridSum partials sized by
// vec_blocks suffice).  Fewer, fuller threads keep enough loads in flight and halve the
// FP64 work of the block reductions relative to one wave of 8 CTAs per SM.
static thread_local int g_hot_ctas_per_sm = 4;   // set from the handle before its launches
void set_hot_ctas_per_sm(int c) { g_hot_ctas_per_sm = c < 1 ? 1 : (c > 8 ? 8 : c); }
int hot_ctas_per_sm() { return g_hot_ctas_per_sm; }
int hot_blocks(int64_t work) {
    const int64_t cap = (int64_t)g_hot_ctas_per_sm * g_sms;
    int64_t g = (work + VEC_BS - 1) / VEC_BS;
    return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

#define GRID_STRIDE(i, n) \
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// dst[k] = src[perm[k]] / dst[perm[k]] = src[k], column blockIdx.y at the given strides
__global__ void k_gather(int64_t n, const int32_t* __restrict__ perm, const double* __restrict__ src,
                         int64_t lds, double* __restrict__ dst, int64_t ldd) {
    src += blockIdx.y * lds;
    dst += blockIdx.y * ldd;
    GRID_STRIDE(k, n) dst[k] = src[perm[k]];
}

__global__ void k_scatter(int64_t n, const int32_t* __restrict__ perm, const double* __restrict__ src,
                          int64_t lds, double* __restrict__ dst, int64_t ldd) {
    src += blockIdx.y * lds;
    dst += blockIdx.y * ldd;
    GRID_STRIDE(k, n) dst[perm[k]] = src[k];
}

__global__ void k_scatter_values(int64_t n, const int64_t* __restrict__ idx, const double* __restrict__ v,
                                 double* __restrict__ dst) {
    GRID_STRIDE(k, n) dst[idx[k]] = v[k];
}

// b_eta[I] = -1/4 sum_k G[k, I] pbar_k = sum_{(k,l) in E_I} |a_kl| (pbar_k + pbar_l)/2 --
// the interface right-hand side of Eq. (interface-problem-alg), one warp per interface,
// written at position omap[I] (the interface solve's ordering) when omap is given.
__global__ void k_restrict(int L, const int64_t* __restrict__ rptr, const int32_t* __restrict__ rcell,
                           const double* __restrict__ rcoef, const double* __restrict__ pbar,
                           double* __restrict__ beta, const int32_t* __restrict__ omap, ColStrides cs,
                           float* __restrict__ beta32, int64_t fl, const int32_t* __restrict__ p32) {
    const int col = blockIdx.y;
    if (cs.done && cs.done[col * cs.done_stride]) return;
    pbar += col * cs.v;
    beta += col * cs.l;
    if (beta32) beta32 += col * fl;
    int I = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    int lane = threadIdx.x & 31;
    if (I >= L) return;
    double s = 0.0;
    for (int64_t t = rptr[I] + lane; t < rptr[I + 1]; t += 32) s += rcoef[t] * pbar[rcell[t]];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        const int o = omap ? omap[I] : I;
        beta[o] = s;
        if (beta32) beta32[p32 ? p32[o] : o] = (float)s;   // the FP32 interface solve's copy
    }
}

// z_k = pbar_k + sum_{m in I_i} eta_m p_hat_i^(m)_k  (Eq. p-decomposition-alg).  One warp
// per chunk of <= 32 rows of one subdomain i, one row per lane, chunks grid-strided over
// the warps.  The panels are read row-major (ProlongChunk): lane k loads its row's k_i
// entries as 16-byte vectors, so a warp streams one contiguous block of the panel array.
// Lane c holds the interface values eta_m of list entries c and c + 32 and passes them
// to the products by shuffles, so warps never wait on one another; the next chunk's
// descriptor and interface indices are loaded while the current chunk's loads are in
// flight.  Inside PCG (`psc` given) also rho = r . z and, in the CTA that completes it,
// the next beta (one thread: scalar FP64 divisions stay off the per-row path, B300's
// FP64 pipe being ~1/64 of its FP32 rate).
template <typename TP>
struct Vec16;
template <>
struct Vec16<float> {
    using T = float4;
};
template <>
struct Vec16<double> {
    using T = double2;
};

template <typename TP>
__global__ void __launch_bounds__(VEC_BS) k_prolong(const ProlongChunk* __restrict__ chunks, int nchunks,
                                                     const int32_t* __restrict__ if_list,
                                                     const TP* __restrict__ phi, const double* __restrict__ eta,
                                                     const double* __restrict__ pbar,
                                                     const double* base, double* z,   // may alias
                                                     const double* __restrict__ r, GridSum gs,
                                                     PcgScalars* psc, ColStrides cs) {
    // the correction sum_m eta_m p_hat^(m) is accumulated in the panel's arithmetic
    // (FP64 panels: FP64; FP32 panels: FP32), then added to pbar in FP64
    using TV = typename Vec16<TP>::T;
    constexpr int VW = 16 / sizeof(TP);   // entries per vector
    constexpr int NV = 24 / VW;           // vectors per row loaded before the first product
    const int col = blockIdx.y;
    if (cs.done && cs.done[col * cs.done_stride]) return;
    __shared__ double sh[VEC_BS];
    eta += col * cs.l;
    pbar += col * cs.v;
    z += col * cs.v;
    if (base) base += col * cs.v;
    if (r) r += col * cs.v;
    if (psc) psc += col;
    gs.part += col * gridDim.x;
    gs.ticket += col;
    const int lane = threadIdx.x & 31;
    const int nw = blockDim.x >> 5;
    const int ws = gridDim.x * nw;
    int ch = blockIdx.x * nw + (threadIdx.x >> 5);
    double acc = 0.0;
    ProlongChunk cur{};
    int ia = -1, ib = -1;   // interface positions of list entries lane, lane + 32
    if (ch < nchunks) {
        cur = chunks[ch];
        if (lane < cur.kk) ia = if_list[cur.i0 + lane];
        if (lane + 32 < cur.kk) ib = if_list[cur.i0 + lane + 32];
    }
    for (; ch < nchunks; ch += ws) {
        const int kk = cur.kk;   // warp-uniform, as is every field of cur
        const int i0 = cur.i0;
        const int nv = (kk + VW - 1) / VW;
        const bool row = lane < cur.nrow;
        const TP* ph = phi + cur.phi0 + (int64_t)lane * cur.ld;
        TV pv[NV];
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            if (row && j < nv) {
                pv[j] = *reinterpret_cast<const TV*>(ph + j * VW);
            } else {
                TP* q = reinterpret_cast<TP*>(&pv[j]);
#pragma unroll
                for (int u = 0; u < VW; ++u) q[u] = (TP)0;
            }
        }
        const int64_t g = cur.row0 + lane;
        const double pb = row ? pbar[g] : 0.0;
        const double bs = (row && base) ? base[g] : 0.0;
        const double rv = (row && psc) ? r[g] : 0.0;
        // entries past k_i: zero panel padding times a zero interface value
        const TP ea = ia >= 0 ? (TP)eta[ia] : (TP)0;
        const TP eb = ib >= 0 ? (TP)eta[ib] : (TP)0;
        // the next chunk's descriptor and indices, overlapping the loads above
        const int nx = ch + ws;
        if (nx < nchunks) {
            cur = chunks[nx];
            ia = lane < cur.kk ? if_list[cur.i0 + lane] : -1;
            ib = lane + 32 < cur.kk ? if_list[cur.i0 + lane + 32] : -1;
        }
        TP a4[4] = {(TP)0, (TP)0, (TP)0, (TP)0};
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            if (j < nv) {
                const TP* q = reinterpret_cast<const TP*>(&pv[j]);
#pragma unroll
                for (int u = 0; u < VW; ++u) a4[(j * VW + u) & 3] += q[u] * __shfl_sync(0xffffffffu, ea, j * VW + u);
            }
        }
        for (int j = NV; j < nv; ++j) {
            TV w;
            if (row) {
                w = *reinterpret_cast<const TV*>(ph + j * VW);
            } else {
                TP* q = reinterpret_cast<TP*>(&w);
#pragma unroll
                for (int u = 0; u < VW; ++u) q[u] = (TP)0;
            }
            const TP* q = reinterpret_cast<const TP*>(&w);
#pragma unroll
            for (int u = 0; u < VW; ++u) {
                const int c = j * VW + u;
                TP ev;
                if (c < 64) {
                    ev = __shfl_sync(0xffffffffu, c < 32 ? ea : eb, c & 31);
                } else {
                    // subdomains with more than 64 interfaces: values beyond from global memory
                    ev = c < kk ? (TP)eta[if_list[i0 + c]] : (TP)0;
                }
                a4[u & 3] += q[u] * ev;
            }
        }
        if (row) {
            double v = pb + (double)((a4[0] + a4[1]) + (a4[2] + a4[3]));
            if (base) v += bs;   // smoothed application: x + M^{-1} (r - A x)
            z[g] = v;
            if (psc) acc += rv * v;
        }
    }
    if (psc && grid_sum(acc, sh, gs, &psc->rz_next) && threadIdx.x == 0) {
        const double rn = psc->rz_next;
        psc->beta = (psc->iter == 0 || psc->restart)
                        ? 0.0
                        : (psc->flexible ? (rn - psc->rz_mix) / psc->rz : rn / psc->rz);
    }
}

// Row-major copy (layout of ProlongChunk) of the column-major FP64 panels, one warp per
// 32-row chunk: lane = row, 16 columns at a time read as coalesced column segments and
// written as 16-byte row segments; the padding columns up to ld are zero.
template <typename TP>
__global__ void __launch_bounds__(256) k_panel_rows(int nchunks, const ProlongChunk* __restrict__ chunks,
                                                    const int32_t* __restrict__ chunk_sub,
                                                    const int64_t* __restrict__ sub_off,
                                                    const int64_t* __restrict__ phi_off,
                                                    const double* __restrict__ phi, TP* __restrict__ out) {
    constexpr int VW = 16 / sizeof(TP);
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int ch = blockIdx.x * nw + (threadIdx.x >> 5); ch < nchunks; ch += gridDim.x * nw) {
        const ProlongChunk cu = chunks[ch];
        if (lane >= cu.nrow) continue;
        const int s = chunk_sub[ch];
        const int64_t ns = sub_off[s + 1] - sub_off[s], o = cu.row0 - sub_off[s] + lane;
        const double* src = phi + phi_off[s] + o;
        TP* dst = out + cu.phi0 + (int64_t)lane * cu.ld;
        for (int cb = 0; cb < cu.ld; cb += 16) {
            TP v[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = cb + j < cu.kk ? (TP)src[(int64_t)(cb + j) * ns] : (TP)0;
#pragma unroll
            for (int j = 0; j < 16; j += VW) {
                if (cb + j < cu.ld) {
                    if constexpr (VW == 4)
                        *reinterpret_cast<float4*>(dst + cb + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                    else
                        *reinterpret_cast<double2*>(dst + cb + j) = make_double2(v[j], v[j + 1]);
                }
            }
        }
    }
}

// s = r - A x (sliced ELL) for the block-Jacobi smoothing steps (Sec. 5.4).
__global__ void __launch_bounds__(VEC_BS) k_smooth_residual(int64_t n, const int64_t* __restrict__ ell_ptr,
                                                             const int32_t* __restrict__ ell_col,
                                                             const double* __restrict__ ell_val,
                                                             const double* __restrict__ x, const double* __restrict__ r,
                                                             double* __restrict__ s, ColStrides cs) {
    const int col = blockIdx.y;
    if (cs.done && cs.done[col * cs.done_stride]) return;
    x += col * cs.v;
    r += col * cs.v;
    s += col * cs.v;
    GRID_STRIDE(k, n) {
        const int64_t sl = k >> 5;
        const int rr = (int)(k & 31);
        const int64_t b = __ldg(ell_ptr + sl), w = (__ldg(ell_ptr + sl + 1) - b) >> 5;
        const double* v = ell_val + b + rr;
        const int32_t* c = ell_col + b + rr;
        double acc = r[k];
        for (int64_t e = 0; e < w; ++e) acc -= __ldg(v + e * 32) * __ldg(x + __ldg(c + e * 32));
        s[k] = acc;
    }
}

// Completion of the preconditioned residual (smoothed path): rho = r . z and the next
// beta (as in k_prolong's tail).
__global__ void __launch_bounds__(VEC_BS) k_pcg_rho(int64_t n, const double* __restrict__ r,
                                                     const double* __restrict__ z, PcgScalars* psc, GridSum gs,
                                                     ColStrides cs) {
    const int col = blockIdx.y;
    if (cs.done && cs.done[col * cs.done_stride]) return;
    __shared__ double sh[VEC_BS];
    r += col * cs.v;
    z += col * cs.v;
    psc += col;
    gs.part += col * gridDim.x;
    gs.ticket += col;
    double acc = 0.0;
    GRID_STRIDE(k, n) acc += r[k] * z[k];
    if (grid_sum(acc, sh, gs, &psc->rz_next) && threadIdx.x == 0) {
        const double rn = psc->rz_next;
        psc->beta = (psc->iter == 0 || psc->restart)
                        ? 0.0
                        : (psc->flexible ? (rn - psc->rz_mix) / psc->rz : rn / psc->rz);
    }
}

// ------------------------------------------------------------------------------ PCG
// x = 0, r = b, ||b||^2; the CTA that completes the sum initialises the PCG state.
__global__ void __launch_bounds__(VEC_BS) k_pcg_init(int64_t n, const double* __restrict__ b,
                                                      double* __restrict__ x, double* __restrict__ r, int64_t ld,
                                                      PcgScalars* __restrict__ sc, GridSum gs, double tol,
                                                      int max_it, int flexible, double* hist, int hist_len) {
    __shared__ double sh[VEC_BS];
    const int col = blockIdx.y;
    b += col * ld;
    x += col * ld;
    r += col * ld;
    sc += col;
    gs.part += col * gridDim.x;
    gs.ticket += col;
    double acc = 0.0;
    GRID_STRIDE(k, n) {
        const double v = b[k];
        r[k] = v;
        x[k] = 0.0;
        acc += v * v;
    }
    if (grid_sum(acc, sh, gs, &sc->bb) && threadIdx.x == 0) {
        const double bb = sc->bb;
        sc->rr = bb;
        sc->rr_new = bb;
        sc->tol2 = tol * tol * bb;
        sc->iter = 0;
        sc->done = bb == 0.0 ? 1 : 0;
        sc->status = 0;
        sc->max_it = max_it;
        sc->rz = 0.0;
        sc->rz_next = 0.0;
        sc->rz_mix = 0.0;
        sc->alpha = sc->beta = sc->pq = 0.0;
        sc->flexible = flexible;
        sc->restart = 0;
        if (hist && hist_len > 0) hist[(int64_t)col * hist_len] = bb;
    }
}

// p = z + beta p; beta (set where rho_new is completed, in the prolongation) is
// rho_new / rho (Fletcher-Reeves form of CG) or the flexible (Polak-Ribiere)
// (rho_new - r_new . z_old) / rho, which tolerates a slightly non-symmetric
// preconditioner; 0 on the first iteration and right after a residual replacement.
// V = 2: rows in 16-byte pairs (n and the column stride even, bases 16-byte aligned).
template <int V>
__global__ void __launch_bounds__(VEC_BS, 4) k_pcg_p(int64_t n, const double* __restrict__ z, double* __restrict__ p,
                                                   int64_t ld, const PcgScalars* __restrict__ sc) {
    const int col = blockIdx.y;
    sc += col;
    if (sc->done) return;
    z += col * ld;
    p += col * ld;
    const double beta = sc->beta;
    if (V == 2) {
        const double2* z2 = reinterpret_cast<const double2*>(z);
        double2* p2 = reinterpret_cast<double2*>(p);
        GRID_STRIDE(i, n >> 1) {
            const double2 zz = z2[i];
            double2 pp = p2[i];
            pp.x = zz.x + beta * pp.x;
            pp.y = zz.y + beta * pp.y;
            p2[i] = pp;
        }
    } else {
        GRID_STRIDE(k, n) p[k] = z[k] + beta * p[k];
    }
}

// q = A p on the sliced-ELL copy and p . q -> sc->pq; the CTA that completes p . q sets
// alpha = rho / p . q once.  CTA 0 moves rho to the new direction's value (read by the
// following kernels only).
//
// A warp takes two 32-row slices at a time (lane = row of each), so each load of values
// and columns is one contiguous 128/256-byte segment, and the two rows' product chains are
// independent.  Columns and values of EB entries of both rows are loaded before the
// gathers of p they index, and those before any product, giving every lane up to 4 EB
// independent loads in flight.  A slice's width is the same for all its lanes, so entries
// past it are skipped by a uniform branch (no FP64 work on padding beyond the width;
// B300's FP64 rate, about two lanes per SM and clock, bounds this kernel more than HBM
// does).  Padding inside the width and rows past n read column min(row, n - 1) with
// value 0.  WF > 0: a pair of slices that are both WF entries wide (the common width of
// a stencil matrix, e.g. 7 for a 3D seven-point stencil) takes a fully unrolled path
// with the fewest FP64 instructions: 2 WF loads of each kind in flight per lane, one FMA
// chain per row, no predicated slot past the width (WF = 7 in steps of EB = 4 spends
// one) and no add joining split chains.
template <int EB, int WF>
__global__ void __launch_bounds__(VEC_BS, WF > 0 ? 3 : 4) k_pcg_spmv_ell(int64_t n, const int64_t* __restrict__ ell_ptr,
                                                          const int32_t* __restrict__ ell_col,
                                                          const double* __restrict__ ell_val,
                                                          const double* __restrict__ p, double* __restrict__ q,
                                                          int64_t ld, PcgScalars* __restrict__ sc, GridSum gs) {
    const int col = blockIdx.y;
    sc += col;
    if (sc->done) return;
    __shared__ double sh[VEC_BS];
    p += col * ld;
    q += col * ld;
    gs.part += col * gridDim.x;
    gs.ticket += col;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        sc->rz = sc->rz_next;
        sc->restart = 0;
    }
    const int lane = threadIdx.x & 31;
    const int64_t nsl = (n + 31) >> 5, npair = (nsl + 1) >> 1;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double acc = 0.0, acc1 = 0.0;
    for (int64_t sp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; sp < npair; sp += nwarp) {
        const int64_t sa = 2 * sp, sb = sa + 1;
        const bool hb = sb < nsl;
        const int64_t ba = __ldg(ell_ptr + sa), bb = __ldg(ell_ptr + sa + 1);
        const int64_t eb = hb ? __ldg(ell_ptr + sb + 1) : bb;
        const int wa = (int)((bb - ba) >> 5), wb = (int)((eb - bb) >> 5);
        const int wm = wa > wb ? wa : wb;
        const int32_t* ca = ell_col + ba + lane;
        const int32_t* cb = ell_col + bb + lane;
        const double* va = ell_val + ba + lane;
        const double* vb = ell_val + bb + lane;
        double s0, s1;
        constexpr int WA = WF > 0 ? WF : 1;
        if (WF > 0 && wa == WF && wb == WF) {
            // one FMA chain per row: 2 per lane, and the many resident warps, keep the
            // FP64 unit fed, and no add joins split chains (the SpMV is FP64-bound)
            int32_t ia[WA], ib[WA];
            double xa[WA], xb[WA], ga[WA], gb[WA];
#pragma unroll
            for (int j = 0; j < WF; ++j) {
                ia[j] = __ldg(ca + j * 32);
                ib[j] = __ldg(cb + j * 32);
            }
#pragma unroll
            for (int j = 0; j < WF; ++j) {
                xa[j] = __ldg(va + j * 32);
                xb[j] = __ldg(vb + j * 32);
            }
#pragma unroll
            for (int j = 0; j < WF; ++j) {
                ga[j] = __ldg(p + ia[j]);
                gb[j] = __ldg(p + ib[j]);
            }
            s0 = xa[0] * ga[0];
            s1 = xb[0] * gb[0];
#pragma unroll
            for (int j = 1; j < WF; ++j) {
                s0 = fma(xa[j], ga[j], s0);
                s1 = fma(xb[j], gb[j], s1);
            }
        } else {
            // four independent FP64 chains per lane (even / odd entries of each row)
            double t0 = 0.0, t1 = 0.0;
            s0 = 0.0;
            s1 = 0.0;
            for (int e0 = 0; e0 < wm; e0 += EB) {
                int32_t ia[EB], ib[EB];
                double xa[EB], xb[EB], ga[EB], gb[EB];
#pragma unroll
                for (int j = 0; j < EB; ++j) {
                    const int e = e0 + j;
                    ia[j] = e < wa ? __ldg(ca + (int64_t)e * 32) : 0;
                    ib[j] = e < wb ? __ldg(cb + (int64_t)e * 32) : 0;
                }
#pragma unroll
                for (int j = 0; j < EB; ++j) {
                    const int e = e0 + j;
                    xa[j] = e < wa ? __ldg(va + (int64_t)e * 32) : 0.0;
                    xb[j] = e < wb ? __ldg(vb + (int64_t)e * 32) : 0.0;
                }
#pragma unroll
                for (int j = 0; j < EB; ++j) {
                    const int e = e0 + j;
                    ga[j] = e < wa ? __ldg(p + ia[j]) : 0.0;
                    gb[j] = e < wb ? __ldg(p + ib[j]) : 0.0;
                }
#pragma unroll
                for (int j = 0; j < EB; j += 2) {
                    const int e = e0 + j;
                    if (e < wa) s0 += xa[j] * ga[j];
                    if (e < wb) s1 += xb[j] * gb[j];
                    if (e + 1 < wa) t0 += xa[j + 1] * ga[j + 1];
                    if (e + 1 < wb) t1 += xb[j + 1] * gb[j + 1];
                }
            }
            s0 += t0;
            s1 += t1;
        }
        const int64_t ka = sa * 32 + lane, kb = sb * 32 + lane;
        if (ka < n) {
            q[ka] = s0;
            acc += p[ka] * s0;
        }
        if (hb && kb < n) {
            q[kb] = s1;
            acc1 += p[kb] * s1;
        }
    }
    acc += acc1;
    if (grid_sum(acc, sh, gs, &sc->pq) && threadIdx.x == 0) {
        const double pq = sc->pq, al = sc->rz_next / pq;
        sc->alpha = al;
        sc->step_ok = (pq > 0.0 && isfinite(al)) ? 1 : 0;
    }
}

// Stop test on the device (breakdown, convergence, iteration cap), run by the thread that
// completes ||r||^2.
__device__ __forceinline__ void pcg_stop_test(PcgScalars* sc) {
    sc->iter += 1;
    const double rr = sc->rr_new;
    if (!sc->step_ok || !isfinite(rr)) {
        sc->done = 1;
        sc->status = 6;
    } else {
        sc->rr = rr;
        if (rr <= sc->tol2) {
            sc->done = 1;
            sc->status = 0;
        } else if (sc->iter >= sc->max_it) {
            sc->done = 1;
            sc->status = 5;
        }
    }
}

// Rows of k_pcg_xr in 16-byte pairs: with UPD, x += alpha p and r -= alpha q; then
// ||r||^2 (and with FLEX r . z) into two independent FP64 chains each.  Separate loop
// bodies per case keep the per-row path free of branches.
template <bool FLEX, bool UPD>
__device__ __forceinline__ void xr_pairs(int64_t np, double2* __restrict__ x2, double2* __restrict__ r2,
                                         const double2* __restrict__ p2, const double2* __restrict__ q2,
                                         const double2* __restrict__ z2, double al, double& acc, double& acc2) {
    double ay = 0.0, a2y = 0.0;
#pragma unroll 1   // unrolled, the loop spills at the 64 registers of 4 CTAs per SM
    GRID_STRIDE(i, np) {
        double2 rk = r2[i];
        if (UPD) {
            const double2 pk = p2[i], qk = q2[i];
            double2 xk = x2[i];
            xk.x += al * pk.x;
            xk.y += al * pk.y;
            rk.x -= al * qk.x;
            rk.y -= al * qk.y;
            x2[i] = xk;
            r2[i] = rk;
        }
        acc += rk.x * rk.x;
        ay += rk.y * rk.y;
        if (FLEX) {
            const double2 zk = z2[i];
            acc2 += rk.x * zk.x;
            a2y += rk.y * zk.y;
        }
    }
    acc += ay;
    acc2 += a2y;
}
template <bool FLEX, bool UPD>
__device__ __forceinline__ void xr_rows(int64_t n, double* __restrict__ x, double* __restrict__ r,
                                        const double* __restrict__ p, const double* __restrict__ q,
                                        const double* __restrict__ z, double al, double& acc, double& acc2) {
    GRID_STRIDE(k, n) {
        double rk = r[k];
        if (UPD) {
            x[k] += al * p[k];
            rk -= al * q[k];
            r[k] = rk;
        }
        acc += rk * rk;
        if (FLEX) acc2 += rk * z[k];
    }
}

// x += alpha p;  r -= alpha q;  ||r||^2 -> sc->rr_new (and, for the flexible beta,
// r_new . z_old -> sc->rz_mix, z still holding z_old), then the stop test.  After a
// breakdown (step_ok == 0) x and r stay as they are.  V = 2: rows in 16-byte pairs, as
// in k_pcg_p.
template <int V>
__global__ void __launch_bounds__(VEC_BS, 4) k_pcg_xr(int64_t n, double* __restrict__ x, double* __restrict__ r,
                                                    const double* __restrict__ p, const double* __restrict__ q,
                                                    const double* __restrict__ z, int64_t ld,
                                                    PcgScalars* __restrict__ sc, GridSum gs, double* hist,
                                                    int hist_len) {
    const int col = blockIdx.y;
    sc += col;
    if (sc->done) return;
    __shared__ double sh[VEC_BS];
    x += col * ld;
    r += col * ld;
    p += col * ld;
    q += col * ld;
    z += col * ld;
    const bool flex = sc->flexible != 0;
    gs.part += col * (flex ? 2 : 1) * gridDim.x;
    gs.ticket += col;
    const double al = sc->alpha;
    const bool ok = sc->step_ok != 0;
    double acc = 0.0, acc2 = 0.0;
    if (V == 2) {
        double2* x2 = reinterpret_cast<double2*>(x);
        double2* r2 = reinterpret_cast<double2*>(r);
        const double2* p2 = reinterpret_cast<const double2*>(p);
        const double2* q2 = reinterpret_cast<const double2*>(q);
        const double2* z2 = reinterpret_cast<const double2*>(z);
        const int64_t np = n >> 1;
        if (ok) {
            if (flex) xr_pairs<true, true>(np, x2, r2, p2, q2, z2, al, acc, acc2);
            else xr_pairs<false, true>(np, x2, r2, p2, q2, z2, al, acc, acc2);
        } else {
            if (flex) xr_pairs<true, false>(np, x2, r2, p2, q2, z2, al, acc, acc2);
            else xr_pairs<false, false>(np, x2, r2, p2, q2, z2, al, acc, acc2);
        }
    } else {
        if (ok) {
            if (flex) xr_rows<true, true>(n, x, r, p, q, z, al, acc, acc2);
            else xr_rows<false, true>(n, x, r, p, q, z, al, acc, acc2);
        } else {
            if (flex) xr_rows<true, false>(n, x, r, p, q, z, al, acc, acc2);
            else xr_rows<false, false>(n, x, r, p, q, z, al, acc, acc2);
        }
    }
    const bool last = flex ? grid_sum2(acc, acc2, sh, gs, &sc->rr_new, &sc->rz_mix)
                           : grid_sum(acc, sh, gs, &sc->rr_new);
    if (last && threadIdx.x == 0) {
        pcg_stop_test(sc);
        if (hist && sc->iter < hist_len) hist[(int64_t)col * hist_len + sc->iter] = sc->rr_new;   // residual history
    }
}

// Residual replacement for columns that restart (done == 0): r = b - A x, ||r||^2 ->
// rr and rr_new, and the next beta is 0 (CSR copy of A).
__global__ void __launch_bounds__(VEC_BS) k_pcg_replace(int64_t n, const int32_t* __restrict__ rowptr,
                                                         const int32_t* __restrict__ cidx,
                                                         const double* __restrict__ val,
                                                         const double* __restrict__ x, const double* __restrict__ b,
                                                         double* __restrict__ r, int64_t ld,
                                                         PcgScalars* __restrict__ sc, GridSum gs) {
    const int col = blockIdx.y;
    sc += col;
    if (sc->done) return;
    __shared__ double sh[VEC_BS];
    x += col * ld;
    b += col * ld;
    r += col * ld;
    gs.part += col * gridDim.x;
    gs.ticket += col;
    double acc = 0.0;
    GRID_STRIDE(k, n) {
        double s = b[k];
        for (int32_t e = rowptr[k]; e < rowptr[k + 1]; ++e) s -= val[e] * x[cidx[e]];
        r[k] = s;
        acc += s * s;
    }
    if (grid_sum(acc, sh, gs, &sc->rr_new) && threadIdx.x == 0) {
        sc->rr = sc->rr_new;
        sc->restart = 1;
    }
}

// ||b - A x||^2 -> sc->res2 (true residual, CSR copy of A).
__global__ void __launch_bounds__(VEC_BS) k_residual(int64_t n, const int32_t* __restrict__ rowptr,
                                                      const int32_t* __restrict__ cidx,
                                                      const double* __restrict__ val,
                                                      const double* __restrict__ x, const double* __restrict__ b,
                                                      int64_t ld, PcgScalars* __restrict__ sc, GridSum gs) {
    __shared__ double sh[VEC_BS];
    const int col = blockIdx.y;
    x += col * ld;
    b += col * ld;
    sc += col;
    gs.part += col * gridDim.x;
    gs.ticket += col;
    double acc = 0.0;
    GRID_STRIDE(k, n) {
        double s = b[k];
        for (int32_t e = rowptr[k]; e < rowptr[k + 1]; ++e) s -= val[e] * x[cidx[e]];
        acc += s * s;
    }
    grid_sum(acc, sh, gs, &sc->res2);
}

// ell_val[t] = val[src[t]] (0 for padding)
__global__ void k_ell_values(int64_t nell, const int32_t* __restrict__ src, const double* __restrict__ val,
                             double* __restrict__ ell_val) {
    GRID_STRIDE(t, nell) {
        const int32_t s = src[t];
        ell_val[t] = s >= 0 ? val[s] : 0.0;
    }
}

// ------------------------------------------------------------------------- adjoint
// dL/d lnK for a TPFA matrix (harmonic-mean transmissibilities T_kl = -a_kl between
// cells k, l; Dirichlet half-faces folded into per-cell sums tb_k = sum_b T_b,
// tbp_k = sum_b T_b p_bc), given the state p (A p = f) and the adjoint lambda
// (A lambda = dL/dp):
//   dL/dT_kl = -(lambda_k - lambda_l)(p_k - p_l),   dT_kl/dlnK_k = T_kl K_l / (K_k + K_l)
//   dL/dT_b  =  lambda_k (p_bc - p_k),              dT_b/dlnK_k  = T_b
// One thread per cell gathers over its row: deterministic, no atomics.  All vectors in
// the CSR's own ordering.
__global__ void k_tpfa_grad(int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                            const double* __restrict__ val, const double* __restrict__ K,
                            const double* __restrict__ tb, const double* __restrict__ tbp,
                            const double* __restrict__ p, const double* __restrict__ lam,
                            double* __restrict__ grad) {
    GRID_STRIDE(k, n) {
        const double pk = p[k], lk = lam[k], Kk = K[k];
        double g = lk * (tbp[k] - pk * tb[k]);
        for (int32_t e = rowptr[k]; e < rowptr[k + 1]; ++e) {
            const int32_t l = col[e];
            if (l == k) continue;
            const double T = -val[e];
            const double dLdT = -(lk - lam[l]) * (pk - p[l]);
            g += dLdT * T * K[l] / (Kk + K[l]);
        }
        grad[k] = g;
    }
}

// ------------------------------------------------------------------------ launchers
static inline int grid_for(int64_t n, int bs) {
    int64_t g = (n + bs - 1) / bs;
    return (int)(g < 1 ? 1 : (g > 65535 * 4 ? 65535 * 4 : g));
}

void launch_gather(int64_t n, const int32_t* perm, const double* src, double* dst, cudaStream_t st) {
    launch_gather_cols(n, 1, perm, src, n, dst, n, st);
}
void launch_gather_cols(int64_t n, int ncols, const int32_t* perm, const double* src, int64_t lds, double* dst,
                        int64_t ldd, cudaStream_t st) {
    count_launch();
    k_gather<<<dim3(grid_for(n, 256), ncols), 256, 0, st>>>(n, perm, src, lds, dst, ldd);
}
void launch_scatter_values(int64_t n, const int64_t* idx, const double* v, double* dst, cudaStream_t st) {
    if (n > 0) {
        count_launch();
        k_scatter_values<<<grid_for(n, 256), 256, 0, st>>>(n, idx, v, dst);
    }
}
void launch_scatter(int64_t n, const int32_t* perm, const double* src, double* dst, cudaStream_t st) {
    launch_scatter_cols(n, 1, perm, src, n, dst, n, st);
}
void launch_scatter_cols(int64_t n, int ncols, const int32_t* perm, const double* src, int64_t lds, double* dst,
                         int64_t ldd, cudaStream_t st) {
    count_launch();
    k_scatter<<<dim3(grid_for(n, 256), ncols), 256, 0, st>>>(n, perm, src, lds, dst, ldd);
}
void launch_restrict(int L, const int64_t* rptr, const int32_t* rcell, const double* rcoef, const double* pbar,
                     double* beta, const int32_t* omap, ColStrides cs, int ncols, float* beta32, int64_t fl,
                     const int32_t* p32, cudaStream_t st) {
    if (L > 0) {
        count_launch();
        k_restrict<<<dim3((L + 7) / 8, ncols), 256, 0, st>>>(L, rptr, rcell, rcoef, pbar, beta, omap, cs, beta32, fl,
                                                             p32);
    }
}
// CTAs of the prolongation: one wave at the kernel's occupancy (every CTA's arrival at
// the grid-wide sum delays its retirement, so extra waves cost), at most one warp per
// chunk and at most vec_blocks of the widest vector (the GridSum partials).
static int g_prolong_ctas_per_sm[2] = {0, 0};
template <typename TP>
static int prolong_ctas_per_sm() {
    int& c = g_prolong_ctas_per_sm[sizeof(TP) == 8 ? 1 : 0];
    if (c == 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_prolong<TP>, VEC_BS, 0) != cudaSuccess || b < 1)
            b = 1;
        c = b;
    }
    return c;
}
int prolong_blocks(int nchunks) {
    const int64_t want = ((int64_t)nchunks + (VEC_BS / 32) - 1) / (VEC_BS / 32);
    return vec_blocks(want * VEC_BS);
}
template <typename TP>
void launch_prolong(int nchunks, const ProlongChunk* chunks, const int32_t* if_list, const TP* phi,
                    const double* eta, const double* pbar, const double* base, double* z, const double* r,
                    GridSum gs, PcgScalars* sc, ColStrides cs, int ncols, cudaStream_t st) {
    count_launch();
    int g = prolong_blocks(nchunks);
    const int cap = prolong_ctas_per_sm<TP>() * g_sms;
    if (g > cap) g = cap;
    k_prolong<TP><<<dim3(g > 0 ? g : 1, ncols), VEC_BS, 0, st>>>(chunks, nchunks, if_list, phi, eta, pbar, base, z,
                                                                  r, gs, sc, cs);
}
template <typename TP>
void launch_panel_rows(int nchunks, const ProlongChunk* chunks, const int32_t* chunk_sub, const int64_t* sub_off,
                       const int64_t* phi_off, const double* phi, TP* out, cudaStream_t st) {
    if (nchunks <= 0) return;
    count_launch();
    k_panel_rows<TP><<<prolong_blocks(nchunks), 256, 0, st>>>(nchunks, chunks, chunk_sub, sub_off, phi_off, phi, out);
}
void launch_smooth_residual(int64_t n, int ncols, const int64_t* ell_ptr, const int32_t* ell_col,
                            const double* ell_val, const double* x, const double* r, double* s, ColStrides cs,
                            cudaStream_t st) {
    count_launch();
    k_smooth_residual<<<dim3(vec_blocks(n), ncols), VEC_BS, 0, st>>>(n, ell_ptr, ell_col, ell_val, x, r, s, cs);
}
void launch_pcg_rho(int64_t n, int ncols, const double* r, const double* z, PcgScalars* sc, GridSum gs,
                    ColStrides cs, cudaStream_t st) {
    count_launch();
    k_pcg_rho<<<dim3(vec_blocks(n), ncols), VEC_BS, 0, st>>>(n, r, z, sc, gs, cs);
}
void launch_pcg_init(int64_t n, int ncols, int64_t ld, const double* b, double* x, double* r, PcgScalars* sc,
                     GridSum gs, double tol, int max_it, int flexible, double* hist, int hist_len, cudaStream_t st) {
    count_launch();
    k_pcg_init<<<dim3(vec_blocks(n), ncols), VEC_BS, 0, st>>>(n, b, x, r, ld, sc, gs, tol, max_it, flexible, hist,
                                                               hist_len);
}
void launch_pcg_replace(int64_t n, int ncols, int64_t ld, const int32_t* rowptr, const int32_t* col,
                        const double* val, const double* x, const double* b, double* r, PcgScalars* sc, GridSum gs,
                        cudaStream_t st) {
    count_launch();
    k_pcg_replace<<<dim3(vec_blocks(n), ncols), VEC_BS, 0, st>>>(n, rowptr, col, val, x, b, r, ld, sc, gs);
}
// 16-byte row pairs when every column of every operand starts 16-byte aligned
static bool pairs_ok(int64_t n, int64_t ld, std::initializer_list<const void*> ptrs) {
    if ((n & 1) || (ld & 1)) return false;
    for (const void* q : ptrs)
        if (reinterpret_cast<uintptr_t>(q) & 15) return false;
    return true;
}
void launch_pcg_p(int64_t n, int ncols, int64_t ld, const double* z, double* p, const PcgScalars* sc,
                  cudaStream_t st) {
    count_launch();
    if (pairs_ok(n, ld, {z, p}))
        k_pcg_p<2><<<dim3(hot_blocks(n >> 1), ncols), VEC_BS, 0, st>>>(n, z, p, ld, sc);
    else
        k_pcg_p<1><<<dim3(hot_blocks(n), ncols), VEC_BS, 0, st>>>(n, z, p, ld, sc);
}
// resident CTAs per SM of an SpMV instantiation (its register budget), cached
template <int WF>
static int spmv_ctas_per_sm() {
    static int c = 0;
    if (c == 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_pcg_spmv_ell<4, WF>, VEC_BS, 0) != cudaSuccess || b < 1)
            b = 1;
        c = b;
    }
    return c;
}
template <int WF>
static void spmv_launch(int64_t n, int ncols, int64_t ld, const int64_t* ell_ptr, const int32_t* ell_col,
                        const double* ell_val, const double* p, double* q, PcgScalars* sc, GridSum gs,
                        cudaStream_t st) {
    const int64_t warps = (((n + 31) >> 5) + 1) >> 1;   // one warp per pair of slices
    int g = hot_blocks(warps * 32);
    g = std::min(g, spmv_ctas_per_sm<WF>() * g_sms);   // one wave: no CTA waits for a slot
    k_pcg_spmv_ell<4, WF><<<dim3(g, ncols), VEC_BS, 0, st>>>(n, ell_ptr, ell_col, ell_val, p, q, ld, sc, gs);
}
void launch_pcg_spmv_ell(int64_t n, int ncols, int64_t ld, const int64_t* ell_ptr, const int32_t* ell_col,
                         const double* ell_val, const double* p, double* q, PcgScalars* sc, GridSum gs, int wf,
                         cudaStream_t st) {
    count_launch();
    if (wf == 7)
        spmv_launch<7>(n, ncols, ld, ell_ptr, ell_col, ell_val, p, q, sc, gs, st);
    else if (wf == 5)
        spmv_launch<5>(n, ncols, ld, ell_ptr, ell_col, ell_val, p, q, sc, gs, st);
    else
        spmv_launch<0>(n, ncols, ld, ell_ptr, ell_col, ell_val, p, q, sc, gs, st);
}
// the slice width that takes the SpMV's unrolled path: 7 or 5 when at least half of the
// 32-row slices have it, else 0
int spmv_fast_width(const int64_t* ell_ptr_host, int64_t nslices) {
    int64_t c5 = 0, c7 = 0;
    for (int64_t s = 0; s < nslices; ++s) {
        const int64_t w = (ell_ptr_host[s + 1] - ell_ptr_host[s]) >> 5;
        c5 += w == 5;
        c7 += w == 7;
    }
    if (2 * c7 >= nslices && nslices > 0) return 7;
    if (2 * c5 >= nslices && nslices > 0) return 5;
    return 0;
}
void launch_ell_values(int64_t nell, const int32_t* src, const double* val, double* ell_val, cudaStream_t st) {
    count_launch();
    k_ell_values<<<grid_for(nell, 256), 256, 0, st>>>(nell, src, val, ell_val);
}
void launch_pcg_xr(int64_t n, int ncols, int64_t ld, double* x, double* r, const double* p, const double* q,
                   const double* z, PcgScalars* sc, GridSum gs, double* hist, int hist_len, cudaStream_t st) {
    count_launch();
    if (pairs_ok(n, ld, {x, r, p, q, z}))
        k_pcg_xr<2><<<dim3(hot_blocks(n >> 1), ncols), VEC_BS, 0, st>>>(n, x, r, p, q, z, ld, sc, gs, hist, hist_len);
    else
        k_pcg_xr<1><<<dim3(hot_blocks(n), ncols), VEC_BS, 0, st>>>(n, x, r, p, q, z, ld, sc, gs, hist, hist_len);
}
void launch_residual(int64_t n, int ncols, int64_t ld, const int32_t* rowptr, const int32_t* col, const double* val,
                     const double* x, const double* b, PcgScalars* sc, GridSum gs, cudaStream_t st) {
    count_launch();
    k_residual<<<dim3(vec_blocks(n), ncols), VEC_BS, 0, st>>>(n, rowptr, col, val, x, b, ld, sc, gs);
}
void launch_tpfa_grad(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val, const double* K,
                      const double* tb, const double* tbp, const double* p, const double* lam, double* grad,
                      cudaStream_t st) {
    count_launch();
    k_tpfa_grad<<<grid_for(n, 256), 256, 0, st>>>(n, rowptr, col, val, K, tb, tbp, p, lam, grad);
}

#define INST_PROLONG(TP)                                                                                     \
    template void launch_prolong<TP>(int, const ProlongChunk*, const int32_t*, const TP*, const double*,         \
                                     const double*, const double*, double*, const double*, GridSum, PcgScalars*, \
                                     ColStrides, int, cudaStream_t);
#define INST_PANEL_ROWS(TP)                                                                                  \
    template void launch_panel_rows<TP>(int, const ProlongChunk*, const int32_t*, const int64_t*, const int64_t*, \
                                        const double*, TP*, cudaStream_t);
INST_PANEL_ROWS(double)
INST_PANEL_ROWS(float)
INST_PROLONG(double)
INST_PROLONG(float)

}  // namespace am
