// Local-diagonal and tile-profile kernels of AlgMortar on sm_103a: the diagonal of the
// modified blocks A_i (Eq. A_i) with their symmetric scaling, the MBF right-hand sides
// (Eq. def-phat-local), and the FP64 tile-profile sweep streams and batched triangular
// solves used for the explicit inverses of the interface blocks (kernels_coarse.cu).
// The local factors themselves are supernodal (kernels_snode.cu).
#include "common.cuh"
#include "kernels.h"
#include "tma.cuh"

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

// ---------------------------------------------------------------------------------
// Sweep streams of a tile-profile factor (the FP64 interface blocks): forward rows
// [L_I,lo .. L_I,I-1 | L_II^{-1}], backward rows [(L_I+1,I)^T .. (L_hi,I)^T | L_II^{-T}].
// Every 32x32 tile M is stored row-major with its 16-byte chunks XOR-swizzled
// (swz_index), so that the solve reads row `lane` of a tile with conflict-free 128-bit
// shared loads.
// ---------------------------------------------------------------------------------
template <typename TW, typename TS>
__global__ void __launch_bounds__(256) k_finalize(Profile pf, const TW* __restrict__ work,
                                                  const TW* __restrict__ dinv,
                                                  TS* __restrict__ fwdS, TS* __restrict__ bwdS) {
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
    const int tid = threadIdx.x;
    for (int I = blockIdx.y; I < T; I += gridDim.y) {
        const int nt = I - lo[I];
        const int64_t fo = (base + fwd[I]) * TILE2;
        // forward: M = L_IJ (column-major source: M[r][c] at c*32 + r), then L_II^{-1}
        for (int t = 0; t <= nt; ++t) {
            const TW* src = t < nt ? Wb + (fwd[I] + t) * TILE2 : Db + (int64_t)I * TILE2;
            for (int e = tid; e < TILE2; e += blockDim.x) {
                const int r = e >> 5, c = e & 31;
                fwdS[fo + (int64_t)t * TILE2 + swz_index<TS>(r, c)] = stf<TS>((double)src[c * TILE + r]);
            }
        }
        // backward: M = (L_JI)^T (M[r][c] = L_JI[c][r] at r*32 + c), then L_II^{-T}
        const int nb = hi[I] - I;
        const int64_t bo = (base + bwd[I]) * TILE2;
        for (int t = 0; t <= nb; ++t) {
            const TW* src = t < nb ? Wb + (fwd[I + 1 + t] + (I - lo[I + 1 + t])) * TILE2 : Db + (int64_t)I * TILE2;
            for (int e = tid; e < TILE2; e += blockDim.x) {
                const int r = e >> 5, c = e & 31;
                bwdS[bo + (int64_t)t * TILE2 + swz_index<TS>(r, c)] = stf<TS>((double)src[r * TILE + c]);
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

__device__ __forceinline__ void named_barrier(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
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

template <typename TS, typename TA>
cudaError_t launch_tile_solve(const SolveArgs& a, int njobs, int max_tiles, cudaStream_t st, int ncols) {
    static_assert(sizeof(TA) == 8, "the tile-profile chain solve serves the FP64 interface blocks");
    constexpr int G = group_tiles<TS>();
    return launch_ring<TS, TA, G, 4, 2>(a, njobs, max_tiles, st, ncols);   // 4 far groups, 2 critical pairs
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

template void launch_finalize<double, double>(int, const Profile&, const double*, const double*, double*,
                                              double*, cudaStream_t);
template cudaError_t launch_tile_solve<double, double>(const SolveArgs&, int, int, cudaStream_t, int);
template void launch_convert<float>(int64_t, const double*, float*, cudaStream_t);

}  // namespace am
