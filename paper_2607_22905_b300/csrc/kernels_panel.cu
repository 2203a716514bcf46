// Multi-column local solves for the FP32 / BF16 sweep streams: out = S L^{-T} L^{-1} S in
// for up to PANEL_NC right-hand sides of one subdomain at once, used for the multiscale
// basis functions of Algorithm 1 (Eq. def-phat-local: the k_i columns -B_i psi_m of one
// subdomain share its factor, which is therefore streamed once per PANEL_NC columns).
//
// One CTA (4 warps) per job walks the subdomain's tile rows in stream order, forward then
// backward, a block of 32 rows x PANEL_NC columns per step.  Thread (lane r, warp w) owns
// row r of columns 8w .. 8w+7: it reads its tile row as 16-byte chunks (the streams'
// swizzle makes those reads conflict-free) and the operand rows from shared memory as
// broadcast 16-byte loads.  Per step:
//   t_I = b_I - sum_J M_IJ x_J      (M: the stream's off-diagonal tiles, x_J of the rows
//                                    within the profile band, kept in a ring of wm blocks)
//   x_I = D_I t_I (+ C t_prev)      (the pair coupling of the FP32 / BF16 streams: row b's
//                                    coupling tile C multiplies the previous row's t)
// The right-hand sides come scaled in FP32 (`w32`, written by k_mbf_rhs32); the forward
// results overwrite them in place and come back as the backward right-hand side, loaded
// one step ahead; the step's tiles are copied by 16-byte asynchronous copies one step
// ahead; the results go to the FP64 output with an exact float -> double conversion in
// integer arithmetic (B300 runs the conversion instruction on its FP64 pipe).
#include <cstdint>
#include <type_traits>

#include "async.cuh"
#include "common.cuh"
#include "kernels.h"

namespace am {

namespace {

constexpr int XS = PANEL_NC + 4;   // row stride (floats) of the operand blocks in shared memory

// acc[j] += sum_t M(r, t) X(t, c0 + j), j < 8, for the tile M (stream format) and the
// 32 x PANEL_NC block X (row t at X + t * XS)
__device__ __forceinline__ void tile_rows_acc(const float* tile, const float* X, int r, int c0, float (&acc)[8]) {
    const float4* row = reinterpret_cast<const float4*>(tile + r * TILE);
    const int key = swz_row_key<float>(r);
#pragma unroll
    for (int ch = 0; ch < 8; ++ch) {
        const float4 m = row[ch ^ key];
        const float mv[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float* xr = X + (ch * 4 + u) * XS + c0;
            const float4 x0 = *reinterpret_cast<const float4*>(xr);
            const float4 x1 = *reinterpret_cast<const float4*>(xr + 4);
            acc[0] = fmaf(mv[u], x0.x, acc[0]);
            acc[1] = fmaf(mv[u], x0.y, acc[1]);
            acc[2] = fmaf(mv[u], x0.z, acc[2]);
            acc[3] = fmaf(mv[u], x0.w, acc[3]);
            acc[4] = fmaf(mv[u], x1.x, acc[4]);
            acc[5] = fmaf(mv[u], x1.y, acc[5]);
            acc[6] = fmaf(mv[u], x1.z, acc[6]);
            acc[7] = fmaf(mv[u], x1.w, acc[7]);
        }
    }
}
__device__ __forceinline__ void tile_rows_acc(const __nv_bfloat16* tile, const float* X, int r, int c0,
                                              float (&acc)[8]) {
    const uint4* row = reinterpret_cast<const uint4*>(tile + r * TILE);
    const int key = swz_row_key<__nv_bfloat16>(r);
#pragma unroll
    for (int ch = 0; ch < 4; ++ch) {
        const uint4 m = row[ch ^ key];
        const uint32_t w4[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const float2 p = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w4[h]));
            const float mv[2] = {p.x, p.y};
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const float* xr = X + (ch * 8 + h * 2 + u) * XS + c0;
                const float4 x0 = *reinterpret_cast<const float4*>(xr);
                const float4 x1 = *reinterpret_cast<const float4*>(xr + 4);
                acc[0] = fmaf(mv[u], x0.x, acc[0]);
                acc[1] = fmaf(mv[u], x0.y, acc[1]);
                acc[2] = fmaf(mv[u], x0.z, acc[2]);
                acc[3] = fmaf(mv[u], x0.w, acc[3]);
                acc[4] = fmaf(mv[u], x1.x, acc[4]);
                acc[5] = fmaf(mv[u], x1.y, acc[5]);
                acc[6] = fmaf(mv[u], x1.z, acc[6]);
                acc[7] = fmaf(mv[u], x1.w, acc[7]);
            }
        }
    }
}

// float -> double, exact for normal numbers and zeros (denormals become signed zeros)
__device__ __forceinline__ double f2d_exact(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xffu;
    uint64_t bits = (uint64_t)(u & 0x80000000u) << 32;
    if (e == 0xffu) bits |= 0x7ff0000000000000ull | ((uint64_t)(u & 0x7fffffu) << 29);
    else if (e != 0) bits |= ((uint64_t)(e + 896u) << 52) | ((uint64_t)(u & 0x7fffffu) << 29);
    return __longlong_as_double((long long)bits);
}

}  // namespace

// w32[phi_off[s] + col * n_s + row] = (float)(-g_val) * scale32 of the row: the MBF right-hand
// sides -B_i psi_m of Eq. (def-phat-local), scaled (w32 zeroed beforehand)
__global__ void k_mbf_rhs32(int m, const int64_t* __restrict__ g_off, const int32_t* __restrict__ g_row,
                            const int32_t* __restrict__ g_col, const double* __restrict__ g_val,
                            const int32_t* __restrict__ rows, const int64_t* __restrict__ phi_off,
                            const float* __restrict__ sc32, const int64_t* __restrict__ sc_off,
                            float* __restrict__ w32) {
    const int s = blockIdx.x;
    if (s >= m) return;
    const int64_t ns = rows[s];
    for (int64_t t = g_off[s] + threadIdx.x; t < g_off[s + 1]; t += blockDim.x)
        w32[phi_off[s] + g_col[t] * ns + g_row[t]] = (float)(-g_val[t]) * sc32[sc_off[s] + g_row[t]];
}

void launch_mbf_rhs32(int m, const int64_t* g_off, const int32_t* g_row, const int32_t* g_col, const double* g_val,
                      const int32_t* rows, const int64_t* phi_off, const float* sc32, const int64_t* sc_off,
                      float* w32, cudaStream_t st) {
    if (m <= 0) return;
    count_launch();
    k_mbf_rhs32<<<m, 128, 0, st>>>(m, g_off, g_row, g_col, g_val, rows, phi_off, sc32, sc_off, w32);
}

// IN64: the right-hand sides come from a.in (FP64, scaled here; batched PCG columns with
// their stop flags, column c of the job being column job_col0 + c), w32 then only holds
// the forward results; a.accumulate adds the result to a.out.  Otherwise (the MBFs) w32
// holds the scaled FP32 right-hand sides.
template <typename TS, bool IN64>
__global__ void __launch_bounds__(128) k_panel_solve(SolveArgs a, float* __restrict__ w32, int wm) {
    constexpr int NT = 128;
    constexpr uint32_t TB = TILE2 * sizeof(TS);
    const int job = blockIdx.x;
    const int s = a.job_sub[job];
    const int nc = a.job_nc[job];
    const int64_t ld = a.job_ld[job];
    const int col0 = IN64 && a.job_col0 ? a.job_col0[job] : 0;
    // columns of the job that still run (PCG stop flags); none: nothing to do
    uint32_t live = 0;
    for (int c = 0; c < nc; ++c)
        if (!(IN64 && a.done && a.done[(int64_t)(col0 + c) * a.done_stride])) live |= 1u << c;
    if (!live) return;
    const Profile pf = a.pf;
    const int n = pf.rows[s], T = pf.ntiles[s];
    const int64_t r0 = pf.row0[s];
    const int64_t nts = pf.fwd[r0 + T - 1] + (T - 1 - pf.lo[r0 + T - 1]) + 1;   // tiles per stream
    const TS* F = (const TS*)a.fwdS + pf.base[s] * TILE2;
    const TS* Bk = (const TS*)a.bwdS + pf.base[s] * TILE2;
    const float* sc32 = a.scale32 ? a.scale32 + a.scale_off[s] : nullptr;
    float* wv = w32 + a.job_in[job];
    double* out = a.out + a.job_in[job];
    const double* in = IN64 ? a.in + a.job_in[job] : nullptr;
    const int tid = threadIdx.x, r = tid & 31, w = tid >> 5, c0 = 8 * w;

    extern __shared__ __align__(16) unsigned char pn_raw[];
    TS* stage = reinterpret_cast<TS*>(pn_raw);                                   // [2][wm] tiles
    float* ring = reinterpret_cast<float*>(pn_raw + (size_t)2 * wm * TB);         // [wm][32][XS]
    float* tb = ring + (size_t)wm * TILE * XS;                                   // [2][32][XS]
    int32_t* lo_s = reinterpret_cast<int32_t*>(tb + 2 * TILE * XS);
    int32_t* hi_s = lo_s + T;
    for (int i = tid; i < T; i += NT) {
        lo_s[i] = pf.lo[r0 + i];
        hi_s[i] = pf.hi[r0 + i];
    }
    for (int i = tid; i < 2 * TILE * XS; i += NT) tb[i] = 0.0f;
    __syncthreads();
    // step k (0 .. 2T-1): row I, its off-diagonal count nt, first stream tile q
    auto step_rows = [&](int k, int& I, int& nt) {
        if (k < T) {
            I = k;
            nt = I - lo_s[I];
        } else {
            I = 2 * T - 1 - k;
            nt = hi_s[I] - I;
        }
    };
    auto issue = [&](int k, int64_t q, int buf) {
        int I, nt;
        step_rows(k, I, nt);
        const TS* src = q < nts ? F + q * TILE2 : Bk + (q - nts) * TILE2;
        const char* g = reinterpret_cast<const char*>(src);
        const uint32_t dst = smem_u32(stage + (size_t)buf * wm * TILE2);
        const int nch = (nt + 1) * (int)(TB / 16);
        for (int i = tid; i < nch; i += NT)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + 16u * i), "l"(g + 16 * (int64_t)i)
                         : "memory");
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    auto on = [&](int j) { return ((live >> (c0 + j)) & 1u) != 0; };
    // right-hand side block of step k (row `lane` of its 8 columns): the scaled input
    // (forward) or the forward result (backward), from w32; FP64 inputs are loaded raw
    // here and converted when used, so that the load's latency falls in the step before
    auto load_rhs = [&](int k, float (&v)[8], double (&vd)[8]) {
        int I, nt;
        step_rows(k, I, nt);
        const int row = I * TILE + r;
        if (IN64 && k < T) {
#pragma unroll
            for (int j = 0; j < 8; ++j) vd[j] = (row < n && on(j)) ? in[(int64_t)(c0 + j) * ld + row] : 0.0;
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = (row < n && on(j)) ? wv[(int64_t)(c0 + j) * ld + row] : 0.0f;
        }
    };
    int64_t q = 0;
    issue(0, 0, 0);
    float bvn[8];
    double bvd[8];
    load_rhs(0, bvn, bvd);
    int cur = 0;
    for (int k = 0; k < 2 * T; ++k) {
        int I, nt;
        step_rows(k, I, nt);
        const bool fwd = k < T;
        const int64_t qn = q + nt + 1;
        if (k + 1 < 2 * T) issue(k + 1, qn, (k + 1) & 1);
        else asm volatile("cp.async.commit_group;" ::: "memory");
        const int row = I * TILE + r;
        float bv[8];
        if (IN64 && fwd) {
            const float f = (row < n && sc32) ? sc32[row] : 1.0f;
#pragma unroll
            for (int j = 0; j < 8; ++j) bv[j] = (float)bvd[j] * f;
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) bv[j] = bvn[j];
        }
        // the next step's block, one step ahead (the first backward step's is the last
        // forward result, still in registers)
        if (k + 1 < 2 * T && k + 1 != T) load_rhs(k + 1, bvn, bvd);
        asm volatile("cp.async.wait_group 1;" ::: "memory");
        __syncthreads();
        const TS* st = stage + (size_t)(k & 1) * wm * TILE2;
        // coupling tile of the pair (forward: row b's last off-diagonal; backward: row a's first)
        const int tc = nt == 0 ? -1 : (fwd ? ((I & 1) ? nt - 1 : -1) : ((I & 1) ? -1 : 0));
        const int j0 = fwd ? lo_s[I] : I + 1;
        float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int t = 0; t < nt; ++t) {
            if (t == tc) continue;
            tile_rows_acc(st + (size_t)t * TILE2, ring + (size_t)((j0 + t) % wm) * TILE * XS, r, c0, acc);
        }
        float* tn = tb + (size_t)cur * TILE * XS;
        float tv[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) tv[j] = bv[j] - acc[j];
        *reinterpret_cast<float4*>(tn + r * XS + c0) = make_float4(tv[0], tv[1], tv[2], tv[3]);
        *reinterpret_cast<float4*>(tn + r * XS + c0 + 4) = make_float4(tv[4], tv[5], tv[6], tv[7]);
        __syncthreads();
        float x[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        tile_rows_acc(st + (size_t)nt * TILE2, tn, r, c0, x);
        if (tc >= 0) tile_rows_acc(st + (size_t)tc * TILE2, tb + (size_t)(cur ^ 1) * TILE * XS, r, c0, x);
        float* xs = ring + (size_t)(I % wm) * TILE * XS + r * XS + c0;
        *reinterpret_cast<float4*>(xs) = make_float4(x[0], x[1], x[2], x[3]);
        *reinterpret_cast<float4*>(xs + 4) = make_float4(x[4], x[5], x[6], x[7]);
        if (row < n) {
            if (fwd) {
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (on(j)) wv[(int64_t)(c0 + j) * ld + row] = x[j];
            } else {
                const float f = sc32 ? sc32[row] : 1.0f;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if (!on(j)) continue;
                    double* o = out + (int64_t)(c0 + j) * ld + row;
                    const double y = f2d_exact(x[j] * f);
                    if (IN64 && a.accumulate) *o += y;
                    else *o = y;
                }
            }
        }
        if (k + 1 == T) {
#pragma unroll
            for (int j = 0; j < 8; ++j) bvn[j] = (row < n && on(j)) ? x[j] : 0.0f;
        }
        __syncthreads();
        cur ^= 1;
        q = qn;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

size_t panel_solve_smem(int wm, int max_tiles, size_t ts) {
    return (size_t)2 * wm * TILE2 * ts + ((size_t)wm + 2) * TILE * XS * sizeof(float) +
           (size_t)2 * max_tiles * sizeof(int32_t) + 16;
}
bool panel_solve_fits(int wm, int max_tiles, size_t ts) { return panel_solve_smem(wm, max_tiles, ts) <= 227 * 1024; }

template <typename TS, bool IN64>
static cudaError_t launch_panel(const SolveArgs& a, float* w32, int njobs, int max_tiles, int wm, cudaStream_t st) {
    if (njobs <= 0) return cudaSuccess;
    const size_t smem = panel_solve_smem(wm, max_tiles, sizeof(TS));
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    cudaError_t e =
        cudaFuncSetAttribute(k_panel_solve<TS, IN64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    count_launch();
    k_panel_solve<TS, IN64><<<njobs, 128, smem, st>>>(a, w32, wm);
    return cudaGetLastError();
}
template <typename TS>
cudaError_t launch_panel_solve(const SolveArgs& a, float* w32, int njobs, int max_tiles, int wm, cudaStream_t st) {
    return launch_panel<TS, false>(a, w32, njobs, max_tiles, wm, st);
}
template <typename TS>
cudaError_t launch_panel_solve_cols(const SolveArgs& a, float* w32, int njobs, int max_tiles, int wm, cudaStream_t st) {
    return launch_panel<TS, true>(a, w32, njobs, max_tiles, wm, st);
}

template cudaError_t launch_panel_solve<float>(const SolveArgs&, float*, int, int, int, cudaStream_t);
template cudaError_t launch_panel_solve<__nv_bfloat16>(const SolveArgs&, float*, int, int, int, cudaStream_t);
template cudaError_t launch_panel_solve_cols<float>(const SolveArgs&, float*, int, int, int, cudaStream_t);
template cudaError_t launch_panel_solve_cols<__nv_bfloat16>(const SolveArgs&, float*, int, int, int, cudaStream_t);

}  // namespace am
