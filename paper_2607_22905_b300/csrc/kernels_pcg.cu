// Global-vector kernels of AlgMortar-PCG on sm_103a: CSR SpMV, the fused FP64 CG vector
// updates and dot products (Sec. 7: x0 = 0, Euclidean relative-residual stop), the
// interface restriction and prolongation of Algorithm 2, and the coarse interface solve
// as a product with the explicit (symmetrised) inverse.
//
// Dot products are deterministic: every partial-producing kernel runs with exactly
// vec_grid() CTAs, writes one partial per CTA, and consumers sum the partials in a fixed
// order (warp_sum_partials), so repeated runs give bit-identical scalars.
#include <atomic>
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace am {

static std::atomic<int64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void add_launches(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

static int g_vec_grid = 4 * 148;
int vec_grid() { return g_vec_grid; }
void set_vec_grid(int sms) { g_vec_grid = 4 * (sms > 0 ? sms : 148); }

#define GRID_STRIDE(i, n) \
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

__global__ void k_gather(int64_t n, const int32_t* __restrict__ perm, const double* __restrict__ src,
                         double* __restrict__ dst) {
    GRID_STRIDE(k, n) dst[k] = src[perm[k]];
}

__global__ void k_scatter_values(int64_t n, const int64_t* __restrict__ idx, const double* __restrict__ v,
                                 double* __restrict__ dst) {
    GRID_STRIDE(k, n) dst[idx[k]] = v[k];
}

__global__ void k_scatter(int64_t n, const int32_t* __restrict__ perm, const double* __restrict__ src,
                          double* __restrict__ dst) {
    GRID_STRIDE(k, n) dst[perm[k]] = src[k];
}

// b_eta[I] = -1/4 sum_k G[k, I] pbar_k = sum_{(k,l) in E_I} |a_kl| (pbar_k + pbar_l)/2 --
// the interface right-hand side of Eq. (interface-problem-alg), one warp per interface.
__global__ void k_restrict(int L, const int64_t* __restrict__ rptr, const int32_t* __restrict__ rcell,
                           const double* __restrict__ rcoef, const double* __restrict__ pbar,
                           double* __restrict__ beta, const int32_t* __restrict__ omap,
                           const int32_t* __restrict__ done) {
    if (done && *done) return;
    int I = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    int lane = threadIdx.x & 31;
    if (I >= L) return;
    double s = 0.0;
    for (int64_t t = rptr[I] + lane; t < rptr[I + 1]; t += 32) s += rcoef[t] * pbar[rcell[t]];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) beta[omap ? omap[I] : I] = s;
}

// eta = S_eta^{-1} b_eta, one warp per row of the explicit inverse (FP64).
__global__ void k_coarse_gemv(int L, const double* __restrict__ Sinv, const double* __restrict__ b,
                              double* __restrict__ eta, const int32_t* __restrict__ done) {
    if (done && *done) return;
    int I = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    int lane = threadIdx.x & 31;
    if (I >= L) return;
    const double* row = Sinv + (int64_t)I * L;
    double s = 0.0;
    for (int J = lane; J < L; J += 32) s += row[J] * __ldg(b + J);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) eta[I] = s;
}

// z_k = pbar_k + sum_{m in I_i} eta_m p_hat_i^(m)_k  (Eq. p-decomposition-alg), fused with
// the partial of r . z when r is given.
template <typename TP>
__global__ void __launch_bounds__(VEC_BS) k_prolong(int64_t n, const int32_t* __restrict__ row_sub,
                                                     const int64_t* __restrict__ sub_off,
                                                     const int64_t* __restrict__ if_off,
                                                     const int32_t* __restrict__ if_list,
                                                     const int64_t* __restrict__ phi_off,
                                                     const TP* __restrict__ phi, const double* __restrict__ eta,
                                                     const double* __restrict__ pbar, double* __restrict__ z,
                                                     const double* __restrict__ r, double* __restrict__ part,
                                                     const int32_t* __restrict__ done) {
    if (done && *done) return;
    __shared__ double sh[32];
    double acc = 0.0;
    GRID_STRIDE(k, n) {
        int32_t s = row_sub[k];
        int64_t a = sub_off[s];
        int64_t ns = sub_off[s + 1] - a;
        int64_t i0 = if_off[s];
        int kk = (int)(if_off[s + 1] - i0);
        const TP* ph = phi + phi_off[s] + (k - a);
        // the correction sum_m eta_m p_hat^(m) is accumulated in the panel's arithmetic
        // (FP64 panels: FP64; FP32/BF16 panels: FP32), then added to pbar in FP64
        using TA = typename std::conditional<sizeof(TP) == 8, double, float>::type;
        TA corr = 0;
        for (int c = 0; c < kk; ++c) corr += ldf<TA>(ph + c * ns) * (TA)eta[if_list[i0 + c]];
        double v = pbar[k] + (double)corr;
        z[k] = v;
        if (r) acc += r[k] * v;
    }
    if (part) {
        double s = block_sum(acc, sh);
        if (threadIdx.x == 0) part[blockIdx.x] = s;
    }
}

// ------------------------------------------------------------------------------ PCG
__global__ void __launch_bounds__(VEC_BS) k_pcg_init(int64_t n, const double* __restrict__ b,
                                                      double* __restrict__ x, double* __restrict__ r,
                                                      double* __restrict__ part) {
    __shared__ double sh[32];
    double acc = 0.0;
    GRID_STRIDE(k, n) {
        double v = b[k];
        r[k] = v;
        x[k] = 0.0;
        acc += v * v;
    }
    double s = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_pcg_start(PcgScalars* sc, const double* __restrict__ part, int np, double tol, int max_it,
                            int flexible) {
    double bb = warp_sum_partials(part, np);
    if (threadIdx.x == 0) {
        sc->bb = bb;
        sc->rr = bb;
        sc->tol2 = tol * tol * bb;
        sc->iter = 0;
        sc->done = bb == 0.0 ? 1 : 0;
        sc->status = 0;
        sc->max_it = max_it;
        sc->flexible = flexible;
        sc->rz = 0.0;
        sc->rz_prev = 0.0;
        sc->alpha = sc->beta = sc->pq = 0.0;
    }
}

// p = z + beta p, beta = rho_k / rho_{k-1} (0 on the first iteration).
__global__ void __launch_bounds__(VEC_BS) k_pcg_p(int64_t n, const double* __restrict__ z, double* __restrict__ p,
                                                   PcgScalars* __restrict__ sc, const double* __restrict__ part_rz,
                                                   int np) {
    if (sc->done) return;
    __shared__ double s_beta;
    if (threadIdx.x < 32) {
        double rz = warp_sum_partials(part_rz, np);
        if (threadIdx.x == 0) s_beta = sc->iter == 0 ? 0.0 : rz / sc->rz;
    }
    __syncthreads();
    const double beta = s_beta;
    GRID_STRIDE(k, n) p[k] = z[k] + beta * p[k];
}

// q = A p (CSR, one thread per row) and the partial of p . q; CTA 0 records rho_k.
__global__ void __launch_bounds__(VEC_BS) k_pcg_spmv(int64_t n, const int32_t* __restrict__ rowptr,
                                                      const int32_t* __restrict__ col,
                                                      const double* __restrict__ val,
                                                      const double* __restrict__ p, double* __restrict__ q,
                                                      double* __restrict__ part_pq, PcgScalars* __restrict__ sc,
                                                      const double* __restrict__ part_rz, int np) {
    if (sc->done) return;
    __shared__ double sh[32];
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        double rz = warp_sum_partials(part_rz, np);
        if (threadIdx.x == 0) {
            sc->rz_prev = sc->rz;
            sc->rz = rz;
        }
    }
    double acc = 0.0;
    GRID_STRIDE(k, n) {
        double s = 0.0;
        for (int32_t e = rowptr[k]; e < rowptr[k + 1]; ++e) s += val[e] * __ldg(p + col[e]);
        q[k] = s;
        acc += p[k] * s;
    }
    double s = block_sum(acc, sh);
    if (threadIdx.x == 0) part_pq[blockIdx.x] = s;
}

// Same product on the sliced-ELL copy: one thread per row, the warp = one 32-row slice,
// every load of values/columns is one contiguous 256/128-byte segment.
__global__ void __launch_bounds__(VEC_BS) k_pcg_spmv_ell(int64_t n, const int64_t* __restrict__ ell_ptr,
                                                          const int32_t* __restrict__ ell_col,
                                                          const double* __restrict__ ell_val,
                                                          const double* __restrict__ p, double* __restrict__ q,
                                                          double* __restrict__ part_pq, PcgScalars* __restrict__ sc,
                                                          const double* __restrict__ part_rz, int np) {
    if (sc->done) return;
    __shared__ double sh[32];
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        double rz = warp_sum_partials(part_rz, np);
        if (threadIdx.x == 0) {
            sc->rz_prev = sc->rz;
            sc->rz = rz;
        }
    }
    double acc = 0.0;
    GRID_STRIDE(k, n) {
        const int64_t sl = k >> 5;
        const int r = (int)(k & 31);
        const int64_t b = ell_ptr[sl], w = (ell_ptr[sl + 1] - b) >> 5;
        const double* v = ell_val + b + r;
        const int32_t* c = ell_col + b + r;
        double s = 0.0;
        for (int64_t e = 0; e < w; ++e) s += __ldg(v + e * 32) * __ldg(p + __ldg(c + e * 32));
        q[k] = s;
        acc += p[k] * s;
    }
    double s = block_sum(acc, sh);
    if (threadIdx.x == 0) part_pq[blockIdx.x] = s;
}

// ell_val[t] = val[src[t]] (0 for padding)
__global__ void k_ell_values(int64_t nell, const int32_t* __restrict__ src, const double* __restrict__ val,
                             double* __restrict__ ell_val) {
    GRID_STRIDE(t, nell) {
        const int32_t s = src[t];
        ell_val[t] = s >= 0 ? val[s] : 0.0;
    }
}

// alpha = rho_k / (p . q);  x += alpha p;  r -= alpha q;  partial of ||r||^2.
__global__ void __launch_bounds__(VEC_BS) k_pcg_xr(int64_t n, double* __restrict__ x, double* __restrict__ r,
                                                    const double* __restrict__ p, const double* __restrict__ q,
                                                    PcgScalars* __restrict__ sc, const double* __restrict__ part_pq,
                                                    double* __restrict__ part_rr, int np) {
    if (sc->done) return;
    __shared__ double sh[32];
    __shared__ double s_alpha;
    __shared__ int s_ok;
    if (threadIdx.x < 32) {
        double pq = warp_sum_partials(part_pq, np);
        if (threadIdx.x == 0) {
            double al = sc->rz / pq;
            s_ok = (pq > 0.0 && isfinite(al)) ? 1 : 0;
            s_alpha = al;
        }
    }
    __syncthreads();
    const double al = s_alpha;
    const int ok = s_ok;
    double acc = 0.0;
    GRID_STRIDE(k, n) {
        double rk = r[k];
        if (ok) {
            x[k] += al * p[k];
            rk -= al * q[k];
            r[k] = rk;
        }
        acc += rk * rk;
    }
    double s = block_sum(acc, sh);
    if (threadIdx.x == 0) part_rr[blockIdx.x] = s;
}

__global__ void k_pcg_check(PcgScalars* sc, const double* __restrict__ part_pq, const double* __restrict__ part_rr,
                            int np) {
    if (sc->done) return;
    double pq = warp_sum_partials(part_pq, np);
    double rr = warp_sum_partials(part_rr, np);
    if (threadIdx.x == 0) {
        sc->iter += 1;
        sc->pq = pq;
        double al = sc->rz / pq;
        sc->alpha = al;
        if (!(pq > 0.0) || !isfinite(al) || !isfinite(rr)) {
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
}

// partials of ||b - A x||^2 (true residual)
__global__ void __launch_bounds__(VEC_BS) k_residual(int64_t n, const int32_t* __restrict__ rowptr,
                                                      const int32_t* __restrict__ col,
                                                      const double* __restrict__ val,
                                                      const double* __restrict__ x, const double* __restrict__ b,
                                                      double* __restrict__ part) {
    __shared__ double sh[32];
    double acc = 0.0;
    GRID_STRIDE(k, n) {
        double s = b[k];
        for (int32_t e = rowptr[k]; e < rowptr[k + 1]; ++e) s -= val[e] * x[col[e]];
        acc += s * s;
    }
    double s = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_sum_partials(const double* __restrict__ part, int np, double* __restrict__ out) {
    double s = warp_sum_partials(part, np);
    if (threadIdx.x == 0) *out = s;
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
    count_launch();
    k_gather<<<grid_for(n, 256), 256, 0, st>>>(n, perm, src, dst);
}
void launch_scatter_values(int64_t n, const int64_t* idx, const double* v, double* dst, cudaStream_t st) {
    if (n > 0) {
        count_launch();
        k_scatter_values<<<grid_for(n, 256), 256, 0, st>>>(n, idx, v, dst);
    }
}
void launch_scatter(int64_t n, const int32_t* perm, const double* src, double* dst, cudaStream_t st) {
    count_launch();
    k_scatter<<<grid_for(n, 256), 256, 0, st>>>(n, perm, src, dst);
}
void launch_restrict(int L, const int64_t* rptr, const int32_t* rcell, const double* rcoef, const double* pbar,
                     double* beta, const int32_t* omap, const int32_t* done, cudaStream_t st) {
    if (L > 0) {
        count_launch();
        k_restrict<<<(L + 7) / 8, 256, 0, st>>>(L, rptr, rcell, rcoef, pbar, beta, omap, done);
    }
}
void launch_coarse_gemv(int L, const double* Sinv, const double* b, double* eta, const int32_t* done,
                        cudaStream_t st) {
    if (L > 0) {
        count_launch();
        k_coarse_gemv<<<(L + 7) / 8, 256, 0, st>>>(L, Sinv, b, eta, done);
    }
}
template <typename TP>
void launch_prolong(int64_t n, const int32_t* row_sub, const int64_t* sub_off, const int64_t* if_off,
                    const int32_t* if_list, const int64_t* phi_off, const TP* phi, const double* eta,
                    const double* pbar, double* z, const double* r, double* part, const int32_t* done,
                    cudaStream_t st) {
    count_launch();
    k_prolong<TP><<<vec_grid(), VEC_BS, 0, st>>>(n, row_sub, sub_off, if_off, if_list, phi_off, phi, eta, pbar, z,
                                                 r, part, done);
}
void launch_pcg_init(int64_t n, const double* b, double* x, double* r, double* part, cudaStream_t st) {
    count_launch();
    k_pcg_init<<<vec_grid(), VEC_BS, 0, st>>>(n, b, x, r, part);
}
void launch_pcg_start(PcgScalars* sc, const double* part_bb, double tol, int max_it, int flexible,
                      cudaStream_t st) {
    count_launch();
    k_pcg_start<<<1, 32, 0, st>>>(sc, part_bb, vec_grid(), tol, max_it, flexible);
}
void launch_pcg_p(int64_t n, const double* z, double* p, const double* r, double* r_old, PcgScalars* sc,
                  const double* part_rz, cudaStream_t st) {
    (void)r;
    (void)r_old;
    count_launch();
    k_pcg_p<<<vec_grid(), VEC_BS, 0, st>>>(n, z, p, sc, part_rz, vec_grid());
}
void launch_pcg_spmv(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                     const double* p, double* q, double* part_pq, PcgScalars* sc, const double* part_rz,
                     cudaStream_t st) {
    count_launch();
    k_pcg_spmv<<<vec_grid(), VEC_BS, 0, st>>>(n, rowptr, col, val, p, q, part_pq, sc, part_rz, vec_grid());
}
void launch_pcg_spmv_ell(int64_t n, const int64_t* ell_ptr, const int32_t* ell_col, const double* ell_val,
                         const double* p, double* q, double* part_pq, PcgScalars* sc, const double* part_rz,
                         cudaStream_t st) {
    count_launch();
    k_pcg_spmv_ell<<<vec_grid(), VEC_BS, 0, st>>>(n, ell_ptr, ell_col, ell_val, p, q, part_pq, sc, part_rz,
                                                  vec_grid());
}
void launch_ell_values(int64_t nell, const int32_t* src, const double* val, double* ell_val, cudaStream_t st) {
    count_launch();
    k_ell_values<<<grid_for(nell, 256), 256, 0, st>>>(nell, src, val, ell_val);
}
void launch_pcg_xr(int64_t n, double* x, double* r, const double* p, const double* q, PcgScalars* sc,
                   const double* part_pq, double* part_rr, cudaStream_t st) {
    count_launch();
    k_pcg_xr<<<vec_grid(), VEC_BS, 0, st>>>(n, x, r, p, q, sc, part_pq, part_rr, vec_grid());
}
void launch_pcg_check(PcgScalars* sc, const double* part_pq, const double* part_rr, cudaStream_t st) {
    count_launch();
    k_pcg_check<<<1, 32, 0, st>>>(sc, part_pq, part_rr, vec_grid());
}
void launch_residual(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                     const double* x, const double* b, double* part, cudaStream_t st) {
    count_launch();
    k_residual<<<vec_grid(), VEC_BS, 0, st>>>(n, rowptr, col, val, x, b, part);
}
void launch_tpfa_grad(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val, const double* K,
                      const double* tb, const double* tbp, const double* p, const double* lam, double* grad,
                      cudaStream_t st) {
    count_launch();
    k_tpfa_grad<<<grid_for(n, 256), 256, 0, st>>>(n, rowptr, col, val, K, tb, tbp, p, lam, grad);
}
void launch_sum_partials(const double* part, double* out, cudaStream_t st) {
    count_launch();
    k_sum_partials<<<1, 32, 0, st>>>(part, vec_grid(), out);
}

template void launch_prolong<double>(int64_t, const int32_t*, const int64_t*, const int64_t*, const int32_t*,
                                     const int64_t*, const double*, const double*, const double*, double*,
                                     const double*, double*, const int32_t*, cudaStream_t);
template void launch_prolong<float>(int64_t, const int32_t*, const int64_t*, const int64_t*, const int32_t*,
                                    const int64_t*, const float*, const double*, const double*, double*,
                                    const double*, double*, const int32_t*, cudaStream_t);
template void launch_prolong<__nv_bfloat16>(int64_t, const int32_t*, const int64_t*, const int64_t*,
                                            const int32_t*, const int64_t*, const __nv_bfloat16*, const double*,
                                            const double*, double*, const double*, double*, const int32_t*,
                                            cudaStream_t);

}  // namespace am
