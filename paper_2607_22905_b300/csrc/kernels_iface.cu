// Inexact interface solve of AlgMortar on sm_103a (Sec. 7 solver settings: the interface
// system of Algorithm 2 solved by PCG with a block-Jacobi preconditioner to a relative
// tolerance, inside a flexible outer CG).
//
//   setup:  S_eta = diag(T) + 1/4 G^T Phi  in CSR (interfaces in their natural order,
//           i.e. pairs (i, j), i < j, lexicographic), and the explicit inverse of each
//           block-Jacobi block (interfaces (i, j) with equal i / g), formed in FP64 and
//           stored in FP32.
//   apply:  the whole inner PCG in ONE launch per right-hand side: a thread-block cluster
//           of up to 16 CTAs, each owning a contiguous, block-aligned range of rows.  Every
//           CTA keeps a full copy of the search direction p in shared memory; after each
//           update a CTA writes its own rows of p into every CTA's copy through distributed
//           shared memory, and the hardware cluster barrier orders those writes before the
//           next product.  Dot products: FP32 within a warp, FP64 across warps and CTAs, each
//           CTA adding the CTAs' partials in the same fixed order, so all CTAs take the same
//           stop decision.  S_eta rows and block inverses are staged in shared memory when
//           they fit.  No spin-waits: every wait is a cluster or CTA barrier.
//
// FP32 is the working precision of the inner solve (its tolerance is 1e-2); on B300 the
// FP64 pipe runs at 1/64 of FP32, and a cluster is too few SMs for FP64 products.
#include <cooperative_groups.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace am {

// CSR values of S_eta: off-diagonal (I, J) from the one subdomain the two interfaces share
// (pv[csr_src[e]], symmetrised at assembly), diagonal T_I + both sides' contributions in
// the order used by the exact path.
__global__ void k_iface_csr_values(int L, const int32_t* __restrict__ s_ptr, const int32_t* __restrict__ s_col,
                                   const int64_t* __restrict__ csr_src, const double* __restrict__ pv,
                                   const double* __restrict__ T, const double* __restrict__ diagc,
                                   double* __restrict__ s_val64, float2* __restrict__ s_ent) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= L) return;
    for (int32_t e = s_ptr[I]; e < s_ptr[I + 1]; ++e) {
        const int J = s_col[e];
        const double v = (J == I) ? T[I] + diagc[2 * I] + diagc[2 * I + 1] : pv[csr_src[e]];
        s_val64[e] = v;
        s_ent[e] = make_float2((float)v, __int_as_float(J));   // FP32 value, column bits
    }
}

// Explicit inverse of each block-Jacobi block (rows [b0, b1) of S_eta, nb <= IFACE_MAX_BLOCK)
// by Gauss-Jordan elimination without pivoting (S_eta is SPD, so every pivot is a positive
// Schur complement); symmetrised (X + X^T) / 2 and stored row-major in FP32.  One CTA per
// block.  A pivot <= 0 or non-finite sets err[0] = 1, err[1] = the block (first one wins).
__global__ void k_iface_block_inv(const int32_t* __restrict__ blk_row0, const int64_t* __restrict__ blk_off,
                                  const int32_t* __restrict__ s_ptr, const int32_t* __restrict__ s_col,
                                  const double* __restrict__ s_val64, float* __restrict__ binv, int* err) {
    extern __shared__ double A[];
    const int b = blockIdx.x;
    const int b0 = blk_row0[b], nb = blk_row0[b + 1] - b0;
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) A[e] = 0.0;
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x)
        for (int32_t e = s_ptr[b0 + i]; e < s_ptr[b0 + i + 1]; ++e) {
            const int j = s_col[e] - b0;
            if (j >= 0 && j < nb) A[i * nb + j] = s_val64[e];
        }
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int k = 0; k < nb; ++k) {
        const double piv = A[k * nb + k];
        if (!(piv > 0.0) || !isfinite(piv)) {
            if (threadIdx.x == 0) bad = 1;
            break;   // uniform: every thread read the same pivot
        }
        const double inv = 1.0 / piv;
        __syncthreads();
        // row k /= pivot (its diagonal becomes 1 / pivot)
        for (int j = threadIdx.x; j < nb; j += blockDim.x) A[k * nb + j] = (j == k) ? inv : A[k * nb + j] * inv;
        __syncthreads();
        // every other row: row_i -= a_ik * row_k, column k becomes -a_ik / pivot
        for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
            const int i = e / nb, j = e % nb;
            if (i == k) continue;
            const double f = A[i * nb + k];
            if (j == k) continue;
            A[e] -= f * A[k * nb + j];
        }
        __syncthreads();
        for (int i = threadIdx.x; i < nb; i += blockDim.x)
            if (i != k) A[i * nb + k] = -A[i * nb + k] * inv;
        __syncthreads();
    }
    __syncthreads();
    if (bad) {
        if (threadIdx.x == 0 && atomicCAS(err, 0, 1) == 0) err[1] = b;
        return;
    }
    float* out = binv + blk_off[b];
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        const int i = e / nb, j = e % nb;
        out[e] = (float)(0.5 * (A[i * nb + j] + A[j * nb + i]));
    }
}

// Sum of a float over the CTA: FP32 inside each warp, FP64 across the warps (one warp);
// result in every thread.  `sh` holds >= 32 doubles; the call ends with a CTA barrier.
__device__ __forceinline__ double cta_sum_f(float v, double* sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[w] = (double)v;
    __syncthreads();
    if (w == 0) {
        double s = lane < nw ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) sh[32] = s;
    }
    __syncthreads();
    const double s = sh[32];
    __syncthreads();
    return s;
}

// One inner PCG per right-hand side (gridDim.y = columns; blockIdx.x = rank in the
// cluster).  b: FP64 interface right-hand sides (natural order); eta: FP64 solutions.
__global__ void __launch_bounds__(IFACE_BS, 1) k_iface_pcg(IfaceArgs a, const double* __restrict__ b,
                                                           double* __restrict__ eta, ColStrides cs) {
    cg::cluster_group cluster = cg::this_cluster();
    const int col = blockIdx.y;
    if (cs.done && cs.done[col * cs.done_stride]) return;   // uniform over the cluster
    b += col * cs.l;
    eta += col * cs.l;
    const int me = (int)cluster.block_rank(), nc = (int)cluster.num_blocks();
    const int L = a.L;
    const int R0 = a.cta_row0[me], R1 = a.cta_row0[me + 1], nr = R1 - R0;
    const int B0 = a.cta_blk0[me], B1 = a.cta_blk0[me + 1];
    const int32_t e0 = a.s_ptr[R0], e1 = a.s_ptr[R1];
    const int64_t q0 = a.blk_off[B0], q1 = a.blk_off[B1];

    // shared memory: CTA partials, sums, the full copy of p, this CTA's vectors, per-row
    // metadata (always), and -- when they fit -- its rows of S_eta as packed (value,
    // column) pairs and its block inverses
    extern __shared__ __align__(16) unsigned char smem[];
    double* red = reinterpret_cast<double*>(smem);              // 4 * IFACE_MAX_CLUSTER partials
    double* sh = red + 4 * IFACE_MAX_CLUSTER;                  // 33 doubles (CTA sums)
    float* pf = reinterpret_cast<float*>(sh + 40);             // L: full copy of p
    const int MR = (a.max_rows + 3) & ~3;
    float* xv = pf + ((L + 3) & ~3);                           // nr each: x, r, z, q
    float* rv = xv + MR;
    float* zv = rv + MR;
    float* qv = zv + MR;
    int32_t* rp = reinterpret_cast<int32_t*>(qv + MR);         // nr + 1 local entry offsets
    int2* rinfo = reinterpret_cast<int2*>(rp + MR + 4);        // per row: (block start - R0) | nb << 16,
                                                                // offset of its inverse row
    const float2* ent;                                          // (value, column bits)
    const float* binv;                                          // this CTA's block inverses
    if (a.stage) {
        float2* st_ent = reinterpret_cast<float2*>(rinfo + MR);
        float* st_inv = reinterpret_cast<float*>(st_ent + a.max_nnz);
        for (int32_t e = threadIdx.x; e < e1 - e0; e += blockDim.x) st_ent[e] = a.s_ent[e0 + e];
        for (int64_t e = threadIdx.x; e < q1 - q0; e += blockDim.x) st_inv[e] = a.binv[q0 + e];
        ent = st_ent;
        binv = st_inv;
    } else {
        ent = a.s_ent + e0;
        binv = a.binv + q0;
    }
    for (int i = threadIdx.x; i <= nr; i += blockDim.x) rp[i] = a.s_ptr[R0 + i] - e0;
    for (int i = threadIdx.x; i < nr; i += blockDim.x) rinfo[i] = a.row_info[R0 + i];
    double* red_bb = red;
    double* red_pq = red + IFACE_MAX_CLUSTER;
    double* red_rr = red + 2 * IFACE_MAX_CLUSTER;
    double* red_rz = red + 3 * IFACE_MAX_CLUSTER;
    // all CTAs of the cluster are running before any distributed shared-memory access
    // (the barrier also publishes the staged data inside the CTA)
    cluster.sync();

    // 8 lanes per row, 4 rows per warp and step; the step loop is uniform over the warp,
    // so every lane reaches the shuffles
    const int lane8 = threadIdx.x & 7, sub = (threadIdx.x >> 3) & 3;
    const int wrp = threadIdx.x >> 5, nwrp = blockDim.x >> 5;
    // z = Binv r on this CTA's rows; returns this thread's r . z part
    auto precond = [&]() -> float {
        float part = 0.0f;
        for (int i0 = wrp * 4; i0 < nr; i0 += nwrp * 4) {
            const int i = i0 + sub;
            float s = 0.0f;
            if (i < nr) {
                const int2 ri = rinfo[i];
                const int nb = ri.x >> 16;
                const float* Bi = binv + ri.y;
                const float* rb = rv + (ri.x & 0xffff);
                for (int j = lane8; j < nb; j += 8) s = fmaf(Bi[j], rb[j], s);
            }
            s += __shfl_xor_sync(0xffffffffu, s, 4);
            s += __shfl_xor_sync(0xffffffffu, s, 2);
            s += __shfl_xor_sync(0xffffffffu, s, 1);
            if (i < nr && lane8 == 0) {
                zv[i] = s;
                part = fmaf(rv[i], s, part);
            }
        }
        return part;
    };
    // own rows of p (values already in pf[R0..R1)) to every other CTA's copy
    // (16-byte stores for the aligned body of the range; every CTA's pf sits at the same
    // 16-byte-aligned offset, so source and destination alignments agree)
    const int hd = min(nr, (4 - (R0 & 3)) & 3), nv4 = (nr - hd) >> 2, tl = hd + 4 * nv4;
    auto broadcast_p = [&]() {
        const float4* s4 = reinterpret_cast<const float4*>(pf + R0 + hd);
        for (int u = threadIdx.x; u < nc * nv4; u += blockDim.x) {
            const int c = u / nv4, i = u - c * nv4;
            if (c != me) reinterpret_cast<float4*>(cluster.map_shared_rank(pf, c) + R0 + hd)[i] = s4[i];
        }
        for (int u = threadIdx.x; u < nc * (hd + nr - tl); u += blockDim.x) {
            const int c = u / (hd + nr - tl), k = u - c * (hd + nr - tl);
            const int i = k < hd ? k : tl + (k - hd);
            if (c != me) cluster.map_shared_rank(pf, c)[R0 + i] = pf[R0 + i];
        }
    };
    auto push = [&](double* slot, double v) {   // thread 0: this CTA's partial to all CTAs
        if (threadIdx.x == 0)
            for (int c = 0; c < nc; ++c) cluster.map_shared_rank(slot, c)[me] = v;
    };
    auto total = [&](const double* slot) {       // fixed order over the CTAs (thread 0 only)
        double s = 0.0;
        for (int c = 0; c < nc; ++c) s += slot[c];
        return s;
    };
    // scalar FP64 work (sums over the CTAs, divisions, the stop test) is done by thread 0
    // and handed to the others through shared memory: B300 runs FP64 at 1/64 of FP32, so
    // 512 threads repeating it cost more than the inner iteration's products
    float* scal = reinterpret_cast<float*>(sh + 36);           // [0] alpha or beta, [1] flag

    // ---- eta_0 = 0, r_0 = b, z_0 = Binv r_0, p_0 = z_0
    float bpart = 0.0f;
    for (int i = threadIdx.x; i < nr; i += blockDim.x) {
        const float bf = (float)b[R0 + i];
        rv[i] = bf;
        xv[i] = 0.0f;
        bpart = fmaf(bf, bf, bpart);
    }
    __syncthreads();
    const float rzpart = precond();
    __syncthreads();
    for (int i = threadIdx.x; i < nr; i += blockDim.x) pf[R0 + i] = zv[i];
    __syncthreads();
    broadcast_p();
    const double bbc = cta_sum_f(bpart, sh);
    const double rzc = cta_sum_f(rzpart, sh);
    push(red_bb, bbc);
    push(red_rz, rzc);
    cluster.sync();
    double rz = 0.0, tol2 = 0.0;                            // thread 0's copies
    if (threadIdx.x == 0) {
        const double bb = total(red_bb);
        rz = total(red_rz);
        tol2 = a.rtol * a.rtol * bb;
        scal[1] = bb > 0.0 ? 1.0f : 0.0f;
    }
    __syncthreads();
    int it = 0;
    if (scal[1] != 0.0f) {
        for (;;) {
            ++it;
            // q = S p (8 lanes per row), p . q
            float pqpart = 0.0f;
            for (int i0 = wrp * 4; i0 < nr; i0 += nwrp * 4) {
                const int i = i0 + sub;
                float s = 0.0f;
                if (i < nr)
                    for (int32_t e = rp[i] + lane8; e < rp[i + 1]; e += 8) {
                        const float2 v = ent[e];
                        s = fmaf(v.x, pf[__float_as_int(v.y)], s);
                    }
                s += __shfl_xor_sync(0xffffffffu, s, 4);
                s += __shfl_xor_sync(0xffffffffu, s, 2);
                s += __shfl_xor_sync(0xffffffffu, s, 1);
                if (i < nr && lane8 == 0) {
                    qv[i] = s;
                    pqpart = fmaf(pf[R0 + i], s, pqpart);
                }
            }
            push(red_pq, cta_sum_f(pqpart, sh));
            cluster.sync();                                   // B1: p . q complete
            if (threadIdx.x == 0) {
                const double pq = total(red_pq);
                const bool ok = pq > 0.0 && isfinite(pq);     // same decision in every CTA
                scal[0] = ok ? (float)(rz / pq) : 0.0f;
                scal[1] = ok ? 1.0f : 0.0f;
            }
            __syncthreads();
            if (scal[1] == 0.0f) break;
            const float al = scal[0];
            float rrpart = 0.0f;
            for (int i = threadIdx.x; i < nr; i += blockDim.x) {
                xv[i] = __fadd_rn(xv[i], __fmul_rn(al, pf[R0 + i]));
                const float rn = __fsub_rn(rv[i], __fmul_rn(al, qv[i]));
                rv[i] = rn;
                rrpart = fmaf(rn, rn, rrpart);
            }
            __syncthreads();
            const float rz2part = precond();
            push(red_rr, cta_sum_f(rrpart, sh));
            push(red_rz, cta_sum_f(rz2part, sh));
            cluster.sync();                                   // B2: ||r||^2, r . z complete
            if (threadIdx.x == 0) {
                const double rr = total(red_rr), rzn = total(red_rz);
                const bool stop = rr <= tol2 || it >= a.max_it;
                scal[0] = stop ? 0.0f : (float)(rzn / rz);
                scal[1] = stop ? 0.0f : 1.0f;
                rz = rzn;
            }
            __syncthreads();
            if (scal[1] == 0.0f) break;
            const float be = scal[0];
            for (int i = threadIdx.x; i < nr; i += blockDim.x)
                pf[R0 + i] = __fadd_rn(zv[i], __fmul_rn(be, pf[R0 + i]));
            __syncthreads();
            broadcast_p();
            cluster.sync();                                   // B3: new p in every copy
        }
    }
    for (int i = threadIdx.x; i < nr; i += blockDim.x) eta[R0 + i] = (double)xv[i];
    if (me == 0 && threadIdx.x == 0) {
        a.its[col] = it;
        a.its_total[col] += it;
    }
    cluster.sync();   // no CTA leaves while another may still write into its shared memory
}

// ------------------------------------------------------------------------ launchers
void launch_iface_csr_values(int L, const int32_t* s_ptr, const int32_t* s_col, const int64_t* csr_src,
                             const double* pv, const double* T, const double* diagc, double* s_val64, float2* s_ent,
                             cudaStream_t st) {
    if (L <= 0) return;
    count_launch();
    k_iface_csr_values<<<(L + 255) / 256, 256, 0, st>>>(L, s_ptr, s_col, csr_src, pv, T, diagc, s_val64, s_ent);
}

cudaError_t launch_iface_block_inv(int nblk, int max_nb, const int32_t* blk_row0, const int64_t* blk_off,
                                   const int32_t* s_ptr, const int32_t* s_col, const double* s_val64, float* binv,
                                   int* err, cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    const size_t smem = (size_t)max_nb * max_nb * sizeof(double);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_iface_block_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    count_launch();
    k_iface_block_inv<<<nblk, 256, smem, st>>>(blk_row0, blk_off, s_ptr, s_col, s_val64, binv, err);
    return cudaGetLastError();
}

size_t iface_smem_bytes(int L, int max_rows, int64_t max_nnz, int64_t max_inv, bool stage) {
    const size_t MR = (size_t)((max_rows + 3) & ~3);
    size_t bytes = (4 * IFACE_MAX_CLUSTER + 40) * sizeof(double) + (size_t)((L + 3) & ~3) * sizeof(float) +
                   4 * MR * sizeof(float) + (MR + 4) * sizeof(int32_t) + MR * sizeof(int2);
    if (stage) bytes += (size_t)max_nnz * sizeof(float2) + (size_t)max_inv * sizeof(float);
    return bytes;
}

cudaError_t prepare_iface_pcg(int cluster, size_t smem, int* active_clusters) {
    cudaError_t e = cudaFuncSetAttribute(k_iface_pcg, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (cluster > 8) {
        e = cudaFuncSetAttribute(k_iface_pcg, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(cluster, 1, 1);
    cfg.blockDim = dim3(IFACE_BS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(active_clusters, k_iface_pcg, &cfg);
}

cudaError_t launch_iface_pcg(const IfaceArgs& a, int cluster, size_t smem, const double* b, double* eta,
                             ColStrides cs, int ncols, cudaStream_t st) {
    count_launch();
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(cluster, ncols, 1);
    cfg.blockDim = dim3(IFACE_BS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_iface_pcg, a, b, eta, cs);
}

}  // namespace am
