// Launch interfaces of the AlgMortar CUDA kernels (host-callable, no torch types).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "common.cuh"

namespace am {

// Process-wide count of kernels this library has launched (graph replays included).
void count_launch();
void add_launches(int64_t k);
int64_t launch_count();

struct SolveArgs {
    Profile pf;
    const void* fwdS;          // forward sweep stream (TS)
    const void* bwdS;          // backward sweep stream (TS)
    const double* scale;       // symmetric scaling per row, or null (= 1); FP64 solves
    const float* scale32;      // the same scaling rounded to FP32 (FP32 / BF16 solves)
    const int64_t* scale_off;  // first scale entry of item s
    const int32_t* job_sub;    // item of each job
    const int64_t* job_in;     // offset of the job's input vector in `in`
    const int64_t* job_out;    // offset of the job's output vector in `out`
    const double* in;
    double* out;
    const int32_t* done;       // early exit when *done != 0 (PCG), or null
    int* err;                  // set to 1 if a bulk copy never completed (bounded wait)
    const int32_t* job_t0;     // per job: tile row where the right-hand side starts (rows
                               // above are zero) and below which no result is needed; or null
    int64_t ldin, ldout;       // column strides of in / out (gridDim.y = columns)
    int done_stride;           // int32 stride between columns' stop flags
    int col_fast;              // set by the launcher: grid (columns, jobs) instead of (jobs)
    int deep_ring;             // launch variant (ring / warp shape) of the chain solves, 0..4
                               // (defaults, or the autotuner's choice); all compute the solve
    int accumulate;            // 1: out += result instead of out = result
    // column-block jobs (launch_tile_solve_cols): up to NW columns of one item per job,
    // column c at job_in[job] + c * job_ld[job] (in and out), the first job_nc[job] valid,
    // and for PCG columns the stop flag of column job_col0[job] + c
    const int64_t* job_ld;
    const int32_t* job_nc;
    const int32_t* job_col0;
};

struct NdAssembleArgs {
    const int32_t* rows;
    const int64_t* if_off;
    const int32_t* if_list;
    const int64_t* phi_off;
    const double* phi;         // FP64 MBF panels
    const int64_t* g_cptr;
    const int32_t* g_row;
    const double* g_val;
    const int32_t* pairs;
    const int32_t* nd_pos;     // interface id -> ND position
    double* Sd;                // dense ND-ordered interface matrix (row-major), or null:
    double* pv;                //   per-subdomain blocks pv[pv_off[s] + a k_s + b] instead
    const int64_t* pv_off;     //   (off-diagonal entries only; the inexact solve's CSR)
    double* diagc;             // 2 * n_lambda
    int64_t L;
};

// Inexact interface solve (kernels_iface.cu): one thread-block cluster per right-hand side.
constexpr int IFACE_BS = 512;           // threads per CTA
constexpr int IFACE_MAX_CLUSTER = 16;   // CTAs per cluster (non-portable size on sm_10x)
constexpr int IFACE_MAX_BLOCK = 128;    // largest block-Jacobi block (FP64 inverse in smem)
struct IfaceArgs {
    int L;
    int max_rows;              // most rows of one CTA
    int64_t max_nnz;           // most S_eta entries of one CTA's rows
    int64_t max_inv;           // most block-inverse entries of one CTA
    int stage;                 // 1: the CTA's rows of S_eta and inverses in shared memory
    int max_it;                // inner iteration cap
    double rtol;               // inner relative tolerance (Euclidean, recurrence residual)
    const int32_t* cta_row0;   // cluster + 1 row ranges (block-aligned)
    const int32_t* cta_blk0;   // cluster + 1 block ranges
    const int32_t* s_ptr;      // CSR of S_eta (natural interface order)
    const int32_t* s_col;
    const float2* s_ent;       // its entries as (FP32 value, column bits)
    const int32_t* row_blk;    // row -> block
    const int2* row_info;      // per row: (block start - CTA's first row) | nb << 16, offset of
                               // the row's inverse row from the CTA's first inverse entry
    const int32_t* blk_row0;   // nblk + 1
    const int64_t* blk_off;    // nblk + 1 offsets of the row-major block inverses
    const float* binv;
    int32_t* its;              // per column: inner iterations of the latest solve
    int64_t* its_total;        // per column: running sum
};
void launch_iface_csr_values(int L, const int32_t* s_ptr, const int32_t* s_col, const int64_t* csr_src,
                             const double* pv, const double* T, const double* diagc, double* s_val64, float2* s_ent,
                             cudaStream_t st);
cudaError_t launch_iface_block_inv(int nblk, int max_nb, const int32_t* blk_row0, const int64_t* blk_off,
                                   const int32_t* s_ptr, const int32_t* s_col, const double* s_val64, float* binv,
                                   int* err, cudaStream_t st);
size_t iface_smem_bytes(int L, int max_rows, int64_t max_nnz, int64_t max_inv, bool stage);
cudaError_t prepare_iface_pcg(int cluster, size_t smem, int* active_clusters);
cudaError_t launch_iface_pcg(const IfaceArgs& a, int cluster, size_t smem, const double* b, double* eta,
                             ColStrides cs, int ncols, cudaStream_t st);

struct NdSolveArgs {
    int G;                     // groups
    int nsep;                  // separator unknowns
    int64_t nin;               // interior unknowns (= goff[G])
    int64_t np;                // sum_g a_g (= aoff[G])
    const int64_t* goff;       // G + 1
    const int64_t* aoff;       // G + 1
    const int32_t* alist;      // separator-local indices adjacent to each group
    const int32_t* sg;         // 2 * nsep groups of each separator unknown
    const int32_t* sidx;       // 2 * nsep index inside A_g
    const int32_t* row_g;      // interior ND row -> group
    const int32_t* prow_g;     // row of P -> group
    const double* Ginv;        // per group n_g x n_g symmetric inverse
    const int64_t* gioff;      // G offsets into Ginv
    const double* Wcm;         // per group n_g x a_g, column-major
    const double* Wrm;         // same, row-major
    const int64_t* woff;       // G offsets into W
    const double* Cinv;        // nsep x nsep symmetric inverse of the separator Schur complement
    // FP32 copies of Ginv, Wcm, Wrm, Cinv (rounded once from FP64): when set, the solve
    // multiplies in FP32 (the FP32 / BF16 factor variants)
    const float* Ginv32 = nullptr;
    const float* Wcm32 = nullptr;
    const float* Wrm32 = nullptr;
    const float* Cinv32 = nullptr;
    // FP32 layout: rows of Ginv32, columns of Wcm32 and rows of Cinv32 padded with zeros to
    // a multiple of 4 floats (16-byte loads); the FP32 right-hand side holds each group's
    // interior unknowns and then the separator's at 16-byte-aligned positions (zeros between)
    const int64_t* gioff32 = nullptr;   // G offsets into Ginv32 (row stride n_g rounded up to 4)
    const int64_t* woff32 = nullptr;    // G offsets into Wcm32 (column stride likewise)
    const int64_t* gpo32 = nullptr;     // G positions of the groups in the FP32 right-hand side
    const int32_t* p32 = nullptr;       // ND position -> position in the FP32 right-hand side
    int64_t spo32 = 0;                  // the separator's position there
    int64_t L32 = 0;                    // its length
    int nsep4 = 0;                      // nsep rounded up to 4 (row stride of Cinv32)
};

// interface system (kernels_coarse.cu)
void launch_iface_tables(int L, int64_t nr, const int64_t* rp_ptr, const int32_t* rp_pos, const double* val,
                         const int64_t* r_ptr, double* rcoef, double* T, int64_t ng, const int32_t* g_from_r,
                         double* gval, cudaStream_t st);
void launch_nd_assemble(int m, const NdAssembleArgs& a, cudaStream_t st);
void launch_nd_diag(int L, const double* T, const double* diagc, const int32_t* nd_pos, double* Sd, cudaStream_t st);
// dense tiles of the interface blocks in the setup's arithmetic TW (FP64, or FP32 for the
// FP32 / BF16 factor variants)
template <typename TW>
void launch_dense_to_tiles(int64_t ntiles, const double* src, int64_t ld, const int64_t* src_off, const int32_t* rows,
                           const int64_t* base, const int32_t* tile_item, const int32_t* tile_I,
                           const int32_t* tile_J, TW* work, cudaStream_t st);
// Cholesky of dense items advancing together (T_host: host copy of T): right-looking
// tile updates (planes == null), or -- FP32 with `planes` (2 TF32 operand planes per
// tile, same tile indexing as work) -- left-looking with the column updates on tcgen05
// Workspace of the K-split tensor-core column update: partial products of up to
// max_ctas CTAs (4 tiles each) and one zeroed ticket per row block (up to max_blocks).
struct TcSplit {
    float* part = nullptr;
    unsigned int* ticket = nullptr;
    int64_t max_ctas = 0;
    int64_t max_blocks = 0;
};
template <typename TW>
void launch_dense_cholesky(int nitems, const std::vector<int32_t>& T_host, const int32_t* T, const int64_t* base,
                           const int64_t* row0, TW* work, TW* dinv, int* err, cudaStream_t st,
                           TW* planes = nullptr, int* kerr = nullptr, TcSplit tcs = TcSplit{});
// Explicit FP32 inverse of dense tile-factored items, S^{-1} = W^T W, W = L^{-1}: each launch
// runs one batch of int4 jobs {item, I << 16 | J, k0 << 16 | k1, type} (0: W_II = dinv_I,
// 1: P_IJ = sum L_IK W_KJ, 2: W_IJ = -sum W_IK P_KJ, 3: lower tile of W^T W into the dense
// FP64 column-major out + out_off[item], leading dimension nrows[item]).
void launch_tile_inv(const int4* jobs, int njobs, const float* L, const float* dinv, float* Wt, float* Pt,
                     double* out, const int64_t* base, const int64_t* row0, const int32_t* nrows,
                     const int64_t* out_off, cudaStream_t st);
void launch_mirror_lower(const int32_t* rows, const int64_t* off, int nitems, double* M, cudaStream_t st);
void launch_transpose_blocks(const int64_t* goff, const int64_t* aoff, const int64_t* woff, int G, const double* Wcm,
                             double* Wrm, cudaStream_t st);
void launch_nd_w_sparse(int64_t np, int64_t L, const double* Sd, const int64_t* goff, const int64_t* aoff,
                        const int32_t* alist, int64_t sep0, const int32_t* prow_g, const int64_t* wc_ptr,
                        const int32_t* wc_row, const int64_t* gioff, const double* Ginv, const int64_t* woff,
                        double* Wcm, cudaStream_t st);
void launch_nd_schur_sparse(int64_t np, int64_t L, const double* Sd, const int64_t* goff, const int64_t* aoff,
                            const int32_t* alist, int64_t sep0, const int32_t* prow_g, const int64_t* wc_ptr,
                            const int32_t* wc_row, const int64_t* woff, const double* Wrm, const int64_t* doff,
                            double* D, cudaStream_t st);
template <typename TW>
void launch_nd_schur_tiles(int64_t ntiles, int64_t L, int nsep, int64_t sep0, const double* Sd, const int32_t* sg,
                           const int32_t* sidx, const int64_t* aoff, const int64_t* doff, const double* D,
                           TW* work, cudaStream_t st);
// f32: FP32 side vectors for the FP32 copies ([b: L32 | c: nsep4 | separator eta: nsep] per
// column, column stride fl; null for FP64); b32_ready: the restriction already wrote the
// FP32 copy of b (else it is converted here)
void launch_nd_solve(const NdSolveArgs& a, const double* b, double* eta, double* P, float* f32, int64_t fl,
                     bool b32_ready, ColStrides cs, int ncols, cudaStream_t st);
cudaError_t prepare_nd_solve(int nsep);
// FP32 copy with zero padding: nlines lines of len doubles (source stride ss) to lines of
// ds >= len floats
void launch_pad_convert(int64_t nlines, int64_t len, const double* src, int64_t ss, float* dst, int64_t ds,
                        cudaStream_t st);

// local factor
void launch_local_diag(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                       const int32_t* row_sub, int diag_scale, int modified, double* dloc, double* sc, float* sc32,
                       cudaStream_t st);
template <typename TW>
void launch_scatter_local(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                          const int32_t* row_sub, const int64_t* sub_off, const Profile& pf,
                          const double* dloc, const double* sc, TW* work, int nitems, cudaStream_t st);
template <typename TW>
void launch_pad_diag(int nitems, const Profile& pf, TW* work, cudaStream_t st);
// wm: widest tile row over all items, max_I (I - lo(I) + 1)
template <typename TW>
void launch_tile_chol(int nitems, const Profile& pf, const int32_t* order, TW* work, TW* dinv, int* err, int wm,
                      cudaStream_t st);
template <typename TW, typename TS>
void launch_finalize(int nitems, const Profile& pf, const TW* work, const TW* dinv, TS* fwdS, TS* bwdS,
                     cudaStream_t st);
template <typename TS, typename TA>
cudaError_t launch_tile_solve(const SolveArgs& a, int njobs, int max_tiles, cudaStream_t st, int ncols = 1);
// Column-block jobs: each of the 4 consumer warps of a CTA solves one column of the job
// with the same factor tile stream (each tile copied once per job, read by every warp).
constexpr int COLS_PER_JOB = 4;
// Multi-column local solves of up to PANEL_NC right-hand sides of one subdomain per CTA
// (FP32 / BF16 streams; jobs as launch_tile_solve_cols: job_sub, job_in (= offset in w32
// and in out), job_ld, job_nc); the scaled FP32 right-hand sides in w32 (overwritten),
// the results in a.out (FP64); wm = widest tile row.  cudaErrorInvalidValue when its
// shared memory does not fit an SM (the caller then uses launch_tile_solve_cols).
constexpr int PANEL_NC = 32;
template <typename TS>
cudaError_t launch_panel_solve(const SolveArgs& a, float* w32, int njobs, int max_tiles, int wm, cudaStream_t st);
bool panel_solve_fits(int wm, int max_tiles, size_t ts);   // its shared memory fits one SM
// The same for batched PCG columns: FP64 right-hand sides in a.in (scaled by a.scale32 in the
// solve), column c of a job being column job_col0[job] + c with its stop flag (a.done); w32
// (same indexing as in / out, FP32) holds the forward results; a.accumulate adds to a.out.
template <typename TS>
cudaError_t launch_panel_solve_cols(const SolveArgs& a, float* w32, int njobs, int max_tiles, int wm,
                                    cudaStream_t st);
// w32 (zeroed) <- the scaled FP32 MBF right-hand sides -B_i psi_m (as launch_mbf_rhs, times
// sc32[sc_off[i] + row])
void launch_mbf_rhs32(int m, const int64_t* g_off, const int32_t* g_row, const int32_t* g_col, const double* g_val,
                      const int32_t* rows, const int64_t* phi_off, const float* sc32, const int64_t* sc_off,
                      float* w32, cudaStream_t st);
template <typename TS, typename TA>
cudaError_t launch_tile_solve_cols(const SolveArgs& a, int njobs, int max_tiles, cudaStream_t st);
void launch_mbf_rhs(int m, const int64_t* g_off, const int32_t* g_row, const int32_t* g_col,
                    const double* g_val, const int32_t* rows, const int64_t* phi_off, double* rhs,
                    cudaStream_t st);
template <typename TS>
void launch_convert(int64_t n, const double* src, TS* dst, cudaStream_t st);
void launch_eye(int L, double* E, cudaStream_t st);

// vector / PCG kernels (kernels_pcg.cu)
constexpr int VEC_BS = 256;
int vec_blocks(int64_t n);                    // CTAs of the grid-strided vector kernels
void set_vec_sms(int sms);
void set_hot_ctas_per_sm(int c);              // CTAs per SM of the per-iteration PCG kernels
int hot_ctas_per_sm();
int hot_blocks(int64_t work);
void launch_gather(int64_t n, const int32_t* perm, const double* src, double* dst, cudaStream_t st);
void launch_scatter(int64_t n, const int32_t* perm, const double* src, double* dst, cudaStream_t st);
void launch_gather_cols(int64_t n, int ncols, const int32_t* perm, const double* src, int64_t lds, double* dst,
                        int64_t ldd, cudaStream_t st);
void launch_scatter_cols(int64_t n, int ncols, const int32_t* perm, const double* src, int64_t lds, double* dst,
                         int64_t ldd, cudaStream_t st);
void launch_scatter_values(int64_t n, const int64_t* idx, const double* v, double* dst, cudaStream_t st);
void launch_restrict(int L, const int64_t* rptr, const int32_t* rcell, const double* rcoef, const double* pbar,
                     double* beta, const int32_t* omap, ColStrides cs, int ncols, float* beta32, int64_t fl,
                     const int32_t* p32, cudaStream_t st);
// One prolongation work item: up to 32 consecutive rows of one subdomain i (one warp).
// The prolongation reads the MBF panels of subdomain i row-major: row k's k_i entries
// p_hat^(m)_k are contiguous, padded with zeros to ld = k_i rounded up to 16 bytes.
struct __align__(16) ProlongChunk {
    int64_t row0;   // first row (subdomain-contiguous numbering)
    int64_t phi0;   // offset of the first row's panel entries in the row-major panels
    int32_t ld;     // panel entries per row (k_i padded to a multiple of 16 bytes)
    int32_t nrow;   // rows in this chunk, 1..32
    int32_t i0;     // first entry of subdomain i in the interface list
    int32_t kk;     // interfaces of subdomain i
};
template <typename TP>
void launch_prolong(int nchunks, const ProlongChunk* chunks, const int32_t* if_list, const TP* phi,
                    const double* eta, const double* pbar, const double* base, double* z, const double* r,
                    GridSum gs, PcgScalars* sc, ColStrides cs, int ncols, cudaStream_t st);
// Row-major padded copy (layout of ProlongChunk) of the column-major FP64 panels phi
// (subdomain i's column m at phi_off[i] + m n_i); chunk_sub = subdomain of each chunk.
template <typename TP>
void launch_panel_rows(int nchunks, const ProlongChunk* chunks, const int32_t* chunk_sub, const int64_t* sub_off,
                       const int64_t* phi_off, const double* phi, TP* out, cudaStream_t st);
int prolong_blocks(int nchunks);   // CTAs of launch_prolong (<= vec_blocks of the widest vector)
void launch_smooth_residual(int64_t n, int ncols, const int64_t* ell_ptr, const int32_t* ell_col,
                            const double* ell_val, const double* x, const double* r, double* s, ColStrides cs,
                            cudaStream_t st);
void launch_pcg_rho(int64_t n, int ncols, const double* r, const double* z, PcgScalars* sc, GridSum gs,
                    ColStrides cs, cudaStream_t st);
void launch_pcg_init(int64_t n, int ncols, int64_t ld, const double* b, double* x, double* r, PcgScalars* sc,
                     GridSum gs, double tol, int max_it, int flexible, double* hist, int hist_len, cudaStream_t st);
void launch_pcg_replace(int64_t n, int ncols, int64_t ld, const int32_t* rowptr, const int32_t* col,
                        const double* val, const double* x, const double* b, double* r, PcgScalars* sc, GridSum gs,
                        cudaStream_t st);
void launch_pcg_p(int64_t n, int ncols, int64_t ld, const double* z, double* p, const PcgScalars* sc,
                  cudaStream_t st);
// wf: the slice width of the unrolled path (spmv_fast_width), 0 for none
void launch_pcg_spmv_ell(int64_t n, int ncols, int64_t ld, const int64_t* ell_ptr, const int32_t* ell_col,
                         const double* ell_val, const double* p, double* q, PcgScalars* sc, GridSum gs, int wf,
                         cudaStream_t st);
int spmv_fast_width(const int64_t* ell_ptr_host, int64_t nslices);
void launch_ell_values(int64_t nell, const int32_t* src, const double* val, double* ell_val, cudaStream_t st);
void launch_pcg_xr(int64_t n, int ncols, int64_t ld, double* x, double* r, const double* p, const double* q,
                   const double* z, PcgScalars* sc, GridSum gs, double* hist, int hist_len, cudaStream_t st);
void launch_residual(int64_t n, int ncols, int64_t ld, const int32_t* rowptr, const int32_t* col, const double* val,
                     const double* x, const double* b, PcgScalars* sc, GridSum gs, cudaStream_t st);
void launch_tpfa_grad(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val, const double* K,
                      const double* tb, const double* tbp, const double* p, const double* lam, double* grad,
                      cudaStream_t st);

}  // namespace am
