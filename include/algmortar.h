/*
 * algmortar.h -- C ABI of the B300-native AlgMortar-PCG library (libalgmortar.so).
 *
 * AlgMortar (arxiv 2607.22905) is an algebraic multiscale mortar preconditioner for an
 * SPD matrix A whose off-diagonal couplings between subdomains are negative
 * (Sec. 3.2, the sign assumption on the weights W).  From A alone it
 *   - partitions the adjacency graph G(A) into m subdomains Omega_i (Sec. 3.1),
 *   - forms the diagonally modified local blocks A_i = A_ii - sum_j D_ij (Eq. A_i),
 *   - builds one multiscale basis function per neighbouring interface (Eq. def-phat-local)
 *     with the piecewise-constant mortar space of Sec. 5.5,
 *   - assembles the interface system (Eq. interface-problem-alg),
 * and applies z = cal_M^{-1} r of Eq. (eq-m-reduced-p) by Algorithm 2 inside
 * preconditioned CG (Sec. 7: x0 = 0, Euclidean relative-residual stop).
 *
 * Conventions for every entry point below:
 *   - Return value: 0 (ALGMORTAR_OK) or an algmortar_status code; nothing traps or
 *     aborts.  algmortar_last_error() returns a thread-local message for the last
 *     failure (which block, which row, which CUDA call).
 *   - "host" pointers are read (or written) during the call only and are never retained.
 *   - "device" pointers are CUDA global-memory pointers on the handle's device.  They
 *     are owned by the caller, must stay valid for the call, and are not retained.
 *   - Vectors of the public API are in the caller's ORIGINAL row ordering.
 *   - All device work is issued on opts.stream (NULL = the legacy default stream);
 *     calls that return results to the host synchronise that stream before returning.
 *   - A handle may be used by one host thread at a time.
 */
#ifndef ALGMORTAR_H
#define ALGMORTAR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
enum {
    ALGMORTAR_OK = 0,
    ALGMORTAR_INVALID_ARG = 1,     /* null pointer, bad size, malformed CSR (unsorted or
                                      out-of-range columns, missing diagonal, NaN/Inf)  */
    ALGMORTAR_NOT_SYMMETRIC = 2,   /* a_kl != a_lk for some stored entry                 */
    ALGMORTAR_INTERFACE_SIGN = 3,  /* a_kl >= 0 across two subdomains: W not negative
                                      definite, the hypothesis of Sec. 3.2 / Thm. Q-psd  */
    ALGMORTAR_NOT_SPD = 4,         /* non-positive pivot in a local or interface Cholesky
                                      factor (block id in algmortar_last_error())        */
    ALGMORTAR_NO_CONVERGENCE = 5,  /* max_it reached; x holds the last iterate           */
    ALGMORTAR_BREAKDOWN = 6,       /* p^T A p <= 0 or a non-finite CG scalar             */
    ALGMORTAR_CUDA = 7,            /* a CUDA runtime call failed                        */
    ALGMORTAR_OOM = 8,             /* device or host allocation failed                  */
    ALGMORTAR_TOO_LARGE = 9        /* a subdomain above ALGMORTAR_MAX_PART rows, or an
                                      interface system larger than the static scratch of
                                      algmortar_interface_solve_noalloc                 */
};

/* Largest subdomain the batched local kernels accept (rows). */
#define ALGMORTAR_MAX_PART 16384

/* Right-hand sides one batched PCG iteration carries (algmortar_pcg_solve_multi splits
 * larger requests into batches of this many columns). */
#define ALGMORTAR_MAX_BATCH 32

/* Precision of the local factors L_i, their triangular solves and the MBF panels.
 * The outer PCG recurrences, dot products, SpMV, interface restriction, the coarse
 * interface solve and the true-residual check are FP64 in every mode. */
enum {
    ALGMORTAR_FP64 = 0,            /* factors and solves in FP64                         */
    ALGMORTAR_FP32 = 1,            /* factors stored and applied in FP32                 */
    ALGMORTAR_BF16 = 2             /* factors stored in BF16, applied with FP32 accumulation */
};

/* Interface solve of Algorithm 2 (opts.interface_solve). */
enum {
    ALGMORTAR_IFACE_EXACT = 0,     /* FP64, exact                                         */
    ALGMORTAR_IFACE_INEXACT = 1    /* block-Jacobi PCG in FP32 to opts.iface_rtol          */
};

/* Host CSR matrix, square, full symmetric pattern, columns strictly ascending within
 * each row, explicit diagonal, int32 indices (nnz < 2^31).  Read during setup only. */
typedef struct {
    int64_t n;
    int64_t nnz;
    const int32_t* rowptr;         /* host, n + 1 entries, rowptr[0] = 0, rowptr[n] = nnz */
    const int32_t* col;            /* host, nnz entries                                   */
    const double* val;             /* host, nnz entries                                   */
} algmortar_csr;

typedef struct {
    int32_t precision;             /* ALGMORTAR_FP64 / FP32 / BF16 (default FP64)         */
    int32_t diag_scale;            /* 1: factor D^-1/2 A_i D^-1/2 (D = diag A_i); default 1 */
    int32_t max_it;                /* PCG iteration cap (default 10000)                   */
    int32_t use_graph;             /* 1: replay each PCG iteration as a captured CUDA graph */
    int32_t check_every;           /* iterations between host convergence reads (>= 1)    */
    int32_t flexible;              /* 1: Polak-Ribiere beta (r_{k+1}.(z_{k+1} - z_k) / rho_k,
                                      for slightly non-symmetric low-precision M^{-1})    */
    int32_t verbose;               /* 1: stage timings to stderr                          */
    int32_t device;                /* CUDA device ordinal (default 0)                      */
    const int32_t* part_sizes;     /* host, n_parts target sizes summing to n, or NULL for
                                      sizes differing by at most one (larger ones first)  */
    void* stream;                  /* cudaStream_t for all device work (NULL = default)   */
    int32_t nd_depth;              /* interface solve: depth of the nested-dissection split
                                      (2^depth groups from the partition's bisection tree);
                                      -1 (default) picks ~1000-unknown interior blocks    */
    int32_t autotune;              /* 1: during setup, time the launch variants of the hot
                                      kernels (ring and warp shapes of the batched local
                                      triangular solves, CTAs per SM of the PCG vector
                                      kernels) on this handle's own data and keep the
                                      fastest; results are cached per process by precision
                                      and factor-profile shape.  0 (default): built-in
                                      defaults.  Every variant computes the same result.  */
    int32_t interface_solve;       /* ALGMORTAR_IFACE_EXACT (default): the interface system of
                                      Algorithm 2 solved exactly in FP64 (one-level nested
                                      dissection with explicit inverses); ALGMORTAR_IFACE_
                                      INEXACT: block-Jacobi PCG on S_eta in FP32 to
                                      iface_rtol (Sec. 7 solver settings), which makes M^{-1}
                                      non-linear, so the outer PCG then always uses the
                                      flexible beta                                       */
    int32_t smooth_steps;          /* nu >= 0 block-Jacobi smoothing steps before and after
                                      the AlgMortar correction (Sec. 5.4), composed
                                      multiplicatively; blocks = the subdomains, each
                                      solved with an exact factor of the unmodified
                                      A_ii in the factor precision; default 0            */
    int32_t iface_block_parts;     /* inexact interface solve: block-Jacobi block of interface
                                      (i, j), i < j, is i / iface_block_parts (default 1:
                                      the interfaces each subdomain owns as the smaller
                                      id; larger groups cut few inner iterations at config
                                      3 -- 48 at 1, 41 at 4, 32 at 32 -- for 3.5x-25x the
                                      block-inverse work);
                                      every block must hold <= 128 interfaces              */
    int32_t iface_max_it;          /* inexact interface solve: inner iteration cap (200)    */
    int32_t stage_times;           /* 1: the PCG iteration records CUDA events between its
                                      stages and algmortar_stats.stage_ms reports them for
                                      the last iteration; the iterations then run stream-
                                      ordered even with use_graph (launch gaps included);
                                      0 (default): no events                              */
    double iface_rtol;             /* inexact interface solve: stop when ||b - S eta||_2 <=
                                      iface_rtol ||b||_2 (recurrence residual; 1e-2)       */
    uint64_t seed;                 /* algmortar_setup with part_sizes == NULL: 0 (default)
                                      even target sizes; otherwise uneven target sizes
                                      drawn from this seed (algmortar_part_sizes)          */
} algmortar_opts;

/* Solver statistics of one right-hand side.  history / history_len are INPUTS (set them,
 * or leave both 0): when history is a host array of history_len doubles, the solve
 * writes ||r_k||_2 / ||b||_2 of the CG recurrence for k = 0, 1, ... into it (k = 0 is 1)
 * and the count written into history_count. */
typedef struct {
    int32_t status;                /* status of the solve                                 */
    int32_t iterations;            /* products with A in the CG loop                      */
    double rel_residual;           /* true ||b - A x||_2 / ||b||_2 at exit                */
    double recursive_residual;     /* CG recurrence ||r_k||_2 / ||b||_2 at exit           */
    double solve_ms;               /* wall time of the solve call, device-synchronised    */
    double host_ms;                /* host-side part of the call (setup: partition etc.)  */
    double stage_ms[6];            /* opts.stage_times = 1: device ms of the last PCG
                                      iteration's stages -- [0] SpMV, [1] CG vector
                                      updates, [2] local solves, [3] restriction,
                                      [4] interface solve, [5] prolongation; else 0       */
    int64_t iface_iterations;      /* inexact interface solve: inner iterations summed over
                                      the solve's preconditioner applications; else 0     */
    double* history;               /* in: host buffer or NULL                             */
    int32_t history_len;           /* in: its length                                      */
    int32_t history_count;         /* out: entries written                                */
} algmortar_stats;

typedef struct {
    int64_t n;                     /* rows                                               */
    int32_t n_parts;               /* subdomains m                                       */
    int32_t n_lambda;              /* interface unknowns N_Lambda (one per pair i~j)     */
    int32_t max_part;              /* largest subdomain                                  */
    int32_t min_part;              /* smallest subdomain                                 */
    int32_t precision;
    int64_t n_interface_edges;     /* |E|                                                */
    int64_t factor_entries;        /* stored entries of one triangular sweep (all L_i)   */
    int64_t factor_bytes;          /* bytes of both sweep streams                        */
    int64_t phi_entries;           /* sum_i N_i |I_i| (MBF panel entries)                */
    double setup_ms[8];            /* [0] partition + tables (host), [1] upload,
                                      [2] local factors, [3] MBFs, [4] interface assembly,
                                      [5] interface factor + inverse, [6] interface factor
                                      alone, [7] total of algmortar_setup               */
    int64_t kernel_launches;       /* kernels this library has launched in this process
                                      so far (graph replays counted per kernel)           */
    int32_t interface_solve;       /* ALGMORTAR_IFACE_EXACT / _INEXACT                    */
    int32_t iface_blocks;          /* inexact: block-Jacobi blocks                        */
    int32_t iface_cluster;         /* inexact: CTAs of the inner-PCG cluster               */
    int32_t iface_staged;          /* inexact: 1 if S_eta rows and block inverses are held
                                      in shared memory during the inner solve             */
    int32_t iface_last_iterations; /* inexact: inner iterations of the latest single-right-
                                      hand-side preconditioner application (read from the
                                      device when algmortar_get_info is called)           */
    int32_t tuned_ring;            /* launch variant of the batched local solves in use   */
    int32_t tuned_vec_ctas;        /* CTAs per SM of the PCG vector kernels in use        */
    int32_t tuned_job_order;       /* local-solve job order in use: 0 rows, 1 stored tiles,
                                      2 tile rows (each longest first)                    */
    int32_t pad_;
} algmortar_info;

typedef struct algmortar_handle algmortar_t;

/* Fill *opts with the defaults listed above. */
void algmortar_default_opts(algmortar_opts* opts);

/* Host only: the uneven target sizes algmortar_setup uses when opts.part_sizes is NULL and
 * opts.seed != 0.  With lo = 3n/(10m), hi = 3n/m (integer division) and, for j < m,
 * a_j, b_j = SplitMix64((seed << 32) ^ 2j), SplitMix64((seed << 32) ^ (2j + 1)) mod 2^20,
 * weight w_j = lo 2^40 + (hi - lo) a_j b_j (a right-skewed spread with mean near
 * lo + (hi - lo) / 4); sizes_out[j] = floor(n C_j / W) - floor(n C_{j-1} / W) over the
 * cumulative weights C_j (C_{-1} = 0, W = C_{m-1}), so the sizes sum to n.  sizes_out:
 * host, m entries.  INVALID_ARG if m < 1, n < m, or a size would be 0. */
int algmortar_part_sizes(int64_t n, int32_t m, uint64_t seed, int32_t* sizes_out);

/* Host only (no GPU needed): the deterministic graph partition of Sec. 3.1 used by
 * algmortar_setup.  part_out (host, n entries) receives labels in [0, n_parts).
 * part_sizes as in algmortar_opts (NULL = even).  Rule: recursive bisection; a node set
 * S assigned to parts lo..hi-1 is put in breadth-first order (neighbours ascending,
 * started at the George-Liu pseudo-peripheral node of the component of min(S), then at
 * the smallest unvisited node of each further component) and its first
 * sizes[lo] + ... + sizes[lo + k/2 - 1] nodes go to the first k/2 parts. */
int algmortar_partition(const algmortar_csr* A, int32_t n_parts, const int32_t* part_sizes,
                        int32_t* part_out);

/* Algorithm 1 (AlgMortarSetup) on the device.  Validates A (symmetry, interface sign),
 * partitions it (Sec. 3.1), permutes it, factors every A_i, computes the MBFs, assembles
 * and factors the interface system, and allocates the PCG workspace.  *out receives a
 * handle owning all device state; release it with algmortar_destroy.  On error *out is
 * NULL and nothing is leaked. */
int algmortar_setup(const algmortar_csr* A, int32_t n_parts, const algmortar_opts* opts,
                    algmortar_t** out);

/* As algmortar_setup with caller-given labels part (host, n entries in [0, n_parts),
 * every part non-empty) in place of the built-in partitioner -- e.g. to reuse a
 * partition across time steps. */
int algmortar_setup_with_parts(const algmortar_csr* A, const int32_t* part, int32_t n_parts,
                               const algmortar_opts* opts, algmortar_t** out);

/* Algorithm 2 (AlgMortarApply): z = cal_M^{-1} r (Eq. eq-m-reduced-p).  r_dev, z_dev:
 * device, n doubles each, original ordering; they may not alias. */
int algmortar_apply(algmortar_t* h, const double* r_dev, double* z_dev);

/* Stages of Algorithm 2 in the handle's internal (permuted) ordering, for testing:
 * pbar = A_hat^{-1} r (Eq. def-pbar-local), b_eta = interface right-hand side,
 * eta = interface solution, z = pbar + sum_m eta_m p_hat^(m) (Eq. p-decomposition-alg).
 * r_dev is in the ORIGINAL ordering; pbar_dev, z_dev: n doubles (internal ordering);
 * beta_dev, eta_dev: n_lambda doubles (interfaces numbered lexicographically by (i, j)). */
int algmortar_apply_stages(algmortar_t* h, const double* r_dev, double* pbar_dev,
                           double* beta_dev, double* eta_dev, double* z_dev);

/* PCG with x0 = 0 for A x = b, preconditioned by AlgMortar; stops when
 * ||r_k||_2 <= tol ||b||_2 and the true residual confirms it (Sec. 7).  When it does
 * not, the recursive residual is replaced by b - A x and the search directions restart
 * (at most 8 times).  opts.flexible selects the Polak-Ribiere beta.  b_dev, x_dev:
 * device, n doubles, original ordering.  st may be NULL.  Returns OK, NO_CONVERGENCE
 * or BREAKDOWN (x_dev holds the last iterate in the latter two cases). */
int algmortar_pcg_solve(algmortar_t* h, const double* b_dev, double* x_dev, double tol,
                        algmortar_stats* st);

/* As algmortar_pcg_solve with HOST b and x (n doubles each): copies b to the device,
 * solves, copies x back; the copies are part of the call. */
int algmortar_pcg_solve_host(algmortar_t* h, const double* b_host, double* x_host, double tol,
                             algmortar_stats* st);

/* nrhs independent systems A X[:, j] = B[:, j] (column-major, leading dimension ld >= n,
 * device), solved as batches of up to ALGMORTAR_MAX_BATCH columns: every kernel of a
 * PCG iteration covers all columns of the batch in one launch; the local solves run as
 * column-block jobs (4 columns of one subdomain per CTA, each factor tile read once per
 * block).  Each column runs its own CG scalars and stops on its own tolerance (stopped
 * columns are skipped).  The batched local solve sums a tile row's contributions in a
 * different order than the single-RHS kernel, so columns agree with algmortar_pcg_solve
 * to rounding, not bit for bit.  st (may be NULL) points to nrhs stats.  The batch
 * workspace (8 n + 2 L doubles per column) is allocated on first use and kept.  Returns
 * OK, NO_CONVERGENCE or BREAKDOWN (the worst column). */
int algmortar_pcg_solve_multi(algmortar_t* h, const double* B_dev, double* X_dev, int32_t nrhs,
                              int64_t ld, double tol, algmortar_stats* st);

/* New values for the same sparsity pattern (host, nnz doubles in the CSR order given at
 * setup): keeps the partition, the permutation and every device buffer (so a captured
 * PCG graph stays valid) and re-runs the numeric part of Algorithm 1 (local factors,
 * MBFs, interface system).  The values must keep A symmetric with negative couplings
 * between subdomains; they are not re-validated (a non-SPD block still returns NOT_SPD). */
int algmortar_update_values(algmortar_t* h, const double* val_host);

/* As algmortar_update_values with the nnz values in DEVICE memory (CSR order of setup). */
int algmortar_update_values_device(algmortar_t* h, const double* val_dev);

/* Adjoint gradient for TPFA matrices (not in the paper).  With the handle's current
 * matrix A (values from setup or the last update) read as a two-point flux system --
 * off-diagonal a_kl = -T_kl, T_kl = c 2 K_k K_l / (K_k + K_l) for any face factor c --
 * plus Dirichlet half-faces summarised per cell (tb_k = sum_b T_b, tbp_k = sum_b T_b
 * p_bc, so f_k = tbp_k), the state p (A p = f) and the adjoint lambda (A lambda = dL/dp),
 * writes grad_k = dL/d ln K_k:
 *   sum_l -(lambda_k - lambda_l)(p_k - p_l) T_kl K_l / (K_k + K_l) + lambda_k (tbp_k - p_k tb_k).
 * All pointers: device, n doubles, original ordering.  Uses the handle's work vectors
 * (do not call it between the stages of another call on the same handle). */
int algmortar_tpfa_grad_lnK(algmortar_t* h, const double* K_dev, const double* tb_dev, const double* tbp_dev,
                            const double* p_dev, const double* lam_dev, double* grad_dev);

/* Interface solve eta = S^{-1} b for the handle's interface system, WITHOUT any device
 * allocation.  The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory when they need the solve (a fixed memory budget or a
 * caller-owned pool, real-time loops that must stay out of the allocator, hosts that
 * forbid cudaMalloc after start-up).  It computes the same eta as algmortar_apply_stages
 * returns for b = b_eta (same kernels, same order), but keeps its temporaries in a
 * file-scope device array of 2^20 doubles (8 MiB) that every GPU loading the library
 * holds until the process exits.
 *   b_dev, eta_dev: device, n_lambda doubles each, natural interface order (pairs
 *   (i, j) lexicographic); caller-owned, not retained.  Work goes on the handle's stream.
 * Limits and sharing: needs 2 n_lambda + sum_g |A_g| doubles of the array (the sizes of
 * the nested-dissection layout in algmortar_info terms: at most ~3 n_lambda); larger
 * systems return ALGMORTAR_TOO_LARGE with a message.  All calls share the one array,
 * which keeps the previous call's contents (every entry this call reads is written by
 * it first); calls whose device work overlaps -- other streams, other threads, other
 * handles on the same GPU -- race on it and must be serialised by the caller.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress,
 * no allocation); make that first call before any stream capture on that device.
 * The call makes the handle's device current for its launches and restores the
 * caller's current device before it returns. */
int algmortar_interface_solve_noalloc(const algmortar_t* h, const double* b_dev, double* eta_dev);

/* Labels of the handle's partition (host, n entries). */
int algmortar_get_partition(const algmortar_t* h, int32_t* part_out);

/* perm_out[new] = old for the handle's internal ordering (host, n entries). */
int algmortar_get_permutation(const algmortar_t* h, int32_t* perm_out);

/* Interface pairs (host, 2 * n_lambda entries: i, j with i < j, lexicographic). */
int algmortar_get_interfaces(const algmortar_t* h, int32_t* pairs_out);

int algmortar_get_info(const algmortar_t* h, algmortar_info* info);

/* Measurement: average device time (CUDA events on the handle's stream, ms) of each
 * stage of one PCG iteration over `reps` repetitions, on the handle's current vectors:
 * ms_out[0] SpMV (+ p.q), [1] CG vector updates, [2] local solves (Eq. def-pbar-local),
 * [3] restriction, [4] interface solve, [5] prolongation (+ r.z), [6] a whole iteration
 * as launched by algmortar_pcg_solve (graph or stream), [7] reserved (0).
 * Kernels run exactly as inside the solver.  The handle's work vectors are overwritten
 * (the next solve re-initialises them); its results from earlier calls are not kept. */
int algmortar_time_stages(algmortar_t* h, int32_t reps, double* ms_out);

/* Releases all device and host state of h (NULL is ignored). */
void algmortar_destroy(algmortar_t* h);

const char* algmortar_strerror(int status);
const char* algmortar_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ALGMORTAR_H */
