// C ABI of libalgmortar (include/algmortar.h): handle lifetime, Algorithm 1 on the device,
// Algorithm 2 and the PCG loop.
#include <algorithm>
#include <array>
#include <functional>
#include <map>
#include <mutex>
#include <chrono>
#include <cmath>
#include <type_traits>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "algmortar.h"
#include "host_setup.h"
#include "kernels.h"

using namespace am;

namespace am {
int interface_solve_noalloc(int device, cudaStream_t st, int L, const NdSolveArgs& nd, const int32_t* d_ndpos,
                            const double* b_dev, double* eta_dev, std::string& err);
}

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

#define CU(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail(e_ == cudaErrorMemoryAllocation ? ALGMORTAR_OOM : ALGMORTAR_CUDA,           \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                        \
    } while (0)

}  // namespace

// Device buffers of Algorithm 1 that survive between numeric setups (value updates
// reuse them, so captured graphs and pointers stay valid).
// Column-block jobs of the multi-column chain solve: up to COLS_PER_JOB columns of one
// item at a constant stride, the smallest start row of the block (identity columns).
struct BlockJobs {
    std::vector<int32_t> sub, nc, t0;
    std::vector<int64_t> in, ld;
    void add(int32_t item, int64_t base, int64_t stride, int64_t ncols, bool identity_t0) {
        for (int64_t c = 0; c < ncols; c += COLS_PER_JOB) {
            sub.push_back(item);
            in.push_back(base + c * stride);
            ld.push_back(stride);
            nc.push_back((int32_t)std::min<int64_t>(COLS_PER_JOB, ncols - c));
            t0.push_back(identity_t0 ? (int32_t)(c / TILE) : 0);
        }
    }
    int size() const { return (int)sub.size(); }
};
struct DevBlockJobs {
    int n = 0;
    int32_t *sub = nullptr, *nc = nullptr, *t0 = nullptr;
    int64_t *in = nullptr, *ld = nullptr;
};

struct NumWs {
    bool ready = false;
    int njobs_mbf = 0;
    DevBlockJobs bj_mbf;                      // column-block jobs of the MBF solves
    DevBlockJobs pj_mbf;                      // the same in blocks of PANEL_NC (FP32 / BF16)
    float* w32 = nullptr;                     // FP32 / BF16: scaled FP32 MBF right-hand sides
    int32_t *d_js = nullptr, *d_grow = nullptr, *d_gcol = nullptr, *d_pairs = nullptr;
    int64_t *d_jo = nullptr, *d_goff = nullptr, *d_gcptr = nullptr;
    double* d_gval = nullptr;
    double* d_T = nullptr;
    void *work = nullptr, *dinv = nullptr;
    int* d_err = nullptr;
    double *rhs = nullptr, *phi64 = nullptr, *diagc = nullptr, *Sd = nullptr;
    // interface groups as factor items (non-empty groups only)
    int nitems = 0;
    std::vector<int32_t> item_group;           // item -> group
    std::vector<int64_t> item_row0, item_base; // host copies
    std::vector<std::vector<int32_t>> item_hi; // host hi[] per item (right-looking launcher)
    int32_t *d_irows = nullptr, *d_int = nullptr, *d_ilo = nullptr, *d_ihi = nullptr;
    int64_t *d_irow0 = nullptr, *d_ibase = nullptr, *d_ifwd = nullptr, *d_ibwd = nullptr, *d_isrc = nullptr;
    int32_t *d_titem = nullptr, *d_tI = nullptr, *d_tJ = nullptr;
    int64_t ntiles_items = 0, trows_items = 0;
    int max_tiles_items = 0;
    void *gwork = nullptr, *gdinv = nullptr, *gf = nullptr, *gb = nullptr;   // interface arithmetic
    float *gplanes = nullptr, *cplanes = nullptr;   // FP32: TF32 operand planes of the factor tiles
    TcSplit tcs;                                     // FP32: K-split workspace of the tensor-core update
    double* gE = nullptr;
    // FP32 setup: explicit inverses by batched tile products (launch_tile_inv), one job
    // range per launch, for the group items and for the separator
    int4 *d_ginv_jobs = nullptr, *d_cinv_jobs = nullptr;
    std::vector<std::pair<int, int>> ginv_ranges, cinv_ranges;
    int64_t* d_iout = nullptr;                 // per group item: offset of its inverse in Ginv
    int32_t *d_gjob = nullptr, *d_gjt0 = nullptr, *d_cjt0 = nullptr;
    int64_t* d_gjin = nullptr;
    int njobs_g = 0;
    int64_t* d_doff = nullptr;
    int64_t* d_wc_ptr = nullptr;   // coupling pattern of S_{g,A_g}: per W column, interior rows
    int32_t* d_wc_row = nullptr;
    double* D = nullptr;
    // separator Schur complement as a single dense item
    int cT = 0;
    std::vector<int32_t> c_hi;
    int32_t *d_crows = nullptr, *d_cnt = nullptr, *d_clo = nullptr, *d_chi = nullptr, *d_cjob = nullptr;
    int64_t *d_czero = nullptr, *d_cfwd = nullptr, *d_cbwd = nullptr, *d_cjin = nullptr;
    void *cwork = nullptr, *cdinv = nullptr, *cf = nullptr, *cb = nullptr;
    double* cE = nullptr;
    int32_t* d_crowsq = nullptr;
    int64_t* d_czerooff = nullptr;
    int64_t n_ginv = 0, n_w = 0;            // entries of the interface inverses Ginv, W
    std::vector<int64_t> h_gioff, h_woff, h_gioff32, h_woff32;   // host copies of their offsets
    // inexact interface solve: per-subdomain blocks of 1/4 G^T Phi, CSR values of S_eta
    double* pv = nullptr;
    int64_t* d_pv_off = nullptr;
    int64_t* d_csr_src = nullptr;
    double* s_val64 = nullptr;
};

// PCG / apply vectors of k right-hand sides, column-major: cell vectors with leading
// dimension n, interface vectors with leading dimension max(L, 1), and per column one PCG
// state, one grid-sum ticket and its block partials.  The captured iteration graph
// belongs to the batch (its launches carry the column count).
struct Vecs {
    int k = 0, cap = 0;
    double *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *pbar = nullptr;
    double *b = nullptr, *t = nullptr, *w = nullptr;   // w: smoother residuals
    double *beta = nullptr, *eta = nullptr, *P = nullptr;
    PcgScalars* sc = nullptr;
    GridSum gs{};
    cudaGraphExec_t graph = nullptr;
    int graph_k = 0;                   // column count the graph was captured with
    DevBlockJobs bj;                   // column-block jobs of the batched local solves
    int32_t* bj_col0 = nullptr;
    int bj_k = 0;                      // column count bj was built for
    DevBlockJobs pj;                   // the same in blocks of PANEL_NC (FP32 / BF16 panel solves)
    int32_t* pj_col0 = nullptr;
    float* w32 = nullptr;              // their forward results (k * n floats), or null
    int64_t graph_kernels = 0;         // kernels in one replay of the iteration graph
    int32_t* iits = nullptr;           // inexact interface solve: per column, inner iterations
    int64_t* iits_total = nullptr;     //   of the latest application / summed since reset
    float* f32 = nullptr;              // FP32 interface solve: side vectors per column
    int64_t fl = 0;                    //   (b: L | P: np | separator eta: nsep), column stride
    double* hist = nullptr;            // per column: ||r_k||^2 of iterations 0..hist_len-1
    int hist_len = 0;
    cudaEvent_t sev[8] = {};           // stage boundaries of one PCG iteration (stage_times)
    bool sev_ok = false;
};

struct algmortar_handle {
    int device = 0;
    cudaStream_t st = nullptr;
    cudaStream_t own_st = nullptr;   // created when the caller passes no stream
    algmortar_opts opts{};
    Plan P;
    int64_t n = 0;
    int m = 0, L = 0;
    std::vector<void*> allocs;
    // permuted matrix and maps
    int32_t *d_rowptr = nullptr, *d_col = nullptr, *d_perm = nullptr, *d_row_sub = nullptr;
    double* d_val = nullptr;
    int64_t* d_sub_off = nullptr;
    int nchunks = 0;                   // prolongation: row chunks (<= 32 rows of one subdomain)
    ProlongChunk* d_chunks = nullptr;
    int32_t* d_chunk_sub = nullptr;    // subdomain of each chunk
    int tile_wm = 1;                   // widest tile row of the local profiles (tiles)
    int64_t nprm = 0;                  // entries of the row-major panels
    // local factor profile and streams
    Profile pf{};
    int32_t *d_rows = nullptr, *d_ntiles = nullptr;
    void *d_fwdS = nullptr, *d_bwdS = nullptr;
    // block-Jacobi smoother (Sec. 5.4): factors of the unmodified blocks A_ii on the same
    // tile profiles, and their symmetric scaling
    void *d_fwdS2 = nullptr, *d_bwdS2 = nullptr;
    double *d_dloc2 = nullptr, *d_sc2 = nullptr;
    float* d_sc2_32 = nullptr;
    double *d_dloc = nullptr, *d_sc = nullptr;
    float* d_sc32 = nullptr;
    int32_t* d_job_sub = nullptr;
    int64_t* d_job_off = nullptr;
    // interfaces
    int64_t* d_rptr = nullptr;
    int32_t* d_rcell = nullptr;
    double* d_rcoef = nullptr;
    int64_t *d_if_off = nullptr, *d_phi_off = nullptr;
    int32_t* d_if_list = nullptr;
    void* d_phi = nullptr;
    // interface solve by nested dissection (ND order inside the handle)
    NdSolveArgs nd{};
    int32_t* nd_grows = nullptr;       // rows of each interface group (symmetrisation)
    int32_t* d_ndpos = nullptr;        // interface id -> ND position
    int32_t* d_ifpos = nullptr;        // if_list entries as ND positions (prolongation)
    // inexact interface solve (block-Jacobi PCG on S_eta in a thread-block cluster)
    bool inexact = false;
    IfaceArgs iface{};
    int iface_cluster = 0;
    size_t iface_smem = 0;
    int iface_nblk = 0, iface_max_nb = 0;
    // launch variants in use (defaults, or the autotuner's choice)
    int tuned_ring = 0;
    int tuned_vec_ctas = 4;
    int tuned_order = 0;               // local-solve job order: 0 rows, 1 stored tiles, 2 tile rows
    int32_t* d_job_sub_v[3] = {nullptr, nullptr, nullptr};
    int64_t* d_job_off_v[3] = {nullptr, nullptr, nullptr};
    // workspace: single right-hand side (v1) and the batched solves' columns (vk)
    Vecs v1, vk;
    double* d_scalar = nullptr;
    int* d_kerr = nullptr;             // kernel error word (stuck bulk copy)
    NumWs* ws = nullptr;               // persistent numeric-setup buffers
    int32_t* d_psrc = nullptr;         // permuted CSR value t = original value psrc[t]
    int64_t* d_rp_ptr = nullptr;       // restriction entry -> CSR positions of its couplings
    int32_t* d_rp_pos = nullptr;
    int32_t* d_g_from_r = nullptr;     // G entry -> restriction entry
    int64_t* d_ell_ptr = nullptr;      // sliced-ELL copy of the matrix (SpMV)
    int32_t *d_ell_col = nullptr, *d_ell_src = nullptr;
    double* d_ell_val = nullptr;
    int64_t n_ell = 0;
    int ell_wf = 0;                    // slice width of the SpMV's unrolled path (0: none)
    double* d_vtmp = nullptr;          // staging for value updates (original CSR order)
    // FP32 interface inverses (G_g^-1, W_g in both layouts, C^-1) and the restriction
    // tables in one block, kept in L2 across PCG iterations by an access-policy window on
    // the iteration graph's kernels
    float* ifw32 = nullptr;
    size_t ifw32_bytes = 0;
    int64_t ifw_cinv = 0;   // offset (floats) of C^-1 in the block
    int64_t ifw_ifpos = 0;  // offset (floats) of the ND interface positions
    cudaAccessPolicyWindow l2w{};
    algmortar_info info{};

    template <typename T>
    T* alloc(size_t count) {
        if (count == 0) count = 1;
        void* p = nullptr;
        if (cudaMalloc(&p, count * sizeof(T)) != cudaSuccess) return nullptr;
        allocs.push_back(p);
        return (T*)p;
    }
    void release(void* p) {
        for (auto& q : allocs)
            if (q == p) {
                cudaFree(q);
                q = nullptr;
            }
    }
    ~algmortar_handle() {
        if (v1.graph) cudaGraphExecDestroy(v1.graph);
        if (vk.graph) cudaGraphExecDestroy(vk.graph);
        for (Vecs* v : {&v1, &vk})
            for (cudaEvent_t e : v->sev)
                if (e) cudaEventDestroy(e);
        if (l2w.num_bytes) cudaCtxResetPersistingL2Cache();   // its lines back to normal
        for (void* p : allocs)
            if (p) cudaFree(p);
        if (own_st) cudaStreamDestroy(own_st);
        delete ws;
    }
};

namespace {

// Storage type of the MBF panels Phi: FP64 with FP64 factors, else FP32.  BF16 panels
// would round Phi apart from the A_i^{-1} that the interface matrix was built with, and
// that mismatch makes M^{-1} visibly non-symmetric (~1e-4 relative); FP32 keeps it at
// rounding level for 32 MB more per iteration at config 3.

template <typename TS>
using PanelT = typename std::conditional<std::is_same<TS, double>::value, double, float>::type;

template <typename T>
int upload(algmortar_t* h, T*& dst, const std::vector<T>& src) {
    dst = h->alloc<T>(src.size());
    if (!dst) return fail(ALGMORTAR_OOM, "device allocation failed");
    if (!src.empty()) CU(cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, h->st));
    return 0;
}

#define TRY(x)              \
    do {                    \
        int rc_ = (x);      \
        if (rc_) return rc_; \
    } while (0)

int upload_jobs(algmortar_t* h, DevBlockJobs& d, const BlockJobs& b) {
    d.n = b.size();
    TRY(upload(h, d.sub, b.sub));
    TRY(upload(h, d.nc, b.nc));
    TRY(upload(h, d.t0, b.t0));
    TRY(upload(h, d.in, b.in));
    TRY(upload(h, d.ld, b.ld));
    return 0;
}

// A solve over column-block jobs (SolveArgs.job_* set from d; in/out offsets shared).
template <typename TS, typename TA>
int solve_cols(SolveArgs a, const DevBlockJobs& d, bool identity, int max_tiles, cudaStream_t st) {
    a.job_sub = d.sub;
    a.job_in = d.in;
    a.job_out = d.in;
    a.job_ld = d.ld;
    a.job_nc = d.nc;
    a.job_t0 = identity ? d.t0 : nullptr;
    CU((launch_tile_solve_cols<TS, TA>(a, d.n, max_tiles, st)));
    return 0;
}

// Jobs of launch_tile_inv for items with T[it] tile rows: the diagonal inverses, then per
// level of a recursive halving of [0, T) (children first) the products P = L21 W11 and
// W21 = -W22 P of every node of that height, then the lower tiles of W^T W.  Every range
// is one launch; its jobs only read tiles finished by earlier launches.
void build_inv_jobs(const std::vector<int32_t>& T, std::vector<int4>& jobs, std::vector<std::pair<int, int>>& ranges) {
    jobs.clear();
    ranges.clear();
    auto job = [](int it, int I, int J, int k0, int k1, int type) {
        return make_int4(it, (I << 16) | J, (k0 << 16) | k1, type);
    };
    // nodes [a, b) by height, all items
    std::vector<std::vector<std::array<int, 4>>> byh;   // {item, a, m, b}
    std::function<int(int, int, int)> walk = [&](int it, int a, int b) -> int {
        if (b - a <= 1) return 0;
        const int m = a + (b - a) / 2;
        const int h = 1 + std::max(walk(it, a, m), walk(it, m, b));
        if ((int)byh.size() < h) byh.resize(h);
        byh[h - 1].push_back({it, a, m, b});
        return h;
    };
    int start = 0;
    for (int it = 0; it < (int)T.size(); ++it)
        for (int I = 0; I < T[it]; ++I) jobs.push_back(job(it, I, I, 0, 0, 0));
    ranges.push_back({start, (int)jobs.size() - start});
    for (int it = 0; it < (int)T.size(); ++it) walk(it, 0, T[it]);
    for (const auto& lev : byh) {
        start = (int)jobs.size();
        for (const auto& nd : lev)
            for (int I = nd[2]; I < nd[3]; ++I)
                for (int J = nd[1]; J < nd[2]; ++J) jobs.push_back(job(nd[0], I, J, J, nd[2], 1));
        ranges.push_back({start, (int)jobs.size() - start});
        start = (int)jobs.size();
        for (const auto& nd : lev)
            for (int I = nd[2]; I < nd[3]; ++I)
                for (int J = nd[1]; J < nd[2]; ++J) jobs.push_back(job(nd[0], I, J, nd[2], I + 1, 2));
        ranges.push_back({start, (int)jobs.size() - start});
    }
    start = (int)jobs.size();
    for (int it = 0; it < (int)T.size(); ++it)
        for (int I = 0; I < T[it]; ++I)
            for (int J = 0; J <= I; ++J) jobs.push_back(job(it, I, J, I, T[it], 3));
    ranges.push_back({start, (int)jobs.size() - start});
}

int read_err_flag(algmortar_t* h, int* d_err, const char* what) {
    int e[2];
    CU(cudaMemcpyAsync(e, d_err, sizeof(e), cudaMemcpyDeviceToHost, h->st));
    CU(cudaStreamSynchronize(h->st));
    if (e[0]) return fail(ALGMORTAR_NOT_SPD, std::string("non-positive pivot in the ") + what + " factor, block " +
                                                 std::to_string(e[1]));
    return 0;
}

// Symbolic part of the inexact interface solve: the CSR pattern of S_eta (I ~ J when the
// two interfaces share a subdomain; natural interface order, columns ascending), where
// each off-diagonal value comes from (the per-subdomain block of the one shared
// subdomain), the block-Jacobi blocks (I = (i, j) -> block i / g, contiguous because
// interfaces are numbered lexicographically), and a block-aligned split of the rows over
// the CTAs of one cluster, balanced by S_eta entries plus block-inverse entries.
int prepare_inexact(algmortar_t* h, NumWs& W) {
    const Plan& P = h->P;
    const int L = h->L, m = h->m;
    const int g = h->opts.iface_block_parts > 0 ? h->opts.iface_block_parts : 1;
    // per-subdomain block offsets and each interface's position in its subdomains' lists
    std::vector<int64_t> pv_off(m + 1, 0);
    for (int sb = 0; sb < m; ++sb) {
        const int64_t k = P.if_off[sb + 1] - P.if_off[sb];
        pv_off[sb + 1] = pv_off[sb] + k * k;
    }
    std::vector<std::vector<std::pair<int32_t, int64_t>>> rows(L);   // (J, source)
    for (int sb = 0; sb < m; ++sb) {
        const int64_t i0 = P.if_off[sb], k = P.if_off[sb + 1] - i0;
        for (int64_t a = 0; a < k; ++a)
            for (int64_t b = 0; b < k; ++b) {
                if (a == b) continue;
                rows[P.if_list[i0 + a]].push_back({P.if_list[i0 + b], pv_off[sb] + a * k + b});
            }
    }
    std::vector<int32_t> s_ptr(L + 1, 0), s_col;
    std::vector<int64_t> src;
    for (int I = 0; I < L; ++I) {
        auto& r = rows[I];
        r.push_back({I, -1});
        std::sort(r.begin(), r.end());
        for (size_t t = 0; t < r.size(); ++t) {
            if (t > 0 && r[t].first == r[t - 1].first)
                return fail(ALGMORTAR_INVALID_ARG, "two interfaces share more than one subdomain");
            s_col.push_back(r[t].first);
            src.push_back(r[t].second);
        }
        if ((int64_t)s_col.size() > INT32_MAX) return fail(ALGMORTAR_TOO_LARGE, "interface matrix too large");
        s_ptr[I + 1] = (int32_t)s_col.size();
        std::vector<std::pair<int32_t, int64_t>>().swap(r);
    }
    // blocks
    std::vector<int32_t> blk_row0{0}, row_blk(L);
    for (int I = 1; I <= L; ++I)
        if (I == L || P.pairs[2 * (size_t)I] / g != P.pairs[2 * (size_t)(I - 1)] / g) blk_row0.push_back(I);
    const int nblk = (int)blk_row0.size() - 1;
    std::vector<int64_t> blk_off(nblk + 1, 0);
    int max_nb = 0;
    for (int b = 0; b < nblk; ++b) {
        const int nb = blk_row0[b + 1] - blk_row0[b];
        max_nb = std::max(max_nb, nb);
        blk_off[b + 1] = blk_off[b] + (int64_t)nb * nb;
        for (int I = blk_row0[b]; I < blk_row0[b + 1]; ++I) row_blk[I] = b;
    }
    if (L >= (1 << 24)) return fail(ALGMORTAR_TOO_LARGE, "inexact interface solve: n_lambda too large");
    if (max_nb > IFACE_MAX_BLOCK)
        return fail(ALGMORTAR_INVALID_ARG, "inexact interface solve: a block-Jacobi block has " +
                                               std::to_string(max_nb) + " interfaces (at most " +
                                               std::to_string(IFACE_MAX_BLOCK) + "); lower iface_block_parts");
    // cluster: 16 CTAs where the device runs such clusters, else 8, never more than blocks
    int cl = std::min(IFACE_MAX_CLUSTER, nblk);
    std::vector<int32_t> cta_row0, cta_blk0;
    size_t smem = 0;
    bool stage = false;
    int max_rows = 0;
    int64_t max_nnz = 0, max_inv = 0;
    auto split = [&](int c) {
        // greedy block-aligned split: close a CTA once it reaches its share of the work
        std::vector<int64_t> wblk(nblk);
        int64_t tot = 0;
        for (int b = 0; b < nblk; ++b) {
            wblk[b] = (s_ptr[blk_row0[b + 1]] - s_ptr[blk_row0[b]]) + (blk_off[b + 1] - blk_off[b]);
            tot += wblk[b];
        }
        cta_blk0.assign(1, 0);
        int64_t acc = 0;
        for (int b = 0; b < nblk; ++b) {
            acc += wblk[b];
            const int done = (int)cta_blk0.size();
            const int left_blocks = nblk - (b + 1), left_ctas = c - done;
            if (done < c && (acc * c >= tot * done || left_blocks <= left_ctas)) cta_blk0.push_back(b + 1);
        }
        while ((int)cta_blk0.size() < c + 1) cta_blk0.push_back(nblk);
        cta_blk0.back() = nblk;
        cta_row0.resize(c + 1);
        max_rows = 0;
        max_nnz = max_inv = 0;
        for (int t = 0; t <= c; ++t) cta_row0[t] = blk_row0[cta_blk0[t]];
        for (int t = 0; t < c; ++t) {
            max_rows = std::max(max_rows, cta_row0[t + 1] - cta_row0[t]);
            max_nnz = std::max<int64_t>(max_nnz, s_ptr[cta_row0[t + 1]] - s_ptr[cta_row0[t]]);
            max_inv = std::max<int64_t>(max_inv, blk_off[cta_blk0[t + 1]] - blk_off[cta_blk0[t]]);
        }
    };
    int sm_optin = 0;
    CU(cudaDeviceGetAttribute(&sm_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
    for (;;) {
        split(cl);
        if (max_rows >= (1 << 16))
            return fail(ALGMORTAR_TOO_LARGE, "inexact interface solve: too many interfaces for one cluster");
        stage = iface_smem_bytes(L, max_rows, max_nnz, max_inv, true) <= (size_t)sm_optin;
        smem = iface_smem_bytes(L, max_rows, max_nnz, max_inv, stage);
        if (smem > (size_t)sm_optin)
            return fail(ALGMORTAR_TOO_LARGE, "inexact interface solve: n_lambda too large for one cluster");
        int active = 0;
        cudaError_t e = prepare_iface_pcg(cl, smem, &active);
        if (e == cudaSuccess && active > 0) break;
        cudaGetLastError();
        if (cl <= 1) return fail(ALGMORTAR_CUDA, "inexact interface solve: no cluster shape fits the device");
        cl = cl > 8 ? 8 : cl / 2;
    }
    if (h->opts.verbose)
        std::fprintf(stderr,
                     "[algmortar] inexact interface solve: n_lambda=%d blocks=%d (max %d) cluster=%d smem=%zu B "
                     "staged=%d rows/CTA<=%d entries/CTA<=%lld inverse/CTA<=%lld\n",
                     L, nblk, max_nb, cl, smem, stage ? 1 : 0, max_rows, (long long)max_nnz, (long long)max_inv);
    std::vector<int2> row_info(L);
    for (int c = 0; c < cl; ++c)
        for (int I = cta_row0[c]; I < cta_row0[c + 1]; ++I) {
            const int bk = row_blk[I], b0 = blk_row0[bk], nb = blk_row0[bk + 1] - b0;
            row_info[I] = make_int2((b0 - cta_row0[c]) | (nb << 16),
                                    (int)(blk_off[bk] - blk_off[cta_blk0[c]] + (int64_t)(I - b0) * nb));
        }
    IfaceArgs& a = h->iface;
    a.L = L;
    a.max_rows = max_rows;
    a.max_nnz = max_nnz;
    a.max_inv = max_inv;
    a.stage = stage ? 1 : 0;
    a.max_it = h->opts.iface_max_it > 0 ? h->opts.iface_max_it : 200;
    a.rtol = h->opts.iface_rtol > 0 ? h->opts.iface_rtol : 1e-2;
    int32_t *d_sptr = nullptr, *d_scol = nullptr, *d_rowblk = nullptr, *d_blk0 = nullptr, *d_crow = nullptr,
            *d_cblk = nullptr;
    int64_t* d_boff = nullptr;
    TRY(upload(h, d_sptr, s_ptr));
    TRY(upload(h, d_scol, s_col));
    TRY(upload(h, d_rowblk, row_blk));
    int2* d_rinfo = nullptr;
    TRY(upload(h, d_rinfo, row_info));
    TRY(upload(h, d_blk0, blk_row0));
    TRY(upload(h, d_boff, blk_off));
    TRY(upload(h, d_crow, cta_row0));
    TRY(upload(h, d_cblk, cta_blk0));
    TRY(upload(h, W.d_csr_src, src));
    TRY(upload(h, W.d_pv_off, pv_off));
    W.pv = h->alloc<double>((size_t)std::max<int64_t>(pv_off[m], 1));
    W.s_val64 = h->alloc<double>(s_col.size());
    float2* s_ent = h->alloc<float2>(s_col.size());
    float* binv = h->alloc<float>((size_t)std::max<int64_t>(blk_off[nblk], 1));
    if (!W.pv || !W.s_val64 || !s_ent || !binv) return fail(ALGMORTAR_OOM, "inexact interface buffers");
    a.cta_row0 = d_crow;
    a.cta_blk0 = d_cblk;
    a.s_ptr = d_sptr;
    a.s_col = d_scol;
    a.s_ent = s_ent;
    a.row_blk = d_rowblk;
    a.row_info = d_rinfo;
    a.blk_row0 = d_blk0;
    a.blk_off = d_boff;
    a.binv = binv;
    h->iface_cluster = cl;
    h->iface_smem = smem;
    h->iface_nblk = nblk;
    h->iface_max_nb = max_nb;
    h->d_ifpos = h->d_if_list;   // interface values in natural order
    return 0;
}

// Symbolic uploads and persistent buffers (first numeric setup only).
template <typename TW, typename TS>
int numeric_prepare(algmortar_t* h, NumWs& W) {
    if (W.ready) return 0;
    Plan& P = h->P;
    const int m = h->m, L = h->L;
    const int64_t tiles = P.total_tiles, trows = P.trow_off[m], nphi = P.phi_off[m];
    std::vector<int32_t> js;
    std::vector<int64_t> jo;
    for (int s = 0; s < m; ++s) {
        int64_t ns = P.sub_off[s + 1] - P.sub_off[s];
        for (int64_t a = 0; a < P.if_off[s + 1] - P.if_off[s]; ++a) {
            js.push_back(s);
            jo.push_back(P.phi_off[s] + a * ns);
        }
    }
    W.njobs_mbf = (int)js.size();
    {
        BlockJobs b;
        for (int s = 0; s < m; ++s) {
            const int64_t ns = P.sub_off[s + 1] - P.sub_off[s];
            b.add(s, P.phi_off[s], ns, P.if_off[s + 1] - P.if_off[s], false);
        }
        TRY(upload_jobs(h, W.bj_mbf, b));
        // PANEL_NC columns per job, subdomains with the longest tile chains first
        std::vector<int32_t> ord(m);
        for (int s = 0; s < m; ++s) ord[s] = s;
        std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return P.ntiles[x] > P.ntiles[y]; });
        BlockJobs pb;
        for (int s : ord) {
            const int64_t ns = P.sub_off[s + 1] - P.sub_off[s], kk = P.if_off[s + 1] - P.if_off[s];
            for (int64_t c = 0; c < kk; c += PANEL_NC) {
                pb.sub.push_back(s);
                pb.in.push_back(P.phi_off[s] + c * ns);
                pb.ld.push_back(ns);
                pb.nc.push_back((int32_t)std::min<int64_t>(PANEL_NC, kk - c));
                pb.t0.push_back(0);
            }
        }
        TRY(upload_jobs(h, W.pj_mbf, pb));
    }
    std::vector<int64_t> gcptr;
    gcptr.reserve(P.if_off[m] + m);
    for (int s = 0; s < m; ++s) {
        int k = (int)(P.if_off[s + 1] - P.if_off[s]);
        int64_t t = P.g_off[s];
        for (int a = 0; a <= k; ++a) {
            while (t < P.g_off[s + 1] && P.g_col[t] < a) ++t;
            gcptr.push_back(t);
        }
    }
    TRY(upload(h, W.d_js, js));
    TRY(upload(h, W.d_jo, jo));
    TRY(upload(h, W.d_goff, P.g_off));
    TRY(upload(h, W.d_gcptr, gcptr));
    TRY(upload(h, W.d_grow, P.g_row));
    TRY(upload(h, W.d_gcol, P.g_col));
    TRY(upload(h, W.d_gval, P.g_val));
    TRY(upload(h, W.d_pairs, P.pairs));
    W.work = h->alloc<TW>((size_t)tiles * TILE2);
    W.dinv = h->alloc<TW>((size_t)trows * TILE2);
    W.d_err = h->alloc<int>(2);
    W.rhs = h->alloc<double>(nphi);
    W.phi64 = h->alloc<double>(nphi);
    if (!std::is_same<TS, double>::value && panel_solve_fits(h->tile_wm, P.max_tiles, sizeof(TS))) {
        W.w32 = h->alloc<float>((size_t)std::max<int64_t>(nphi, 1));
        if (!W.w32) return fail(ALGMORTAR_OOM, "MBF right-hand sides");
    }
    h->d_fwdS = h->alloc<TS>((size_t)tiles * TILE2);
    h->d_bwdS = h->alloc<TS>((size_t)tiles * TILE2);
    if (h->opts.smooth_steps > 0) {
        h->d_fwdS2 = h->alloc<TS>((size_t)tiles * TILE2);
        h->d_bwdS2 = h->alloc<TS>((size_t)tiles * TILE2);
        if (!h->d_fwdS2 || !h->d_bwdS2) return fail(ALGMORTAR_OOM, "smoother factor buffers");
    }
    h->d_phi = (void*)h->alloc<PanelT<TS>>((size_t)std::max<int64_t>(h->nprm, 1));   // row-major (prolongation)
    if (!W.work || !W.dinv || !W.d_err || !W.rhs || !W.phi64 || !h->d_fwdS || !h->d_bwdS || !h->d_phi)
        return fail(ALGMORTAR_OOM, "factor / MBF buffers");
    if (L > 0 && h->inexact) {
        TRY(upload(h, W.d_T, P.T));
        W.diagc = h->alloc<double>(2 * (size_t)L);
        if (!W.diagc) return fail(ALGMORTAR_OOM, "interface matrix");
        TRY(prepare_inexact(h, W));
    } else if (L > 0) {
        TRY(upload(h, W.d_T, P.T));
        W.diagc = h->alloc<double>(2 * (size_t)L);
        W.Sd = h->alloc<double>((size_t)L * L);
        if (!W.diagc || !W.Sd) return fail(ALGMORTAR_OOM, "interface matrix");
        // ---- groups (interior blocks) as dense factor items ----
        const int G = P.nd_G;
        const int64_t nin = P.nd_goff[G];
        const int nsep = P.nd_nsep;
        std::vector<int32_t> irows, int_, ilo, ihi, titem, tI, tJ, gjob, gjt0, row_g, prow_g;
        std::vector<int64_t> irow0, ibase, ifwd, ibwd, isrc, gjin, gioff(G, 0), woff(G, 0), doff(G, 0);
        int64_t trow = 0, tb = 0, gi = 0, wo = 0, dof = 0;
        for (int g = 0; g < G; ++g) {
            const int64_t ng = P.nd_goff[g + 1] - P.nd_goff[g], ag = P.nd_aoff[g + 1] - P.nd_aoff[g];
            gioff[g] = gi;
            woff[g] = wo;
            doff[g] = dof;
            for (int64_t t = 0; t < ng; ++t) row_g.push_back(g);
            for (int64_t t = 0; t < ag; ++t) prow_g.push_back(g);
            if (ng > 0) {
                const int it = (int)irows.size();
                const int T = (int)((ng + TILE - 1) / TILE);
                W.item_group.push_back(g);
                W.item_row0.push_back(trow);
                W.item_base.push_back(tb);
                irows.push_back((int32_t)ng);
                int_.push_back(T);
                irow0.push_back(trow);
                ibase.push_back(tb);
                isrc.push_back(P.nd_goff[g] * L + P.nd_goff[g]);
                std::vector<int32_t> hi(T, T - 1);
                W.item_hi.push_back(hi);
                for (int I = 0; I < T; ++I) {
                    ilo.push_back(0);
                    ihi.push_back(T - 1);
                    ifwd.push_back((int64_t)I * (I + 1) / 2);
                    ibwd.push_back((int64_t)(T - 1 - I) * (T - I) / 2);
                    for (int J = 0; J <= I; ++J) {
                        titem.push_back(it);
                        tI.push_back(I);
                        tJ.push_back(J);
                    }
                }
                W.max_tiles_items = std::max(W.max_tiles_items, T);
                trow += T;
                tb += (int64_t)T * (T + 1) / 2;
                for (int64_t c = 0; c < ng; ++c) {
                    gjob.push_back(it);
                    gjt0.push_back((int32_t)(c / TILE));
                    gjin.push_back(gi + c * ng);
                }
            }
            gi += ng * ng;
            wo += ng * ag;
            dof += ag * ag;
        }
        W.nitems = (int)irows.size();
        W.ntiles_items = tb;
        W.trows_items = trow;
        W.njobs_g = (int)gjob.size();
        TRY(upload(h, W.d_irows, irows));
        TRY(upload(h, W.d_int, int_));
        TRY(upload(h, W.d_irow0, irow0));
        TRY(upload(h, W.d_ibase, ibase));
        TRY(upload(h, W.d_ilo, ilo));
        TRY(upload(h, W.d_ihi, ihi));
        TRY(upload(h, W.d_ifwd, ifwd));
        TRY(upload(h, W.d_ibwd, ibwd));
        TRY(upload(h, W.d_isrc, isrc));
        TRY(upload(h, W.d_titem, titem));
        TRY(upload(h, W.d_tI, tI));
        TRY(upload(h, W.d_tJ, tJ));
        TRY(upload(h, W.d_gjob, gjob));
        TRY(upload(h, W.d_gjin, gjin));
        TRY(upload(h, W.d_gjt0, gjt0));
        TRY(upload(h, W.d_doff, doff));
        // the interface blocks are factored and inverted in FP64 for FP64 factors and in FP32
        // for FP32 / BF16 factors (the FP32 pipeline reproduces eta to ~4e-6 relative at
        // config 3, below those variants' local-solve error; B300's FP32 rate is 64x FP64)
        const bool lowp = h->opts.precision != ALGMORTAR_FP64;
        const size_t isz = lowp ? sizeof(float) : sizeof(double);
        W.gwork = h->alloc<unsigned char>((size_t)std::max<int64_t>(tb, 1) * TILE2 * isz);
        W.gdinv = h->alloc<unsigned char>((size_t)std::max<int64_t>(trow, 1) * TILE2 * isz);
        W.gf = h->alloc<unsigned char>((size_t)std::max<int64_t>(tb, 1) * TILE2 * isz);
        W.gb = h->alloc<unsigned char>((size_t)std::max<int64_t>(tb, 1) * TILE2 * isz);
        if (lowp) {
            W.gplanes = h->alloc<float>((size_t)std::max<int64_t>(tb, 1) * 2 * TILE2);
            if (!W.gplanes) return fail(ALGMORTAR_OOM, "interface planes");
            {
                // two CTAs of the update per SM; row blocks: at most those of column 0
                int sms = 148;
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
                int64_t nb = 0;
                for (int it = 0; it < W.nitems; ++it) nb += ((int64_t)W.item_hi[it].size() + 3) / 4;
                nb = std::max<int64_t>(nb, ((int64_t)P.nd_nsep + TILE - 1) / TILE / 4 + 1);
                W.tcs.max_ctas = 2 * (int64_t)sms;
                W.tcs.max_blocks = nb;
                W.tcs.part = h->alloc<float>((size_t)W.tcs.max_ctas * 4 * TILE2);
                W.tcs.ticket = h->alloc<unsigned int>((size_t)nb);
                if (!W.tcs.part || !W.tcs.ticket) return fail(ALGMORTAR_OOM, "interface update workspace");
                CU(cudaMemsetAsync(W.tcs.ticket, 0, (size_t)nb * sizeof(unsigned int), h->st));
            }
            // explicit S_gg^{-1} by tile products (gf / gb hold W = L^{-1} and P)
            std::vector<int32_t> Ts;
            std::vector<int64_t> iout;
            for (int it = 0; it < (int)W.item_group.size(); ++it) {
                Ts.push_back((int32_t)W.item_hi[it].size());
                iout.push_back(gioff[W.item_group[it]]);
            }
            std::vector<int4> jobs;
            build_inv_jobs(Ts, jobs, W.ginv_ranges);
            TRY(upload(h, W.d_ginv_jobs, jobs));
            TRY(upload(h, W.d_iout, iout));
        }
        W.gE = h->alloc<double>((size_t)std::max<int64_t>(gi, 1));
        W.D = h->alloc<double>((size_t)std::max<int64_t>(dof, 1));
        double* Ginv = h->alloc<double>((size_t)std::max<int64_t>(gi, 1));
        double* Wcm = h->alloc<double>((size_t)std::max<int64_t>(wo, 1));
        double* Wrm = h->alloc<double>((size_t)std::max<int64_t>(wo, 1));
        if (!W.gwork || !W.gdinv || !W.gf || !W.gb || !W.gE || !W.D || !Ginv || !Wcm || !Wrm)
            return fail(ALGMORTAR_OOM, "interface group buffers");
        // FP32 / BF16 factor variants also apply the interface inverses in FP32 (FP32
        // copies): half the bytes of the solve, and FP32 products
        float *Ginv32 = nullptr, *Wcm32 = nullptr, *Wrm32 = nullptr;
        std::vector<int64_t> gioff32(G, 0), woff32(G, 0), gpo32(G, 0);
        int64_t gi32 = 0, wo32 = 0, pos32 = 0;
        for (int g = 0; g < G; ++g) {
            const int64_t ng = P.nd_goff[g + 1] - P.nd_goff[g], ag = P.nd_aoff[g + 1] - P.nd_aoff[g];
            const int64_t ng4 = (ng + 3) & ~int64_t(3);
            gioff32[g] = gi32;
            woff32[g] = wo32;
            gpo32[g] = pos32;
            gi32 += ng * ng4;
            wo32 += ag * ng4;
            pos32 += ng4;
        }
        const int nsep4 = (nsep + 3) & ~3;
        if (lowp) {
            // One block, 256-byte aligned parts: G^-1 | W (column-major) | W (row-major) |
            // C^-1, then tables every iteration re-reads, moved here from their own
            // allocations: restriction pointers, cells and coefficients, the local solves'
            // FP32 row scales, tile-profile descriptors and job lists (sizes in floats).
            auto up = [](int64_t bytes) { return ((std::max<int64_t>(bytes, 1) + 3) / 4 + 63) & ~int64_t(63); };
            const int64_t R = (int64_t)P.r_cell.size(), trw = P.trow_off[m];
            const int64_t o1 = up(4 * gi32), o2 = o1 + up(4 * wo32), o3 = o2 + up(4 * wo);
            const int64_t o4 = o3 + up(4 * (int64_t)nsep * nsep4);
            // the moved tables, in the order of the move_in calls below
            const int64_t moved = up(8 * ((int64_t)L + 1)) + up(4 * R) + up(8 * R) + up(4 * h->n) + 2 * up(4 * m) +
                                  2 * up(8 * ((int64_t)m + 1)) + 2 * up(4 * trw) + 2 * up(8 * trw) +
                                  3 * (up(4 * (int64_t)m) + up(8 * (int64_t)m)) +
                                  up((int64_t)sizeof(ProlongChunk) * h->nchunks) + up(8 * (int64_t)P.ell_ptr.size()) +
                                  up(4 * (int64_t)P.if_list.size());
            const int64_t tot = o4 + moved;
            h->ifw32 = h->alloc<float>((size_t)tot);
            if (!h->ifw32) return fail(ALGMORTAR_OOM, "interface group buffers");
            h->ifw32_bytes = (size_t)tot * sizeof(float);
            h->ifw_cinv = o3;
            Ginv32 = h->ifw32;
            Wcm32 = h->ifw32 + o1;
            Wrm32 = h->ifw32 + o2;
            int64_t off = o4;
            bool moved_ok = true;
            // copy a table into the block, free its old allocation, return the new address
            auto move_in = [&](auto* src, int64_t count) -> decltype(src) {
                using T = std::remove_cv_t<std::remove_pointer_t<decltype(src)>>;
                T* dst = reinterpret_cast<T*>(h->ifw32 + off);
                off += up((int64_t)sizeof(T) * count);
                if (count > 0 && cudaMemcpyAsync(dst, src, (size_t)count * sizeof(T), cudaMemcpyDeviceToDevice,
                                                 h->st) != cudaSuccess)
                    moved_ok = false;
                if (cudaStreamSynchronize(h->st) != cudaSuccess) moved_ok = false;
                h->release(const_cast<T*>(src));
                return dst;
            };
            h->d_rptr = move_in(h->d_rptr, (int64_t)L + 1);
            h->d_rcell = move_in(h->d_rcell, R);
            h->d_rcoef = move_in(h->d_rcoef, R);
            h->d_sc32 = move_in(h->d_sc32, h->n);
            h->d_rows = move_in(h->d_rows, m);
            h->d_ntiles = move_in(h->d_ntiles, m);
            h->pf.rows = h->d_rows;
            h->pf.ntiles = h->d_ntiles;
            h->pf.row0 = move_in(h->pf.row0, (int64_t)m + 1);
            h->pf.base = move_in(h->pf.base, (int64_t)m + 1);
            h->pf.lo = move_in(h->pf.lo, trw);
            h->pf.hi = move_in(h->pf.hi, trw);
            h->pf.fwd = move_in(h->pf.fwd, trw);
            h->pf.bwd = move_in(h->pf.bwd, trw);
            for (int v = 0; v < 3; ++v) {
                const bool cur = h->d_job_sub == h->d_job_sub_v[v];
                h->d_job_sub_v[v] = move_in(h->d_job_sub_v[v], m);
                h->d_job_off_v[v] = move_in(h->d_job_off_v[v], (int64_t)m);
                if (cur) {
                    h->d_job_sub = h->d_job_sub_v[v];
                    h->d_job_off = h->d_job_off_v[v];
                }
            }
            h->d_chunks = move_in(h->d_chunks, h->nchunks);
            h->d_ell_ptr = move_in(h->d_ell_ptr, (int64_t)P.ell_ptr.size());
            h->ifw_ifpos = off;   // filled below, with the interface positions in ND order
            off += up(4 * (int64_t)P.if_list.size());
            if (!moved_ok) return fail(ALGMORTAR_CUDA, "moving tables into the interface block");
        }
        W.n_ginv = gi;
        W.n_w = wo;
        W.h_gioff = gioff;
        W.h_woff = woff;
        W.h_gioff32 = gioff32;
        W.h_woff32 = woff32;
        // blocks of groups without interior unknowns are never written: keep them zero
        CU(cudaMemsetAsync(W.D, 0, (size_t)std::max<int64_t>(dof, 1) * sizeof(double), h->st));
        // identity right-hand sides of each group (column-major n_g x n_g)
        {
            std::vector<double> eye;
            CU(cudaMemsetAsync(W.gE, 0, (size_t)std::max<int64_t>(gi, 1) * sizeof(double), h->st));
            std::vector<int64_t> diag_idx;
            for (int g = 0; g < G; ++g) {
                const int64_t ng = P.nd_goff[g + 1] - P.nd_goff[g];
                for (int64_t c = 0; c < ng; ++c) diag_idx.push_back(gioff[g] + c * ng + c);
            }
            std::vector<double> ones(diag_idx.size(), 1.0);
            double* d_ones = nullptr;
            int64_t* d_didx = nullptr;
            TRY(upload(h, d_ones, ones));
            TRY(upload(h, d_didx, diag_idx));
            launch_scatter_values((int64_t)diag_idx.size(), d_didx, d_ones, W.gE, h->st);
        }
        // per-iteration ND solve arguments
        int64_t *d_goff = nullptr, *d_aoff = nullptr, *d_gioff = nullptr, *d_woff = nullptr;
        int32_t *d_alist = nullptr, *d_sg = nullptr, *d_sidx = nullptr, *d_rowg = nullptr, *d_prowg = nullptr;
        TRY(upload(h, d_goff, P.nd_goff));
        TRY(upload(h, d_aoff, P.nd_aoff));
        TRY(upload(h, d_gioff, gioff));
        TRY(upload(h, d_woff, woff));
        TRY(upload(h, d_alist, P.nd_alist));
        TRY(upload(h, d_sg, P.nd_sg));
        TRY(upload(h, d_sidx, P.nd_sidx));
        TRY(upload(h, d_rowg, row_g));
        TRY(upload(h, d_prowg, prow_g));
        {
            // nonzeros of S_{g,A_g}: interior interface i couples to separator interface a
            // exactly when they share a subdomain (Eq. interface-problem-alg)
            std::vector<int64_t> wc_ptr{0};
            std::vector<int32_t> wc_row, tmp;
            for (int g = 0; g < G; ++g) {
                const int64_t g0 = P.nd_goff[g], g1 = P.nd_goff[g + 1];
                for (int64_t j = P.nd_aoff[g]; j < P.nd_aoff[g + 1]; ++j) {
                    const int32_t I = P.nd_id[P.nd_goff[G] + P.nd_alist[j]];
                    tmp.clear();
                    for (int e = 0; e < 2; ++e) {
                        const int32_t sb = P.pairs[2 * (size_t)I + e];
                        for (int64_t t = P.if_off[sb]; t < P.if_off[sb + 1]; ++t) {
                            const int32_t pos = P.nd_pos[P.if_list[t]];
                            if (pos >= g0 && pos < g1) tmp.push_back((int32_t)(pos - g0));
                        }
                    }
                    std::sort(tmp.begin(), tmp.end());
                    tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
                    wc_row.insert(wc_row.end(), tmp.begin(), tmp.end());
                    wc_ptr.push_back((int64_t)wc_row.size());
                }
            }
            TRY(upload(h, W.d_wc_ptr, wc_ptr));
            TRY(upload(h, W.d_wc_row, wc_row));
        }
        TRY(upload(h, h->d_ndpos, P.nd_pos));
        {
            std::vector<int32_t> gr(G);
            for (int g = 0; g < G; ++g) gr[g] = (int32_t)(P.nd_goff[g + 1] - P.nd_goff[g]);
            TRY(upload(h, h->nd_grows, gr));
        }
        {
            std::vector<int32_t> ifpos(P.if_list.size());
            for (size_t t = 0; t < ifpos.size(); ++t) ifpos[t] = P.nd_pos[P.if_list[t]];
            if (h->ifw32) {
                h->d_ifpos = reinterpret_cast<int32_t*>(h->ifw32 + h->ifw_ifpos);
                if (!ifpos.empty())
                    CU(cudaMemcpyAsync(h->d_ifpos, ifpos.data(), ifpos.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                                       h->st));
                CU(cudaStreamSynchronize(h->st));
            } else {
                TRY(upload(h, h->d_ifpos, ifpos));
            }
        }
        NdSolveArgs& a = h->nd;
        a.G = G;
        a.nsep = nsep;
        a.nin = nin;
        a.np = P.nd_aoff[G];
        a.goff = d_goff;
        a.aoff = d_aoff;
        a.alist = d_alist;
        a.sg = d_sg;
        a.sidx = d_sidx;
        a.row_g = d_rowg;
        a.prow_g = d_prowg;
        a.Ginv = Ginv;
        a.gioff = d_gioff;
        a.Wcm = Wcm;
        a.Wrm = Wrm;
        a.woff = d_woff;
        a.Ginv32 = Ginv32;
        a.Wcm32 = Wcm32;
        a.Wrm32 = Wrm32;
        if (lowp) {
            std::vector<int32_t> p32(std::max<int64_t>(L, 1), 0);
            for (int64_t q = 0; q < nin; ++q) p32[q] = (int32_t)(gpo32[row_g[q]] + (q - P.nd_goff[row_g[q]]));
            for (int t = 0; t < nsep; ++t) p32[nin + t] = (int32_t)(pos32 + t);
            int64_t *d_gio32 = nullptr, *d_wo32 = nullptr, *d_gpo32 = nullptr;
            int32_t* d_p32 = nullptr;
            TRY(upload(h, d_gio32, gioff32));
            TRY(upload(h, d_wo32, woff32));
            TRY(upload(h, d_gpo32, gpo32));
            TRY(upload(h, d_p32, p32));
            a.gioff32 = d_gio32;
            a.woff32 = d_wo32;
            a.gpo32 = d_gpo32;
            a.p32 = d_p32;
            a.spo32 = pos32;
            a.L32 = pos32 + nsep4;
            a.nsep4 = nsep4;
        }

        // ---- separator Schur complement C as one dense item ----
        if (nsep > 0) {
            const int T = (nsep + TILE - 1) / TILE;
            W.cT = T;
            W.c_hi.assign(T, T - 1);
            std::vector<int32_t> clo(T, 0), chi(T, T - 1), cj(nsep, 0);
            std::vector<int64_t> cfwd(T), cbwd(T), cjin(nsep), czero{0};
            std::vector<int32_t> cjt0(nsep);
            for (int q = 0; q < nsep; ++q) cjt0[q] = q / TILE;
            for (int I = 0; I < T; ++I) {
                cfwd[I] = (int64_t)I * (I + 1) / 2;
                cbwd[I] = (int64_t)(T - 1 - I) * (T - I) / 2;
            }
            for (int q = 0; q < nsep; ++q) cjin[q] = (int64_t)q * nsep;
            std::vector<int32_t> crows{nsep}, cnt{T};
            TRY(upload(h, W.d_crows, crows));
            TRY(upload(h, W.d_cnt, cnt));
            TRY(upload(h, W.d_czero, czero));
            TRY(upload(h, W.d_clo, clo));
            TRY(upload(h, W.d_chi, chi));
            TRY(upload(h, W.d_cfwd, cfwd));
            TRY(upload(h, W.d_cbwd, cbwd));
            TRY(upload(h, W.d_cjob, cj));
            TRY(upload(h, W.d_cjin, cjin));
            TRY(upload(h, W.d_cjt0, cjt0));
            const int64_t ct = (int64_t)T * (T + 1) / 2;
            W.cwork = h->alloc<unsigned char>((size_t)ct * TILE2 * isz);
            W.cdinv = h->alloc<unsigned char>((size_t)T * TILE2 * isz);
            W.cf = h->alloc<unsigned char>((size_t)ct * TILE2 * isz);
            W.cb = h->alloc<unsigned char>((size_t)ct * TILE2 * isz);
            if (lowp) {
                W.cplanes = h->alloc<float>((size_t)ct * 2 * TILE2);
                if (!W.cplanes) return fail(ALGMORTAR_OOM, "separator planes");
                std::vector<int4> jobs;
                build_inv_jobs(std::vector<int32_t>{T}, jobs, W.cinv_ranges);
                TRY(upload(h, W.d_cinv_jobs, jobs));
            }
            W.cE = h->alloc<double>((size_t)nsep * nsep);
            double* Cinv = h->alloc<double>((size_t)nsep * nsep);
            if (!W.cwork || !W.cdinv || !W.cf || !W.cb || !W.cE || !Cinv)
                return fail(ALGMORTAR_OOM, "separator buffers");
            if (lowp) {
                a.Cinv32 = h->ifw32 + h->ifw_cinv;   // part of the interface block
            }
            CU(cudaMemsetAsync(W.cE, 0, (size_t)nsep * nsep * sizeof(double), h->st));
            launch_eye(nsep, W.cE, h->st);
            std::vector<int32_t> sq{nsep};
            std::vector<int64_t> z0{0};
            TRY(upload(h, W.d_crowsq, sq));
            TRY(upload(h, W.d_czerooff, z0));
            a.Cinv = Cinv;
            CU(prepare_nd_solve(nsep));
        }
    }
    W.ready = true;
    return 0;
}

// Interface system by one level of nested dissection, in arithmetic TI (FP64, or FP32 for
// FP32 / BF16 factors): dense tiles of the group blocks S_gg, their right-looking tile
// Cholesky and sweep streams, S_gg^{-1} from identity columns, W_g = S_gg^{-1} S_{g,A_g},
// the separator Schur complement C, its factor and C^{-1}.  Inverses are stored in FP64.
template <typename TI>
int nd_factor_inverse(algmortar_t* h, NumWs& W, cudaStream_t st) {
    const Plan& P = h->P;
    const int G = P.nd_G, nsep = P.nd_nsep, L = h->L;
    const int64_t sep0 = P.nd_goff[G];
    const int err_init[2] = {0, -1};
    Profile gpf{W.d_irows, W.d_int, W.d_irow0, W.d_ibase, W.d_ilo, W.d_ihi, W.d_ifwd, W.d_ibwd};
    launch_dense_to_tiles<TI>(W.ntiles_items, W.Sd, L, W.d_isrc, W.d_irows, W.d_ibase, W.d_titem, W.d_tI, W.d_tJ,
                              (TI*)W.gwork, st);
    CU(cudaMemcpyAsync(W.d_err, err_init, sizeof(err_init), cudaMemcpyHostToDevice, st));
    {
        std::vector<int32_t> Th(W.nitems);
        for (int it = 0; it < W.nitems; ++it) Th[it] = (int32_t)W.item_hi[it].size();
        launch_dense_cholesky<TI>(W.nitems, Th, W.d_int, W.d_ibase, W.d_irow0, (TI*)W.gwork, (TI*)W.gdinv, W.d_err,
                                  st, (TI*)W.gplanes, h->d_kerr, W.tcs);
    }
    CU(cudaGetLastError());
    TRY(read_err_flag(h, W.d_err, "interface (interior block)"));
    // S_gg^{-1}, then W_g = S_gg^{-1} S_{g,A_g} from its sparse pattern
    if constexpr (std::is_same<TI, double>::value) {
        // FP64: identity columns through the sweep streams, one job per column (measured
        // faster than column blocks for FP64: the FP64 work of a job is spread over four
        // warps and the grids are larger)
        launch_finalize<TI, TI>(W.nitems, gpf, (const TI*)W.gwork, (const TI*)W.gdinv, (TI*)W.gf, (TI*)W.gb, st);
        SolveArgs sa{};
        sa.pf = gpf;
        sa.fwdS = W.gf;
        sa.bwdS = W.gb;
        sa.err = h->d_kerr;
        sa.in = W.gE;
        sa.out = (double*)h->nd.Ginv;
        sa.job_sub = W.d_gjob;
        sa.job_in = W.d_gjin;
        sa.job_out = W.d_gjin;
        sa.job_t0 = W.d_gjt0;   // identity columns: lower triangle of S_gg^{-1} only
        CU((launch_tile_solve<TI, TI>(sa, W.njobs_g, W.max_tiles_items, st)));
    } else {
        // FP32: lower triangle of W^T W, W = L^{-1}, by batched tile products
        for (const auto& r : W.ginv_ranges)
            launch_tile_inv(W.d_ginv_jobs + r.first, r.second, (const float*)W.gwork, (const float*)W.gdinv,
                            (float*)W.gf, (float*)W.gb, (double*)h->nd.Ginv, W.d_ibase, W.d_irow0, W.d_irows,
                            W.d_iout, st);
    }
    launch_mirror_lower(h->nd_grows, h->nd.gioff, G, (double*)h->nd.Ginv, st);
    launch_nd_w_sparse(h->nd.np, L, W.Sd, h->nd.goff, h->nd.aoff, h->nd.alist, sep0, h->nd.prow_g, W.d_wc_ptr,
                       W.d_wc_row, h->nd.gioff, h->nd.Ginv, h->nd.woff, (double*)h->nd.Wcm, st);
    launch_transpose_blocks(h->nd.goff, h->nd.aoff, h->nd.woff, G, h->nd.Wcm, (double*)h->nd.Wrm, st);
    if (nsep > 0) {
        launch_nd_schur_sparse(h->nd.np, L, W.Sd, h->nd.goff, h->nd.aoff, h->nd.alist, sep0, h->nd.prow_g,
                               W.d_wc_ptr, W.d_wc_row, h->nd.woff, h->nd.Wrm, W.d_doff, W.D, st);
        const int64_t ct = (int64_t)W.cT * (W.cT + 1) / 2;
        launch_nd_schur_tiles<TI>(ct, L, nsep, sep0, W.Sd, h->nd.sg, h->nd.sidx, h->nd.aoff, W.d_doff, W.D,
                                  (TI*)W.cwork, st);
        CU(cudaMemcpyAsync(W.d_err, err_init, sizeof(err_init), cudaMemcpyHostToDevice, st));
        launch_dense_cholesky<TI>(1, std::vector<int32_t>{W.cT}, W.d_cnt, W.d_czero, W.d_czero, (TI*)W.cwork,
                                  (TI*)W.cdinv, W.d_err, st, (TI*)W.cplanes, h->d_kerr, W.tcs);
        CU(cudaGetLastError());
        TRY(read_err_flag(h, W.d_err, "interface (separator)"));
        if constexpr (std::is_same<TI, double>::value) {
            Profile cpf{W.d_crows, W.d_cnt, W.d_czero, W.d_czero, W.d_clo, W.d_chi, W.d_cfwd, W.d_cbwd};
            launch_finalize<TI, TI>(1, cpf, (const TI*)W.cwork, (const TI*)W.cdinv, (TI*)W.cf, (TI*)W.cb, st);
            SolveArgs ca{};
            ca.pf = cpf;
            ca.fwdS = W.cf;
            ca.bwdS = W.cb;
            ca.err = h->d_kerr;
            ca.in = W.cE;
            ca.out = (double*)h->nd.Cinv;
            ca.job_sub = W.d_cjob;
            ca.job_in = W.d_cjin;
            ca.job_out = W.d_cjin;
            ca.job_t0 = W.d_cjt0;   // lower triangle of C^{-1} only
            CU((launch_tile_solve<TI, TI>(ca, nsep, W.cT, st)));
        } else {
            for (const auto& r : W.cinv_ranges)
                launch_tile_inv(W.d_cinv_jobs + r.first, r.second, (const float*)W.cwork, (const float*)W.cdinv,
                                (float*)W.cf, (float*)W.cb, (double*)h->nd.Cinv, W.d_czero, W.d_czero, W.d_crows,
                                W.d_czerooff, st);
        }
        launch_mirror_lower(W.d_crowsq, W.d_czerooff, 1, (double*)h->nd.Cinv, st);
    }
    return 0;
}

// Numeric part of Algorithm 1 on the device: local blocks A_i and their factors, MBFs,
// interface system, its factor and explicit inverse.  Re-runnable for new values.
template <typename TW, typename TS, typename TA>
int numeric_setup(algmortar_t* h) {
    NumWs& W = *h->ws;
    TRY((numeric_prepare<TW, TS>(h, W)));
    Plan& P = h->P;
    cudaStream_t st = h->st;
    cudaEvent_t ev[8];
    for (auto& e : ev) cudaEventCreate(&e);
    cudaEventRecord(ev[0], st);
    const int m = h->m, L = h->L;
    const int64_t tiles = P.total_tiles, nphi = P.phi_off[m];
    TW* work = (TW*)W.work;
    TW* dinv = (TW*)W.dinv;
    // value-dependent interface tables (restriction coefficients, T_I, G entries)
    launch_iface_tables(L, (int64_t)P.r_cell.size(), h->d_rp_ptr, h->d_rp_pos, h->d_val, h->d_rptr, h->d_rcoef,
                        W.d_T ? W.d_T : h->d_scalar, (int64_t)P.g_val.size(), h->d_g_from_r, W.d_gval, st);
    // --- local factors (Algorithm 1: extract A_ii, modify its diagonal, factor) ---
    int err_init[2] = {0, -1};
    CU(cudaMemcpyAsync(W.d_err, err_init, sizeof(err_init), cudaMemcpyHostToDevice, st));
    CU(cudaMemsetAsync(work, 0, (size_t)tiles * TILE2 * sizeof(TW), st));
    launch_local_diag(h->n, h->d_rowptr, h->d_col, h->d_val, h->d_row_sub, h->opts.diag_scale, 1, h->d_dloc,
                      h->d_sc, h->d_sc32, st);
    launch_scatter_local<TW>(h->n, h->d_rowptr, h->d_col, h->d_val, h->d_row_sub, h->d_sub_off, h->pf, h->d_dloc,
                             h->d_sc, work, m, st);
    launch_tile_chol<TW>(m, h->pf, h->d_job_sub, work, dinv, W.d_err, h->tile_wm, st);
    CU(cudaGetLastError());
    TRY(read_err_flag(h, W.d_err, "local"));
    launch_finalize<TW, TS>(m, h->pf, work, dinv, (TS*)h->d_fwdS, (TS*)h->d_bwdS, st);
    CU(cudaGetLastError());
    if (h->opts.smooth_steps > 0) {
        // smoother blocks = the subdomains, unmodified A_ii (same sparsity, same profile)
        CU(cudaMemcpyAsync(W.d_err, err_init, sizeof(err_init), cudaMemcpyHostToDevice, st));
        CU(cudaMemsetAsync(work, 0, (size_t)tiles * TILE2 * sizeof(TW), st));
        launch_local_diag(h->n, h->d_rowptr, h->d_col, h->d_val, h->d_row_sub, h->opts.diag_scale, 0, h->d_dloc2,
                          h->d_sc2, h->d_sc2_32, st);
        launch_scatter_local<TW>(h->n, h->d_rowptr, h->d_col, h->d_val, h->d_row_sub, h->d_sub_off, h->pf,
                                 h->d_dloc2, h->d_sc2, work, m, st);
        launch_tile_chol<TW>(m, h->pf, h->d_job_sub, work, dinv, W.d_err, h->tile_wm, st);
        CU(cudaGetLastError());
        TRY(read_err_flag(h, W.d_err, "smoother block"));
        launch_finalize<TW, TS>(m, h->pf, work, dinv, (TS*)h->d_fwdS2, (TS*)h->d_bwdS2, st);
        CU(cudaGetLastError());
    }
    cudaEventRecord(ev[1], st);
    // --- MBFs (Eq. def-phat-local): Phi_i = A_i^{-1} (-B_i psi_m), one job per (i, m) ---
    const bool panel = W.w32 != nullptr && sizeof(TA) == 4;
    if (panel) {
        CU(cudaMemsetAsync(W.w32, 0, nphi * sizeof(float), st));
        launch_mbf_rhs32(m, W.d_goff, W.d_grow, W.d_gcol, W.d_gval, h->d_rows, h->d_phi_off, h->d_sc32, h->d_sub_off,
                         W.w32, st);
    } else {
        CU(cudaMemsetAsync(W.rhs, 0, nphi * sizeof(double), st));
        launch_mbf_rhs(m, W.d_goff, W.d_grow, W.d_gcol, W.d_gval, h->d_rows, h->d_phi_off, W.rhs, st);
    }
    {
        SolveArgs a{};
        a.pf = h->pf;
        a.fwdS = h->d_fwdS;
        a.bwdS = h->d_bwdS;
        a.scale = h->d_sc;
        a.scale32 = h->d_sc32;
        a.scale_off = h->d_sub_off;
        a.in = W.rhs;
        a.out = W.phi64;
        a.done = nullptr;
        a.err = h->d_kerr;
        if constexpr (sizeof(TA) == 4) {
            if (panel) {
                // all of a subdomain's MBF columns (up to PANEL_NC) against one pass of its factor
                SolveArgs b = a;
                b.job_sub = W.pj_mbf.sub;
                b.job_in = W.pj_mbf.in;
                b.job_out = W.pj_mbf.in;
                b.job_ld = W.pj_mbf.ld;
                b.job_nc = W.pj_mbf.nc;
                CU(launch_panel_solve<TS>(b, W.w32, W.pj_mbf.n, P.max_tiles, h->tile_wm, st));
            }
        }
        if (!panel) TRY((solve_cols<TS, TA>(a, W.bj_mbf, false, P.max_tiles, st)));
    }
    launch_panel_rows<PanelT<TS>>(h->nchunks, h->d_chunks, h->d_chunk_sub, h->d_sub_off, h->d_phi_off, W.phi64,
                                  (PanelT<TS>*)h->d_phi, st);
    cudaEventRecord(ev[2], st);
    // --- interface system S_eta = diag(T) + 1/4 G^T Phi (Eq. interface-problem-alg),
    //     solved exactly by one level of nested dissection (kernels_coarse.cu) ---
    if (L > 0 && h->inexact) {
        // S_eta in CSR (the same values as the exact path's dense matrix) and the explicit
        // FP64 inverses of the block-Jacobi blocks, stored in FP32
        NdAssembleArgs ia{};
        ia.rows = h->d_rows;
        ia.if_off = h->d_if_off;
        ia.if_list = h->d_if_list;
        ia.phi_off = h->d_phi_off;
        ia.phi = W.phi64;
        ia.g_cptr = W.d_gcptr;
        ia.g_row = W.d_grow;
        ia.g_val = W.d_gval;
        ia.pairs = W.d_pairs;
        ia.pv = W.pv;
        ia.pv_off = W.d_pv_off;
        ia.diagc = W.diagc;
        ia.L = L;
        launch_nd_assemble(m, ia, st);
        launch_iface_csr_values(L, h->iface.s_ptr, h->iface.s_col, W.d_csr_src, W.pv, W.d_T, W.diagc, W.s_val64,
                                (float2*)h->iface.s_ent, st);
        cudaEventRecord(ev[3], st);
        CU(cudaMemcpyAsync(W.d_err, err_init, sizeof(err_init), cudaMemcpyHostToDevice, st));
        CU(launch_iface_block_inv(h->iface_nblk, h->iface_max_nb, h->iface.blk_row0, h->iface.blk_off,
                                  h->iface.s_ptr, h->iface.s_col, W.s_val64, (float*)h->iface.binv, W.d_err, st));
        TRY(read_err_flag(h, W.d_err, "interface (block-Jacobi block)"));
        cudaEventRecord(ev[5], st);
    } else if (L > 0) {
        const int G = P.nd_G, nsep = P.nd_nsep;
        const int64_t sep0 = P.nd_goff[G];
        CU(cudaMemsetAsync(W.Sd, 0, (size_t)L * L * sizeof(double), st));
        NdAssembleArgs ia{};
        ia.rows = h->d_rows;
        ia.if_off = h->d_if_off;
        ia.if_list = h->d_if_list;
        ia.phi_off = h->d_phi_off;
        ia.phi = W.phi64;
        ia.g_cptr = W.d_gcptr;
        ia.g_row = W.d_grow;
        ia.g_val = W.d_gval;
        ia.pairs = W.d_pairs;
        ia.nd_pos = h->d_ndpos;
        ia.Sd = W.Sd;
        ia.diagc = W.diagc;
        ia.L = L;
        launch_nd_assemble(m, ia, st);
        launch_nd_diag(L, W.d_T, W.diagc, h->d_ndpos, W.Sd, st);
        cudaEventRecord(ev[3], st);
        if (h->opts.precision == ALGMORTAR_FP64) TRY(nd_factor_inverse<double>(h, W, st));
        else TRY(nd_factor_inverse<float>(h, W, st));
        if (h->nd.Ginv32) {   // FP32 copies, padded rows (see NdSolveArgs)
            for (int g = 0; g < G; ++g) {
                const int64_t ng = P.nd_goff[g + 1] - P.nd_goff[g], ag = P.nd_aoff[g + 1] - P.nd_aoff[g];
                const int64_t ng4 = (ng + 3) & ~int64_t(3);
                launch_pad_convert(ng, ng, h->nd.Ginv + W.h_gioff[g], ng, (float*)h->nd.Ginv32 + W.h_gioff32[g], ng4,
                                   st);
                launch_pad_convert(ag, ng, h->nd.Wcm + W.h_woff[g], ng, (float*)h->nd.Wcm32 + W.h_woff32[g], ng4, st);
            }
            launch_convert<float>(W.n_w, h->nd.Wrm, (float*)h->nd.Wrm32, st);
        }
        if (h->nd.Cinv32) launch_pad_convert(nsep, nsep, h->nd.Cinv, nsep, (float*)h->nd.Cinv32, h->nd.nsep4, st);
        CU(cudaGetLastError());
        cudaEventRecord(ev[5], st);
    } else {
        cudaEventRecord(ev[3], st);
        cudaEventRecord(ev[5], st);
    }
    cudaEventRecord(ev[4], st);
    CU(cudaStreamSynchronize(st));
    int kerr = 0;
    CU(cudaMemcpy(&kerr, h->d_kerr, sizeof(int), cudaMemcpyDeviceToHost));
    if (kerr) return fail(ALGMORTAR_CUDA, "a bulk copy of the triangular solves did not complete");
    float t01, t12, t23, t34, t35;
    cudaEventElapsedTime(&t01, ev[0], ev[1]);
    cudaEventElapsedTime(&t12, ev[1], ev[2]);
    cudaEventElapsedTime(&t23, ev[2], ev[3]);
    cudaEventElapsedTime(&t34, ev[3], ev[4]);
    cudaEventElapsedTime(&t35, ev[3], ev[5]);
    h->info.setup_ms[2] = t01;
    h->info.setup_ms[3] = t12;
    h->info.setup_ms[4] = t23;
    h->info.setup_ms[5] = t34;
    h->info.setup_ms[6] = t35;
    for (auto& e : ev) cudaEventDestroy(e);
    return 0;
}

int numeric_dispatch(algmortar_t* h) {
    switch (h->opts.precision) {
        case ALGMORTAR_FP64: return numeric_setup<double, double, double>(h);
        case ALGMORTAR_FP32: return numeric_setup<float, float, float>(h);
        case ALGMORTAR_BF16: return numeric_setup<float, __nv_bfloat16, float>(h);
        default: return fail(ALGMORTAR_INVALID_ARG, "unknown precision");
    }
}

// Column strides of a batch; `pcg` makes the kernels skip columns whose PCG has stopped.
ColStrides col_strides(const algmortar_t* h, const Vecs& v, bool pcg) {
    ColStrides cs{};
    cs.v = h->n;
    cs.l = h->L > 0 ? h->L : 1;
    cs.done = pcg ? &v.sc->done : nullptr;
    cs.done_stride = (int)(sizeof(PcgScalars) / sizeof(int32_t));
    cs.sc_stride = (int)(sizeof(PcgScalars) / sizeof(double));
    return cs;
}

// Stages of Algorithm 2 on internal-order vectors, all columns of the batch per launch.
// Local particular solutions pbar_i = A_i^{-1} r_i for all subdomains (one launch).
// With `smoother`, the same batched solve with the block-Jacobi factors of the
// unmodified A_ii into `out` (accumulating when asked): out (+)= B^{-1} r.
template <typename TS, typename TA>
int stage_local(algmortar_t* h, Vecs& v, const double* r, const ColStrides& cs, bool smoother = false,
                double* out = nullptr, bool accumulate = false) {
    SolveArgs a{};
    a.pf = h->pf;
    a.fwdS = smoother ? h->d_fwdS2 : h->d_fwdS;
    a.bwdS = smoother ? h->d_bwdS2 : h->d_bwdS;
    a.scale = smoother ? h->d_sc2 : h->d_sc;
    a.scale32 = smoother ? h->d_sc2_32 : h->d_sc32;
    a.scale_off = h->d_sub_off;
    a.job_sub = h->d_job_sub;
    a.job_in = h->d_job_off;
    a.job_out = h->d_job_off;
    a.in = r;
    a.out = out ? out : v.pbar;
    a.accumulate = accumulate ? 1 : 0;
    a.done = cs.done;
    a.done_stride = cs.done_stride;
    a.ldin = a.ldout = h->n;
    a.deep_ring = h->tuned_ring;
    a.err = h->d_kerr;
    if (v.k > 1) {
        if constexpr (sizeof(TA) == 4) {
            if (v.w32) {
                // batched FP32 / BF16 columns: one job per (subdomain, block of PANEL_NC
                // columns), the factor streamed once per block
                a.job_sub = v.pj.sub;
                a.job_in = v.pj.in;
                a.job_out = v.pj.in;
                a.job_ld = v.pj.ld;
                a.job_nc = v.pj.nc;
                a.job_col0 = v.pj_col0;
                CU(launch_panel_solve_cols<TS>(a, v.w32, v.pj.n, h->P.max_tiles, h->tile_wm, h->st));
                return 0;
            }
        }
        // batched columns: one job per (subdomain, block of COLS_PER_JOB columns), each
        // factor tile read once per block
        a.job_col0 = v.bj_col0;
        return solve_cols<TS, TA>(a, v.bj, false, h->P.max_tiles, h->st);
    }
    CU((launch_tile_solve<TS, TA>(a, h->m, h->P.max_tiles, h->st, v.k)));
    return 0;
}

// Stage boundary i of one PCG iteration (opts.stage_times): a stream-ordered event; the
// solve does not replay the iteration graph while stage times are requested.
int mark(algmortar_t* h, Vecs& v, int i) {
    if (!v.sev_ok) return 0;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CU(cudaStreamIsCapturing(h->st, &cs));
    if (cs != cudaStreamCaptureStatusNone) return 0;   // graph capture: no stage events
    CU(cudaEventRecord(v.sev[i], h->st));
    return 0;
}

// Interface right-hand side and interface solve: b_eta from pbar, eta = S^{-1} b_eta.
void stage_restrict(algmortar_t* h, Vecs& v, const ColStrides& cs) {
    // the FP32 interface solve reads an FP32 copy of b_eta, written here with it
    const bool f32 = !h->inexact && h->nd.Ginv32;
    launch_restrict(h->L, h->d_rptr, h->d_rcell, h->d_rcoef, v.pbar, v.beta, h->d_ndpos, cs, v.k,
                    f32 ? v.f32 : nullptr, v.fl, h->nd.p32, h->st);
}
int stage_coarse(algmortar_t* h, Vecs& v, const ColStrides& cs) {
    if (h->L <= 0) return 0;
    if (h->inexact) {
        IfaceArgs a = h->iface;
        a.its = v.iits;
        a.its_total = v.iits_total;
        CU(launch_iface_pcg(a, h->iface_cluster, h->iface_smem, v.beta, v.eta, cs, v.k, h->st));
    } else {
        launch_nd_solve(h->nd, v.beta, v.eta, v.P, v.f32, v.fl, true, cs, v.k, h->st);
    }
    return 0;
}

// z = base + pbar + Phi eta (base may be null); inside PCG (sc given) also r . z and the
// next beta per column.
template <typename TS>
void stage_prolong(algmortar_t* h, Vecs& v, const double* r, double* z, const ColStrides& cs, PcgScalars* sc,
                   const double* base = nullptr) {
    launch_prolong<TS>(h->nchunks, h->d_chunks, h->L > 0 ? h->d_ifpos : h->d_if_list, (const TS*)h->d_phi, v.eta,
                       v.pbar, base, z, r, v.gs, sc, cs, v.k, h->st);
}

template <typename TS, typename TA>
int apply_t(algmortar_t* h, Vecs& v, const double* r, double* z, bool pcg) {
    const ColStrides cs = col_strides(h, v, pcg);
    const int nu = h->opts.smooth_steps;
    if (nu <= 0) {
        TRY((stage_local<TS, TA>(h, v, r, cs)));
        if (pcg) TRY(mark(h, v, 4));
        stage_restrict(h, v, cs);
        if (pcg) TRY(mark(h, v, 5));
        TRY(stage_coarse(h, v, cs));
        if (pcg) TRY(mark(h, v, 6));
        stage_prolong<PanelT<TS>>(h, v, r, z, cs, pcg ? v.sc : nullptr);
        CU(cudaGetLastError());
        return 0;
    }
    // Sec. 5.4: nu block-Jacobi steps, the AlgMortar correction, nu block-Jacobi steps,
    // composed multiplicatively on x (= z): x = B^{-1} r first, then x += B^{-1} (r - A x)
    const int64_t n = h->n;
    auto resid = [&]() {
        launch_smooth_residual(n, v.k, h->d_ell_ptr, h->d_ell_col, h->d_ell_val, z, r, v.w, cs, h->st);
    };
    TRY((stage_local<TS, TA>(h, v, r, cs, true, z, false)));
    for (int k = 1; k < nu; ++k) {
        resid();
        TRY((stage_local<TS, TA>(h, v, v.w, cs, true, z, true)));
    }
    resid();
    TRY((stage_local<TS, TA>(h, v, v.w, cs)));
    stage_restrict(h, v, cs);
    TRY(stage_coarse(h, v, cs));
    stage_prolong<PanelT<TS>>(h, v, nullptr, z, cs, nullptr, z);
    for (int k = 0; k < nu; ++k) {
        resid();
        TRY((stage_local<TS, TA>(h, v, v.w, cs, true, z, true)));
    }
    if (pcg) launch_pcg_rho(n, v.k, r, z, v.sc, v.gs, cs, h->st);
    CU(cudaGetLastError());
    return 0;
}

// z = M^{-1} r for the batch's columns; with `pcg`, stopped columns are skipped and
// r . z goes to each column's rz_next.
int apply_internal(algmortar_t* h, Vecs& v, const double* r, double* z, bool pcg) {
    switch (h->opts.precision) {
        case ALGMORTAR_FP64: return apply_t<double, double>(h, v, r, z, pcg);
        case ALGMORTAR_FP32: return apply_t<float, float>(h, v, r, z, pcg);
        default: return apply_t<__nv_bfloat16, float>(h, v, r, z, pcg);
    }
}

int pcg_iteration(algmortar_t* h, Vecs& v) {
    cudaStream_t st = h->st;
    const int64_t n = h->n;
    set_hot_ctas_per_sm(h->tuned_vec_ctas);
    TRY(mark(h, v, 0));
    launch_pcg_p(n, v.k, n, v.z, v.p, v.sc, st);
    TRY(mark(h, v, 1));
    launch_pcg_spmv_ell(n, v.k, n, h->d_ell_ptr, h->d_ell_col, h->d_ell_val, v.p, v.q, v.sc, v.gs, h->ell_wf, st);
    TRY(mark(h, v, 2));
    launch_pcg_xr(n, v.k, n, v.x, v.r, v.p, v.q, v.z, v.sc, v.gs, v.hist, v.hist_len, st);
    TRY(mark(h, v, 3));
    TRY(apply_internal(h, v, v.r, v.z, true));
    return mark(h, v, 7);
}

// The FP32 interface inverses are re-read every iteration, while the local solves stream
// ~0.5 GB of factor tiles between two reads and would evict them: where the device offers
// persisting L2 lines, the iteration graph's kernels carry an access-policy window over
// the interface block (hit ratio = the persisting set-aside / the window), so the three
// interface stages read L2.  The set-aside belongs to this process's context; it is only
// ever raised.  A hint: failures are ignored.
void set_l2_window(algmortar_t* h, cudaGraph_t g) {
    if (!h->ifw32 || h->ifw32_bytes == 0) return;
    if (h->l2w.num_bytes == 0) {
        int maxp = 0, maxw = 0;
        if (cudaDeviceGetAttribute(&maxp, cudaDevAttrMaxPersistingL2CacheSize, h->device) != cudaSuccess ||
            cudaDeviceGetAttribute(&maxw, cudaDevAttrMaxAccessPolicyWindowSize, h->device) != cudaSuccess ||
            maxp <= 0 || maxw <= 0) {
            cudaGetLastError();
            return;
        }
        const size_t win = std::min(h->ifw32_bytes, (size_t)maxw);
        size_t lim = 0;
        if (cudaDeviceGetLimit(&lim, cudaLimitPersistingL2CacheSize) != cudaSuccess) lim = 0;
        const size_t want = std::min(win, (size_t)maxp);
        if (lim < want && cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want) == cudaSuccess) lim = want;
        cudaGetLastError();
        if (lim == 0) return;
        h->l2w.base_ptr = h->ifw32;
        h->l2w.num_bytes = win;
        h->l2w.hitRatio = (float)std::min(1.0, (double)lim / (double)win);
        h->l2w.hitProp = cudaAccessPropertyPersisting;
        h->l2w.missProp = cudaAccessPropertyStreaming;
    }
    size_t nn = 0;
    if (cudaGraphGetNodes(g, nullptr, &nn) != cudaSuccess || nn == 0) {
        cudaGetLastError();
        return;
    }
    std::vector<cudaGraphNode_t> nodes(nn);
    if (cudaGraphGetNodes(g, nodes.data(), &nn) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    cudaKernelNodeAttrValue av{};
    av.accessPolicyWindow = h->l2w;
    for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel)
            cudaGraphKernelNodeSetAttribute(nd, cudaKernelNodeAttributeAccessPolicyWindow, &av);
    }
    cudaGetLastError();
}

int ensure_graph(algmortar_t* h, Vecs& v) {
    if (v.graph && v.graph_k == v.k) return 0;
    if (v.graph) {
        cudaGraphExecDestroy(v.graph);
        v.graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    CU(cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal));
    const int64_t c0 = launch_count();
    int rc = pcg_iteration(h, v);
    cudaError_t e = cudaStreamEndCapture(h->st, &g);
    v.graph_kernels = launch_count() - c0;
    add_launches(-v.graph_kernels);   // captured, not executed
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(ALGMORTAR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    set_l2_window(h, g);
    e = cudaGraphInstantiate(&v.graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        v.graph = nullptr;
        return fail(ALGMORTAR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    v.graph_k = v.k;
    return 0;
}

// Workspace of a batch with room for `cap` columns (first use, or growth).
int alloc_vecs(algmortar_t* h, Vecs& v, int cap) {
    if (v.cap >= cap) return 0;
    void* old[] = {v.x,         v.r,    v.z,    v.p,          v.q,    v.pbar, v.b,  v.t,
                   v.w,         v.beta, v.eta,  v.P,          v.sc,   v.gs.part,    v.gs.ticket,
                   v.iits,      v.iits_total,   v.hist,       v.f32};
    for (void* p : old)
        if (p) h->release(p);
    if (v.graph) {
        cudaGraphExecDestroy(v.graph);
        v.graph = nullptr;
    }
    const size_t n = (size_t)h->n * cap;
    const size_t l = (size_t)std::max(h->L, 1) * cap;
    const int64_t np = h->P.nd_aoff.empty() ? 1 : std::max<int64_t>(h->P.nd_aoff.back(), 1);
    // grid-sum partials: two per CTA (flexible beta) of the widest grid (vector kernels or
    // the prolongation's warp-per-chunk grid)
    const size_t nb = 2 * (size_t)std::max(vec_blocks(h->n), prolong_blocks(h->nchunks)) * cap;
    v.x = h->alloc<double>(n);
    v.r = h->alloc<double>(n);
    v.z = h->alloc<double>(n);
    v.p = h->alloc<double>(n);
    v.q = h->alloc<double>(n);
    v.pbar = h->alloc<double>(n);
    v.b = h->alloc<double>(n);
    v.t = h->alloc<double>(n);
    v.w = h->opts.smooth_steps > 0 ? h->alloc<double>(n) : nullptr;
    v.beta = h->alloc<double>(l);
    v.eta = h->alloc<double>(l);
    v.P = h->alloc<double>((size_t)np * cap);
    v.sc = h->alloc<PcgScalars>(cap);
    v.gs.part = h->alloc<double>(nb);
    v.gs.ticket = h->alloc<unsigned int>(cap);
    {   // FP32 side vectors of the interface solve: padded b (groups, separator), c, separator eta
        int64_t l32 = 0;
        const Plan& Q = h->P;
        for (size_t g = 0; g + 1 < Q.nd_goff.size(); ++g) l32 += (Q.nd_goff[g + 1] - Q.nd_goff[g] + 3) & ~int64_t(3);
        const int64_t ns4 = (Q.nd_nsep + 3) & ~3;
        v.fl = ((std::max<int64_t>(l32 + ns4, 1) + ns4 + Q.nd_nsep + 3) / 4) * 4;
    }
    v.f32 = h->alloc<float>((size_t)v.fl * cap);
    v.iits = h->alloc<int32_t>(cap);
    v.iits_total = h->alloc<int64_t>(cap);
    // ||r_k||^2 of every iteration (k <= max_it) per column, written by the stop test
    v.hist_len = std::max(h->opts.max_it, 1) + 1;
    v.hist = h->alloc<double>((size_t)v.hist_len * cap);
    if (!v.x || !v.r || !v.z || !v.p || !v.q || !v.pbar || !v.b || !v.t || (h->opts.smooth_steps > 0 && !v.w) ||
        !v.beta || !v.eta || !v.P || !v.sc || !v.gs.part || !v.gs.ticket || !v.iits || !v.iits_total || !v.hist ||
        !v.f32) {
        v.cap = 0;
        return fail(ALGMORTAR_OOM, "vector workspace");
    }
    CU(cudaMemsetAsync(v.p, 0, n * sizeof(double), h->st));
    CU(cudaMemsetAsync(v.sc, 0, cap * sizeof(PcgScalars), h->st));
    CU(cudaMemsetAsync(v.gs.ticket, 0, cap * sizeof(unsigned int), h->st));
    CU(cudaMemsetAsync(v.iits, 0, cap * sizeof(int32_t), h->st));
    CU(cudaMemsetAsync(v.f32, 0, (size_t)v.fl * cap * sizeof(float), h->st));   // padding stays zero
    CU(cudaMemsetAsync(v.iits_total, 0, cap * sizeof(int64_t), h->st));
    if (h->opts.stage_times && !v.sev_ok) {
        for (cudaEvent_t& e : v.sev) CU(cudaEventCreate(&e));
        v.sev_ok = true;
    }
    v.cap = cap;
    v.k = cap;
    return 0;
}

// Column-block jobs for a batch of k > 1 columns: per subdomain (largest first) blocks of
// COLS_PER_JOB consecutive columns at stride n.
int ensure_batch_jobs(algmortar_t* h, Vecs& v) {
    if (v.k <= 1 || v.bj_k == v.k) return 0;
    std::vector<int32_t> rows(h->m), order(h->m);
    for (int s = 0; s < h->m; ++s) {
        rows[s] = (int32_t)(h->P.sub_off[s + 1] - h->P.sub_off[s]);
        order[s] = s;
    }
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return rows[x] > rows[y]; });
    BlockJobs b;
    std::vector<int32_t> col0;
    for (int s : order) {
        const size_t before = b.sub.size();
        b.add(s, h->P.sub_off[s], h->n, v.k, false);
        for (size_t j = before; j < b.sub.size(); ++j) col0.push_back((int32_t)((j - before) * COLS_PER_JOB));
    }
    void* old[] = {v.bj.sub, v.bj.nc, v.bj.t0, v.bj.in, v.bj.ld, v.bj_col0,
                   v.pj.sub, v.pj.nc, v.pj.t0, v.pj.in, v.pj.ld, v.pj_col0, v.w32};
    for (void* p : old)
        if (p) h->release(p);
    v.pj = DevBlockJobs{};
    v.pj_col0 = nullptr;
    v.w32 = nullptr;
    TRY(upload_jobs(h, v.bj, b));
    TRY(upload(h, v.bj_col0, col0));
    if (h->opts.precision != ALGMORTAR_FP64 && panel_solve_fits(h->tile_wm, h->P.max_tiles, h->opts.precision ==
                                                                                  ALGMORTAR_FP32 ? 4 : 2)) {
        // PANEL_NC columns per job, subdomains with the longest tile chains first
        std::vector<int32_t> ord(h->m);
        for (int s = 0; s < h->m; ++s) ord[s] = s;
        std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return h->P.ntiles[x] > h->P.ntiles[y]; });
        BlockJobs pb;
        std::vector<int32_t> pc0;
        for (int s : ord)
            for (int c = 0; c < v.k; c += PANEL_NC) {
                pb.sub.push_back(s);
                pb.in.push_back(h->P.sub_off[s] + (int64_t)c * h->n);
                pb.ld.push_back(h->n);
                pb.nc.push_back(std::min(PANEL_NC, v.k - c));
                pb.t0.push_back(0);
                pc0.push_back(c);
            }
        TRY(upload_jobs(h, v.pj, pb));
        TRY(upload(h, v.pj_col0, pc0));
        v.w32 = h->alloc<float>((size_t)h->n * v.k);
        if (!v.w32) return fail(ALGMORTAR_OOM, "panel solve scratch");
    }
    v.bj_k = v.k;
    return 0;
}

// PCG in the internal ordering on v.b -> v.x for the batch's k columns; stats[j] per column.
// Returns the worst column status.
int pcg_internal(algmortar_t* h, Vecs& v, double tol, algmortar_stats* stt) {
    cudaStream_t st = h->st;
    double t0 = now_ms();
    if (!(tol > 0.0)) return fail(ALGMORTAR_INVALID_ARG, "tol must be positive");
    const int k = v.k;
    const int64_t n = h->n;
    TRY(ensure_batch_jobs(h, v));
    // stage timing brackets the kernels with stream-ordered events: no graph replay then
    // (event nodes inside an instantiated graph do not mark its kernels' boundaries)
    const bool graph = h->opts.use_graph && !h->opts.stage_times;
    if (graph) TRY(ensure_graph(h, v));
    // the inexact interface solve makes M^{-1} non-linear: always the flexible beta then
    const int flex = (h->opts.flexible || h->inexact) ? 1 : 0;
    CU(cudaMemsetAsync(v.iits_total, 0, k * sizeof(int64_t), st));
    launch_pcg_init(n, k, n, v.b, v.x, v.r, v.sc, v.gs, tol, h->opts.max_it, flex, v.hist, v.hist_len, st);
    TRY(apply_internal(h, v, v.r, v.z, true));
    std::vector<PcgScalars> hs(k);
    std::vector<int> restarts(k, 0);
    std::vector<double> true_rel(k, 0.0);
    std::vector<char> fin(k, 0);
    const int every = h->opts.check_every > 0 ? h->opts.check_every : 1;
    static const int zero = 0;
    for (;;) {
        for (int c = 0; c < every; ++c) {
            if (graph && v.graph) {
                CU(cudaGraphLaunch(v.graph, st));
                add_launches(v.graph_kernels);
            } else {
                TRY(pcg_iteration(h, v));
            }
        }
        CU(cudaMemcpyAsync(hs.data(), v.sc, k * sizeof(PcgScalars), cudaMemcpyDeviceToHost, st));
        CU(cudaStreamSynchronize(st));
        bool all = true;
        for (int j = 0; j < k; ++j) all = all && hs[j].done;
        if (!all) continue;
        launch_residual(n, k, n, h->d_rowptr, h->d_col, h->d_val, v.x, v.b, v.sc, v.gs, st);
        CU(cudaMemcpyAsync(hs.data(), v.sc, k * sizeof(PcgScalars), cudaMemcpyDeviceToHost, st));
        CU(cudaStreamSynchronize(st));
        bool again = false;
        for (int j = 0; j < k; ++j) {
            if (fin[j]) continue;
            true_rel[j] = hs[j].bb > 0 ? std::sqrt(hs[j].res2 / hs[j].bb) : 0.0;
            if (hs[j].status == 0 && hs[j].bb > 0 && !(true_rel[j] <= tol) && restarts[j] < 8 &&
                hs[j].iter < hs[j].max_it) {
                // the recurrence converged but the true residual does not confirm it:
                // replace r by b - A x and restart the directions (below)
                ++restarts[j];
                CU(cudaMemcpyAsync(&v.sc[j].done, &zero, sizeof(int), cudaMemcpyHostToDevice, st));
                again = true;
            } else {
                fin[j] = 1;
            }
        }
        if (!again) break;
        launch_pcg_replace(n, k, n, h->d_rowptr, h->d_col, h->d_val, v.x, v.b, v.r, v.sc, v.gs, st);
        TRY(apply_internal(h, v, v.r, v.z, true));
        CU(cudaStreamSynchronize(st));
    }
    std::vector<int64_t> iits(k, 0);
    CU(cudaMemcpyAsync(iits.data(), v.iits_total, k * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    float sms[7] = {0, 0, 0, 0, 0, 0, 0};
    if (v.sev_ok && h->opts.stage_times) {
        CU(cudaStreamSynchronize(st));
        for (int i = 0; i < 7; ++i)
            if (cudaEventElapsedTime(&sms[i], v.sev[i], v.sev[i + 1]) != cudaSuccess) sms[i] = 0.0f;
        cudaGetLastError();
    }
    int worst = ALGMORTAR_OK;
    for (int j = 0; j < k; ++j) {
        const PcgScalars& s = hs[j];
        if (stt) {
            stt[j].iface_iterations = iits[j];
            const double st_ms[6] = {sms[1], (double)sms[0] + sms[2], sms[3], sms[4], sms[5], sms[6]};
            for (int i = 0; i < 6; ++i) stt[j].stage_ms[i] = v.sev_ok && h->opts.stage_times ? st_ms[i] : 0.0;
            stt[j].history_count = 0;
            if (stt[j].history && stt[j].history_len > 0) {
                const int cnt = std::min(std::min(stt[j].history_len, s.iter + 1), v.hist_len);
                std::vector<double> hb(cnt);
                CU(cudaMemcpy(hb.data(), v.hist + (size_t)j * v.hist_len, cnt * sizeof(double),
                              cudaMemcpyDeviceToHost));
                for (int i = 0; i < cnt; ++i) stt[j].history[i] = s.bb > 0 ? std::sqrt(hb[i] / s.bb) : 0.0;
                stt[j].history_count = cnt;
            }
        }
        int status = s.status == 0 ? (true_rel[j] <= tol || s.bb == 0 ? ALGMORTAR_OK : ALGMORTAR_NO_CONVERGENCE)
                                   : (s.status == 5 ? ALGMORTAR_NO_CONVERGENCE : ALGMORTAR_BREAKDOWN);
        if (stt) {
            stt[j].status = status;
            stt[j].iterations = s.iter;
            stt[j].rel_residual = true_rel[j];
            stt[j].recursive_residual = s.bb > 0 ? std::sqrt(s.rr / s.bb) : 0.0;
            stt[j].solve_ms = now_ms() - t0;
            stt[j].host_ms = 0.0;
        }
        if (status == ALGMORTAR_BREAKDOWN || (status == ALGMORTAR_NO_CONVERGENCE && worst == ALGMORTAR_OK))
            worst = status;
    }
    if (worst == ALGMORTAR_NO_CONVERGENCE) g_err = "PCG reached max_it or the true residual did not confirm";
    if (worst == ALGMORTAR_BREAKDOWN) g_err = "PCG breakdown: p^T A p <= 0 or non-finite scalar";
    return worst;
}

// SplitMix64 (Steele, Lea & Flood 2014): the state advanced by the golden gamma, then the
// published finaliser.
uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Uneven target sizes of the partition (see algmortar_part_sizes).
int uneven_part_sizes(int64_t n, int32_t m, uint64_t seed, int32_t* out, std::string& err) {
    if (m < 1 || n < m) {
        err = "part sizes: need 1 <= m <= n";
        return ALGMORTAR_INVALID_ARG;
    }
    const uint64_t K = 1ull << 20;
    const unsigned __int128 lo = (unsigned __int128)(3 * n / (10 * (int64_t)m)), hi = (unsigned __int128)(3 * n / m);
    std::vector<unsigned __int128> C(m);
    unsigned __int128 acc = 0;
    for (int32_t j = 0; j < m; ++j) {
        const uint64_t a = splitmix64((seed << 32) ^ (uint64_t)(2 * (int64_t)j)) % K;
        const uint64_t b = splitmix64((seed << 32) ^ (uint64_t)(2 * (int64_t)j + 1)) % K;
        acc += lo * K * K + (hi - lo) * a * b;
        C[j] = acc;
    }
    if (acc == 0) {
        err = "part sizes: zero total weight";
        return ALGMORTAR_INVALID_ARG;
    }
    int64_t prev = 0;
    for (int32_t j = 0; j < m; ++j) {
        const int64_t cut = (int64_t)(((unsigned __int128)n * C[j]) / acc);
        if (cut - prev <= 0) {
            err = "part sizes: a part would be empty";
            return ALGMORTAR_INVALID_ARG;
        }
        out[j] = (int32_t)(cut - prev);
        prev = cut;
    }
    return 0;
}

// ------------------------------------------------------------------ autotuner
// Launch variants of the hot kernels, measured on the handle's own data with CUDA events:
// the batched local triangular solves (5 ring / warp shapes x 3 job orders) and the CTAs
// per SM of the PCG vector kernels.  Every local-solve variant must reproduce the default
// variant's output to rounding (else ALGMORTAR_CUDA); the choice is cached per process by
// precision and factor-profile shape, so later setups of the same shape skip the search.
struct TuneVal {
    int ring, order, vec_ctas;
};
std::mutex g_tune_mu;
std::map<std::vector<int64_t>, TuneVal> g_tune_cache;

std::vector<int64_t> tune_key(const algmortar_t* h) {
    const Plan& P = h->P;
    std::vector<int64_t> key{h->opts.precision, h->n, h->m, P.total_tiles, P.max_tiles, h->device};
    // histogram of tile rows per subdomain in buckets of 4
    std::map<int, int64_t> hist;
    for (int s = 0; s < h->m; ++s) hist[P.ntiles[s] / 4] += 1;
    for (auto& kv : hist) {
        key.push_back(kv.first);
        key.push_back(kv.second);
    }
    return key;
}

template <typename F>
int time_ms(algmortar_t* h, int reps, F&& body, float* out) {
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    for (int i = 0; i < 2; ++i) TRY(body());
    std::vector<float> t;
    for (int i = 0; i < reps; ++i) {
        CU(cudaEventRecord(e0, h->st));
        TRY(body());
        CU(cudaEventRecord(e1, h->st));
        CU(cudaEventSynchronize(e1));
        float ms = 0.0f;
        CU(cudaEventElapsedTime(&ms, e0, e1));
        t.push_back(ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::sort(t.begin(), t.end());
    *out = t[t.size() / 2];
    return 0;
}

int autotune(algmortar_t* h) {
    CU(cudaSetDevice(h->device));
    const std::vector<int64_t> key = tune_key(h);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            h->tuned_ring = it->second.ring;
            h->tuned_order = it->second.order;
            h->tuned_vec_ctas = it->second.vec_ctas;
            h->d_job_sub = h->d_job_sub_v[h->tuned_order];
            h->d_job_off = h->d_job_off_v[h->tuned_order];
            return 0;
        }
    }
    Vecs& v = h->v1;
    const int64_t n = h->n;
    const ColStrides cs = col_strides(h, v, false);
    // a fixed, finite right-hand side (SplitMix64 values in [-1, 1))
    std::vector<double> rhs(n);
    for (int64_t i = 0; i < n; ++i) rhs[i] = (double)(splitmix64(0xA1u + (uint64_t)i) >> 11) * 0x1.0p-52 - 1.0;
    CU(cudaMemcpyAsync(v.t, rhs.data(), n * sizeof(double), cudaMemcpyHostToDevice, h->st));
    auto local = [&]() -> int {
        switch (h->opts.precision) {
            case ALGMORTAR_FP64: return stage_local<double, double>(h, v, v.t, cs);
            case ALGMORTAR_FP32: return stage_local<float, float>(h, v, v.t, cs);
            default: return stage_local<__nv_bfloat16, float>(h, v, v.t, cs);
        }
    };
    std::vector<double> ref(n), out(n);
    const double tol = h->opts.precision == ALGMORTAR_FP64 ? 1e-12 : 1e-5;
    int best_ring = 0, best_order = 0;
    float best = 3.4e38f;
    for (int order = 0; order < 3; ++order)
        for (int ring = 0; ring < 5; ++ring) {
            h->tuned_ring = ring;
            h->d_job_sub = h->d_job_sub_v[order];
            h->d_job_off = h->d_job_off_v[order];
            float ms = 0.0f;
            TRY(time_ms(h, 7, local, &ms));
            CU(cudaMemcpyAsync(ring == 0 && order == 0 ? ref.data() : out.data(), v.pbar, n * sizeof(double),
                               cudaMemcpyDeviceToHost, h->st));
            CU(cudaStreamSynchronize(h->st));
            if (ring || order) {
                double dmax = 0.0, rmax = 0.0;
                for (int64_t i = 0; i < n; ++i) {
                    dmax = std::max(dmax, std::fabs(out[i] - ref[i]));
                    rmax = std::max(rmax, std::fabs(ref[i]));
                }
                if (!(dmax <= tol * rmax))
                    return fail(ALGMORTAR_CUDA, "autotune: launch variant " + std::to_string(ring) + "/" +
                                                    std::to_string(order) + " disagrees with the default");
            }
            if (ms < best) {
                best = ms;
                best_ring = ring;
                best_order = order;
            }
        }
    h->tuned_ring = best_ring;
    h->tuned_order = best_order;
    h->d_job_sub = h->d_job_sub_v[best_order];
    h->d_job_off = h->d_job_off_v[best_order];
    // PCG vector kernels on finite vectors with a live scalar state
    PcgScalars live{};
    live.rz = live.rz_next = 1.0;
    live.beta = 0.5;
    live.iter = 1;
    live.max_it = 1 << 30;
    live.step_ok = 1;
    for (double* dst : {v.x, v.r, v.p, v.q, v.z})
        CU(cudaMemcpyAsync(dst, v.t, n * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    int best_c = h->tuned_vec_ctas;
    float best_v = 3.4e38f;
    for (int c : {2, 3, 4, 6, 8}) {
        set_hot_ctas_per_sm(c);
        auto vec = [&]() -> int {
            CU(cudaMemcpyAsync(v.sc, &live, sizeof(live), cudaMemcpyHostToDevice, h->st));
            launch_pcg_p(n, 1, n, v.z, v.p, v.sc, h->st);
            launch_pcg_spmv_ell(n, 1, n, h->d_ell_ptr, h->d_ell_col, h->d_ell_val, v.p, v.q, v.sc, v.gs, h->ell_wf, h->st);
            launch_pcg_xr(n, 1, n, v.x, v.r, v.p, v.q, v.z, v.sc, v.gs, nullptr, 0, h->st);
            CU(cudaGetLastError());
            return 0;
        };
        float ms = 0.0f;
        TRY(time_ms(h, 7, vec, &ms));
        if (ms < best_v) {
            best_v = ms;
            best_c = c;
        }
    }
    h->tuned_vec_ctas = best_c;
    set_hot_ctas_per_sm(best_c);
    CU(cudaMemsetAsync(v.sc, 0, sizeof(PcgScalars), h->st));
    CU(cudaMemsetAsync(v.p, 0, n * sizeof(double), h->st));
    CU(cudaStreamSynchronize(h->st));
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = TuneVal{best_ring, best_order, best_c};
    return 0;
}

int setup_impl(const algmortar_csr* A, const int32_t* part_in, int32_t n_parts, const algmortar_opts* opts_in,
               algmortar_t** out) {
    if (!out) return fail(ALGMORTAR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!A) return fail(ALGMORTAR_INVALID_ARG, "A is NULL");
    double t0 = now_ms();
    algmortar_opts o;
    algmortar_default_opts(&o);
    if (opts_in) o = *opts_in;
    if (o.precision < 0 || o.precision > 2) return fail(ALGMORTAR_INVALID_ARG, "unknown precision");
    if (o.max_it <= 0) o.max_it = 10000;
    if (o.smooth_steps < 0 || o.smooth_steps > 64) return fail(ALGMORTAR_INVALID_ARG, "smooth_steps out of [0, 64]");
    if (o.check_every <= 0) o.check_every = 1;
    if (o.interface_solve != ALGMORTAR_IFACE_EXACT && o.interface_solve != ALGMORTAR_IFACE_INEXACT)
        return fail(ALGMORTAR_INVALID_ARG, "unknown interface_solve");
    if (o.iface_block_parts <= 0) o.iface_block_parts = 1;
    if (o.iface_max_it <= 0) o.iface_max_it = 200;
    if (!(o.iface_rtol > 0.0) || !(o.iface_rtol < 1.0)) o.iface_rtol = 1e-2;
    HostCsr H{A->n, A->nnz, A->rowptr, A->col, A->val};
    std::string err;
    int rc = validate_csr(H, err);
    if (rc) return fail(rc, err);
    std::vector<int32_t> part;
    if (part_in) {
        part.assign(part_in, part_in + A->n);
    } else {
        Graph G = adjacency(H);
        std::vector<int32_t> drawn;
        const int32_t* sizes = o.part_sizes;
        if (!sizes && o.seed != 0) {
            drawn.resize(n_parts > 0 ? n_parts : 1);
            rc = uneven_part_sizes(A->n, n_parts, o.seed, drawn.data(), err);
            if (rc) return fail(rc, err);
            sizes = drawn.data();
        }
        rc = partition_graph(G, n_parts, sizes, part, err);
        if (rc) return fail(rc, err);
    }
    double t_part = now_ms();
    algmortar_t* h = new (std::nothrow) algmortar_handle();
    if (!h) return fail(ALGMORTAR_OOM, "host allocation");
    h->opts = o;
    h->inexact = o.interface_solve == ALGMORTAR_IFACE_INEXACT;
    rc = build_plan(H, part, n_parts, h->P, err);
    if (rc) {
        delete h;
        return fail(rc, err);
    }
    if (o.nd_depth >= 0) plan_interface_nd(h->P, o.nd_depth);
    double t_plan = now_ms();
    auto bail = [&](int code) {
        delete h;
        return code;
    };
    if (cudaSetDevice(o.device) != cudaSuccess) return bail(fail(ALGMORTAR_CUDA, "cudaSetDevice failed"));
    h->device = o.device;
    {
        int sms = 148;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, o.device);
        set_vec_sms(sms);
    }
    h->st = (cudaStream_t)o.stream;
    if (!h->st) {
        // a blocking stream: ordered with the legacy default stream both ways, and
        // capturable into a CUDA graph
        if (cudaStreamCreate(&h->own_st) != cudaSuccess) return bail(fail(ALGMORTAR_CUDA, "cudaStreamCreate"));
        h->st = h->own_st;
    }

    Plan& P = h->P;
    h->n = P.n;
    h->m = P.m;
    h->L = P.n_lambda;
    std::vector<int32_t> rows(h->m);
    for (int s = 0; s < h->m; ++s) rows[s] = (int32_t)(P.sub_off[s + 1] - P.sub_off[s]);
    // apply jobs, longest first by one of three cost proxies (the autotuner picks one):
    // 0 rows, 1 stored tiles (bytes streamed), 2 tile rows (length of the dependent chain)
    std::vector<int32_t> orders[3];
    std::vector<int64_t> joffs[3];
    for (int v = 0; v < 3; ++v) {
        std::vector<int64_t> cost(h->m);
        for (int s = 0; s < h->m; ++s)
            cost[s] = v == 0 ? rows[s] : (v == 1 ? P.tile_base[s + 1] - P.tile_base[s] : (int64_t)P.ntiles[s]);
        orders[v].resize(h->m);
        for (int s = 0; s < h->m; ++s) orders[v][s] = s;
        std::stable_sort(orders[v].begin(), orders[v].end(), [&](int a, int b) { return cost[a] > cost[b]; });
        joffs[v].resize(h->m);
        for (int t = 0; t < h->m; ++t) joffs[v][t] = P.sub_off[orders[v][t]];
    }
    const std::vector<int32_t>& order = orders[0];
    const std::vector<int64_t>& joff = joffs[0];
    int32_t *d_lo = nullptr, *d_hi = nullptr;
    int64_t *d_row0 = nullptr, *d_base = nullptr, *d_fwd = nullptr, *d_bwd = nullptr;
    rc = 0;
    rc = rc ? rc : upload(h, h->d_rowptr, P.p_rowptr);
    rc = rc ? rc : upload(h, h->d_col, P.p_col);
    rc = rc ? rc : upload(h, h->d_val, P.p_val);
    rc = rc ? rc : upload(h, h->d_perm, P.perm);
    rc = rc ? rc : upload(h, h->d_row_sub, P.row_sub);
    rc = rc ? rc : upload(h, h->d_sub_off, P.sub_off);
    {
        // row-major panels padded to 16-byte rows (4 FP32 or 2 FP64 entries)
        const int vw = h->opts.precision == ALGMORTAR_FP64 ? 2 : 4;
        std::vector<ProlongChunk> ch;
        std::vector<int64_t> prm(P.m + 1, 0);
        for (int s = 0; s < P.m; ++s) {
            const int64_t ns = P.sub_off[s + 1] - P.sub_off[s];
            const int32_t kk = (int32_t)(P.if_off[s + 1] - P.if_off[s]);
            const int32_t ld = (kk + vw - 1) / vw * vw;
            for (int64_t o = 0; o < ns; o += 32) {
                ProlongChunk c;
                c.row0 = P.sub_off[s] + o;
                c.phi0 = prm[s] + o * ld;
                c.ld = ld;
                c.nrow = (int32_t)std::min<int64_t>(32, ns - o);
                c.i0 = (int32_t)P.if_off[s];
                c.kk = kk;
                ch.push_back(c);
            }
            prm[s + 1] = prm[s] + ns * ld;
        }
        h->nchunks = (int)ch.size();
        h->nprm = prm[P.m];
        {
            std::vector<int32_t> csub;
            csub.reserve(ch.size());
            for (int s = 0; s < P.m; ++s)
                for (int64_t o = 0; o < P.sub_off[s + 1] - P.sub_off[s]; o += 32) csub.push_back(s);
            rc = rc ? rc : upload(h, h->d_chunk_sub, csub);
        }
        for (int s = 0; s < P.m; ++s)
            for (int I = 0; I < P.ntiles[s]; ++I)
                h->tile_wm = std::max(h->tile_wm, I - P.t_lo[P.trow_off[s] + I] + 1);
        rc = rc ? rc : upload(h, h->d_chunks, ch);
    }
    rc = rc ? rc : upload(h, h->d_rows, rows);
    rc = rc ? rc : upload(h, h->d_ntiles, P.ntiles);
    rc = rc ? rc : upload(h, d_row0, P.trow_off);
    rc = rc ? rc : upload(h, d_base, P.tile_base);
    rc = rc ? rc : upload(h, d_lo, P.t_lo);
    rc = rc ? rc : upload(h, d_hi, P.t_hi);
    rc = rc ? rc : upload(h, d_fwd, P.t_fwd);
    rc = rc ? rc : upload(h, d_bwd, P.t_bwd);
    for (int v = 0; v < 3; ++v) {
        rc = rc ? rc : upload(h, h->d_job_sub_v[v], orders[v]);
        rc = rc ? rc : upload(h, h->d_job_off_v[v], joffs[v]);
    }
    h->d_job_sub = h->d_job_sub_v[0];
    h->d_job_off = h->d_job_off_v[0];
    rc = rc ? rc : upload(h, h->d_rptr, P.r_ptr);
    rc = rc ? rc : upload(h, h->d_rcell, P.r_cell);
    rc = rc ? rc : upload(h, h->d_rcoef, P.r_coef);
    rc = rc ? rc : upload(h, h->d_if_off, P.if_off);
    rc = rc ? rc : upload(h, h->d_if_list, P.if_list);
    rc = rc ? rc : upload(h, h->d_phi_off, P.phi_off);
    {
        std::vector<int32_t> psrc(P.p_src.begin(), P.p_src.end());
        rc = rc ? rc : upload(h, h->d_psrc, psrc);
    }
    if (rc) return bail(rc);
    rc = rc ? rc : upload(h, h->d_rp_ptr, P.rp_ptr);
    rc = rc ? rc : upload(h, h->d_rp_pos, P.rp_pos);
    rc = rc ? rc : upload(h, h->d_g_from_r, P.g_from_r);
    rc = rc ? rc : upload(h, h->d_ell_ptr, P.ell_ptr);
    rc = rc ? rc : upload(h, h->d_ell_col, P.ell_col);
    rc = rc ? rc : upload(h, h->d_ell_src, P.ell_src);
    if (rc) return bail(rc);
    h->n_ell = (int64_t)P.ell_col.size();
    h->ell_wf = spmv_fast_width(P.ell_ptr.data(), (int64_t)P.ell_ptr.size() - 1);
    h->ws = new (std::nothrow) NumWs();
    h->d_vtmp = h->alloc<double>((size_t)A->nnz);
    h->d_ell_val = h->alloc<double>((size_t)h->n_ell);
    if (!h->ws || !h->d_vtmp || !h->d_ell_val) return bail(fail(ALGMORTAR_OOM, "workspace"));
    if (cudaMemcpyAsync(h->d_vtmp, A->val, A->nnz * sizeof(double), cudaMemcpyHostToDevice, h->st) != cudaSuccess)
        return bail(fail(ALGMORTAR_CUDA, "upload values"));
    launch_ell_values(h->n_ell, h->d_ell_src, h->d_vtmp, h->d_ell_val, h->st);
    h->pf = Profile{h->d_rows, h->d_ntiles, d_row0, d_base, d_lo, d_hi, d_fwd, d_bwd};
    const int64_t n = h->n;
    h->d_dloc = h->alloc<double>(n);
    h->d_sc = h->alloc<double>(n);
    h->d_sc32 = h->alloc<float>(n);
    if (o.smooth_steps > 0) {
        h->d_dloc2 = h->alloc<double>(n);
        h->d_sc2 = h->alloc<double>(n);
        h->d_sc2_32 = h->alloc<float>(n);
        if (!h->d_dloc2 || !h->d_sc2 || !h->d_sc2_32) return bail(fail(ALGMORTAR_OOM, "smoother workspace"));
    }
    h->d_scalar = h->alloc<double>(4);
    h->d_kerr = h->alloc<int>(1);
    if (!h->d_dloc || !h->d_sc || !h->d_sc32 || !h->d_scalar || !h->d_kerr) return bail(fail(ALGMORTAR_OOM, "workspace"));
    rc = alloc_vecs(h, h->v1, 1);
    if (rc) return bail(rc);
    if (cudaMemsetAsync(h->d_kerr, 0, sizeof(int), h->st) != cudaSuccess) return bail(fail(ALGMORTAR_CUDA, "memset"));
    double t_up = now_ms();
    rc = numeric_dispatch(h);
    if (rc) return bail(rc);
    if (cudaStreamSynchronize(h->st) != cudaSuccess) return bail(fail(ALGMORTAR_CUDA, "setup synchronize"));
    if (o.autotune) {
        rc = autotune(h);
        if (rc) return bail(rc);
    }
    double t_end = now_ms();
    algmortar_info& I = h->info;
    I.n = n;
    I.n_parts = h->m;
    I.n_lambda = h->L;
    I.max_part = P.max_part;
    I.min_part = P.min_part;
    I.precision = o.precision;
    I.n_interface_edges = P.n_edges;
    I.factor_entries = P.total_tiles * TILE2;
    int es = o.precision == ALGMORTAR_FP64 ? 8 : (o.precision == ALGMORTAR_FP32 ? 4 : 2);
    I.factor_bytes = 2 * P.total_tiles * TILE2 * es;
    I.phi_entries = P.phi_off[h->m];
    I.setup_ms[0] = (t_part - t0) + (t_plan - t_part);
    I.setup_ms[1] = t_up - t_plan;
    I.setup_ms[7] = t_end - t0;
    I.interface_solve = o.interface_solve;
    I.iface_blocks = h->inexact ? h->iface_nblk : 0;
    I.iface_cluster = h->inexact ? h->iface_cluster : 0;
    I.iface_staged = h->inexact ? h->iface.stage : 0;
    I.tuned_ring = h->tuned_ring;
    I.tuned_vec_ctas = h->tuned_vec_ctas;
    if (o.verbose)
        std::fprintf(stderr,
                     "[algmortar] n=%lld m=%d nLam=%d parts %d..%d tiles=%lld | partition %.1f ms plan %.1f ms "
                     "upload %.1f | factor %.2f mbf %.2f iface-asm %.2f iface-factor %.2f iface-factor+inv %.2f | total %.1f ms\n",
                     (long long)n, h->m, h->L, P.min_part, P.max_part, (long long)P.total_tiles, t_part - t0,
                     t_plan - t_part, I.setup_ms[1], I.setup_ms[2], I.setup_ms[3], I.setup_ms[4], I.setup_ms[6], I.setup_ms[5],
                     I.setup_ms[7]);
    *out = h;
    return 0;
}

}  // namespace

extern "C" {

void algmortar_default_opts(algmortar_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = ALGMORTAR_FP64;
    o->diag_scale = 1;
    o->max_it = 10000;
    o->use_graph = 0;
    o->check_every = 1;
    o->flexible = 0;
    o->verbose = 0;
    o->device = 0;
    o->part_sizes = nullptr;
    o->stream = nullptr;
    o->nd_depth = -1;
    o->autotune = 0;
    o->interface_solve = ALGMORTAR_IFACE_EXACT;
    o->smooth_steps = 0;
    o->iface_block_parts = 1;
    o->iface_max_it = 200;
    o->stage_times = 0;
    o->iface_rtol = 1e-2;
    o->seed = 0;
}

int algmortar_part_sizes(int64_t n, int32_t m, uint64_t seed, int32_t* sizes_out) {
    if (!sizes_out) return fail(ALGMORTAR_INVALID_ARG, "null argument");
    std::string err;
    int rc = uneven_part_sizes(n, m, seed, sizes_out, err);
    return rc ? fail(rc, err) : 0;
}

int algmortar_partition(const algmortar_csr* A, int32_t n_parts, const int32_t* part_sizes, int32_t* part_out) {
    if (!A || !part_out) return fail(ALGMORTAR_INVALID_ARG, "null argument");
    HostCsr H{A->n, A->nnz, A->rowptr, A->col, A->val};
    std::string err;
    int rc = validate_csr(H, err);
    if (rc) return fail(rc, err);
    Graph G = adjacency(H);
    std::vector<int32_t> part;
    rc = partition_graph(G, n_parts, part_sizes, part, err);
    if (rc) return fail(rc, err);
    std::memcpy(part_out, part.data(), part.size() * sizeof(int32_t));
    return 0;
}

int algmortar_setup(const algmortar_csr* A, int32_t n_parts, const algmortar_opts* opts, algmortar_t** out) {
    return setup_impl(A, nullptr, n_parts, opts, out);
}

int algmortar_setup_with_parts(const algmortar_csr* A, const int32_t* part, int32_t n_parts,
                               const algmortar_opts* opts, algmortar_t** out) {
    if (!part) return fail(ALGMORTAR_INVALID_ARG, "part is NULL");
    return setup_impl(A, part, n_parts, opts, out);
}

int algmortar_apply(algmortar_t* h, const double* r_dev, double* z_dev) {
    if (!h || !r_dev || !z_dev) return fail(ALGMORTAR_INVALID_ARG, "null argument");
    CU(cudaSetDevice(h->device));
    Vecs& v = h->v1;
    launch_gather(h->n, h->d_perm, r_dev, v.t, h->st);
    TRY(apply_internal(h, v, v.t, v.z, false));
    launch_scatter(h->n, h->d_perm, v.z, z_dev, h->st);
    CU(cudaGetLastError());
    return 0;
}

int algmortar_apply_stages(algmortar_t* h, const double* r_dev, double* pbar_dev, double* beta_dev,
                           double* eta_dev, double* z_dev) {
    if (!h || !r_dev || !pbar_dev || !z_dev || (h->L > 0 && (!beta_dev || !eta_dev)))
        return fail(ALGMORTAR_INVALID_ARG, "null argument");
    CU(cudaSetDevice(h->device));
    Vecs& v = h->v1;
    launch_gather(h->n, h->d_perm, r_dev, v.t, h->st);
    TRY(apply_internal(h, v, v.t, v.z, false));
    CU(cudaMemcpyAsync(pbar_dev, v.pbar, h->n * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    if (h->L > 0 && h->inexact) {   // natural interface order inside the handle
        CU(cudaMemcpyAsync(beta_dev, v.beta, h->L * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
        CU(cudaMemcpyAsync(eta_dev, v.eta, h->L * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    } else if (h->L > 0) {
        // ND order inside the handle -> natural interface order
        launch_gather(h->L, h->d_ndpos, v.beta, beta_dev, h->st);
        launch_gather(h->L, h->d_ndpos, v.eta, eta_dev, h->st);
    }
    CU(cudaMemcpyAsync(z_dev, v.z, h->n * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    return 0;
}

int algmortar_pcg_solve(algmortar_t* h, const double* b_dev, double* x_dev, double tol, algmortar_stats* st) {
    if (!h || !b_dev || !x_dev) return fail(ALGMORTAR_INVALID_ARG, "null argument");
    CU(cudaSetDevice(h->device));
    Vecs& v = h->v1;
    launch_gather(h->n, h->d_perm, b_dev, v.b, h->st);
    int rc = pcg_internal(h, v, tol, st);
    if (rc != ALGMORTAR_OK && rc != ALGMORTAR_NO_CONVERGENCE && rc != ALGMORTAR_BREAKDOWN) return rc;
    launch_scatter(h->n, h->d_perm, v.x, x_dev, h->st);
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(h->st));
    return rc;
}

int algmortar_pcg_solve_host(algmortar_t* h, const double* b_host, double* x_host, double tol,
                             algmortar_stats* st) {
    if (!h || !b_host || !x_host) return fail(ALGMORTAR_INVALID_ARG, "null argument");
    CU(cudaSetDevice(h->device));
    double t0 = now_ms();
    Vecs& v = h->v1;
    CU(cudaMemcpyAsync(v.t, b_host, h->n * sizeof(double), cudaMemcpyHostToDevice, h->st));
    launch_gather(h->n, h->d_perm, v.t, v.b, h->st);
    int rc = pcg_internal(h, v, tol, st);
    if (rc != ALGMORTAR_OK && rc != ALGMORTAR_NO_CONVERGENCE && rc != ALGMORTAR_BREAKDOWN) return rc;
    launch_scatter(h->n, h->d_perm, v.x, v.t, h->st);
    CU(cudaMemcpyAsync(x_host, v.t, h->n * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CU(cudaStreamSynchronize(h->st));
    if (st) st->solve_ms = now_ms() - t0;
    return rc;
}

int algmortar_pcg_solve_multi(algmortar_t* h, const double* B_dev, double* X_dev, int32_t nrhs, int64_t ld,
                              double tol, algmortar_stats* st) {
    if (!h || !B_dev || !X_dev || nrhs <= 0 || ld < h->n) return fail(ALGMORTAR_INVALID_ARG, "bad argument");
    CU(cudaSetDevice(h->device));
    // batches of up to ALGMORTAR_MAX_BATCH columns: every launch of the iteration covers
    // all columns of the batch (gridDim.y), each column with its own PCG state
    const int kmax = nrhs < ALGMORTAR_MAX_BATCH ? nrhs : ALGMORTAR_MAX_BATCH;
    TRY(alloc_vecs(h, h->vk, kmax));
    Vecs& v = h->vk;
    int worst = ALGMORTAR_OK;
    for (int j0 = 0; j0 < nrhs; j0 += kmax) {
        v.k = nrhs - j0 < kmax ? nrhs - j0 : kmax;
        launch_gather_cols(h->n, v.k, h->d_perm, B_dev + j0 * ld, ld, v.b, h->n, h->st);
        int rc = pcg_internal(h, v, tol, st ? st + j0 : nullptr);
        if (rc != ALGMORTAR_OK && rc != ALGMORTAR_NO_CONVERGENCE && rc != ALGMORTAR_BREAKDOWN) return rc;
        launch_scatter_cols(h->n, v.k, h->d_perm, v.x, h->n, X_dev + j0 * ld, ld, h->st);
        CU(cudaGetLastError());
        if (rc == ALGMORTAR_BREAKDOWN || (rc == ALGMORTAR_NO_CONVERGENCE && worst == ALGMORTAR_OK)) worst = rc;
    }
    CU(cudaStreamSynchronize(h->st));
    return worst;
}

int algmortar_update_values(algmortar_t* h, const double* val_host) {
    if (!h || !val_host) return fail(ALGMORTAR_INVALID_ARG, "null argument");
    CU(cudaSetDevice(h->device));
    const int64_t nnz = (int64_t)h->P.p_val.size();
    CU(cudaMemcpyAsync(h->d_vtmp, val_host, nnz * sizeof(double), cudaMemcpyHostToDevice, h->st));
    launch_gather(nnz, h->d_psrc, h->d_vtmp, h->d_val, h->st);
    launch_ell_values(h->n_ell, h->d_ell_src, h->d_vtmp, h->d_ell_val, h->st);
    CU(cudaGetLastError());
    return numeric_dispatch(h);
}

int algmortar_update_values_device(algmortar_t* h, const double* val_dev) {
    if (!h || !val_dev) return fail(ALGMORTAR_INVALID_ARG, "null argument");
    CU(cudaSetDevice(h->device));
    const int64_t nnz = (int64_t)h->P.p_val.size();
    launch_gather(nnz, h->d_psrc, val_dev, h->d_val, h->st);
    launch_ell_values(h->n_ell, h->d_ell_src, val_dev, h->d_ell_val, h->st);
    CU(cudaGetLastError());
    return numeric_dispatch(h);
}

int algmortar_tpfa_grad_lnK(algmortar_t* h, const double* K_dev, const double* tb_dev, const double* tbp_dev,
                            const double* p_dev, const double* lam_dev, double* grad_dev) {
    if (!h || !K_dev || !tb_dev || !tbp_dev || !p_dev || !lam_dev || !grad_dev)
        return fail(ALGMORTAR_INVALID_ARG, "null argument");
    CU(cudaSetDevice(h->device));
    const int64_t n = h->n;
    // internal ordering: gather the per-cell inputs, run the row gather, scatter back
    Vecs& v = h->v1;
    double* buf[5] = {v.x, v.r, v.z, v.p, v.q};
    const double* src[5] = {K_dev, tb_dev, tbp_dev, p_dev, lam_dev};
    for (int i = 0; i < 5; ++i) launch_gather(n, h->d_perm, src[i], buf[i], h->st);
    launch_tpfa_grad(n, h->d_rowptr, h->d_col, h->d_val, buf[0], buf[1], buf[2], buf[3], buf[4], v.t, h->st);
    launch_scatter(n, h->d_perm, v.t, grad_dev, h->st);
    CU(cudaGetLastError());
    return 0;
}

int algmortar_interface_solve_noalloc(const algmortar_t* h, const double* b_dev, double* eta_dev) {
    if (!h) return fail(ALGMORTAR_INVALID_ARG, "null handle");
    if (h->L > 0 && (!b_dev || !eta_dev)) return fail(ALGMORTAR_INVALID_ARG, "null argument");
    if (h->inexact)
        return fail(ALGMORTAR_INVALID_ARG, "the allocation-free interface solve is the exact one; this handle was set "
                                           "up with the inexact interface solve");
    std::string err;
    int rc = am::interface_solve_noalloc(h->device, h->st, h->L, h->nd, h->d_ndpos, b_dev, eta_dev, err);
    if (rc) return fail(rc, err);
    return 0;
}

int algmortar_get_partition(const algmortar_t* h, int32_t* part_out) {
    if (!h || !part_out) return fail(ALGMORTAR_INVALID_ARG, "null argument");
    std::memcpy(part_out, h->P.part.data(), h->P.part.size() * sizeof(int32_t));
    return 0;
}

int algmortar_get_permutation(const algmortar_t* h, int32_t* perm_out) {
    if (!h || !perm_out) return fail(ALGMORTAR_INVALID_ARG, "null argument");
    std::memcpy(perm_out, h->P.perm.data(), h->P.perm.size() * sizeof(int32_t));
    return 0;
}

int algmortar_get_interfaces(const algmortar_t* h, int32_t* pairs_out) {
    if (!h || !pairs_out) return fail(ALGMORTAR_INVALID_ARG, "null argument");
    if (!h->P.pairs.empty()) std::memcpy(pairs_out, h->P.pairs.data(), h->P.pairs.size() * sizeof(int32_t));
    return 0;
}

int algmortar_time_stages(algmortar_t* h, int32_t reps, double* ms_out) {
    if (!h || !ms_out || reps <= 0) return fail(ALGMORTAR_INVALID_ARG, "bad argument");
    CU(cudaSetDevice(h->device));
    set_hot_ctas_per_sm(h->tuned_vec_ctas);
    cudaStream_t st = h->st;
    Vecs& v = h->v1;
    const int64_t n = h->n;
    PcgScalars saved;
    CU(cudaMemcpyAsync(&saved, v.sc, sizeof(saved), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    // a live scalar state: not done, beta/alpha finite, so no kernel exits early
    PcgScalars live = saved;
    live.done = 0;
    live.iter = 1;
    live.max_it = 1 << 30;
    live.rz = saved.rz != 0.0 ? saved.rz : 1.0;
    live.tol2 = 0.0;
    const ColStrides cs = col_strides(h, v, false);
    PcgScalars* rz = v.sc;
    if (h->opts.use_graph) TRY(ensure_graph(h, v));
    cudaEvent_t ev[8];
    for (auto& e : ev) CU(cudaEventCreate(&e));
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int it = 0; it <= reps; ++it) {
        CU(cudaMemcpyAsync(v.sc, &live, sizeof(live), cudaMemcpyHostToDevice, st));
        cudaEventRecord(ev[0], st);
        launch_pcg_spmv_ell(n, 1, n, h->d_ell_ptr, h->d_ell_col, h->d_ell_val, v.p, v.q, v.sc, v.gs, h->ell_wf, st);
        cudaEventRecord(ev[1], st);
        launch_pcg_p(n, 1, n, v.z, v.p, v.sc, st);
        launch_pcg_xr(n, 1, n, v.x, v.r, v.p, v.q, v.z, v.sc, v.gs, nullptr, 0, st);
        cudaEventRecord(ev[2], st);
        // stages of Algorithm 2 (same launches as apply_internal, timed one by one)
        switch (h->opts.precision) {
            case ALGMORTAR_FP64: TRY((stage_local<double, double>(h, v, v.r, cs))); break;
            case ALGMORTAR_FP32: TRY((stage_local<float, float>(h, v, v.r, cs))); break;
            default: TRY((stage_local<__nv_bfloat16, float>(h, v, v.r, cs))); break;
        }
        cudaEventRecord(ev[3], st);
        stage_restrict(h, v, cs);
        cudaEventRecord(ev[4], st);
        TRY(stage_coarse(h, v, cs));
        cudaEventRecord(ev[5], st);
        switch (h->opts.precision) {
            case ALGMORTAR_FP64: stage_prolong<double>(h, v, v.r, v.z, cs, rz); break;
            case ALGMORTAR_FP32: stage_prolong<float>(h, v, v.r, v.z, cs, rz); break;
            default: stage_prolong<float>(h, v, v.r, v.z, cs, rz); break;
        }
        cudaEventRecord(ev[6], st);
        CU(cudaMemcpyAsync(v.sc, &live, sizeof(live), cudaMemcpyHostToDevice, st));
        cudaEventRecord(ev[7], st);
        if (v.graph) {
            CU(cudaGraphLaunch(v.graph, st));
            add_launches(v.graph_kernels);
        } else {
            TRY(pcg_iteration(h, v));
        }
        cudaEvent_t e8;
        CU(cudaEventCreate(&e8));
        cudaEventRecord(e8, st);
        CU(cudaEventSynchronize(e8));
        if (it > 0) {
            float t;
            for (int k = 0; k < 6; ++k) {
                cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
                acc[k] += t;
            }
            cudaEventElapsedTime(&t, ev[7], e8);
            acc[6] += t;
        }
        cudaEventDestroy(e8);
    }
    for (int k = 0; k < 7; ++k) ms_out[k] = acc[k] / reps;
    ms_out[7] = 0.0;
    for (auto& e : ev) cudaEventDestroy(e);
    CU(cudaMemcpyAsync(v.sc, &saved, sizeof(saved), cudaMemcpyHostToDevice, st));
    CU(cudaStreamSynchronize(st));
    return 0;
}

int algmortar_get_info(const algmortar_t* h, algmortar_info* info) {
    if (!h || !info) return fail(ALGMORTAR_INVALID_ARG, "null argument");
    *info = h->info;
    info->kernel_launches = launch_count();
    info->iface_last_iterations = 0;
    if (h->inexact && h->v1.iits) {
        CU(cudaSetDevice(h->device));
        CU(cudaMemcpyAsync(&info->iface_last_iterations, h->v1.iits, sizeof(int32_t), cudaMemcpyDeviceToHost, h->st));
        CU(cudaStreamSynchronize(h->st));
    }
    info->tuned_ring = h->tuned_ring;
    info->tuned_vec_ctas = h->tuned_vec_ctas;
    info->tuned_job_order = h->tuned_order;
    return 0;
}

void algmortar_destroy(algmortar_t* h) {
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->st) cudaStreamSynchronize(h->st);
    else cudaDeviceSynchronize();
    delete h;
}

const char* algmortar_strerror(int s) {
    switch (s) {
        case ALGMORTAR_OK: return "ok";
        case ALGMORTAR_INVALID_ARG: return "invalid argument";
        case ALGMORTAR_NOT_SYMMETRIC: return "matrix not symmetric";
        case ALGMORTAR_INTERFACE_SIGN: return "non-negative coupling between subdomains";
        case ALGMORTAR_NOT_SPD: return "non-positive pivot (matrix not SPD)";
        case ALGMORTAR_NO_CONVERGENCE: return "PCG did not converge";
        case ALGMORTAR_BREAKDOWN: return "PCG breakdown";
        case ALGMORTAR_CUDA: return "CUDA error";
        case ALGMORTAR_OOM: return "out of memory";
        case ALGMORTAR_TOO_LARGE: return "subdomain too large";
        default: return "unknown status";
    }
}

const char* algmortar_last_error(void) { return g_err.c_str(); }

}  // extern "C"
