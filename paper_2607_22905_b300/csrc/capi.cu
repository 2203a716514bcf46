// C ABI of libalgmortar (include/algmortar.h): handle lifetime, Algorithm 1 on the device,
// Algorithm 2 and the PCG loop.
#include <algorithm>
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
    double *gwork = nullptr, *gdinv = nullptr, *gf = nullptr, *gb = nullptr, *gE = nullptr;
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
    double *cwork = nullptr, *cdinv = nullptr, *cf = nullptr, *cb = nullptr, *cE = nullptr;
    int32_t* d_crowsq = nullptr;
    int64_t* d_czerooff = nullptr;
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
    int64_t graph_kernels = 0;         // kernels in one replay of the iteration graph
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
    int nchunks = 0;                   // prolongation: row chunks (<= VEC_BS rows of one subdomain)
    int32_t *d_chunk_sub = nullptr, *d_chunk_off = nullptr;
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
    double* d_vtmp = nullptr;          // staging for value updates (original CSR order)
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

int read_err_flag(algmortar_t* h, int* d_err, const char* what) {
    int e[2];
    CU(cudaMemcpyAsync(e, d_err, sizeof(e), cudaMemcpyDeviceToHost, h->st));
    CU(cudaStreamSynchronize(h->st));
    if (e[0]) return fail(ALGMORTAR_NOT_SPD, std::string("non-positive pivot in the ") + what + " factor, block " +
                                                 std::to_string(e[1]));
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
    h->d_fwdS = h->alloc<TS>((size_t)tiles * TILE2);
    h->d_bwdS = h->alloc<TS>((size_t)tiles * TILE2);
    if (h->opts.smooth_steps > 0) {
        h->d_fwdS2 = h->alloc<TS>((size_t)tiles * TILE2);
        h->d_bwdS2 = h->alloc<TS>((size_t)tiles * TILE2);
        if (!h->d_fwdS2 || !h->d_bwdS2) return fail(ALGMORTAR_OOM, "smoother factor buffers");
    }
    h->d_phi = std::is_same<TS, double>::value ? (void*)W.phi64 : (void*)h->alloc<PanelT<TS>>(nphi);
    if (!W.work || !W.dinv || !W.d_err || !W.rhs || !W.phi64 || !h->d_fwdS || !h->d_bwdS || !h->d_phi)
        return fail(ALGMORTAR_OOM, "factor / MBF buffers");
    if (L > 0) {
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
        W.gwork = h->alloc<double>((size_t)std::max<int64_t>(tb, 1) * TILE2);
        W.gdinv = h->alloc<double>((size_t)std::max<int64_t>(trow, 1) * TILE2);
        W.gf = h->alloc<double>((size_t)std::max<int64_t>(tb, 1) * TILE2);
        W.gb = h->alloc<double>((size_t)std::max<int64_t>(tb, 1) * TILE2);
        W.gE = h->alloc<double>((size_t)std::max<int64_t>(gi, 1));
        W.D = h->alloc<double>((size_t)std::max<int64_t>(dof, 1));
        double* Ginv = h->alloc<double>((size_t)std::max<int64_t>(gi, 1));
        double* Wcm = h->alloc<double>((size_t)std::max<int64_t>(wo, 1));
        double* Wrm = h->alloc<double>((size_t)std::max<int64_t>(wo, 1));
        if (!W.gwork || !W.gdinv || !W.gf || !W.gb || !W.gE || !W.D || !Ginv || !Wcm || !Wrm)
            return fail(ALGMORTAR_OOM, "interface group buffers");
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
            TRY(upload(h, h->d_ifpos, ifpos));
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
            W.cwork = h->alloc<double>((size_t)ct * TILE2);
            W.cdinv = h->alloc<double>((size_t)T * TILE2);
            W.cf = h->alloc<double>((size_t)ct * TILE2);
            W.cb = h->alloc<double>((size_t)ct * TILE2);
            W.cE = h->alloc<double>((size_t)nsep * nsep);
            double* Cinv = h->alloc<double>((size_t)nsep * nsep);
            if (!W.cwork || !W.cdinv || !W.cf || !W.cb || !W.cE || !Cinv)
                return fail(ALGMORTAR_OOM, "separator buffers");
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
    launch_tile_chol<TW>(m, h->pf, h->d_job_sub, work, dinv, W.d_err, st);
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
        launch_tile_chol<TW>(m, h->pf, h->d_job_sub, work, dinv, W.d_err, st);
        CU(cudaGetLastError());
        TRY(read_err_flag(h, W.d_err, "smoother block"));
        launch_finalize<TW, TS>(m, h->pf, work, dinv, (TS*)h->d_fwdS2, (TS*)h->d_bwdS2, st);
        CU(cudaGetLastError());
    }
    cudaEventRecord(ev[1], st);
    // --- MBFs (Eq. def-phat-local): Phi_i = A_i^{-1} (-B_i psi_m), one job per (i, m) ---
    CU(cudaMemsetAsync(W.rhs, 0, nphi * sizeof(double), st));
    launch_mbf_rhs(m, W.d_goff, W.d_grow, W.d_gcol, W.d_gval, h->d_rows, h->d_phi_off, W.rhs, st);
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
        TRY((solve_cols<TS, TA>(a, W.bj_mbf, false, P.max_tiles, st)));
    }
    if (!std::is_same<TS, double>::value) launch_convert<PanelT<TS>>(nphi, W.phi64, (PanelT<TS>*)h->d_phi, st);
    cudaEventRecord(ev[2], st);
    // --- interface system S_eta = diag(T) + 1/4 G^T Phi (Eq. interface-problem-alg),
    //     solved exactly by one level of nested dissection (kernels_coarse.cu) ---
    if (L > 0) {
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
        // interior blocks: dense tiles, right-looking factor per group, sweep streams
        Profile gpf{W.d_irows, W.d_int, W.d_irow0, W.d_ibase, W.d_ilo, W.d_ihi, W.d_ifwd, W.d_ibwd};
        launch_dense_to_tiles(W.ntiles_items, W.Sd, L, W.d_isrc, W.d_irows, W.d_ibase, W.d_titem, W.d_tI, W.d_tJ,
                              W.gwork, st);
        CU(cudaMemcpyAsync(W.d_err, err_init, sizeof(err_init), cudaMemcpyHostToDevice, st));
        {
            std::vector<int32_t> Th(W.nitems);
            for (int it = 0; it < W.nitems; ++it) Th[it] = (int32_t)W.item_hi[it].size();
            launch_dense_cholesky(W.nitems, Th, W.d_int, W.d_ibase, W.d_irow0, W.gwork, W.gdinv, W.d_err, st);
        }
        CU(cudaGetLastError());
        TRY(read_err_flag(h, W.d_err, "interface (interior block)"));
        launch_finalize<double, double>(W.nitems, gpf, W.gwork, W.gdinv, W.gf, W.gb, st);
        // S_gg^{-1} (identity columns), then W_g = S_gg^{-1} S_{g,A_g} from its sparse pattern
        SolveArgs sa{};
        sa.pf = gpf;
        sa.fwdS = W.gf;
        sa.bwdS = W.gb;
        sa.err = h->d_kerr;
        // one job per column (measured faster than column blocks here: the FP64 work of a
        // job is spread over four warps and the grids are larger)
        sa.job_sub = W.d_gjob;
        sa.job_in = W.d_gjin;
        sa.job_out = W.d_gjin;
        sa.job_t0 = W.d_gjt0;          // identity columns: lower triangle of S_gg^{-1} only
        sa.in = W.gE;
        sa.out = (double*)h->nd.Ginv;
        CU((launch_tile_solve<double, double>(sa, W.njobs_g, W.max_tiles_items, st)));
        launch_mirror_lower(h->nd_grows, h->nd.gioff, G, (double*)h->nd.Ginv, st);
        launch_nd_w_sparse(h->nd.np, L, W.Sd, h->nd.goff, h->nd.aoff, h->nd.alist, sep0, h->nd.prow_g, W.d_wc_ptr,
                           W.d_wc_row, h->nd.gioff, h->nd.Ginv, h->nd.woff, (double*)h->nd.Wcm, st);
        launch_transpose_blocks(h->nd.goff, h->nd.aoff, h->nd.woff, G, h->nd.Wcm, (double*)h->nd.Wrm, st);
        if (nsep > 0) {
            launch_nd_schur_sparse(h->nd.np, L, W.Sd, h->nd.goff, h->nd.aoff, h->nd.alist, sep0, h->nd.prow_g,
                                   W.d_wc_ptr, W.d_wc_row, h->nd.woff, h->nd.Wrm, W.d_doff, W.D, st);
            const int64_t ct = (int64_t)W.cT * (W.cT + 1) / 2;
            launch_nd_schur_tiles(ct, L, nsep, sep0, W.Sd, h->nd.sg, h->nd.sidx, h->nd.aoff, W.d_doff, W.D, W.cwork, st);
            CU(cudaMemcpyAsync(W.d_err, err_init, sizeof(err_init), cudaMemcpyHostToDevice, st));
            launch_dense_cholesky(1, std::vector<int32_t>{W.cT}, W.d_cnt, W.d_czero, W.d_czero, W.cwork, W.cdinv,
                                  W.d_err, st);
            CU(cudaGetLastError());
            TRY(read_err_flag(h, W.d_err, "interface (separator)"));
            Profile cpf{W.d_crows, W.d_cnt, W.d_czero, W.d_czero, W.d_clo, W.d_chi, W.d_cfwd, W.d_cbwd};
            launch_finalize<double, double>(1, cpf, W.cwork, W.cdinv, W.cf, W.cb, st);
            SolveArgs ca{};
            ca.pf = cpf;
            ca.fwdS = W.cf;
            ca.bwdS = W.cb;
            ca.err = h->d_kerr;
            ca.job_sub = W.d_cjob;
            ca.job_in = W.d_cjin;
            ca.job_out = W.d_cjin;
            ca.job_t0 = W.d_cjt0;      // lower triangle of C^{-1} only
            ca.in = W.cE;
            ca.out = (double*)h->nd.Cinv;
            CU((launch_tile_solve<double, double>(ca, nsep, W.cT, st)));
            launch_mirror_lower(W.d_crowsq, W.d_czerooff, 1, (double*)h->nd.Cinv, st);
        }
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
    a.deep_ring = h->opts.deep_ring;
    a.err = h->d_kerr;
    if (v.k > 1) {
        // batched columns: one job per (subdomain, block of COLS_PER_JOB columns), each
        // factor tile read once per block
        a.job_col0 = v.bj_col0;
        return solve_cols<TS, TA>(a, v.bj, false, h->P.max_tiles, h->st);
    }
    CU((launch_tile_solve<TS, TA>(a, h->m, h->P.max_tiles, h->st, v.k)));
    return 0;
}

// Interface right-hand side and interface solve: b_eta from pbar, eta = S^{-1} b_eta.
void stage_restrict(algmortar_t* h, Vecs& v, const ColStrides& cs) {
    launch_restrict(h->L, h->d_rptr, h->d_rcell, h->d_rcoef, v.pbar, v.beta, h->d_ndpos, cs, v.k, h->st);
}
void stage_coarse(algmortar_t* h, Vecs& v, const ColStrides& cs) {
    if (h->L > 0) launch_nd_solve(h->nd, v.beta, v.eta, v.P, cs, v.k, h->st);
}

// z = base + pbar + Phi eta (base may be null); inside PCG (sc given) also r . z and the
// next beta per column.
template <typename TS>
void stage_prolong(algmortar_t* h, Vecs& v, const double* r, double* z, const ColStrides& cs, PcgScalars* sc,
                   const double* base = nullptr) {
    launch_prolong<TS>(h->nchunks, h->d_chunk_sub, h->d_chunk_off, h->P.max_k, h->d_sub_off, h->d_if_off,
                       h->L > 0 ? h->d_ifpos : h->d_if_list, h->d_phi_off, (const TS*)h->d_phi, v.eta, v.pbar, base,
                       z, r, v.gs, sc, cs, v.k, h->st);
}

template <typename TS, typename TA>
int apply_t(algmortar_t* h, Vecs& v, const double* r, double* z, bool pcg) {
    const ColStrides cs = col_strides(h, v, pcg);
    const int nu = h->opts.smooth_steps;
    if (nu <= 0) {
        TRY((stage_local<TS, TA>(h, v, r, cs)));
        stage_restrict(h, v, cs);
        stage_coarse(h, v, cs);
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
    stage_coarse(h, v, cs);
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
    launch_pcg_p(n, v.k, n, v.z, v.p, v.sc, st);
    launch_pcg_spmv_ell(n, v.k, n, h->d_ell_ptr, h->d_ell_col, h->d_ell_val, v.p, v.q, v.sc, v.gs, st);
    launch_pcg_xr(n, v.k, n, v.x, v.r, v.p, v.q, v.z, v.sc, v.gs, st);
    return apply_internal(h, v, v.r, v.z, true);
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
    void* old[] = {v.x, v.r, v.z, v.p, v.q, v.pbar, v.b, v.t, v.w, v.beta, v.eta, v.P, v.sc, v.gs.part, v.gs.ticket};
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
    // one CTA per row chunk of a subdomain)
    const size_t nb = 2 * (size_t)std::max(vec_blocks(h->n), h->nchunks) * cap;
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
    if (!v.x || !v.r || !v.z || !v.p || !v.q || !v.pbar || !v.b || !v.t || (h->opts.smooth_steps > 0 && !v.w) ||
        !v.beta || !v.eta || !v.P || !v.sc ||
        !v.gs.part || !v.gs.ticket) {
        v.cap = 0;
        return fail(ALGMORTAR_OOM, "vector workspace");
    }
    CU(cudaMemsetAsync(v.p, 0, n * sizeof(double), h->st));
    CU(cudaMemsetAsync(v.sc, 0, cap * sizeof(PcgScalars), h->st));
    CU(cudaMemsetAsync(v.gs.ticket, 0, cap * sizeof(unsigned int), h->st));
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
    void* old[] = {v.bj.sub, v.bj.nc, v.bj.t0, v.bj.in, v.bj.ld, v.bj_col0};
    for (void* p : old)
        if (p) h->release(p);
    TRY(upload_jobs(h, v.bj, b));
    TRY(upload(h, v.bj_col0, col0));
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
    if (h->opts.use_graph) TRY(ensure_graph(h, v));
    launch_pcg_init(n, k, n, v.b, v.x, v.r, v.sc, v.gs, tol, h->opts.max_it, h->opts.flexible ? 1 : 0, st);
    TRY(apply_internal(h, v, v.r, v.z, true));
    std::vector<PcgScalars> hs(k);
    std::vector<int> restarts(k, 0);
    std::vector<double> true_rel(k, 0.0);
    std::vector<char> fin(k, 0);
    const int every = h->opts.check_every > 0 ? h->opts.check_every : 1;
    static const int zero = 0;
    for (;;) {
        for (int c = 0; c < every; ++c) {
            if (v.graph) {
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
    int worst = ALGMORTAR_OK;
    for (int j = 0; j < k; ++j) {
        const PcgScalars& s = hs[j];
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
    HostCsr H{A->n, A->nnz, A->rowptr, A->col, A->val};
    std::string err;
    int rc = validate_csr(H, err);
    if (rc) return fail(rc, err);
    std::vector<int32_t> part;
    if (part_in) {
        part.assign(part_in, part_in + A->n);
    } else {
        Graph G = adjacency(H);
        rc = partition_graph(G, n_parts, o.part_sizes, part, err);
        if (rc) return fail(rc, err);
    }
    double t_part = now_ms();
    algmortar_t* h = new (std::nothrow) algmortar_handle();
    if (!h) return fail(ALGMORTAR_OOM, "host allocation");
    h->opts = o;
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
    // apply jobs: largest subdomains first
    std::vector<int32_t> order(h->m);
    for (int s = 0; s < h->m; ++s) order[s] = s;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return rows[a] > rows[b]; });
    std::vector<int64_t> joff(h->m);
    for (int t = 0; t < h->m; ++t) joff[t] = P.sub_off[order[t]];
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
        std::vector<int32_t> cs, co;
        for (int s = 0; s < P.m; ++s)
            for (int64_t o = 0; o < P.sub_off[s + 1] - P.sub_off[s]; o += VEC_BS) {
                cs.push_back(s);
                co.push_back((int32_t)o);
            }
        h->nchunks = (int)cs.size();
        rc = rc ? rc : upload(h, h->d_chunk_sub, cs);
        rc = rc ? rc : upload(h, h->d_chunk_off, co);
    }
    rc = rc ? rc : upload(h, h->d_rows, rows);
    rc = rc ? rc : upload(h, h->d_ntiles, P.ntiles);
    rc = rc ? rc : upload(h, d_row0, P.trow_off);
    rc = rc ? rc : upload(h, d_base, P.tile_base);
    rc = rc ? rc : upload(h, d_lo, P.t_lo);
    rc = rc ? rc : upload(h, d_hi, P.t_hi);
    rc = rc ? rc : upload(h, d_fwd, P.t_fwd);
    rc = rc ? rc : upload(h, d_bwd, P.t_bwd);
    rc = rc ? rc : upload(h, h->d_job_sub, order);
    rc = rc ? rc : upload(h, h->d_job_off, joff);
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
    o->l2_prefetch = -1;
    o->deep_ring = 0;
    o->smooth_steps = 0;
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
    if (h->L > 0) {
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
        launch_pcg_spmv_ell(n, 1, n, h->d_ell_ptr, h->d_ell_col, h->d_ell_val, v.p, v.q, v.sc, v.gs, st);
        cudaEventRecord(ev[1], st);
        launch_pcg_p(n, 1, n, v.z, v.p, v.sc, st);
        launch_pcg_xr(n, 1, n, v.x, v.r, v.p, v.q, v.z, v.sc, v.gs, st);
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
        stage_coarse(h, v, cs);
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
