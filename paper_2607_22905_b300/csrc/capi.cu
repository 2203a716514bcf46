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
struct NumWs {
    bool ready = false;
    int njobs_mbf = 0;
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
    double *gwork = nullptr, *gdinv = nullptr, *gf = nullptr, *gb = nullptr, *gE = nullptr, *RHS = nullptr;
    int32_t *d_gjob = nullptr, *d_gjt0 = nullptr, *d_cjt0 = nullptr;
    int64_t *d_gjin = nullptr, *d_wjin = nullptr;
    int32_t* d_wjob = nullptr;
    int njobs_g = 0, njobs_w = 0;
    int32_t *d_colitem = nullptr, *d_cola = nullptr;
    int64_t ncols_w = 0;
    int64_t *d_doff = nullptr, *d_entbase = nullptr;
    int32_t* d_entg = nullptr;
    int64_t nent = 0;
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
    // local factor profile and streams
    Profile pf{};
    int32_t *d_rows = nullptr, *d_ntiles = nullptr;
    void *d_fwdS = nullptr, *d_bwdS = nullptr;
    double *d_dloc = nullptr, *d_sc = nullptr;
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
    double* d_P = nullptr;             // sum_g a_g partial products
    double* d_nat = nullptr;           // natural-order staging (stage outputs)
    // workspace
    double *d_x = nullptr, *d_r = nullptr, *d_z = nullptr, *d_p = nullptr, *d_q = nullptr, *d_pbar = nullptr;
    double *d_beta = nullptr, *d_eta = nullptr, *d_b = nullptr, *d_t = nullptr;
    GridSum gs{};                      // partials + ticket of the deterministic grid sums
    double* d_scalar = nullptr;
    PcgScalars* d_pcg = nullptr;
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
    cudaGraphExec_t graph = nullptr;
    int64_t graph_kernels = 0;         // kernels in one replay of the iteration graph
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
        if (graph) cudaGraphExecDestroy(graph);
        for (void* p : allocs)
            if (p) cudaFree(p);
        if (own_st) cudaStreamDestroy(own_st);
        delete ws;
    }
};

namespace {

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
    h->d_phi = std::is_same<TS, double>::value ? (void*)W.phi64 : (void*)h->alloc<TS>(nphi);
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
        std::vector<int32_t> irows, int_, ilo, ihi, titem, tI, tJ, gjob, gjt0, wjob, colitem, cola, entg, row_g,
            prow_g;
        std::vector<int64_t> irow0, ibase, ifwd, ibwd, isrc, gjin, wjin, gioff(G, 0), woff(G, 0), doff(G, 0),
            entbase(G, 0);
        int64_t trow = 0, tb = 0, gi = 0, wo = 0, dof = 0, ent = 0;
        for (int g = 0; g < G; ++g) {
            const int64_t ng = P.nd_goff[g + 1] - P.nd_goff[g], ag = P.nd_aoff[g + 1] - P.nd_aoff[g];
            gioff[g] = gi;
            woff[g] = wo;
            doff[g] = dof;
            entbase[g] = ent;
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
                for (int64_t c = 0; c < ag; ++c) {
                    wjob.push_back(it);
                    wjin.push_back(wo + c * ng);
                    colitem.push_back(g);
                    cola.push_back((int32_t)c);
                }
                for (int64_t e = 0; e < ag * ag; ++e) entg.push_back(g);
            }
            gi += ng * ng;
            wo += ng * ag;
            dof += ag * ag;
            ent += (ng > 0) ? ag * ag : 0;
        }
        W.nitems = (int)irows.size();
        W.ntiles_items = tb;
        W.trows_items = trow;
        W.njobs_g = (int)gjob.size();
        W.njobs_w = (int)wjob.size();
        W.ncols_w = (int64_t)colitem.size();
        W.nent = (int64_t)entg.size();
        // entries of groups without interior rows contribute nothing: rebase ent indices
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
        TRY(upload(h, W.d_wjob, wjob));
        TRY(upload(h, W.d_wjin, wjin));
        TRY(upload(h, W.d_colitem, colitem));
        TRY(upload(h, W.d_cola, cola));
        TRY(upload(h, W.d_entg, entg));
        // ent_base must index the compacted entry list: recompute from entg
        {
            std::vector<int64_t> eb(G, 0);
            int64_t o = 0;
            for (int g = 0; g < G; ++g) {
                eb[g] = o;
                const int64_t ng = P.nd_goff[g + 1] - P.nd_goff[g], ag = P.nd_aoff[g + 1] - P.nd_aoff[g];
                if (ng > 0) o += ag * ag;
            }
            TRY(upload(h, W.d_entbase, eb));
        }
        TRY(upload(h, W.d_doff, doff));
        W.gwork = h->alloc<double>((size_t)std::max<int64_t>(tb, 1) * TILE2);
        W.gdinv = h->alloc<double>((size_t)std::max<int64_t>(trow, 1) * TILE2);
        W.gf = h->alloc<double>((size_t)std::max<int64_t>(tb, 1) * TILE2);
        W.gb = h->alloc<double>((size_t)std::max<int64_t>(tb, 1) * TILE2);
        W.gE = h->alloc<double>((size_t)std::max<int64_t>(gi, 1));
        W.RHS = h->alloc<double>((size_t)std::max<int64_t>(wo, 1));
        W.D = h->alloc<double>((size_t)std::max<int64_t>(dof, 1));
        double* Ginv = h->alloc<double>((size_t)std::max<int64_t>(gi, 1));
        double* Wcm = h->alloc<double>((size_t)std::max<int64_t>(wo, 1));
        double* Wrm = h->alloc<double>((size_t)std::max<int64_t>(wo, 1));
        if (!W.gwork || !W.gdinv || !W.gf || !W.gb || !W.gE || !W.RHS || !W.D || !Ginv || !Wcm || !Wrm)
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
        h->d_P = h->alloc<double>((size_t)std::max<int64_t>(P.nd_aoff[G], 1));
        h->d_nat = h->alloc<double>((size_t)L);
        if (!h->d_P || !h->d_nat) return fail(ALGMORTAR_OOM, "interface vectors");
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
    launch_local_diag(h->n, h->d_rowptr, h->d_col, h->d_val, h->d_row_sub, h->opts.diag_scale, h->d_dloc, h->d_sc, st);
    launch_scatter_local<TW>(h->n, h->d_rowptr, h->d_col, h->d_val, h->d_row_sub, h->d_sub_off, h->pf, h->d_dloc,
                             h->d_sc, work, m, st);
    launch_tile_chol<TW>(m, h->pf, h->d_job_sub, work, dinv, W.d_err, st);
    CU(cudaGetLastError());
    TRY(read_err_flag(h, W.d_err, "local"));
    launch_finalize<TW, TS>(m, h->pf, work, dinv, (TS*)h->d_fwdS, (TS*)h->d_bwdS, st);
    CU(cudaGetLastError());
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
        a.scale_off = h->d_sub_off;
        a.job_sub = W.d_js;
        a.job_in = W.d_jo;
        a.job_out = W.d_jo;
        a.in = W.rhs;
        a.out = W.phi64;
        a.alpha = 1.0;
        a.done = nullptr;
        a.err = h->d_kerr;
        CU((launch_tile_solve<TS, TA>(a, W.njobs_mbf, P.max_tiles, st)));
    }
    if (!std::is_same<TS, double>::value) launch_convert<TS>(nphi, W.phi64, (TS*)h->d_phi, st);
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
        for (int it = 0; it < W.nitems; ++it) {
            const int64_t r0 = W.item_row0[it], b0 = W.item_base[it];
            launch_rl_cholesky<double>((int)W.item_hi[it].size(), W.d_ilo + r0, W.d_ifwd + r0, W.item_hi[it].data(),
                                       W.gwork + b0 * TILE2, W.gdinv + r0 * TILE2, W.d_err, st);
        }
        CU(cudaGetLastError());
        TRY(read_err_flag(h, W.d_err, "interface (interior block)"));
        launch_finalize<double, double>(W.nitems, gpf, W.gwork, W.gdinv, W.gf, W.gb, st);
        // S_gg^{-1} (identity columns) and W_g = S_gg^{-1} S_{g,A_g}
        launch_nd_rhs(W.ncols_w, L, W.Sd, h->nd.goff, h->nd.aoff, h->nd.alist, sep0, h->nd.woff, W.d_colitem,
                      W.d_cola, W.RHS, st);
        SolveArgs sa{};
        sa.pf = gpf;
        sa.fwdS = W.gf;
        sa.bwdS = W.gb;
        sa.alpha = 1.0;
        sa.err = h->d_kerr;
        sa.job_sub = W.d_gjob;
        sa.job_in = W.d_gjin;
        sa.job_out = W.d_gjin;
        sa.job_t0 = W.d_gjt0;          // lower triangle of S_gg^{-1} only
        sa.in = W.gE;
        sa.out = (double*)h->nd.Ginv;
        CU((launch_tile_solve<double, double>(sa, W.njobs_g, W.max_tiles_items, st)));
        sa.job_t0 = nullptr;
        sa.job_sub = W.d_wjob;
        sa.job_in = W.d_wjin;
        sa.job_out = W.d_wjin;
        sa.in = W.RHS;
        sa.out = (double*)h->nd.Wcm;
        CU((launch_tile_solve<double, double>(sa, W.njobs_w, W.max_tiles_items, st)));
        launch_mirror_lower(h->nd_grows, h->nd.gioff, G, (double*)h->nd.Ginv, st);
        launch_transpose_blocks(h->nd.goff, h->nd.aoff, h->nd.woff, G, h->nd.Wcm, (double*)h->nd.Wrm, st);
        if (nsep > 0) {
            launch_nd_schur_blocks(W.nent, h->nd.goff, h->nd.aoff, h->nd.woff, W.d_doff, W.d_entg, W.d_entbase, W.RHS,
                                   h->nd.Wcm, W.D, st);
            const int64_t ct = (int64_t)W.cT * (W.cT + 1) / 2;
            launch_nd_schur_tiles(ct, L, nsep, sep0, W.Sd, h->nd.sg, h->nd.sidx, h->nd.aoff, W.d_doff, W.D, W.cwork, st);
            CU(cudaMemcpyAsync(W.d_err, err_init, sizeof(err_init), cudaMemcpyHostToDevice, st));
            launch_rl_cholesky<double>(W.cT, W.d_clo, W.d_cfwd, W.c_hi.data(), W.cwork, W.cdinv, W.d_err, st);
            CU(cudaGetLastError());
            TRY(read_err_flag(h, W.d_err, "interface (separator)"));
            Profile cpf{W.d_crows, W.d_cnt, W.d_czero, W.d_czero, W.d_clo, W.d_chi, W.d_cfwd, W.d_cbwd};
            launch_finalize<double, double>(1, cpf, W.cwork, W.cdinv, W.cf, W.cb, st);
            SolveArgs ca{};
            ca.pf = cpf;
            ca.fwdS = W.cf;
            ca.bwdS = W.cb;
            ca.alpha = 1.0;
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

// Stages of Algorithm 2 on internal-order vectors.
// Local particular solutions pbar_i = A_i^{-1} r_i for all subdomains (one launch).
template <typename TS, typename TA>
int stage_local(algmortar_t* h, const double* r, const int32_t* done) {
    SolveArgs a{};
    a.pf = h->pf;
    a.fwdS = h->d_fwdS;
    a.bwdS = h->d_bwdS;
    a.scale = h->d_sc;
    a.scale_off = h->d_sub_off;
    a.job_sub = h->d_job_sub;
    a.job_in = h->d_job_off;
    a.job_out = h->d_job_off;
    a.in = r;
    a.out = h->d_pbar;
    a.alpha = 1.0;
    a.done = done;
    a.err = h->d_kerr;
    CU((launch_tile_solve<TS, TA>(a, h->m, h->P.max_tiles, h->st)));
    return 0;
}

// Interface right-hand side and interface solve: b_eta from pbar, eta = S^{-1} b_eta.
void stage_restrict(algmortar_t* h, const int32_t* done) {
    launch_restrict(h->L, h->d_rptr, h->d_rcell, h->d_rcoef, h->d_pbar, h->d_beta, h->d_ndpos, done, h->st);
}
void stage_coarse(algmortar_t* h, const int32_t* done) {
    if (h->L > 0) launch_nd_solve(h->nd, h->d_beta, h->d_eta, h->d_P, done, h->st);
}

// z = pbar + Phi eta, and r . z into *rz when rz is given.
template <typename TS>
void stage_prolong(algmortar_t* h, const double* r, double* z, const int32_t* done, double* rz) {
    launch_prolong<TS>(h->n, h->d_row_sub, h->d_sub_off, h->d_if_off, h->L > 0 ? h->d_ifpos : h->d_if_list,
                       h->d_phi_off, (const TS*)h->d_phi, h->d_eta, h->d_pbar, z, r, h->gs, rz, done, h->st);
}

template <typename TS, typename TA>
int apply_t(algmortar_t* h, const double* r, double* z, const int32_t* done, double* rz) {
    TRY((stage_local<TS, TA>(h, r, done)));
    stage_restrict(h, done);
    stage_coarse(h, done);
    stage_prolong<TS>(h, r, z, done, rz);
    CU(cudaGetLastError());
    return 0;
}

int apply_internal(algmortar_t* h, const double* r, double* z, const int32_t* done, double* rz) {
    switch (h->opts.precision) {
        case ALGMORTAR_FP64: return apply_t<double, double>(h, r, z, done, rz);
        case ALGMORTAR_FP32: return apply_t<float, float>(h, r, z, done, rz);
        default: return apply_t<__nv_bfloat16, float>(h, r, z, done, rz);
    }
}

int pcg_iteration(algmortar_t* h) {
    cudaStream_t st = h->st;
    const int32_t* done = &h->d_pcg->done;
    launch_pcg_p(h->n, h->d_z, h->d_p, h->d_pcg, st);
    launch_pcg_spmv_ell(h->n, h->d_ell_ptr, h->d_ell_col, h->d_ell_val, h->d_p, h->d_q, h->d_pcg, h->gs, st);
    launch_pcg_xr(h->n, h->d_x, h->d_r, h->d_p, h->d_q, h->d_pcg, h->gs, st);
    launch_pcg_check(h->d_pcg, st);
    return apply_internal(h, h->d_r, h->d_z, done, &h->d_pcg->rz_next);
}

int ensure_graph(algmortar_t* h) {
    if (h->graph) return 0;
    cudaGraph_t g = nullptr;
    CU(cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal));
    const int64_t c0 = launch_count();
    int rc = pcg_iteration(h);
    cudaError_t e = cudaStreamEndCapture(h->st, &g);
    h->graph_kernels = launch_count() - c0;
    add_launches(-h->graph_kernels);   // captured, not executed
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(ALGMORTAR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        h->graph = nullptr;
        return fail(ALGMORTAR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    return 0;
}

// PCG in the internal ordering on h->d_b -> h->d_x.
int pcg_internal(algmortar_t* h, double tol, algmortar_stats* stt) {
    cudaStream_t st = h->st;
    double t0 = now_ms();
    if (!(tol > 0.0)) return fail(ALGMORTAR_INVALID_ARG, "tol must be positive");
    if (h->opts.use_graph) TRY(ensure_graph(h));
    launch_pcg_init(h->n, h->d_b, h->d_x, h->d_r, h->d_pcg, h->gs, tol, h->opts.max_it, st);
    TRY(apply_internal(h, h->d_r, h->d_z, &h->d_pcg->done, &h->d_pcg->rz_next));
    PcgScalars hs{};
    int restarts = 0;
    const int every = h->opts.check_every > 0 ? h->opts.check_every : 1;
    double true_rel = 0.0;
    for (;;) {
        for (int c = 0; c < every; ++c) {
            if (h->graph) {
                CU(cudaGraphLaunch(h->graph, st));
                add_launches(h->graph_kernels);
            } else {
                TRY(pcg_iteration(h));
            }
        }
        CU(cudaMemcpyAsync(&hs, h->d_pcg, sizeof(hs), cudaMemcpyDeviceToHost, st));
        CU(cudaStreamSynchronize(st));
        if (!hs.done) continue;
        launch_residual(h->n, h->d_rowptr, h->d_col, h->d_val, h->d_x, h->d_b, h->d_pcg, h->gs, st);
        double res2 = 0.0;
        CU(cudaMemcpyAsync(&res2, &h->d_pcg->res2, sizeof(double), cudaMemcpyDeviceToHost, st));
        CU(cudaStreamSynchronize(st));
        true_rel = hs.bb > 0 ? std::sqrt(res2 / hs.bb) : 0.0;
        if (hs.status == 0 && hs.bb > 0 && !(true_rel <= tol) && restarts < 8 && hs.iter < hs.max_it) {
            // recurrence converged but the true residual does not confirm it: continue
            ++restarts;
            int zero = 0;
            CU(cudaMemcpyAsync(&h->d_pcg->done, &zero, sizeof(int), cudaMemcpyHostToDevice, st));
            CU(cudaStreamSynchronize(st));
            continue;
        }
        break;
    }
    int status = hs.status == 0 ? (true_rel <= tol || hs.bb == 0 ? ALGMORTAR_OK : ALGMORTAR_NO_CONVERGENCE)
                                : (hs.status == 5 ? ALGMORTAR_NO_CONVERGENCE : ALGMORTAR_BREAKDOWN);
    if (stt) {
        stt->status = status;
        stt->iterations = hs.iter;
        stt->rel_residual = true_rel;
        stt->recursive_residual = hs.bb > 0 ? std::sqrt(hs.rr / hs.bb) : 0.0;
        stt->solve_ms = now_ms() - t0;
        stt->host_ms = 0.0;
    }
    if (status == ALGMORTAR_NO_CONVERGENCE) g_err = "PCG reached max_it or the true residual did not confirm";
    if (status == ALGMORTAR_BREAKDOWN) g_err = "PCG breakdown: p^T A p <= 0 or non-finite scalar";
    return status;
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
    const int np = vec_blocks(P.n);
    h->d_dloc = h->alloc<double>(n);
    h->d_sc = h->alloc<double>(n);
    h->d_x = h->alloc<double>(n);
    h->d_r = h->alloc<double>(n);
    h->d_z = h->alloc<double>(n);
    h->d_p = h->alloc<double>(n);
    h->d_q = h->alloc<double>(n);
    h->d_pbar = h->alloc<double>(n);
    h->d_b = h->alloc<double>(n);
    h->d_t = h->alloc<double>(n);
    h->d_beta = h->alloc<double>(h->L);
    h->d_eta = h->alloc<double>(h->L);
    h->gs.part = h->alloc<double>(np);
    h->gs.ticket = h->alloc<unsigned int>(1);
    h->d_scalar = h->alloc<double>(4);
    h->d_pcg = h->alloc<PcgScalars>(1);
    h->d_kerr = h->alloc<int>(1);
    if (!h->d_dloc || !h->d_sc || !h->d_x || !h->d_r || !h->d_z || !h->d_p || !h->d_q || !h->d_pbar || !h->d_b ||
        !h->d_t || !h->d_beta || !h->d_eta || !h->gs.part || !h->gs.ticket ||
        !h->d_scalar || !h->d_pcg || !h->d_kerr)
        return bail(fail(ALGMORTAR_OOM, "workspace"));
    if (cudaMemsetAsync(h->d_p, 0, n * sizeof(double), h->st) != cudaSuccess ||
        cudaMemsetAsync(h->d_pcg, 0, sizeof(PcgScalars), h->st) != cudaSuccess ||
        cudaMemsetAsync(h->d_kerr, 0, sizeof(int), h->st) != cudaSuccess ||
        cudaMemsetAsync(h->gs.ticket, 0, sizeof(unsigned int), h->st) != cudaSuccess)
        return bail(fail(ALGMORTAR_CUDA, "memset"));
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
    launch_gather(h->n, h->d_perm, r_dev, h->d_t, h->st);
    TRY(apply_internal(h, h->d_t, h->d_z, nullptr, nullptr));
    launch_scatter(h->n, h->d_perm, h->d_z, z_dev, h->st);
    CU(cudaGetLastError());
    return 0;
}

int algmortar_apply_stages(algmortar_t* h, const double* r_dev, double* pbar_dev, double* beta_dev,
                           double* eta_dev, double* z_dev) {
    if (!h || !r_dev || !pbar_dev || !z_dev || (h->L > 0 && (!beta_dev || !eta_dev)))
        return fail(ALGMORTAR_INVALID_ARG, "null argument");
    CU(cudaSetDevice(h->device));
    launch_gather(h->n, h->d_perm, r_dev, h->d_t, h->st);
    TRY(apply_internal(h, h->d_t, h->d_z, nullptr, nullptr));
    CU(cudaMemcpyAsync(pbar_dev, h->d_pbar, h->n * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    if (h->L > 0) {
        // ND order inside the handle -> natural interface order
        launch_gather(h->L, h->d_ndpos, h->d_beta, beta_dev, h->st);
        launch_gather(h->L, h->d_ndpos, h->d_eta, eta_dev, h->st);
    }
    CU(cudaMemcpyAsync(z_dev, h->d_z, h->n * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    return 0;
}

int algmortar_pcg_solve(algmortar_t* h, const double* b_dev, double* x_dev, double tol, algmortar_stats* st) {
    if (!h || !b_dev || !x_dev) return fail(ALGMORTAR_INVALID_ARG, "null argument");
    CU(cudaSetDevice(h->device));
    launch_gather(h->n, h->d_perm, b_dev, h->d_b, h->st);
    int rc = pcg_internal(h, tol, st);
    if (rc != ALGMORTAR_OK && rc != ALGMORTAR_NO_CONVERGENCE && rc != ALGMORTAR_BREAKDOWN) return rc;
    launch_scatter(h->n, h->d_perm, h->d_x, x_dev, h->st);
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(h->st));
    return rc;
}

int algmortar_pcg_solve_host(algmortar_t* h, const double* b_host, double* x_host, double tol,
                             algmortar_stats* st) {
    if (!h || !b_host || !x_host) return fail(ALGMORTAR_INVALID_ARG, "null argument");
    CU(cudaSetDevice(h->device));
    double t0 = now_ms();
    CU(cudaMemcpyAsync(h->d_t, b_host, h->n * sizeof(double), cudaMemcpyHostToDevice, h->st));
    launch_gather(h->n, h->d_perm, h->d_t, h->d_b, h->st);
    int rc = pcg_internal(h, tol, st);
    if (rc != ALGMORTAR_OK && rc != ALGMORTAR_NO_CONVERGENCE && rc != ALGMORTAR_BREAKDOWN) return rc;
    launch_scatter(h->n, h->d_perm, h->d_x, h->d_t, h->st);
    CU(cudaMemcpyAsync(x_host, h->d_t, h->n * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CU(cudaStreamSynchronize(h->st));
    if (st) st->solve_ms = now_ms() - t0;
    return rc;
}

int algmortar_pcg_solve_multi(algmortar_t* h, const double* B_dev, double* X_dev, int32_t nrhs, int64_t ld,
                              double tol, algmortar_stats* st) {
    if (!h || !B_dev || !X_dev || nrhs <= 0 || ld < h->n) return fail(ALGMORTAR_INVALID_ARG, "bad argument");
    int worst = 0;
    for (int j = 0; j < nrhs; ++j) {
        int rc = algmortar_pcg_solve(h, B_dev + j * ld, X_dev + j * ld, tol, st ? st + j : nullptr);
        if (rc != ALGMORTAR_OK && rc != ALGMORTAR_NO_CONVERGENCE && rc != ALGMORTAR_BREAKDOWN) return rc;
        if (rc > worst) worst = rc;
    }
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
    double* buf[5] = {h->d_x, h->d_r, h->d_z, h->d_p, h->d_q};
    const double* src[5] = {K_dev, tb_dev, tbp_dev, p_dev, lam_dev};
    for (int i = 0; i < 5; ++i) launch_gather(n, h->d_perm, src[i], buf[i], h->st);
    launch_tpfa_grad(n, h->d_rowptr, h->d_col, h->d_val, buf[0], buf[1], buf[2], buf[3], buf[4], h->d_t, h->st);
    launch_scatter(n, h->d_perm, h->d_t, grad_dev, h->st);
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
    PcgScalars saved;
    CU(cudaMemcpyAsync(&saved, h->d_pcg, sizeof(saved), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    // a live scalar state: not done, beta/alpha finite, so no kernel exits early
    PcgScalars live = saved;
    live.done = 0;
    live.iter = 1;
    live.max_it = 1 << 30;
    live.rz = saved.rz != 0.0 ? saved.rz : 1.0;
    live.tol2 = 0.0;
    cudaEvent_t ev[8];
    for (auto& e : ev) CU(cudaEventCreate(&e));
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int it = 0; it <= reps; ++it) {
        CU(cudaMemcpyAsync(h->d_pcg, &live, sizeof(live), cudaMemcpyHostToDevice, st));
        cudaEventRecord(ev[0], st);
        launch_pcg_spmv_ell(h->n, h->d_ell_ptr, h->d_ell_col, h->d_ell_val, h->d_p, h->d_q, h->d_pcg, h->gs, st);
        cudaEventRecord(ev[1], st);
        launch_pcg_p(h->n, h->d_z, h->d_p, h->d_pcg, st);
        launch_pcg_xr(h->n, h->d_x, h->d_r, h->d_p, h->d_q, h->d_pcg, h->gs, st);
        cudaEventRecord(ev[2], st);
        // stages of Algorithm 2 (same launches as apply_internal, timed one by one)
        switch (h->opts.precision) {
            case ALGMORTAR_FP64: TRY((stage_local<double, double>(h, h->d_r, nullptr))); break;
            case ALGMORTAR_FP32: TRY((stage_local<float, float>(h, h->d_r, nullptr))); break;
            default: TRY((stage_local<__nv_bfloat16, float>(h, h->d_r, nullptr))); break;
        }
        cudaEventRecord(ev[3], st);
        stage_restrict(h, nullptr);
        cudaEventRecord(ev[4], st);
        stage_coarse(h, nullptr);
        cudaEventRecord(ev[5], st);
        switch (h->opts.precision) {
            case ALGMORTAR_FP64: stage_prolong<double>(h, h->d_r, h->d_z, nullptr, &h->d_pcg->rz_next); break;
            case ALGMORTAR_FP32: stage_prolong<float>(h, h->d_r, h->d_z, nullptr, &h->d_pcg->rz_next); break;
            default: stage_prolong<__nv_bfloat16>(h, h->d_r, h->d_z, nullptr, &h->d_pcg->rz_next); break;
        }
        cudaEventRecord(ev[6], st);
        CU(cudaMemcpyAsync(h->d_pcg, &live, sizeof(live), cudaMemcpyHostToDevice, st));
        cudaEventRecord(ev[7], st);
        if (h->graph) {
            CU(cudaGraphLaunch(h->graph, st));
            add_launches(h->graph_kernels);
        } else {
            TRY(pcg_iteration(h));
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
    CU(cudaMemcpyAsync(h->d_pcg, &saved, sizeof(saved), cudaMemcpyHostToDevice, st));
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
