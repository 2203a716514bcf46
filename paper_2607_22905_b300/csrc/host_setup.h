// Host-side symbolic setup of AlgMortar (Algorithm 1, everything before the numeric
// factorisation): CSR validation, graph partition (Sec. 3.1), permutation, interface
// edge sets E_ij (Eq. E), supernodal layout of the local factors, and the index
// tables the device kernels read.  Pure C++; no CUDA types.
#pragma once

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <string>
#include <thread>
#include <vector>

#include "snode_stream.h"
#include "tile.h"

namespace am {

// Runs f(i, t) for every i in [0, n) on up to 16 threads (t = thread index, for per-
// thread scratch), taking indices in chunks from a shared counter.  Every i must write
// only its own outputs, so the result does not depend on the schedule.  If threads cannot
// be started, the calling thread runs everything.
template <typename F>
void parallel_for(int64_t n, int64_t chunk, F f) {
    const unsigned hw = std::thread::hardware_concurrency();
    const int64_t T = std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(hw == 0 ? 1 : hw, 16),
                                                             (n + chunk - 1) / std::max<int64_t>(chunk, 1)));
    std::atomic<int64_t> next{0};
    auto run = [&](int64_t t) {
        for (;;) {
            const int64_t i0 = next.fetch_add(chunk);
            if (i0 >= n) return;
            const int64_t i1 = std::min(n, i0 + chunk);
            for (int64_t i = i0; i < i1; ++i) f(i, t);
        }
    };
    std::vector<std::thread> pool;
    try {
        for (int64_t t = 1; t < T; ++t) pool.emplace_back(run, t);
    } catch (...) {   // fewer threads: the counter hands their indices to the others
    }
    run(0);
    for (auto& th : pool) th.join();
}

struct HostCsr {
    int64_t n = 0, nnz = 0;
    const int32_t* rowptr = nullptr;
    const int32_t* col = nullptr;
    const double* val = nullptr;
};

// Adjacency graph G(A): off-diagonal nonzeros, neighbours ascending (Sec. 3.1).
struct Graph {
    int32_t n = 0;
    std::vector<int64_t> ptr;
    std::vector<int32_t> adj;
};

// Status codes mirror include/algmortar.h.
int validate_csr(const HostCsr& A, std::string& err);
Graph adjacency(const HostCsr& A);
// Recursive BFS bisection with target sizes (larger-first even split when sizes empty).
int partition_graph(const Graph& G, int32_t m, const int32_t* sizes, std::vector<int32_t>& part,
                    std::string& err);

// Supernodal layout of one subdomain's factor (snode_plan.cpp): nested-dissection order,
// supernodes J = local rows [c0[J], c0[J] + w[J]) in postorder, row structures R[J]
// (local rows below the block, ascending), the supernodal elimination tree, levels
// (height above the leaves) and the numeric updates J <- K (rows [a, b) of R[K] in J).
struct SnUpd {
    int32_t K, a, b;
};
struct SnLocal {
    std::vector<int32_t> order;        // local position -> old local id
    std::vector<int32_t> c0, w, parent, lev;
    std::vector<std::vector<int32_t>> R;
    std::vector<std::vector<SnUpd>> upd;
    int32_t nlev = 0;
};
void sn_local_plan(int32_t n, const std::vector<int64_t>& ptr, const std::vector<int32_t>& adj, SnLocal& out);

// Everything the device needs, built from A and a partition.
struct Plan {
    int64_t n = 0;
    int32_t m = 0;
    std::vector<int32_t> part;          // original row -> subdomain
    std::vector<int32_t> perm;          // internal row -> original row
    std::vector<int32_t> iperm;         // original row -> internal row
    std::vector<int64_t> sub_off;       // m + 1: rows of subdomain i = [sub_off[i], sub_off[i+1])
    // permuted matrix (internal ordering), columns ascending
    std::vector<int32_t> p_rowptr, p_col;
    std::vector<double> p_val;
    std::vector<int64_t> p_src;         // p_val[t] = A.val[p_src[t]] (for value updates)
    std::vector<int32_t> row_sub;       // internal row -> subdomain
    // sliced ELL copy of the permuted matrix for the SpMV: slices of 32 rows, width =
    // longest row of the slice, column-major inside the slice; padding has src = -1
    std::vector<int64_t> ell_ptr;       // nslices + 1 element offsets
    std::vector<int32_t> ell_col;       // column (internal), padding -> the row itself
    std::vector<int32_t> ell_src;       // index into the ORIGINAL CSR values, or -1
    // supernodal local factors (global supernode index J over all subdomains)
    std::vector<int32_t> sn_off;        // m + 1: supernodes of subdomain s
    std::vector<int32_t> sn_c0, sn_w, sn_nr;   // first local row, width, |R_J|
    std::vector<int64_t> sn_roff;       // R_J at sn_rows[sn_roff[J] ..)
    std::vector<uint16_t> sn_rows;      // local rows of the R_J
    std::vector<int64_t> sn_poff;       // panel L_{R_J,J}: |R_J| w entries at sn_poff[J]
    std::vector<int64_t> sn_doff;       // inverse diagonal block: w (w + 1) / 2 entries at sn_doff[J]
    std::vector<int64_t> sn_foff;       // factorisation front (w + |R_J|) x w at sn_foff[J]
    std::vector<int64_t> sn_upd_ptr;    // updates J <- K: [sn_upd_ptr[J], sn_upd_ptr[J+1])
    std::vector<int32_t> sn_upd;        // 3 per update: K (global), a, b
    int64_t panel_entries = 0, diag_entries = 0, front_entries = 0;
    std::vector<int32_t> sub_nlev;      // per subdomain: levels
    std::vector<int32_t> sub_lev0;      // per subdomain: first global level
    std::vector<int32_t> lev_du;        // global level + 1 entries: units [lev_du[l], lev_du[l+1])
    std::vector<uint8_t> lev_multi;     // per global level: a supernode of the level is wider than 32
    std::vector<uint32_t> du_list;      // units: (J local << 10) | 32-row chunk
    // forward sweep: row k (internal) receives, for every descendant K with k in R_K, the
    // product of K's panel row for k with x_K; fwd_desc[2 t] = offset of that panel row,
    // fwd_desc[2 t + 1] = c0_K | w_K << 16, for t in [fwd_ptr[k], fwd_ptr[k+1]), K ascending
    std::vector<int32_t> fwd_ptr;       // n + 1
    std::vector<uint32_t> fwd_desc;
    int32_t max_nlev = 0;
    // interfaces (Sec. 3.1 / 5.5): one mortar unknown per pair i < j, lexicographic
    int32_t n_lambda = 0;
    int64_t n_edges = 0;
    std::vector<int32_t> pairs;         // 2 * n_lambda
    std::vector<double> T;              // T_I = sum_{(k,l) in E_I} |a_kl|
    // restriction: b_eta[I] = sum_t rcoef[t] * pbar[rcell[t]],  t in [r_ptr[I], r_ptr[I+1])
    std::vector<int64_t> r_ptr;
    std::vector<int32_t> r_cell;
    std::vector<double> r_coef;         // = -1/4 G[k, I] = -1/2 c_k^(I)  (> 0)
    std::vector<int64_t> rp_ptr;        // restriction entry t: its CSR positions
    std::vector<int32_t> rp_pos;        //   rp_pos[rp_ptr[t] .. rp_ptr[t+1]) (c_k = sum of those values)
    // per subdomain interface lists I_i and MBF panel layout
    std::vector<int64_t> if_off;        // m + 1 into if_list
    std::vector<int32_t> if_list;       // global interface ids, ascending
    std::vector<int64_t> phi_off;       // m + 1: panel of subdomain i starts at phi_off[i]
                                        // (column-major N_i x k_i)
    // sparse G restricted to each subdomain: (panel index, value 2 c_k^(I)), grouped by
    // subdomain; g_col = local column a, g_row = local row
    std::vector<int64_t> g_off;         // m + 1
    std::vector<int32_t> g_row, g_col;
    std::vector<double> g_val;
    std::vector<int32_t> g_from_r;      // G entry -> restriction entry (g_val = -4 r_coef)
    int32_t max_part = 0, min_part = 0, max_k = 0;
    // one-level nested dissection of the interface system: interfaces whose two
    // subdomains lie in the same group g (a subtree of the partition's bisection tree)
    // are interior to g; the rest form the separator.  ND position order: interiors of
    // group 0..G-1, then the separator.
    int32_t nd_G = 1;
    std::vector<int32_t> nd_pos;        // interface id -> ND position
    std::vector<int32_t> nd_id;         // ND position -> interface id
    std::vector<int64_t> nd_goff;       // G + 1: interior of g = positions [goff[g], goff[g+1])
    int32_t nd_nsep = 0;                // separator = positions [goff[G], goff[G] + nsep)
    std::vector<int64_t> nd_aoff;       // G + 1 into nd_alist
    std::vector<int32_t> nd_alist;      // separator-local indices adjacent to group g, ascending
    std::vector<int32_t> nd_sg;         // 2 * nsep: the two groups of separator s (g1 < g2)
    std::vector<int32_t> nd_sidx;       // 2 * nsep: index of s in A_{g1}, A_{g2}
};

int build_plan(const HostCsr& A, const std::vector<int32_t>& part, int32_t m, Plan& P,
               std::string& err);

// Record streams of the batched local solves (snode_stream.h) for CTAs of nw warps and
// factor entries of elem bytes: headers and index lists (entries zero, written on the
// device from the numeric factor by the fill descriptors).  Warp w of subdomain s reads
// bytes [woff[s nw + w], woff[s nw + w + 1]); every warp stream of s holds nbar[s]
// barriers.
struct SnStream {
    int nw = 0, elem = 0;
    std::vector<uint8_t> bytes;
    std::vector<int64_t> woff;
    std::vector<int32_t> nbar;
    std::vector<SnFill> fill;
    int32_t max_record = 0;             // largest record (bytes)
};
int build_sn_stream(const Plan& P, int nw, int elem, SnStream& out, std::string& err);

// Nested-dissection layout of the interface system (fills the nd_* fields of P).
// depth < 0 chooses it from the interface count (interior blocks of ~1000 unknowns).
void plan_interface_nd(Plan& P, int depth);

}  // namespace am
