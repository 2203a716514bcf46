// Host-side symbolic setup of AlgMortar (Algorithm 1, everything before the numeric
// factorisation): CSR validation, graph partition (Sec. 3.1), permutation, interface
// edge sets E_ij (Eq. E), tile-profile layout of the local factors, and the index
// tables the device kernels read.  Pure C++; no CUDA types.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "tile.h"

namespace am {

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
    // tile profile of each local factor
    std::vector<int32_t> ntiles;        // per subdomain
    std::vector<int64_t> trow_off;      // m + 1: tile-row descriptors of subdomain i start here
    std::vector<int32_t> t_lo;          // per tile row (fwd): first tile column
    std::vector<int64_t> t_fwd;         // per tile row: tile offset of (I, lo) in the fwd stream
    std::vector<int32_t> t_hi;          // per tile row (bwd, indexed by I): last tile row below
    std::vector<int64_t> t_bwd;         // per tile row I: tile offset of its bwd step
    std::vector<int64_t> tile_base;     // m + 1: first tile of subdomain i (both streams)
    int64_t total_tiles = 0;
    int32_t max_tiles = 0;
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
    // interface system layout: RCM order of the interface graph and its tile profile
    std::vector<int32_t> s_perm;        // s_perm[pos] = interface id
    std::vector<int32_t> s_iperm;       // interface id -> pos
    int32_t s_ntiles = 0;
    std::vector<int32_t> s_lo, s_hi;
    std::vector<int64_t> s_fwd, s_bwd;
    int64_t s_tiles = 0;
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

// Nested-dissection layout of the interface system (fills the nd_* fields of P).
// depth < 0 chooses it from the interface count (interior blocks of ~1000 unknowns).
void plan_interface_nd(Plan& P, int depth);

// Tile-profile descriptors for a symmetric pattern given as local adjacency lists.
void tile_profile(int32_t n, const std::vector<int64_t>& ptr, const std::vector<int32_t>& adj,
                  int32_t& ntiles, std::vector<int32_t>& lo, std::vector<int32_t>& hi,
                  std::vector<int64_t>& fwd, std::vector<int64_t>& bwd, int64_t& tiles);

// Reverse Cuthill-McKee order (local ids) of a graph given by local adjacency lists.
std::vector<int32_t> rcm_order(int32_t n, const std::vector<int64_t>& ptr,
                               const std::vector<int32_t>& adj);

}  // namespace am
