// Host-side symbolic setup of AlgMortar: see host_setup.h.
#include "host_setup.h"

#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstdio>
#include <condition_variable>
#include <mutex>
#include <numeric>
#include <thread>

namespace am {

static std::string fmt(const char* f, long long a, long long b = 0, long long c = 0) {
    char buf[256];
    std::snprintf(buf, sizeof(buf), f, a, b, c);
    return buf;
}

namespace {

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

}  // namespace

namespace {

// Row checks of validate_csr: 0, or the status code with err set.
int check_row_structure(const HostCsr& A, int64_t i, std::string& err) {
    const int64_t a = A.rowptr[i], b = A.rowptr[i + 1];
    if (b < a || b > A.nnz) {
        err = fmt("CSR: rowptr decreases or exceeds nnz at row %lld", i);
        return 1;
    }
    bool diag = false;
    for (int64_t t = a; t < b; ++t) {
        const int32_t c = A.col[t];
        if (c < 0 || c >= A.n || (t > a && c <= A.col[t - 1])) {
            err = fmt("CSR: column out of range or not strictly ascending in row %lld", i);
            return 1;
        }
        if (!std::isfinite(A.val[t])) {
            err = fmt("CSR: non-finite value in row %lld", i);
            return 1;
        }
        if (c == i) {
            diag = true;
            if (!(A.val[t] > 0.0)) {
                err = fmt("CSR: non-positive diagonal in row %lld", i);
                return 4;
            }
        }
    }
    if (!diag) {
        err = fmt("CSR: missing diagonal in row %lld", i);
        return 1;
    }
    return 0;
}

// Requires every row to have passed check_row_structure.
int check_row_symmetry(const HostCsr& A, int64_t i, std::string& err) {
    for (int64_t t = A.rowptr[i]; t < A.rowptr[i + 1]; ++t) {
        const int32_t j = A.col[t];
        if (j == i) continue;
        const int32_t* first = A.col + A.rowptr[j];
        const int32_t* last = A.col + A.rowptr[j + 1];
        const int32_t* f = std::lower_bound(first, last, (int32_t)i);
        if (f == last || *f != i || A.val[A.rowptr[j] + (f - first)] != A.val[t]) {
            err = fmt("CSR: a(%lld,%lld) has no equal transposed entry", i, j);
            return 2;
        }
    }
    return 0;
}

// First row (lowest index) for which check(row) fails, or -1; rows are checked in
// parallel blocks, and the reported row is the same as a sequential scan's.
template <typename Check>
int64_t first_failing_row(int64_t n, Check check) {
    constexpr int64_t B = 8192;
    const int64_t nb = (n + B - 1) / B;
    std::vector<int64_t> first(nb, -1);
    parallel_for(nb, 1, [&](int64_t bi, int64_t) {
        std::string e;
        for (int64_t i = bi * B; i < std::min(n, bi * B + B); ++i)
            if (check(i, e)) {
                first[bi] = i;
                return;
            }
    });
    for (int64_t bi = 0; bi < nb; ++bi)
        if (first[bi] >= 0) return first[bi];
    return -1;
}

}  // namespace

int validate_csr(const HostCsr& A, std::string& err) {
    if (A.n <= 0 || !A.rowptr || !A.col || !A.val) {
        err = "CSR: null pointer or n <= 0";
        return 1;
    }
    if (A.n >= INT32_MAX || A.nnz >= INT32_MAX || A.nnz < A.n) {
        err = "CSR: n or nnz outside the int32 range, or fewer entries than rows";
        return 1;
    }
    if (A.rowptr[0] != 0 || (int64_t)A.rowptr[A.n] != A.nnz) {
        err = "CSR: rowptr[0] must be 0 and rowptr[n] must equal nnz";
        return 1;
    }
    int64_t i = first_failing_row(A.n, [&](int64_t r, std::string& e) { return check_row_structure(A, r, e); });
    if (i >= 0) return check_row_structure(A, i, err);
    i = first_failing_row(A.n, [&](int64_t r, std::string& e) { return check_row_symmetry(A, r, e); });
    if (i >= 0) return check_row_symmetry(A, i, err);
    return 0;
}

Graph adjacency(const HostCsr& A) {
    Graph G;
    G.n = (int32_t)A.n;
    G.ptr.assign(A.n + 1, 0);
    parallel_for(A.n, 16384, [&](int64_t i, int64_t) {
        int64_t c = 0;
        for (int64_t t = A.rowptr[i]; t < A.rowptr[i + 1]; ++t)
            if (A.col[t] != i && A.val[t] != 0.0) ++c;
        G.ptr[i + 1] = c;
    });
    for (int64_t i = 0; i < A.n; ++i) G.ptr[i + 1] += G.ptr[i];
    G.adj.resize(G.ptr[A.n]);
    parallel_for(A.n, 16384, [&](int64_t i, int64_t) {
        int64_t o = G.ptr[i];
        for (int64_t t = A.rowptr[i]; t < A.rowptr[i + 1]; ++t)
            if (A.col[t] != i && A.val[t] != 0.0) G.adj[o++] = A.col[t];
    });
    return G;
}

// ------------------------------------------------------------------------------------
// Recursive BFS bisection (the rule stated in oracle/partition.py, implemented anew).
// ------------------------------------------------------------------------------------
namespace {

struct SubsetBfs {
    const Graph& G;
    std::vector<int32_t> loc;     // global -> local index in the current subset, -1 if not
    std::vector<int64_t> lptr;    // induced subgraph of the current subset, local indices,
    std::vector<int32_t> ladj;    //   neighbours in the global (ascending) order
    std::vector<int32_t> dist, q, deg;
    explicit SubsetBfs(const Graph& g) : G(g), loc(g.n, -1) {}

    // BFS from local `s` over the induced subgraph; q receives the visit order, dist the
    // levels (nodes of other components keep -1).  Returns the eccentricity of s.
    int32_t bfs(size_t n, int32_t s) {
        std::fill(dist.begin(), dist.begin() + n, -1);
        q.clear();
        q.push_back(s);
        dist[s] = 0;
        size_t h = 0;
        while (h < q.size()) {
            const int32_t u = q[h++];
            const int32_t du = dist[u] + 1;
            for (int64_t e = lptr[u]; e < lptr[u + 1]; ++e) {
                const int32_t v = ladj[e];
                if (dist[v] < 0) {
                    dist[v] = du;
                    q.push_back(v);
                }
            }
        }
        return dist[q.back()];
    }

    // George-Liu pseudo-peripheral node of the component of local node 0.
    int32_t pseudo_peripheral(size_t n) {
        int32_t v = 0;
        int32_t ecc = bfs(n, v);
        for (;;) {
            int32_t u = -1, best = INT32_MAX;
            for (int32_t x : q)
                if (dist[x] == ecc && (deg[x] < best || (deg[x] == best && x < u))) {
                    u = x;
                    best = deg[x];
                }
            int32_t ecc_u = bfs(n, u);
            if (ecc_u > ecc) {
                v = u;
                ecc = ecc_u;
            } else {
                return v;
            }
        }
    }

    // Full BFS order of the subset (local ids).
    void order(const std::vector<int32_t>& S, std::vector<int32_t>& out) {
        const size_t n = S.size();
        if (dist.size() < n) {
            dist.resize(n);
            deg.resize(n);
        }
        for (size_t t = 0; t < n; ++t) loc[S[t]] = (int32_t)t;
        lptr.resize(n + 1);
        ladj.clear();
        lptr[0] = 0;
        for (size_t t = 0; t < n; ++t) {
            const int32_t g = S[t];
            for (int64_t e = G.ptr[g]; e < G.ptr[g + 1]; ++e) {
                const int32_t v = loc[G.adj[e]];
                if (v >= 0) ladj.push_back(v);
            }
            lptr[t + 1] = (int64_t)ladj.size();
            deg[t] = (int32_t)(lptr[t + 1] - lptr[t]);
        }
        for (size_t t = 0; t < n; ++t) loc[S[t]] = -1;
        std::vector<char> seen(n, 0);
        out.clear();
        int32_t start = pseudo_peripheral(n);
        size_t next = 0;
        for (;;) {
            bfs(n, start);
            for (int32_t x : q) seen[x] = 1;
            out.insert(out.end(), q.begin(), q.end());
            while (next < n && seen[next]) ++next;
            if (next == n) break;
            start = (int32_t)next;
        }
    }
};

}  // namespace

int partition_graph(const Graph& G, int32_t m, const int32_t* sizes_in, std::vector<int32_t>& part,
                    std::string& err) {
    if (m <= 0 || m > G.n) {
        err = "partition: n_parts must be in [1, n]";
        return 1;
    }
    std::vector<int64_t> sizes(m);
    if (sizes_in) {
        int64_t s = 0;
        for (int32_t i = 0; i < m; ++i) {
            if (sizes_in[i] <= 0) {
                err = "partition: part sizes must be positive";
                return 1;
            }
            sizes[i] = sizes_in[i];
            s += sizes_in[i];
        }
        if (s != G.n) {
            err = "partition: part sizes must sum to n";
            return 1;
        }
    } else {
        int64_t base = G.n / m, extra = G.n % m;
        for (int32_t i = 0; i < m; ++i) sizes[i] = base + (i < extra ? 1 : 0);
    }
    std::vector<int64_t> pre(m + 1, 0);
    for (int32_t i = 0; i < m; ++i) pre[i + 1] = pre[i] + sizes[i];
    part.assign(G.n, -1);
    // The two halves of a bisection are independent, so subsets are split by a pool of
    // worker threads (each with its own BFS workspace).  A subset's split depends only on
    // the subset, and leaves label disjoint nodes, so the labels do not depend on the
    // schedule.
    struct Item {
        std::vector<int32_t> S;
        int32_t lo, hi;
    };
    std::vector<Item> work;
    {
        Item it;
        it.S.resize(G.n);
        std::iota(it.S.begin(), it.S.end(), 0);
        it.lo = 0;
        it.hi = m;
        work.push_back(std::move(it));
    }
    std::mutex mu;
    std::condition_variable cv;
    int64_t pending = 1;   // items queued or in progress
    auto worker = [&]() {
        SubsetBfs sb(G);
        std::vector<int32_t> ord;
        for (;;) {
            Item it;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv.wait(lk, [&] { return !work.empty() || pending == 0; });
                if (work.empty()) return;
                it = std::move(work.back());
                work.pop_back();
            }
            const int32_t k = it.hi - it.lo;
            if (k == 1) {
                for (int32_t g : it.S) part[g] = it.lo;
            } else {
                const int32_t k1 = k / 2;
                const int64_t n1 = pre[it.lo + k1] - pre[it.lo];
                sb.order(it.S, ord);
                Item a, b;
                a.S.reserve(n1);
                b.S.reserve(it.S.size() - n1);
                for (size_t t = 0; t < ord.size(); ++t)
                    (t < (size_t)n1 ? a.S : b.S).push_back(it.S[ord[t]]);
                std::sort(a.S.begin(), a.S.end());
                std::sort(b.S.begin(), b.S.end());
                a.lo = it.lo;
                a.hi = it.lo + k1;
                b.lo = it.lo + k1;
                b.hi = it.hi;
                std::lock_guard<std::mutex> lk(mu);
                work.push_back(std::move(b));
                work.push_back(std::move(a));
                pending += 2;
            }
            {
                std::lock_guard<std::mutex> lk(mu);
                --pending;
            }
            cv.notify_all();
        }
    };
    const unsigned hw = std::thread::hardware_concurrency();
    const int nthreads = (int)std::max(1u, std::min(std::min(hw == 0 ? 1u : hw, 16u), (unsigned)m));
    std::vector<std::thread> pool;
    try {
        for (int i = 1; i < nthreads; ++i) pool.emplace_back(worker);
    } catch (...) {   // no threads available: the calling thread does all the work
    }
    worker();
    for (auto& t : pool) t.join();
    return 0;
}

// ------------------------------------------------------------------------------------
// Reverse Cuthill-McKee on a local graph (CUDA path only: orders rows inside a subdomain
// so that the Cholesky factor fits a narrow tile profile).
// ------------------------------------------------------------------------------------
std::vector<int32_t> rcm_order(int32_t n, const std::vector<int64_t>& ptr,
                               const std::vector<int32_t>& adj) {
    std::vector<int32_t> deg(n), dist(n, -1), q, out;
    for (int32_t i = 0; i < n; ++i) deg[i] = (int32_t)(ptr[i + 1] - ptr[i]);
    std::vector<char> seen(n, 0);
    auto bfs_levels = [&](int32_t s) {
        for (int32_t x : q) dist[x] = -1;
        q.clear();
        q.push_back(s);
        dist[s] = 0;
        size_t h = 0;
        while (h < q.size()) {
            int32_t u = q[h++];
            for (int64_t e = ptr[u]; e < ptr[u + 1]; ++e) {
                int32_t v = adj[e];
                if (dist[v] < 0) {
                    dist[v] = dist[u] + 1;
                    q.push_back(v);
                }
            }
        }
        return dist[q.back()];
    };
    std::vector<int32_t> nb;
    int32_t next = 0;
    out.reserve(n);
    while ((int32_t)out.size() < n) {
        while (seen[next]) ++next;
        int32_t v = next, ecc = bfs_levels(v);
        for (;;) {
            int32_t u = -1, best = INT32_MAX;
            for (int32_t x : q)
                if (dist[x] == ecc && (deg[x] < best || (deg[x] == best && x < u))) {
                    u = x;
                    best = deg[x];
                }
            int32_t e2 = bfs_levels(u);
            if (e2 > ecc) {
                v = u;
                ecc = e2;
            } else {
                break;
            }
        }
        for (int32_t x : q) dist[x] = -1;
        q.clear();
        size_t h = out.size();
        out.push_back(v);
        seen[v] = 1;
        while (h < out.size()) {
            int32_t u = out[h++];
            nb.clear();
            for (int64_t e = ptr[u]; e < ptr[u + 1]; ++e)
                if (!seen[adj[e]]) nb.push_back(adj[e]);
            std::sort(nb.begin(), nb.end(), [&](int32_t a, int32_t b) {
                return deg[a] != deg[b] ? deg[a] < deg[b] : a < b;
            });
            for (int32_t x : nb)
                if (!seen[x]) {
                    seen[x] = 1;
                    out.push_back(x);
                }
        }
    }
    std::reverse(out.begin(), out.end());
    return out;
}

// Tile profile of the lower Cholesky factor for a pattern in its final local order.
// Row r's envelope starts at f(r) = min(r, min adj(r)); tile row I starts at tile
// lo(I) = min_{r in I} f(r)/TILE, made non-decreasing by a suffix minimum so that tile
// column I of the factor occupies the contiguous rows I..hi(I).
void tile_profile(int32_t n, const std::vector<int64_t>& ptr, const std::vector<int32_t>& adj,
                  int32_t& ntiles, std::vector<int32_t>& lo, std::vector<int32_t>& hi,
                  std::vector<int64_t>& fwd, std::vector<int64_t>& bwd, int64_t& tiles) {
    ntiles = (n + TILE - 1) / TILE;
    lo.assign(ntiles, 0);
    hi.assign(ntiles, 0);
    fwd.assign(ntiles, 0);
    bwd.assign(ntiles, 0);
    for (int32_t I = 0; I < ntiles; ++I) lo[I] = I;
    for (int32_t r = 0; r < n; ++r) {
        int32_t f = r;
        for (int64_t e = ptr[r]; e < ptr[r + 1]; ++e) f = std::min(f, adj[e]);
        lo[r / TILE] = std::min(lo[r / TILE], f / TILE);
    }
    for (int32_t I = ntiles - 2; I >= 0; --I) lo[I] = std::min(lo[I], lo[I + 1]);
    int32_t J = ntiles - 1;
    for (int32_t I = ntiles - 1; I >= 0; --I) {
        while (J > I && lo[J] > I) --J;
        hi[I] = std::max(J, I);
    }
    int64_t o = 0;
    for (int32_t I = 0; I < ntiles; ++I) {
        fwd[I] = o;
        o += I - lo[I] + 1;
    }
    tiles = o;
    o = 0;
    for (int32_t I = ntiles - 1; I >= 0; --I) {
        bwd[I] = o;
        o += hi[I] - I + 1;
    }
}

// ------------------------------------------------------------------------------------
int build_plan(const HostCsr& A, const std::vector<int32_t>& part, int32_t m, Plan& P,
               std::string& err) {
    const int64_t n = A.n;
    P = Plan();
    P.n = n;
    P.m = m;
    P.part = part;
    std::vector<int64_t> cnt(m + 1, 0);
    for (int64_t i = 0; i < n; ++i) {
        if (part[i] < 0 || part[i] >= m) {
            err = fmt("partition label out of range at row %lld", i);
            return 1;
        }
        cnt[part[i] + 1]++;
    }
    P.sub_off.assign(m + 1, 0);
    for (int32_t i = 0; i < m; ++i) {
        if (cnt[i + 1] == 0) {
            err = fmt("subdomain %lld is empty", i);
            return 1;
        }
        if (cnt[i + 1] > 16384) {
            err = fmt("subdomain %lld has %lld rows (limit 16384)", i, cnt[i + 1]);
            return 9;
        }
        P.sub_off[i + 1] = P.sub_off[i] + cnt[i + 1];
    }
    // nodes of each subdomain in ascending original index
    std::vector<int32_t> nodes(n);
    {
        std::vector<int64_t> pos(P.sub_off.begin(), P.sub_off.end() - 1);
        for (int64_t i = 0; i < n; ++i) nodes[pos[part[i]]++] = (int32_t)i;
    }
    // interface sign check (Sec. 3.2: diagonal of W negative)
    for (int64_t i = 0; i < n; ++i)
        for (int64_t t = A.rowptr[i]; t < A.rowptr[i + 1]; ++t) {
            int32_t j = A.col[t];
            if (part[j] != part[i] && A.val[t] > 0.0) {
                err = fmt("positive coupling a(%lld,%lld) between subdomains", i, j);
                return 3;
            }
        }
    // per subdomain RCM order -> internal ordering, subdomains in parallel (each writes
    // its own ranges of perm / iperm and its own profile)
    P.perm.resize(n);
    P.iperm.assign(n, -1);
    P.ntiles.resize(m);
    P.trow_off.assign(m + 1, 0);
    P.tile_base.assign(m + 1, 0);
    std::vector<std::vector<int32_t>> t_lo(m), t_hi(m);
    std::vector<std::vector<int64_t>> t_fwd(m), t_bwd(m);
    std::vector<int64_t> tiles_of(m, 0);
    parallel_for(m, 1, [&](int64_t si, int64_t) {
        const int32_t s = (int32_t)si;
        const int64_t a = P.sub_off[s], b = P.sub_off[s + 1];
        const int32_t ns = (int32_t)(b - a);
        const int32_t* nb = nodes.data() + a;   // ascending original indices
        std::vector<int64_t> lp(ns + 1, 0);
        std::vector<int32_t> la;
        for (int32_t t = 0; t < ns; ++t) {
            const int32_t g = nb[t];
            for (int64_t e = A.rowptr[g]; e < A.rowptr[g + 1]; ++e) {
                const int32_t c = A.col[e];
                if (c != g && part[c] == s && A.val[e] != 0.0)
                    la.push_back((int32_t)(std::lower_bound(nb, nb + ns, c) - nb));
            }
            lp[t + 1] = (int64_t)la.size();
        }
        std::vector<int32_t> ord = rcm_order(ns, lp, la);
        std::vector<int32_t> inv(ns);
        for (int32_t t = 0; t < ns; ++t) {
            inv[ord[t]] = t;
            P.perm[a + t] = nb[ord[t]];
            P.iperm[nb[ord[t]]] = (int32_t)(a + t);
        }
        // relabel local adjacency into the RCM order for the profile
        std::vector<int64_t> rp(ns + 1, 0);
        std::vector<int32_t> ra(la.size());
        for (int32_t t = 0; t < ns; ++t) rp[t + 1] = rp[t] + (lp[ord[t] + 1] - lp[ord[t]]);
        for (int32_t t = 0; t < ns; ++t) {
            int64_t o = rp[t];
            for (int64_t e = lp[ord[t]]; e < lp[ord[t] + 1]; ++e) ra[o++] = inv[la[e]];
        }
        tile_profile(ns, rp, ra, P.ntiles[s], t_lo[s], t_hi[s], t_fwd[s], t_bwd[s], tiles_of[s]);
    });
    P.max_part = 0;
    P.min_part = INT32_MAX;
    for (int32_t s = 0; s < m; ++s) {
        const int32_t ns = (int32_t)(P.sub_off[s + 1] - P.sub_off[s]);
        P.max_part = std::max(P.max_part, ns);
        P.min_part = std::min(P.min_part, ns);
        P.trow_off[s + 1] = P.trow_off[s] + P.ntiles[s];
        P.tile_base[s + 1] = P.tile_base[s] + tiles_of[s];
        P.max_tiles = std::max(P.max_tiles, P.ntiles[s]);
    }
    P.total_tiles = P.tile_base[m];
    P.t_lo.reserve(P.trow_off[m]);
    for (int32_t s = 0; s < m; ++s) {
        P.t_lo.insert(P.t_lo.end(), t_lo[s].begin(), t_lo[s].end());
        P.t_hi.insert(P.t_hi.end(), t_hi[s].begin(), t_hi[s].end());
        for (auto v : t_fwd[s]) P.t_fwd.push_back(v);
        for (auto v : t_bwd[s]) P.t_bwd.push_back(v);
    }
    // permuted CSR: row lengths first, then the rows in parallel (each its own range)
    P.row_sub.resize(n);
    P.p_rowptr.assign(n + 1, 0);
    P.p_col.resize(A.nnz);
    P.p_val.resize(A.nnz);
    P.p_src.resize(A.nnz);
    for (int64_t k = 0; k < n; ++k) {
        const int32_t g = P.perm[k];
        P.p_rowptr[k + 1] = P.p_rowptr[k] + (A.rowptr[g + 1] - A.rowptr[g]);
    }
    parallel_for(n, 4096, [&](int64_t k, int64_t) {
        const int32_t g = P.perm[k];
        P.row_sub[k] = part[g];
        // (new column, source position), sorted by column: insertion sort of a short row
        std::pair<int32_t, int64_t> buf[64];
        std::vector<std::pair<int32_t, int64_t>> big;
        const int64_t len = A.rowptr[g + 1] - A.rowptr[g];
        std::pair<int32_t, int64_t>* row = buf;
        if (len > 64) {
            big.resize(len);
            row = big.data();
        }
        int64_t c = 0;
        for (int64_t e = A.rowptr[g]; e < A.rowptr[g + 1]; ++e) row[c++] = {P.iperm[A.col[e]], e};
        std::sort(row, row + len);
        int64_t o = P.p_rowptr[k];
        for (int64_t t = 0; t < len; ++t, ++o) {
            P.p_col[o] = row[t].first;
            P.p_val[o] = A.val[row[t].second];
            P.p_src[o] = row[t].second;
        }
    });
    // sliced ELL (32-row slices) of the permuted matrix, slices in parallel
    {
        const int64_t ns = (n + 31) / 32;
        P.ell_ptr.assign(ns + 1, 0);
        parallel_for(ns, 1024, [&](int64_t sl, int64_t) {
            int32_t w = 0;
            for (int64_t k = sl * 32; k < std::min<int64_t>(n, sl * 32 + 32); ++k)
                w = std::max(w, P.p_rowptr[k + 1] - P.p_rowptr[k]);
            P.ell_ptr[sl + 1] = 32 * (int64_t)w;
        });
        for (int64_t sl = 0; sl < ns; ++sl) P.ell_ptr[sl + 1] += P.ell_ptr[sl];
        P.ell_col.assign(P.ell_ptr[ns], 0);
        P.ell_src.assign(P.ell_ptr[ns], -1);
        parallel_for(ns, 1024, [&](int64_t sl, int64_t) {
            const int64_t w = (P.ell_ptr[sl + 1] - P.ell_ptr[sl]) / 32;
            for (int r = 0; r < 32; ++r) {
                const int64_t k = sl * 32 + r;
                for (int64_t e = 0; e < w; ++e) {
                    const int64_t o = P.ell_ptr[sl] + e * 32 + r;
                    if (k < n && e < P.p_rowptr[k + 1] - P.p_rowptr[k]) {
                        P.ell_col[o] = P.p_col[P.p_rowptr[k] + e];
                        P.ell_src[o] = (int32_t)P.p_src[P.p_rowptr[k] + e];
                    } else {
                        P.ell_col[o] = (int32_t)std::min<int64_t>(k, n - 1);
                    }
                }
            }
        });
    }
    // interfaces: one per subdomain pair (i < j) with a coupling, lexicographic
    // (rows in parallel blocks; the blocks' outputs are concatenated in row order, so
    // every list below is the one a sequential scan of the rows produces)
    constexpr int64_t RB = 16384;
    const int64_t nrb = (n + RB - 1) / RB;
    std::vector<int64_t> keys;
    {
        std::vector<std::vector<int64_t>> kb(nrb);
        parallel_for(nrb, 1, [&](int64_t bi, int64_t) {
            for (int64_t k = bi * RB; k < std::min(n, bi * RB + RB); ++k) {
                const int32_t i = P.row_sub[k];
                for (int32_t e = P.p_rowptr[k]; e < P.p_rowptr[k + 1]; ++e) {
                    const int32_t j = P.row_sub[P.p_col[e]];
                    if (i < j && P.p_val[e] != 0.0) kb[bi].push_back((int64_t)i * m + j);
                }
            }
        });
        for (auto& v : kb) keys.insert(keys.end(), v.begin(), v.end());
    }
    P.n_edges = (int64_t)keys.size();
    std::sort(keys.begin(), keys.end());
    keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
    P.n_lambda = (int32_t)keys.size();
    P.pairs.resize(2 * (size_t)P.n_lambda);
    for (int32_t I = 0; I < P.n_lambda; ++I) {
        P.pairs[2 * I] = (int32_t)(keys[I] / m);
        P.pairs[2 * I + 1] = (int32_t)(keys[I] % m);
    }
    auto iface = [&](int32_t i, int32_t j) -> int32_t {
        int64_t key = i < j ? (int64_t)i * m + j : (int64_t)j * m + i;
        return (int32_t)(std::lower_bound(keys.begin(), keys.end(), key) - keys.begin());
    };
    P.T.assign(P.n_lambda, 0.0);
    // per row: c_k^(I) = sum_{l in Omega_j} a_kl for each neighbouring subdomain j
    struct RC {
        int32_t I, cell;
        double c;
        int64_t pos0, npos;   // positions of the row's couplings to the other side
    };
    std::vector<RC> rc;
    std::vector<int32_t> row_pos;     // CSR positions, grouped per (row, interface)
    {
        std::vector<std::vector<RC>> rcb(nrb);
        std::vector<std::vector<int32_t>> posb(nrb);
        parallel_for(nrb, 1, [&](int64_t bi, int64_t) {
            std::vector<std::pair<int32_t, std::vector<int32_t>>> acc;
            std::vector<RC>& R = rcb[bi];
            std::vector<int32_t>& Q = posb[bi];
            for (int64_t k = bi * RB; k < std::min(n, bi * RB + RB); ++k) {
                const int32_t i = P.row_sub[k];
                acc.clear();
                for (int32_t e = P.p_rowptr[k]; e < P.p_rowptr[k + 1]; ++e) {
                    const int32_t l = P.p_col[e];
                    const int32_t j = P.row_sub[l];
                    if (j == i || P.p_val[e] == 0.0) continue;
                    const int32_t I = iface(i, j);
                    bool found = false;
                    for (auto& pr : acc)
                        if (pr.first == I) {
                            pr.second.push_back(e);
                            found = true;
                        }
                    if (!found) acc.push_back({I, std::vector<int32_t>{e}});
                }
                for (auto& pr : acc) {
                    double c = 0.0;
                    for (int32_t e : pr.second) c += P.p_val[e];
                    R.push_back({pr.first, (int32_t)k, c, (int64_t)Q.size(), (int64_t)pr.second.size()});
                    Q.insert(Q.end(), pr.second.begin(), pr.second.end());
                }
            }
        });
        for (int64_t bi = 0; bi < nrb; ++bi) {
            const int64_t base = (int64_t)row_pos.size();
            for (RC x : rcb[bi]) {
                x.pos0 += base;
                rc.push_back(x);
            }
            row_pos.insert(row_pos.end(), posb[bi].begin(), posb[bi].end());
        }
    }
    // restriction table, interface-major; rp_* lists each entry's CSR positions so that
    // the value-dependent coefficients can be recomputed on the device for new values
    std::sort(rc.begin(), rc.end(), [](const RC& a, const RC& b) {
        return a.I != b.I ? a.I < b.I : a.cell < b.cell;
    });
    // T_I = sum |a_kl| over E_I, accumulated from the rows of the lower-numbered subdomain
    // of I in ascending row and column order
    for (const RC& x : rc)
        if (P.row_sub[x.cell] == P.pairs[2 * x.I])
            for (int64_t t = x.pos0; t < x.pos0 + x.npos; ++t) P.T[x.I] += std::fabs(P.p_val[row_pos[t]]);
    P.r_ptr.assign(P.n_lambda + 1, 0);
    P.r_cell.resize(rc.size());
    P.r_coef.resize(rc.size());
    P.rp_ptr.assign(rc.size() + 1, 0);
    P.rp_pos.clear();
    for (size_t t = 0; t < rc.size(); ++t) {
        P.r_ptr[rc[t].I + 1]++;
        P.r_cell[t] = rc[t].cell;
        P.r_coef[t] = -0.5 * rc[t].c;
        P.rp_pos.insert(P.rp_pos.end(), row_pos.begin() + rc[t].pos0, row_pos.begin() + rc[t].pos0 + rc[t].npos);
        P.rp_ptr[t + 1] = (int64_t)P.rp_pos.size();
    }
    for (int32_t I = 0; I < P.n_lambda; ++I) P.r_ptr[I + 1] += P.r_ptr[I];
    // per-subdomain interface lists I_i and the sparse G_i
    P.if_off.assign(m + 1, 0);
    {
        std::vector<std::vector<int32_t>> lists(m);
        for (int32_t I = 0; I < P.n_lambda; ++I) {
            lists[P.pairs[2 * I]].push_back(I);
            lists[P.pairs[2 * I + 1]].push_back(I);
        }
        P.max_k = 0;
        for (int32_t s = 0; s < m; ++s) {
            std::sort(lists[s].begin(), lists[s].end());
            P.if_off[s + 1] = P.if_off[s] + (int64_t)lists[s].size();
            P.if_list.insert(P.if_list.end(), lists[s].begin(), lists[s].end());
            P.max_k = std::max(P.max_k, (int32_t)lists[s].size());
        }
    }
    P.phi_off.assign(m + 1, 0);
    for (int32_t s = 0; s < m; ++s)
        P.phi_off[s + 1] = P.phi_off[s] + (P.sub_off[s + 1] - P.sub_off[s]) * (P.if_off[s + 1] - P.if_off[s]);
    {
        std::vector<std::vector<std::pair<RC, int32_t>>> per(m);
        for (size_t t = 0; t < rc.size(); ++t) per[P.row_sub[rc[t].cell]].push_back({rc[t], (int32_t)t});
        P.g_off.assign(m + 1, 0);
        P.g_from_r.clear();
        for (int32_t s = 0; s < m; ++s) {
            std::sort(per[s].begin(), per[s].end(), [](const std::pair<RC, int32_t>& a, const std::pair<RC, int32_t>& b) {
                return a.first.I != b.first.I ? a.first.I < b.first.I : a.first.cell < b.first.cell;
            });
            for (auto& xr : per[s]) {
                const RC& x = xr.first;
                P.g_from_r.push_back(xr.second);
                auto f = std::lower_bound(P.if_list.begin() + P.if_off[s], P.if_list.begin() + P.if_off[s + 1], x.I);
                P.g_col.push_back((int32_t)(f - (P.if_list.begin() + P.if_off[s])));
                P.g_row.push_back((int32_t)(x.cell - P.sub_off[s]));
                P.g_val.push_back(2.0 * x.c);
            }
            P.g_off[s + 1] = (int64_t)P.g_row.size();
        }
    }
    plan_interface_nd(P, -1);
    return 0;
}

// Groups = nodes at depth D of the bisection tree over part ids (the partitioner gives the
// first k/2 of k parts to one side, so every subtree is a contiguous id range).
void plan_interface_nd(Plan& P, int depth) {
    const int32_t L = P.n_lambda, m = P.m;
    if (depth < 0) {
        depth = 0;
        while (depth < 6 && (L >> (depth + 1)) >= 900 && (m >> (depth + 1)) >= 4) ++depth;
    }
    std::vector<int32_t> grp(m, 0);
    int32_t G = 0;
    std::vector<std::pair<int32_t, int32_t>> stack{{0, m}};
    std::vector<std::pair<int32_t, int32_t>> leaves;
    std::vector<int> dep{0};
    while (!stack.empty()) {
        auto r = stack.back();
        int d = dep.back();
        stack.pop_back();
        dep.pop_back();
        if (d == depth || r.second - r.first <= 1) {
            leaves.push_back(r);
            continue;
        }
        int32_t k1 = (r.second - r.first) / 2;
        stack.push_back({r.first + k1, r.second});
        dep.push_back(d + 1);
        stack.push_back({r.first, r.first + k1});
        dep.push_back(d + 1);
    }
    std::sort(leaves.begin(), leaves.end());
    G = (int32_t)leaves.size();
    for (int32_t g = 0; g < G; ++g)
        for (int32_t i = leaves[g].first; i < leaves[g].second; ++i) grp[i] = g;
    P.nd_G = G;
    P.nd_pos.assign(L, -1);
    P.nd_id.clear();
    P.nd_goff.assign(G + 1, 0);
    std::vector<std::vector<int32_t>> inner(G);
    std::vector<int32_t> sep;
    for (int32_t I = 0; I < L; ++I) {
        int32_t gi = grp[P.pairs[2 * I]], gj = grp[P.pairs[2 * I + 1]];
        if (gi == gj) inner[gi].push_back(I);
        else sep.push_back(I);
    }
    for (int32_t g = 0; g < G; ++g) {
        P.nd_goff[g + 1] = P.nd_goff[g] + (int64_t)inner[g].size();
        for (int32_t I : inner[g]) {
            P.nd_pos[I] = (int32_t)P.nd_id.size();
            P.nd_id.push_back(I);
        }
    }
    P.nd_nsep = (int32_t)sep.size();
    std::vector<std::vector<int32_t>> adj(G);
    P.nd_sg.assign(2 * (size_t)P.nd_nsep, 0);
    for (int32_t t = 0; t < P.nd_nsep; ++t) {
        int32_t I = sep[t];
        P.nd_pos[I] = (int32_t)P.nd_id.size();
        P.nd_id.push_back(I);
        int32_t g1 = grp[P.pairs[2 * I]], g2 = grp[P.pairs[2 * I + 1]];
        if (g1 > g2) std::swap(g1, g2);
        P.nd_sg[2 * t] = g1;
        P.nd_sg[2 * t + 1] = g2;
        adj[g1].push_back(t);
        adj[g2].push_back(t);
    }
    P.nd_aoff.assign(G + 1, 0);
    P.nd_alist.clear();
    P.nd_sidx.assign(2 * (size_t)P.nd_nsep, 0);
    for (int32_t g = 0; g < G; ++g) {
        P.nd_aoff[g + 1] = P.nd_aoff[g] + (int64_t)adj[g].size();
        for (size_t a = 0; a < adj[g].size(); ++a) {
            int32_t t = adj[g][a];
            P.nd_alist.push_back(t);
            P.nd_sidx[2 * t + (P.nd_sg[2 * t] == g ? 0 : 1)] = (int32_t)a;
        }
    }
}

}  // namespace am
