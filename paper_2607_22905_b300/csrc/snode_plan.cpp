// Supernodal layout of the local factors L_i (Algorithm 1: "compute the Cholesky
// factorization A_i = L_i L_i^T"), built on the host from the pattern of each subdomain.
//
// Ordering: nested dissection of the subdomain's graph.  A node set is split by the BFS
// level structure from a pseudo-peripheral node: the level with the fewest nodes whose
// lower side holds between 30 % and 70 % of the set becomes the vertex separator (its
// nodes without a neighbour on the upper side move to the lower side), and both sides
// are dissected in turn; sets of at most kLeaf nodes stop.  Disconnected sets are
// dissected per component.  Every leaf and every separator is one supernode: a dense
// diagonal block and one row structure R_J shared by its columns.  The subdomain's
// unknowns are ordered supernode by supernode in postorder (children before parents).
//
// Symbolic factorisation: R_J = (rows of A below J adjacent to J) united with R_K minus J
// for every supernode K whose first row below its block lies in J (the supernodal
// elimination tree); every entry of L_i lies in some J x (J u R_J), and every update
// from a descendant K to an ancestor J lands inside J's front (J u R_J) x J.
//
// Solve schedule: supernodes grouped by their height in the supernodal elimination tree
// (leaves 0).  The forward sweep goes up the levels; at a level every supernode first
// pulls the updates pushed by its descendants (u_K = L_{R_K,K} x_K, stored per K), then
// applies the inverse of its diagonal block, then pushes its own update.  The backward
// sweep goes down the levels.  The pull lists give, for every row, the update entries
// that target it in increasing K order, so the sums have a fixed order.
#include <algorithm>
#include <climits>
#include <numeric>

#include "host_setup.h"

namespace am {

namespace {

constexpr int kLeaf = 32;          // largest set not dissected further (one supernode)
constexpr double kBalance = 0.3;   // separator level: each side gets >= 30 % of the set

struct NdBuilder {
    const std::vector<int64_t>& ptr;
    const std::vector<int32_t>& adj;
    std::vector<int32_t> mem, seen, lev, deg, cmark;
    int32_t stamp = 0;
    std::vector<std::vector<int32_t>> sn_nodes;
    std::vector<int32_t> sn_parent;   // dissection tree (not needed by the solve)

    NdBuilder(int32_t n, const std::vector<int64_t>& p, const std::vector<int32_t>& a)
        : ptr(p), adj(a), mem(n, 0), seen(n, 0), lev(n, -1), deg(n, 0), cmark(n, 0) {}

    int32_t emit(std::vector<int32_t> nodes) {
        std::sort(nodes.begin(), nodes.end());
        sn_nodes.push_back(std::move(nodes));
        sn_parent.push_back(-1);
        return (int32_t)sn_nodes.size() - 1;
    }

    // BFS over the current set (mem == st) from s; returns the visit order, lev = level.
    void bfs(int32_t st, int32_t s, std::vector<int32_t>& q) {
        const int32_t vs = ++stamp;
        q.clear();
        q.push_back(s);
        seen[s] = vs;
        lev[s] = 0;
        for (size_t h = 0; h < q.size(); ++h) {
            const int32_t u = q[h];
            for (int64_t e = ptr[u]; e < ptr[u + 1]; ++e) {
                const int32_t v = adj[e];
                if (mem[v] == st && seen[v] != vs) {
                    seen[v] = vs;
                    lev[v] = lev[u] + 1;
                    q.push_back(v);
                }
            }
        }
    }

    std::vector<int32_t> build(std::vector<int32_t> S) {
        if ((int32_t)S.size() <= kLeaf) return {emit(std::move(S))};
        std::sort(S.begin(), S.end());
        const int32_t st = ++stamp;
        for (int32_t x : S) mem[x] = st;
        std::vector<int32_t> q;
        bfs(st, S[0], q);
        if (q.size() < S.size()) {   // several components: dissect each
            // all components first (the recursion below re-marks the sets it works on)
            const int32_t cs = ++stamp;
            std::vector<std::vector<int32_t>> comps;
            for (int32_t x : S) {
                if (cmark[x] == cs) continue;
                bfs(st, x, q);
                for (int32_t y : q) cmark[y] = cs;
                comps.emplace_back(q.begin(), q.end());
            }
            std::vector<int32_t> roots;
            for (auto& c : comps) {
                std::vector<int32_t> r = build(std::move(c));
                roots.insert(roots.end(), r.begin(), r.end());
            }
            return roots;
        }
        // George-Liu pseudo-peripheral node of the (connected) set
        for (int32_t x : S) {
            int32_t d = 0;
            for (int64_t e = ptr[x]; e < ptr[x + 1]; ++e) d += mem[adj[e]] == st;
            deg[x] = d;
        }
        int32_t s0 = S[0], ecc = lev[q.back()];
        for (int it = 0; it < 16; ++it) {
            int32_t u = -1, best = INT32_MAX;
            for (int32_t x : q)
                if (lev[x] == ecc && (deg[x] < best || (deg[x] == best && x < u))) {
                    u = x;
                    best = deg[x];
                }
            std::vector<int32_t> q2;
            bfs(st, u, q2);
            const int32_t e2 = lev[q2.back()];
            if (e2 > ecc) {
                s0 = u;
                ecc = e2;
                q.swap(q2);
            } else {
                bfs(st, s0, q);
                break;
            }
        }
        const int32_t L = ecc;
        if (L < 2) return {emit(std::move(S))};   // diameter <= 1: no vertex separator
        std::vector<int64_t> cnt(L + 1, 0);
        for (int32_t x : S) cnt[lev[x]]++;
        const int64_t ns = (int64_t)S.size();
        int32_t best = -1;
        int64_t below = cnt[0];
        for (int32_t l = 1; l < L; ++l) {
            const int64_t above = ns - below - cnt[l];
            if (below >= kBalance * ns && above >= kBalance * ns && (best < 0 || cnt[l] < cnt[best])) best = l;
            below += cnt[l];
        }
        if (best < 0) {   // no balanced level: the median level
            int64_t acc = 0;
            for (best = 0; best <= L; ++best) {
                acc += cnt[best];
                if (2 * acc >= ns) break;
            }
            best = std::min(std::max(best, 1), L - 1);
        }
        std::vector<int32_t> A, B, Sep;
        for (int32_t x : S) {
            if (lev[x] < best) {
                A.push_back(x);
            } else if (lev[x] > best) {
                B.push_back(x);
            } else {
                bool toB = false;
                for (int64_t e = ptr[x]; e < ptr[x + 1] && !toB; ++e)
                    toB = mem[adj[e]] == st && lev[adj[e]] == best + 1;
                (toB ? Sep : A).push_back(x);
            }
        }
        std::vector<int32_t> roots = build(std::move(A));
        if (!B.empty()) {
            std::vector<int32_t> rb = build(std::move(B));
            roots.insert(roots.end(), rb.begin(), rb.end());
        }
        if (Sep.empty()) return roots;
        const int32_t id = emit(std::move(Sep));
        for (int32_t r : roots) sn_parent[r] = id;
        return {id};
    }
};

}  // namespace

void sn_local_plan(int32_t n, const std::vector<int64_t>& ptr, const std::vector<int32_t>& adj, SnLocal& out) {
    NdBuilder b(n, ptr, adj);
    std::vector<int32_t> all(n);
    std::iota(all.begin(), all.end(), 0);
    b.build(std::move(all));
    const int32_t nsn = (int32_t)b.sn_nodes.size();
    out = SnLocal();
    out.order.reserve(n);
    out.c0.resize(nsn);
    out.w.resize(nsn);
    std::vector<int32_t> sn_of(n), pos(n);
    for (int32_t J = 0; J < nsn; ++J) {
        out.c0[J] = (int32_t)out.order.size();
        out.w[J] = (int32_t)b.sn_nodes[J].size();
        for (int32_t x : b.sn_nodes[J]) {
            pos[x] = (int32_t)out.order.size();
            sn_of[pos[x]] = J;
            out.order.push_back(x);
        }
    }
    // row structures, supernodal elimination tree, levels
    out.R.assign(nsn, {});
    out.parent.assign(nsn, -1);
    out.lev.assign(nsn, 0);
    std::vector<std::vector<int32_t>> kids(nsn);
    std::vector<int32_t> cand;
    for (int32_t J = 0; J < nsn; ++J) {
        const int32_t end = out.c0[J] + out.w[J];
        cand.clear();
        for (int32_t c = out.c0[J]; c < end; ++c) {
            const int32_t x = out.order[c];
            for (int64_t e = ptr[x]; e < ptr[x + 1]; ++e)
                if (pos[adj[e]] >= end) cand.push_back(pos[adj[e]]);
        }
        for (int32_t K : kids[J]) {
            out.lev[J] = std::max(out.lev[J], out.lev[K] + 1);
            for (int32_t r : out.R[K])
                if (r >= end) cand.push_back(r);
        }
        std::sort(cand.begin(), cand.end());
        cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
        out.R[J].assign(cand.begin(), cand.end());
        if (!cand.empty()) {
            out.parent[J] = sn_of[cand[0]];
            kids[out.parent[J]].push_back(J);
        }
    }
    out.nlev = 0;
    for (int32_t J = 0; J < nsn; ++J) out.nlev = std::max(out.nlev, out.lev[J] + 1);
    // updates of the numeric factorisation: (J <- K, rows [a, b) of R_K in J)
    out.upd.assign(nsn, {});
    for (int32_t K = 0; K < nsn; ++K) {
        const auto& R = out.R[K];
        for (size_t a = 0; a < R.size();) {
            const int32_t J = sn_of[R[a]];
            size_t e = a;
            while (e < R.size() && sn_of[R[e]] == J) ++e;
            out.upd[J].push_back({K, (int32_t)a, (int32_t)e});
            a = e;
        }
    }
}

}  // namespace am
