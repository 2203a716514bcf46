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
#include <atomic>
#include <climits>
#include <cstring>
#include <numeric>
#include <thread>

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

// ------------------------------------------------------------------------------------
// Record streams of the batched local solves (format: snode_stream.h).
// ------------------------------------------------------------------------------------
namespace am {

namespace {

constexpr int64_t kRecData = 2048;   // largest entry block of one record (bytes)

inline int64_t r16(int64_t x) { return (x + 15) & ~int64_t(15); }

struct WarpBuf {
    std::vector<uint8_t> b;
    std::vector<SnFill> f;
    int64_t load = 0;
    int32_t nbar = 0;
    int32_t max_rec = 0;
    void put(SnRec r, const void* idx, int idx_bytes, int64_t data_bytes, SnFill fl, bool has_fill) {
        const int64_t hb = r16(idx_bytes), tot = 16 + hb + r16(data_bytes);
        r.hdr = (uint16_t)hb;
        r.bytes = (uint32_t)tot;
        const size_t o = b.size();
        b.resize(o + tot, 0);
        std::memcpy(b.data() + o, &r, 16);
        if (idx_bytes) std::memcpy(b.data() + o + 16, idx, idx_bytes);
        if (has_fill) {
            fl.off = (int64_t)(o + 16 + hb);
            f.push_back(fl);
        }
        load += tot;
        max_rec = std::max<int32_t>(max_rec, (int32_t)tot);
    }
    void barrier() {
        SnRec r{};
        r.kind = SN_BARRIER;
        put(r, nullptr, 0, 0, SnFill{}, false);
        ++nbar;
    }
};

}  // namespace

int build_sn_stream(const Plan& P, int nw, int elem, SnStream& out, std::string& err) {
    const int32_t m = P.m;
    out = SnStream();
    out.nw = nw;
    out.elem = elem;
    const int32_t V = 8 / elem;   // entries per 8-byte group
    std::vector<std::vector<WarpBuf>> wb(m, std::vector<WarpBuf>(nw));
    std::atomic<int> bad{0};
    parallel_for(m, 1, [&](int64_t si, int64_t) {
        const int32_t s = (int32_t)si;
        const int32_t sn0 = P.sn_off[s];
        std::vector<WarpBuf>& W = wb[s];
        struct Unit {
            int32_t J, q, lanes;
            int64_t work;
        };
        const int64_t fcols = 0;
        (void)fcols;
        auto units_of = [&](int32_t gl) {
            std::vector<Unit> us;
            for (int32_t u = P.lev_du[gl]; u < P.lev_du[gl + 1]; ++u) {
                const int32_t J = sn0 + (int32_t)(P.du_list[u] >> 10), q = (int32_t)(P.du_list[u] & 1023);
                const int32_t lanes = std::min(32, P.sn_w[J] - 32 * q);
                // entries the unit reads in both sweeps: its rows of the descendants' panels,
                // its chunk of D_J twice, its columns of its own panel
                int64_t work = (int64_t)(32 * q + lanes) * lanes + (int64_t)P.sn_nr[J] * lanes;
                for (int64_t t = P.sn_upd_ptr[J]; t < P.sn_upd_ptr[J + 1]; ++t) {
                    const int32_t K = P.sn_upd[3 * t];
                    work += (int64_t)P.sn_w[K] * std::min<int64_t>(lanes, P.sn_upd[3 * t + 2] - P.sn_upd[3 * t + 1]);
                }
                us.push_back({J, q, lanes, work});
            }
            // longest work first onto the least loaded warp; each warp keeps its units in
            // the level's order
            std::vector<int> idx(us.size());
            std::iota(idx.begin(), idx.end(), 0);
            std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return us[a].work > us[b].work; });
            std::vector<int64_t> ld(nw, 0);
            std::vector<std::vector<Unit>> per(nw);
            std::vector<int> owner(us.size());
            for (int i : idx) {
                const int w = (int)(std::min_element(ld.begin(), ld.end()) - ld.begin());
                owner[i] = w;
                ld[w] += us[i].work;
            }
            for (size_t i = 0; i < us.size(); ++i) per[owner[i]].push_back(us[i]);
            return per;
        };
        auto fwd_contrib = [&](WarpBuf& B, const Unit& U) {
            const int32_t J = U.J, c0 = P.sn_c0[J], r_lo = c0 + 32 * U.q, r_hi = r_lo + U.lanes;
            struct Blk {
                int32_t K, a, b;
            };
            std::vector<Blk> blks;
            for (int64_t t = P.sn_upd_ptr[J]; t < P.sn_upd_ptr[J + 1]; ++t) {
                const int32_t K = P.sn_upd[3 * t], a = P.sn_upd[3 * t + 1], b = P.sn_upd[3 * t + 2];
                const uint16_t* RK = P.sn_rows.data() + P.sn_roff[K];
                const int32_t a2 = (int32_t)(std::lower_bound(RK + a, RK + b, (uint16_t)r_lo) - RK);
                const int32_t b2 = (int32_t)(std::lower_bound(RK + a, RK + b, (uint16_t)r_hi) - RK);
                if (b2 > a2) blks.push_back({K, a2, b2});
            }
            std::vector<SnRec> recs;
            std::vector<SnFill> fills;
            std::vector<std::vector<uint8_t>> maps;
            for (const Blk& k : blks) {
                const int32_t rows = k.b - k.a, wK = P.sn_w[k.K];
                const int32_t cmax = V * (int32_t)std::max<int64_t>(1, kRecData / ((int64_t)rows * 8));
                const uint16_t* RK = P.sn_rows.data() + P.sn_roff[k.K];
                std::vector<uint8_t> map(rows);
                for (int32_t i = 0; i < rows; ++i) map[i] = (uint8_t)(RK[k.a + i] - r_lo);
                for (int32_t cs = 0; cs < wK; cs += cmax) {
                    const int32_t nc = std::min(cmax, wK - cs);
                    SnRec r{};
                    r.kind = SN_FCONTRIB;
                    r.lanes = (uint8_t)U.lanes;
                    r.rows = (uint8_t)rows;
                    r.t0 = (uint16_t)r_lo;
                    r.x0 = (uint16_t)(P.sn_c0[k.K] + cs);
                    r.ncols = (uint16_t)nc;
                    SnFill f{};
                    f.sn = k.K;
                    f.kind = SN_FCONTRIB;
                    f.lanes = (uint8_t)U.lanes;
                    f.rows = (uint8_t)rows;
                    f.p0 = (uint16_t)k.a;
                    f.p1 = (uint16_t)cs;
                    f.n = (uint16_t)nc;
                    recs.push_back(r);
                    fills.push_back(f);
                    maps.push_back(map);
                }
            }
            for (size_t i = 0; i < recs.size(); ++i) {
                if (i == 0) recs[i].flags |= SN_FIRST;
                if (i + 1 == recs.size()) recs[i].flags |= SN_LAST;
                B.put(recs[i], maps[i].data(), (int)maps[i].size(),
                      (int64_t)recs[i].rows * ((recs[i].ncols + V - 1) / V) * 8, fills[i], true);
            }
        };
        auto fwd_diag = [&](WarpBuf& B, const Unit& U) {
            const int32_t J = U.J, c0 = P.sn_c0[J], q32 = 32 * U.q, nc = q32 + U.lanes;
            int32_t cA = 0;
            while (cA < nc) {
                int64_t sz = 0;   // bytes
                int32_t cB = cA;
                while (cB < nc) {
                    const int64_t cnt = U.lanes - std::max(0, cB - q32);   // rows of the group
                    if (cB > cA && sz + cnt * 8 > kRecData) break;
                    sz += cnt * 8;
                    cB = std::min(nc, cB + V);
                }
                SnRec r{};
                r.kind = SN_FDIAG;
                r.flags = (uint8_t)((cA == 0 ? SN_FIRST : 0) | (cB == nc ? SN_LAST : 0));
                r.lanes = (uint8_t)U.lanes;
                r.t0 = (uint16_t)(c0 + q32);
                r.x0 = (uint16_t)(c0 + cA);
                r.ncols = (uint16_t)(cB - cA);
                SnFill f{};
                f.sn = J;
                f.kind = SN_FDIAG;
                f.lanes = (uint8_t)U.lanes;
                f.p0 = (uint16_t)q32;
                f.p1 = (uint16_t)cA;
                f.n = (uint16_t)(cB - cA);
                B.put(r, nullptr, 0, sz, f, true);
                cA = cB;
            }
        };
        auto bwd_panel = [&](WarpBuf& B, const Unit& U) {
            const int32_t J = U.J, c0 = P.sn_c0[J], q32 = 32 * U.q, nr = P.sn_nr[J];
            const int32_t rmax = V * (int32_t)std::min<int64_t>(248 / V, std::max<int64_t>(1, kRecData / ((int64_t)U.lanes * 8)));
            const uint16_t* RJ = P.sn_rows.data() + P.sn_roff[J];
            std::vector<uint16_t> ridx;
            for (int32_t iA = 0; iA < nr; iA += rmax) {
                const int32_t rows = std::min(rmax, nr - iA);
                SnRec r{};
                r.kind = SN_BPANEL;
                r.flags = (uint8_t)((iA == 0 ? SN_FIRST : 0) | (iA + rows == nr ? SN_LAST : 0));
                r.lanes = (uint8_t)U.lanes;
                r.rows = (uint8_t)rows;
                r.t0 = (uint16_t)(c0 + q32);
                SnFill f{};
                f.sn = J;
                f.kind = SN_BPANEL;
                f.lanes = (uint8_t)U.lanes;
                f.rows = (uint8_t)rows;
                f.p0 = (uint16_t)iA;
                f.p1 = (uint16_t)q32;
                f.n = (uint16_t)rows;
                const int32_t groups = (rows + V - 1) / V;
                ridx.assign((size_t)groups * V, 0);   // padding rows: index 0, zero entries
                std::copy(RJ + iA, RJ + iA + rows, ridx.begin());
                B.put(r, ridx.data(), (int)ridx.size() * 2, (int64_t)groups * U.lanes * 8, f, true);
            }
        };
        auto bwd_diag = [&](WarpBuf& B, const Unit& U) {
            const int32_t J = U.J, c0 = P.sn_c0[J], q32 = 32 * U.q, w = P.sn_w[J];
            int32_t rA = q32;
            while (rA < w) {
                int64_t sz = 0;   // bytes
                int32_t rB = rA;
                while (rB < w) {
                    const int64_t cnt = std::min(rB - q32 + V, U.lanes);   // columns of the group
                    if (rB > rA && sz + cnt * 8 > kRecData) break;
                    sz += cnt * 8;
                    rB = std::min(w, rB + V);
                }
                SnRec r{};
                r.kind = SN_BDIAG;
                r.flags = (uint8_t)((rA == q32 ? SN_FIRST : 0) | (rB == w ? SN_LAST : 0));
                r.lanes = (uint8_t)U.lanes;
                r.t0 = (uint16_t)(c0 + q32);
                r.x0 = (uint16_t)(c0 + rA);
                r.ncols = (uint16_t)(rB - rA);
                SnFill f{};
                f.sn = J;
                f.kind = SN_BDIAG;
                f.lanes = (uint8_t)U.lanes;
                f.p0 = (uint16_t)q32;
                f.p1 = (uint16_t)rA;
                f.n = (uint16_t)(rB - rA);
                B.put(r, nullptr, 0, sz, f, true);
                rA = rB;
            }
        };
        const int32_t l0 = P.sub_lev0[s], nl = P.sub_nlev[s];
        std::vector<std::vector<std::vector<Unit>>> per(nl);
        for (int32_t lv = 0; lv < nl; ++lv) per[lv] = units_of(l0 + lv);
        for (int32_t lv = 0; lv < nl; ++lv) {
            const bool multi = P.lev_multi[l0 + lv] != 0;
            for (int w = 0; w < nw; ++w) {
                for (const Unit& U : per[lv][w]) {
                    fwd_contrib(W[w], U);
                    if (!multi) fwd_diag(W[w], U);
                }
                if (multi) {
                    W[w].barrier();
                    for (const Unit& U : per[lv][w]) fwd_diag(W[w], U);
                }
                W[w].barrier();
            }
        }
        for (int32_t lv = nl - 1; lv >= 0; --lv) {
            const bool multi = P.lev_multi[l0 + lv] != 0;
            for (int w = 0; w < nw; ++w) {
                for (const Unit& U : per[lv][w]) {
                    bwd_panel(W[w], U);
                    if (!multi) bwd_diag(W[w], U);
                }
                if (multi) {
                    W[w].barrier();
                    for (const Unit& U : per[lv][w]) bwd_diag(W[w], U);
                }
                W[w].barrier();
            }
        }
        for (int w = 0; w < nw; ++w) {
            SnRec r{};
            r.kind = SN_END;
            W[w].put(r, nullptr, 0, 0, SnFill{}, false);
            if (W[w].nbar != W[0].nbar) bad = 1;
        }
    });
    if (bad) {
        err = "local solve streams: unequal barrier counts";
        return 1;
    }
    out.woff.assign((size_t)m * nw + 1, 0);
    out.nbar.assign(m, 0);
    int64_t tot = 0;
    for (int32_t s = 0; s < m; ++s) {
        out.nbar[s] = wb[s][0].nbar;
        for (int w = 0; w < nw; ++w) {
            out.woff[(size_t)s * nw + w] = tot;
            tot += (int64_t)wb[s][w].b.size();
            out.max_record = std::max(out.max_record, wb[s][w].max_rec);
        }
    }
    out.woff[(size_t)m * nw] = tot;
    out.bytes.resize(tot);
    size_t nf = 0;
    for (int32_t s = 0; s < m; ++s)
        for (int w = 0; w < nw; ++w) nf += wb[s][w].f.size();
    out.fill.reserve(nf);
    for (int32_t s = 0; s < m; ++s)
        for (int w = 0; w < nw; ++w) {
            const int64_t base = out.woff[(size_t)s * nw + w];
            std::memcpy(out.bytes.data() + base, wb[s][w].b.data(), wb[s][w].b.size());
            for (SnFill f : wb[s][w].f) {
                f.off += base;
                out.fill.push_back(f);
            }
        }
    return 0;
}

}  // namespace am
