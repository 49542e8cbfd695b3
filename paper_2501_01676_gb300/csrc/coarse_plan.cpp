// Symbolic plan of the coarse problem's sparse factorisation.
//
// The coarse matrix S_Pi of M^-1 = R~^T D~ S~^-1 D~^T R~ (Sect. 3) couples two
// primal unknowns only when their vertices, faces or edges share a subdomain,
// so on a tensor partition it is sparse with the structure of the subdomain
// grid.  The plan orders the primal unknowns by nested dissection of that grid:
// a box of subdomains is cut in half across its longest direction; the primal
// unknowns of the entities lying on the cut plane form the separator (a node of
// the tree) and the two halves are dissected recursively.  Unknowns of the two
// halves never share a subdomain, so the halves are eliminated independently.
//
// Each node becomes one dense front: its own unknowns, then its boundary --
// the unknowns of ancestor separators that its own unknowns or its children's
// boundaries couple to.  Elimination runs from the leaves up (children before
// parents: multifrontal block LU without pivoting; every front's leading block
// is a principal block of a Schur complement of S_Pi, whose symmetric part is
// positive definite); the trailing block of a front is added into its parent.
//
// Host code only: no CUDA calls.
#include <algorithm>
#include <cstring>
#include <vector>

#include "bddc_internal.h"

namespace {
inline int r4(int n) { return (n + 3) & ~3; }
// boxes holding at most this many primal unknowns are not dissected further
constexpr int ND_LEAF_VARS = 160;
}  // namespace

int nd_plan(const HostMesh& hm, int nPi, NDPlan& P) {
    P = NDPlan();
    P.nPi = nPi;
    if (nPi <= 0) return BDDC_OK;
    const int ns0 = hm.nsub[0], ns1 = hm.nsub[1];
    const int nent = (int)hm.ent.size();
    // grid coordinate range of every entity carrying primal unknowns
    std::vector<int> live;
    std::vector<int> cmin(3 * nent, 0), cmax(3 * nent, 0);
    for (int e = 0; e < nent; ++e) {
        const Entity& E = hm.ent[e];
        if (E.k <= 0) continue;
        live.push_back(e);
        int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-1, -1, -1};
        for (int s : E.subs) {
            const int c[3] = {s % ns0, (s / ns0) % ns1, s / (ns0 * ns1)};
            for (int d = 0; d < 3; ++d) {
                lo[d] = std::min(lo[d], c[d]);
                hi[d] = std::max(hi[d], c[d]);
            }
        }
        for (int d = 0; d < 3; ++d) {
            cmin[3 * e + d] = lo[d];
            cmax[3 * e + d] = hi[d];
        }
    }
    // ---- the dissection tree (nodes in pre-order: a parent before its subtree)
    std::vector<std::vector<int>> sep;       // entities of each node
    std::vector<int> parent, end;            // end: one past the last node of the subtree
    struct Box {
        int lo[3], hi[3];                    // subdomain coordinates [lo, hi)
        std::vector<int> ents;
        int parent;
    };
    // explicit stack of pending boxes; a node's subtree is finished once every box
    // pushed below it is done, which `end` records by a post-pass
    std::vector<Box> stack;
    {
        Box b;
        for (int d = 0; d < 3; ++d) {
            b.lo[d] = 0;
            b.hi[d] = hm.nsub[d];
        }
        b.ents = live;
        b.parent = -1;
        stack.push_back(std::move(b));
    }
    while (!stack.empty()) {
        Box b = std::move(stack.back());
        stack.pop_back();
        if (b.ents.empty()) continue;
        int d = 0;
        for (int q = 1; q < 3; ++q)
            if (b.hi[q] - b.lo[q] > b.hi[d] - b.lo[d]) d = q;
        int nvars = 0;
        for (int e : b.ents) nvars += hm.ent[e].k;
        std::vector<int> s, L, R;
        if (b.hi[d] - b.lo[d] <= 1 || nvars <= ND_LEAF_VARS) {
            // a leaf: every unknown of the box in one front (a box that cannot be
            // cut, or one small enough that another level would cost more in the
            // sweeps' dependency chain than its dense front costs to factor)
            s = b.ents;
        } else {
            const int cut = b.lo[d] + (b.hi[d] - b.lo[d]) / 2;
            for (int e : b.ents) {
                if (cmax[3 * e + d] < cut) L.push_back(e);
                else if (cmin[3 * e + d] >= cut) R.push_back(e);
                else s.push_back(e);
            }
            int me = b.parent;
            if (!s.empty()) {
                me = (int)sep.size();
                sep.push_back(s);
                parent.push_back(b.parent);
            }
            Box bl = b, br = b;
            bl.hi[d] = cut;
            br.lo[d] = cut;
            bl.ents = std::move(L);
            br.ents = std::move(R);
            bl.parent = br.parent = me;
            // depth-first: the right box is popped after the whole left subtree
            stack.push_back(std::move(br));
            stack.push_back(std::move(bl));
            continue;
        }
        sep.push_back(s);
        parent.push_back(b.parent);
    }
    const int nn = (int)sep.size();
    // depth-first pre-order: every subtree is a contiguous id range [a, end[a])
    end.assign(nn, 0);
    for (int a = nn - 1; a >= 0; --a) {
        end[a] = std::max(end[a], a + 1);
        if (parent[a] >= 0) end[parent[a]] = std::max(end[parent[a]], end[a]);
    }
    std::vector<int> node_of(nent, -1);
    for (int a = 0; a < nn; ++a)
        for (int e : sep[a]) node_of[e] = a;
    // entities with primal unknowns per subdomain
    std::vector<std::vector<int>> sub_live(hm.nsd);
    for (int e : live)
        for (int s : hm.ent[e].subs) sub_live[s].push_back(e);
    // ---- boundaries, children first (reverse pre-order)
    std::vector<std::vector<int>> bnd(nn);
    std::vector<int> mark(nent, -1);
    std::vector<std::vector<int>> children(nn);
    for (int a = 0; a < nn; ++a)
        if (parent[a] >= 0) children[parent[a]].push_back(a);
    for (int a = nn - 1; a >= 0; --a) {
        std::vector<int>& B = bnd[a];
        auto consider = [&](int x) {
            const int nx = node_of[x];
            if (mark[x] == a) return;
            mark[x] = a;
            if (nx < a && a < end[nx]) B.push_back(x);   // a proper ancestor of node a
        };
        for (int e : sep[a])
            for (int s : hm.ent[e].subs)
                for (int x : sub_live[s]) consider(x);
        for (int c : children[a])
            for (int x : bnd[c]) consider(x);
        std::sort(B.begin(), B.end(), [&](int x, int y) {
            return node_of[x] != node_of[y] ? node_of[x] < node_of[y] : x < y;
        });
    }
    // ---- fronts
    P.fr.resize(nn);
    std::vector<int> height(nn, 0), depth(nn, 0);
    for (int a = nn - 1; a >= 0; --a)
        if (parent[a] >= 0) height[parent[a]] = std::max(height[parent[a]], height[a] + 1);
    for (int a = 0; a < nn; ++a)
        if (parent[a] >= 0) depth[a] = depth[parent[a]] + 1;
    auto vars_of = [&](const std::vector<int>& ents, std::vector<int>& out) {
        for (int e : ents)
            for (int l = 0; l < hm.ent[e].k; ++l) out.push_back(hm.ent[e].prim_off + l);
    };
    std::vector<int>& idx = P.idx;
    long long foff = 0, ooff = 0;
    int maxh = 0, maxd = 0;
    for (int a = 0; a < nn; ++a) {
        NDFront& F = P.fr[a];
        std::vector<int> v;
        vars_of(sep[a], v);
        F.n = (int)v.size();
        vars_of(bnd[a], v);
        F.b = (int)v.size() - F.n;
        F.N = 2 * F.n + F.b;
        F.ld = r4(F.N);
        F.foff = foff;
        foff += (long long)F.N * F.ld;
        F.vars_off = (int)idx.size();
        idx.insert(idx.end(), v.begin(), v.end());
        F.parent = parent[a];
        F.height = height[a];
        F.depth = depth[a];
        F.wf_ld = r4(std::max(F.n, 1));
        F.wf_off = ooff;
        ooff += (long long)F.b * F.wf_ld;
        F.wb_ld = r4(F.b + F.n);
        F.wb_off = ooff;
        ooff += (long long)F.n * F.wb_ld;
        // elimination of the n leading unknowns of the N x N extended front
        for (int p = 0; p < F.n; ++p) {
            const double m = (double)(F.N - p - 1);
            P.flops += 2.0 * m * m + m;
        }
        maxh = std::max(maxh, F.height);
        maxd = std::max(maxd, F.depth);
    }
    P.fpool = std::max(foff, 1LL);
    P.opool = std::max(ooff, 1LL);
    // positions of every child's boundary unknowns in its parent's front
    std::vector<int> posmap(nPi, -1);
    for (int a = 0; a < nn; ++a) {
        NDFront& F = P.fr[a];
        F.map_off = -1;
        if (F.parent < 0 || F.b == 0) continue;
        const NDFront& Pf = P.fr[F.parent];
        for (int q = 0; q < Pf.n + Pf.b; ++q) posmap[idx[Pf.vars_off + q]] = q;
        F.map_off = (int)idx.size();
        for (int q = 0; q < F.b; ++q) {
            const int pq = posmap[idx[F.vars_off + F.n + q]];
            if (pq < 0) return BDDC_EINVAL;          // a boundary unknown missing from the parent's front
            idx.push_back(pq);
        }
        for (int q = 0; q < Pf.n + Pf.b; ++q) posmap[idx[Pf.vars_off + q]] = -1;
    }
    // ---- groups and solve items
    P.by_height.assign(maxh + 1, {});
    P.by_depth.assign(maxd + 1, {});
    for (int a = 0; a < nn; ++a) {
        P.by_height[P.fr[a].height].push_back(a);
        P.by_depth[P.fr[a].depth].push_back(a);
    }
    // solve vector: y (the right-hand side, transformed in place by the forward
    // sweep) at [0, nPi), the solution x at [nPi, 2 nPi)
    // small items (16 rows: one pass of the GEMV's eight two-row warps; 256
    // columns) spread each front of the sweeps' dependency chain over many CTAs
    auto split = [](std::vector<GemvItem>& v, long long moff, int rows, int cols, int ld, int io, int oo) {
        const int RB = ND_ITEM_ROWS, CB = ND_ITEM_COLS;
        for (int c0 = 0; c0 < cols; c0 += CB)
            for (int r0 = 0; r0 < rows; r0 += RB)
                v.push_back(GemvItem{moff, rows, cols, ld, io, oo, r0, std::min(RB, rows - r0), c0,
                                     std::min(CB, cols - c0)});
    };
    P.fwd.assign(maxh + 1, {});
    P.bwd.assign(maxd + 1, {});
    for (int a = 0; a < nn; ++a) {
        NDFront& F = P.fr[a];
        // forward: y[bnd] += (-F21 F11^-1) y[own]
        if (F.b > 0 && F.n > 0) split(P.fwd[F.height], F.wf_off, F.b, F.n, F.wf_ld, F.vars_off, F.vars_off + F.n);
        // backward: x[own] = [-F11^-1 F12 | F11^-1] [x[bnd]; y[own]]
        const int in_off = (int)idx.size();
        for (int q = 0; q < F.b; ++q) idx.push_back(nPi + idx[F.vars_off + F.n + q]);
        for (int q = 0; q < F.n; ++q) idx.push_back(idx[F.vars_off + q]);
        const int out_off = (int)idx.size();
        for (int q = 0; q < F.n; ++q) idx.push_back(nPi + idx[F.vars_off + q]);
        if (F.n > 0) split(P.bwd[F.depth], F.wb_off, F.n, F.b + F.n, F.wb_ld, in_off, out_off);
        P.bytes_solve += 8.0 * ((double)F.b * F.n + (double)F.n * (F.b + F.n)) +
                         12.0 * ((double)F.n + F.b + (F.b + F.n) + F.n);
    }
    // every primal unknown is own to exactly one front
    std::vector<int> seen(nPi, 0);
    for (int a = 0; a < nn; ++a)
        for (int q = 0; q < P.fr[a].n; ++q) ++seen[idx[P.fr[a].vars_off + q]];
    for (int q = 0; q < nPi; ++q)
        if (seen[q] != 1) return BDDC_EINVAL;
    return BDDC_OK;
}
