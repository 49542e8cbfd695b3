// Host-side mesh, tensor partition and interface classification (Sect. 3:
// non-overlapping subdomains meeting in faces, edges and vertices; n(X) is
// the set of subdomains sharing X).
#include <algorithm>
#include <cmath>

#include "bddc_internal.h"

int build_host_boxes(const bddc_mesh* mesh, const bddc_partition* part, HostMesh& hm) {
    if (!part) return BDDC_EINVAL;
    for (int d = 0; d < 3; ++d) {
        if (part->nsub[d] < 1 || !part->elems_per_slab[d]) return BDDC_EINVAL;
        hm.nsub[d] = part->nsub[d];
        hm.off[d].assign(1, 0);
        for (int s = 0; s < part->nsub[d]; ++s) {
            int c = part->elems_per_slab[d][s];
            if (c < 1 || c > 4096) return BDDC_EINVAL;
            hm.off[d].push_back(hm.off[d].back() + c);
        }
        hm.E[d] = hm.off[d].back();
        if (hm.E[d] < 2) return BDDC_EINVAL;
        double lo = 0.0, hi = 1.0;
        if (mesh && (mesh->lo[d] != 0.0 || mesh->hi[d] != 0.0)) {
            lo = mesh->lo[d];
            hi = mesh->hi[d];
        }
        if (!(hi > lo)) return BDDC_EINVAL;
        hm.lo[d] = lo;
        hm.h[d] = (hi - lo) / hm.E[d];
    }
    hm.nsd = hm.nsub[0] * hm.nsub[1] * hm.nsub[2];
    const int Ex = hm.E[0], Ey = hm.E[1], Ez = hm.E[2];
    hm.ndof = (Ex - 1) * (Ey - 1) * (Ez - 1);
    hm.nelem = Ex * Ey * Ez;
    hm.nnodes = (Ex + 1) * (Ey + 1) * (Ez + 1);
    if ((long long)hm.ndof > (1LL << 30)) return BDDC_EINVAL;
    auto dof_of = [&](int ix, int iy, int iz) -> int {
        if (ix <= 0 || iy <= 0 || iz <= 0 || ix >= Ex || iy >= Ey || iz >= Ez) return -1;
        return (ix - 1) + (Ex - 1) * ((iy - 1) + (Ey - 1) * (iz - 1));
    };
    hm.sub.assign(hm.nsd, SubInfo());
    for (int sz = 0; sz < hm.nsub[2]; ++sz)
        for (int sy = 0; sy < hm.nsub[1]; ++sy)
            for (int sx = 0; sx < hm.nsub[0]; ++sx) {
                int s = sx + hm.nsub[0] * (sy + hm.nsub[1] * sz);
                SubInfo& S = hm.sub[s];
                int c[3] = {sx, sy, sz};
                S.max_slab = 0;
                for (int d = 0; d < 3; ++d) {
                    S.box0[d] = hm.off[d][c[d]];
                    S.box1[d] = hm.off[d][c[d] + 1];
                    S.max_slab = std::max(S.max_slab, S.box1[d] - S.box0[d]);
                }
                // the box is walked with x fastest, so both lists come out ascending
                std::vector<int> in, bd;
                const long long nbox = (long long)(S.box1[0] - S.box0[0] + 1) * (S.box1[1] - S.box0[1] + 1) *
                                       (S.box1[2] - S.box0[2] + 1);
                in.reserve((size_t)nbox);
                bd.reserve((size_t)nbox);
                for (int iz = S.box0[2]; iz <= S.box1[2]; ++iz)
                    for (int iy = S.box0[1]; iy <= S.box1[1]; ++iy)
                        for (int ix = S.box0[0]; ix <= S.box1[0]; ++ix) {
                            int d = dof_of(ix, iy, iz);
                            if (d < 0) continue;
                            bool inside = S.box0[0] < ix && ix < S.box1[0] && S.box0[1] < iy &&
                                          iy < S.box1[1] && S.box0[2] < iz && iz < S.box1[2];
                            (inside ? in : bd).push_back(d);
                        }
                S.nI = (int)in.size();
                S.nB = (int)bd.size();
                S.n = S.nI + S.nB;
                S.dofs = std::move(in);
                S.dofs.insert(S.dofs.end(), bd.begin(), bd.end());
            }
    return BDDC_OK;
}

int build_host_interface(HostMesh& hm) {
    const int Ex = hm.E[0], Ey = hm.E[1], Ez = hm.E[2];
    auto dof_of = [&](int ix, int iy, int iz) -> int {
        if (ix <= 0 || iy <= 0 || iz <= 0 || ix >= Ex || iy >= Ey || iz >= Ez) return -1;
        return (ix - 1) + (Ex - 1) * ((iy - 1) + (Ey - 1) * (iz - 1));
    };
    // interface classification by the owner set n(x).  In a tensor partition the
    // owner set of node (ix, iy, iz) is fixed by one code per direction: 2s for
    // the plane between slabs s-1 and s (shared by both), 2s+1 for the inside of
    // slab s; a node on k planes is shared by 2^k subdomains (k = 1 face, 2 edge,
    // 3 vertex).  Nodes are visited in ascending dof order, so every entity's
    // dof list comes out sorted.
    std::vector<int> code[3];
    for (int d = 0; d < 3; ++d) {
        code[d].assign(hm.E[d] + 1, -1);
        for (int s = 0; s < hm.nsub[d]; ++s)
            for (int i = hm.off[d][s] + 1; i < hm.off[d][s + 1]; ++i) code[d][i] = 2 * s + 1;
        for (int s = 1; s < hm.nsub[d]; ++s) code[d][hm.off[d][s]] = 2 * s;
    }
    const int nc0 = 2 * hm.nsub[0] + 1, nc1 = 2 * hm.nsub[1] + 1, nc2 = 2 * hm.nsub[2] + 1;
    std::vector<int> key2ent((size_t)nc0 * nc1 * nc2, -1);
    std::vector<Entity> ents;
    hm.gamma_of_dof.assign(hm.ndof, -1);
    hm.gamma.clear();
    hm.gamma.reserve(hm.ndof);
    for (int iz = 1; iz < Ez; ++iz)
        for (int iy = 1; iy < Ey; ++iy)
            for (int ix = 1; ix < Ex; ++ix) {
                const int cx = code[0][ix], cy = code[1][iy], cz = code[2][iz];
                const int planes = (~cx & 1) + (~cy & 1) + (~cz & 1);
                if (planes == 0) continue;
                const int d = dof_of(ix, iy, iz);
                const size_t key = (size_t)cx + nc0 * ((size_t)cy + (size_t)nc1 * cz);
                int e = key2ent[key];
                if (e < 0) {
                    e = (int)ents.size();
                    key2ent[key] = e;
                    Entity E;
                    E.kind = planes == 3 ? 0 : (planes == 2 ? 1 : 2);
                    int a[2], b[2], c[2], na = 0, nb = 0, ncz = 0;
                    if (cx & 1) a[na++] = cx >> 1; else { a[na++] = (cx >> 1) - 1; a[na++] = cx >> 1; }
                    if (cy & 1) b[nb++] = cy >> 1; else { b[nb++] = (cy >> 1) - 1; b[nb++] = cy >> 1; }
                    if (cz & 1) c[ncz++] = cz >> 1; else { c[ncz++] = (cz >> 1) - 1; c[ncz++] = cz >> 1; }
                    for (int q = 0; q < ncz; ++q)
                        for (int p2 = 0; p2 < nb; ++p2)
                            for (int o = 0; o < na; ++o)
                                E.subs.push_back(a[o] + hm.nsub[0] * (b[p2] + hm.nsub[1] * c[q]));
                    ents.push_back(std::move(E));
                }
                ents[e].dofs.push_back(d);
                hm.gamma_of_dof[d] = (int)hm.gamma.size();
                hm.gamma.push_back(d);
            }
    // entity order: kind, then smallest dof
    std::vector<int> order(ents.size());
    for (size_t e = 0; e < ents.size(); ++e) order[e] = (int)e;
    std::sort(order.begin(), order.end(), [&](int x, int y) {
        if (ents[x].kind != ents[y].kind) return ents[x].kind < ents[y].kind;
        return ents[x].dofs[0] < ents[y].dofs[0];
    });
    hm.ent.clear();
    hm.ent.reserve(ents.size());
    for (int e : order) hm.ent.push_back(std::move(ents[e]));
    for (int k = 0; k < 3; ++k) hm.by_kind[k].clear();
    for (int e = 0; e < (int)hm.ent.size(); ++e) {
        Entity& E = hm.ent[e];
        E.slot = (int)hm.by_kind[E.kind].size();
        hm.by_kind[E.kind].push_back(e);
    }
    for (int s = 0; s < hm.nsd; ++s) {
        SubInfo& S = hm.sub[s];
        S.gidx.resize(S.nB);
        for (int b = 0; b < S.nB; ++b) {
            int g = hm.gamma_of_dof[S.dofs[S.nI + b]];
            if (g < 0) return BDDC_EINVAL;
            S.gidx[b] = g;
        }
    }
    // entity positions within each subdomain's interface list, through a dof ->
    // position table filled for one subdomain at a time
    for (int e = 0; e < (int)hm.ent.size(); ++e) {
        Entity& E = hm.ent[e];
        E.pos.assign(E.subs.size(), std::vector<int>(E.dofs.size()));
        for (size_t a = 0; a < E.subs.size(); ++a) {
            SubInfo& S = hm.sub[E.subs[a]];
            S.ents.push_back(e);
            S.ent_slot.push_back((int)a);
        }
    }
    std::vector<int> loc(hm.ndof, -1);
    for (int s = 0; s < hm.nsd; ++s) {
        SubInfo& S = hm.sub[s];
        for (int b = 0; b < S.nB; ++b) loc[S.dofs[S.nI + b]] = b;
        for (size_t q = 0; q < S.ents.size(); ++q) {
            Entity& E = hm.ent[S.ents[q]];
            std::vector<int>& P = E.pos[S.ent_slot[q]];
            for (size_t l = 0; l < E.dofs.size(); ++l) {
                const int b = loc[E.dofs[l]];
                if (b < 0) return BDDC_EINVAL;
                P[l] = b;
            }
        }
        for (int b = 0; b < S.nB; ++b) loc[S.dofs[S.nI + b]] = -1;
    }
    return BDDC_OK;
}

int build_host_mesh(const bddc_mesh* mesh, const bddc_partition* part, HostMesh& hm) {
    const int rc = build_host_boxes(mesh, part, hm);
    return rc != BDDC_OK ? rc : build_host_interface(hm);
}

int build_local_nd(HostMesh& hm, LocalND& nd) {
    // child slabs and the parent slab of each
    std::vector<int> cs[3], pslab[3];
    for (int d = 0; d < 3; ++d)
        for (int s = 0; s < hm.nsub[d]; ++s) {
            const int c = hm.off[d][s + 1] - hm.off[d][s];
            if (c >= 2) {
                cs[d].push_back(c / 2);
                cs[d].push_back(c - c / 2);
                pslab[d].push_back(s);
                pslab[d].push_back(s);
            } else {
                cs[d].push_back(c);
                pslab[d].push_back(s);
            }
        }
    bddc_partition cp;
    bddc_mesh mesh;
    for (int d = 0; d < 3; ++d) {
        cp.nsub[d] = (int)cs[d].size();
        cp.elems_per_slab[d] = cs[d].data();
        mesh.lo[d] = hm.lo[d];
        mesh.hi[d] = hm.lo[d] + hm.h[d] * hm.E[d];
    }
    BDDC_TRY(build_host_boxes(&mesh, &cp, nd.child));
    const HostMesh& ch = nd.child;
    if (ch.ndof != hm.ndof || ch.E[0] != hm.E[0] || ch.E[1] != hm.E[1] || ch.E[2] != hm.E[2]) return BDDC_EINVAL;
    nd.parent.assign(ch.nsd, -1);
    for (int cz = 0; cz < ch.nsub[2]; ++cz)
        for (int cy = 0; cy < ch.nsub[1]; ++cy)
            for (int cx = 0; cx < ch.nsub[0]; ++cx)
                nd.parent[cx + ch.nsub[0] * (cy + ch.nsub[1] * cz)] =
                    pslab[0][cx] + hm.nsub[0] * (pslab[1][cy] + hm.nsub[1] * pslab[2][cz]);
    const int Ex = hm.E[0], Ey = hm.E[1], Ez = hm.E[2];
    auto dof_of = [&](int ix, int iy, int iz) -> int {
        if (ix <= 0 || iy <= 0 || iz <= 0 || ix >= Ex || iy >= Ey || iz >= Ez) return -1;
        return (ix - 1) + (Ex - 1) * ((iy - 1) + (Ey - 1) * (iz - 1));
    };
    // subdomain numbering [separators, interface], and a node -> new index table per box
    std::vector<std::vector<int>> lidx(hm.nsd);
    for (int s = 0; s < hm.nsd; ++s) {
        SubInfo& S = hm.sub[s];
        int mid[3], n[3];
        for (int d = 0; d < 3; ++d) {
            const int c = S.box1[d] - S.box0[d];
            mid[d] = c >= 2 ? S.box0[d] + c / 2 : -1;
            n[d] = c + 1;
        }
        std::vector<int>& L = lidx[s];
        L.assign((size_t)n[0] * n[1] * n[2], -1);
        std::vector<int> sep;
        for (int pass = 0; pass < 2; ++pass) {       // separators first, then the interface
            int nb = 0;
            for (int iz = S.box0[2]; iz <= S.box1[2]; ++iz)
                for (int iy = S.box0[1]; iy <= S.box1[1]; ++iy)
                    for (int ix = S.box0[0]; ix <= S.box1[0]; ++ix) {
                        const int g = dof_of(ix, iy, iz);
                        if (g < 0) continue;
                        const bool inside = S.box0[0] < ix && ix < S.box1[0] && S.box0[1] < iy && iy < S.box1[1] &&
                                            S.box0[2] < iz && iz < S.box1[2];
                        const long long q = (ix - S.box0[0]) + (long long)n[0] * ((iy - S.box0[1]) +
                                                                                   (long long)n[1] * (iz - S.box0[2]));
                        if (pass == 0 && inside && (ix == mid[0] || iy == mid[1] || iz == mid[2])) {
                            L[q] = (int)sep.size();
                            sep.push_back(g);
                        } else if (pass == 1 && !inside) {
                            L[q] = (int)sep.size() + nb++;
                        }
                    }
            if (pass == 1 && nb != S.nB) return BDDC_EINVAL;
        }
        std::vector<int> dofs = sep;
        dofs.insert(dofs.end(), S.dofs.begin() + S.nI, S.dofs.end());
        S.dofs = std::move(dofs);
        S.nI = (int)sep.size();
        S.n = S.nI + S.nB;
    }
    // child interface dof -> subdomain-local index
    nd.map.assign(ch.nsd, std::vector<int>());
    for (int c = 0; c < ch.nsd; ++c) {
        const SubInfo& K = ch.sub[c];
        const int p = nd.parent[c];
        if (p < 0) return BDDC_EINVAL;
        const SubInfo& S = hm.sub[p];
        const int n0 = S.box1[0] - S.box0[0] + 1, n1 = S.box1[1] - S.box0[1] + 1;
        std::vector<int>& M = nd.map[c];
        M.resize(K.nB);
        for (int j = 0; j < K.nB; ++j) {
            const int g = K.dofs[K.nI + j];
            const int ix = g % (Ex - 1) + 1, iy = (g / (Ex - 1)) % (Ey - 1) + 1, iz = g / ((Ex - 1) * (Ey - 1)) + 1;
            if (ix < S.box0[0] || ix > S.box1[0] || iy < S.box0[1] || iy > S.box1[1] || iz < S.box0[2] ||
                iz > S.box1[2])
                return BDDC_EINVAL;
            const int li = lidx[p][(ix - S.box0[0]) + (long long)n0 * ((iy - S.box0[1]) + (long long)n1 * (iz - S.box0[2]))];
            if (li < 0 || li >= S.n) return BDDC_EINVAL;
            M[j] = li;
        }
    }
    (void)Ez;
    return BDDC_OK;
}
