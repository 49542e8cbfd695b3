// Host-side mesh, tensor partition and interface classification (Sect. 3:
// non-overlapping subdomains meeting in faces, edges and vertices; n(X) is
// the set of subdomains sharing X).
#include <algorithm>
#include <cmath>
#include <map>

#include "bddc_internal.h"

int build_host_mesh(const bddc_mesh* mesh, const bddc_partition* part, HostMesh& hm) {
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
    // slabs holding node index i in direction d
    auto slabs_of = [&](int d, int i, int* out) -> int {
        int c = 0;
        const std::vector<int>& o = hm.off[d];
        for (int s = 0; s < hm.nsub[d]; ++s)
            if (o[s] <= i && i <= o[s + 1]) out[c++] = s;
        return c;
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
                std::vector<int> in, bd;
                for (int iz = S.box0[2]; iz <= S.box1[2]; ++iz)
                    for (int iy = S.box0[1]; iy <= S.box1[1]; ++iy)
                        for (int ix = S.box0[0]; ix <= S.box1[0]; ++ix) {
                            int d = dof_of(ix, iy, iz);
                            if (d < 0) continue;
                            bool inside = S.box0[0] < ix && ix < S.box1[0] && S.box0[1] < iy &&
                                          iy < S.box1[1] && S.box0[2] < iz && iz < S.box1[2];
                            (inside ? in : bd).push_back(d);
                        }
                std::sort(in.begin(), in.end());
                std::sort(bd.begin(), bd.end());
                S.nI = (int)in.size();
                S.nB = (int)bd.size();
                S.n = S.nI + S.nB;
                S.dofs = in;
                S.dofs.insert(S.dofs.end(), bd.begin(), bd.end());
            }
    // interface classification by the owner set n(x)
    hm.gamma_of_dof.assign(hm.ndof, -1);
    std::map<std::vector<int>, int> key2ent;
    std::vector<Entity> ents;
    for (int iz = 1; iz < Ez; ++iz)
        for (int iy = 1; iy < Ey; ++iy)
            for (int ix = 1; ix < Ex; ++ix) {
                int a[2], b[2], c[2];
                int na = slabs_of(0, ix, a), nb = slabs_of(1, iy, b), nc = slabs_of(2, iz, c);
                int cnt = na * nb * nc;
                if (cnt < 2) continue;
                std::vector<int> key;
                for (int q = 0; q < nc; ++q)
                    for (int p = 0; p < nb; ++p)
                        for (int o = 0; o < na; ++o)
                            key.push_back(a[o] + hm.nsub[0] * (b[p] + hm.nsub[1] * c[q]));
                std::sort(key.begin(), key.end());
                int d = dof_of(ix, iy, iz);
                auto it = key2ent.find(key);
                int e;
                if (it == key2ent.end()) {
                    e = (int)ents.size();
                    key2ent[key] = e;
                    Entity E;
                    E.kind = cnt == 8 ? 0 : (cnt == 4 ? 1 : (cnt == 2 ? 2 : -1));
                    if (E.kind < 0) return BDDC_EINVAL;
                    E.subs = key;
                    ents.push_back(E);
                } else {
                    e = it->second;
                }
                ents[e].dofs.push_back(d);
            }
    for (auto& E : ents) std::sort(E.dofs.begin(), E.dofs.end());
    std::sort(ents.begin(), ents.end(), [](const Entity& x, const Entity& y) {
        if (x.kind != y.kind) return x.kind < y.kind;
        return x.dofs[0] < y.dofs[0];
    });
    hm.ent = ents;
    for (int k = 0; k < 3; ++k) hm.by_kind[k].clear();
    for (int e = 0; e < (int)hm.ent.size(); ++e) {
        Entity& E = hm.ent[e];
        E.slot = (int)hm.by_kind[E.kind].size();
        hm.by_kind[E.kind].push_back(e);
        for (int d : E.dofs) hm.gamma.push_back(d);
    }
    std::sort(hm.gamma.begin(), hm.gamma.end());
    for (int g = 0; g < (int)hm.gamma.size(); ++g) hm.gamma_of_dof[hm.gamma[g]] = g;
    for (int s = 0; s < hm.nsd; ++s) {
        SubInfo& S = hm.sub[s];
        S.gidx.resize(S.nB);
        for (int b = 0; b < S.nB; ++b) {
            int g = hm.gamma_of_dof[S.dofs[S.nI + b]];
            if (g < 0) return BDDC_EINVAL;
            S.gidx[b] = g;
        }
    }
    for (int e = 0; e < (int)hm.ent.size(); ++e) {
        Entity& E = hm.ent[e];
        E.pos.resize(E.subs.size());
        for (size_t a = 0; a < E.subs.size(); ++a) {
            SubInfo& S = hm.sub[E.subs[a]];
            auto b0 = S.dofs.begin() + S.nI;
            for (int d : E.dofs) {
                auto it = std::lower_bound(b0, S.dofs.end(), d);
                if (it == S.dofs.end() || *it != d) return BDDC_EINVAL;
                E.pos[a].push_back((int)(it - b0));
            }
            S.ents.push_back(e);
            S.ent_slot.push_back((int)a);
        }
    }
    return BDDC_OK;
}
