// Host check of the nested-dissection plan of the coarse problem (no GPU).
//
// Builds the library's host mesh for a tensor partition, gives every entity a
// random primal count, forms a random coarse matrix with exactly the coupling
// of the method's S_Pi (two primal unknowns couple when their entities share a
// subdomain; every subdomain adds a dense block with a positive definite
// symmetric part), then carries out the plan literally on the CPU -- fill the
// extended fronts, add the children's updates, eliminate the own unknowns
// without pivoting, copy the sweep operators, run the forward and backward
// sweeps as gather/GEMV/scatter-add items -- and compares the result with a
// dense partially pivoted LU solve.
//
// usage: coarse_plan_check nx ny nz m seed   (slabs of m elements; m < 0: random 2..|m|)
// prints "ok <relative error> <fronts> <levels>" and exits 0, or exits 1.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "../paper_2501_01676_gb300/csrc/bddc_internal.h"

void bddc_set_last_error(const char*, const char*, int) {}

int main(int argc, char** argv) {
    if (argc < 6) return 2;
    const int ns[3] = {atoi(argv[1]), atoi(argv[2]), atoi(argv[3])};
    const int m = atoi(argv[4]);
    std::mt19937_64 rng((unsigned long long)atoll(argv[5]));
    std::uniform_real_distribution<double> U(-1.0, 1.0);
    std::vector<int> slabs[3];
    bddc_partition part;
    for (int d = 0; d < 3; ++d) {
        part.nsub[d] = ns[d];
        for (int s = 0; s < ns[d]; ++s) slabs[d].push_back(m > 0 ? m : 2 + (int)(rng() % (unsigned)(-m - 1)));
        part.elems_per_slab[d] = slabs[d].data();
    }
    bddc_mesh mesh = {{0, 0, 0}, {0, 0, 0}};
    HostMesh hm;
    if (build_host_mesh(&mesh, &part, hm) != 0) return 1;
    // primal counts (vertices 1, faces and edges 0..4) and offsets, kinds in the order V, F, E
    for (Entity& E : hm.ent) E.k = E.kind == 0 ? 1 : (int)(rng() % 5) - (E.kind == 1 ? 1 : 0);
    for (Entity& E : hm.ent) E.k = std::max(E.k, 0);
    int nPi = 0;
    for (int kind : {0, 2, 1})
        for (int e : hm.by_kind[kind]) {
            hm.ent[e].prim_off = nPi;
            nPi += hm.ent[e].k;
        }
    // random coarse matrix with the method's coupling
    std::vector<double> S((size_t)nPi * nPi, 0.0);
    for (int s = 0; s < hm.nsd; ++s) {
        std::vector<int> v;
        for (int e : hm.sub[s].ents)
            for (int l = 0; l < hm.ent[e].k; ++l) v.push_back(hm.ent[e].prim_off + l);
        const int q = (int)v.size();
        std::vector<double> G((size_t)q * q), K((size_t)q * q);
        for (auto& x : G) x = U(rng);
        for (auto& x : K) x = U(rng);
        for (int i = 0; i < q; ++i)
            for (int j = 0; j < q; ++j) {
                double a = 0.0;
                for (int t = 0; t < q; ++t) a += G[i * q + t] * G[j * q + t];
                a += 0.5 * (K[i * q + j] - K[j * q + i]) + (i == j ? 0.1 : 0.0);
                S[(size_t)v[i] * nPi + v[j]] += a;
            }
    }
    NDPlan P;
    if (nd_plan(hm, nPi, P) != 0) {
        printf("plan failed\n");
        return 1;
    }
    // ---- numeric factorisation, literally as planned
    std::vector<double> F((size_t)P.fpool, 0.0), W((size_t)P.opool, 0.0);
    const std::vector<int>& idx = P.idx;
    for (size_t h = 0; h < P.by_height.size(); ++h) {
        for (int a : P.by_height[h]) {           // fill
            const NDFront& f = P.fr[a];
            const int n = f.n, mm = f.n + f.b;
            const int* v = idx.data() + f.vars_off;
            for (int r = 0; r < f.N; ++r)
                for (int c = 0; c < f.ld; ++c) {
                    double val = 0.0;
                    if (c < mm && r < mm) {
                        if (r < n || c < n) val = S[(size_t)v[r] * nPi + v[c]];
                    } else if (r < n && c >= mm && c < f.N) {
                        val = (c - mm == r) ? -1.0 : 0.0;
                    } else if (r >= mm && c < n) {
                        val = (r - mm == c) ? 1.0 : 0.0;
                    }
                    F[f.foff + (size_t)r * f.ld + c] = val;
                }
        }
        for (size_t a = 0; a < P.fr.size(); ++a) {   // children's updates
            const NDFront& fc = P.fr[a];
            if (fc.parent < 0 || fc.b == 0 || P.fr[fc.parent].height != (int)h) continue;
            const NDFront& fp = P.fr[fc.parent];
            const int* map = idx.data() + fc.map_off;
            for (int r = 0; r < fc.b; ++r)
                for (int c = 0; c < fc.b; ++c)
                    F[fp.foff + (size_t)map[r] * fp.ld + map[c]] +=
                        F[fc.foff + (size_t)(fc.n + r) * fc.ld + fc.n + c];
        }
        for (int a : P.by_height[h]) {           // eliminate the n leading unknowns
            const NDFront& f = P.fr[a];
            double* A = F.data() + f.foff;
            for (int p = 0; p < f.n; ++p) {
                const double piv = A[(size_t)p * f.ld + p];
                if (!(std::fabs(piv) > 0.0)) return 1;
                for (int i = p + 1; i < f.N; ++i) {
                    const double l = A[(size_t)i * f.ld + p] / piv;
                    A[(size_t)i * f.ld + p] = l;
                    if (l != 0.0)
                        for (int j = p + 1; j < f.N; ++j) A[(size_t)i * f.ld + j] -= l * A[(size_t)p * f.ld + j];
                }
            }
            for (int r = 0; r < f.b; ++r)            // -(F21 F11^-1)
                for (int c = 0; c < f.n; ++c)
                    W[f.wf_off + (size_t)r * f.wf_ld + c] = -A[(size_t)(f.n + r) * f.ld + f.n + f.b + c];
            for (int r = 0; r < f.n; ++r)            // [-F11^-1 F12 | F11^-1]
                for (int c = 0; c < f.b + f.n; ++c)
                    W[f.wb_off + (size_t)r * f.wb_ld + c] = A[(size_t)(f.n + f.b + r) * f.ld + f.n + c];
        }
    }
    // ---- sweeps
    std::vector<double> b(nPi), y2(2 * (size_t)nPi, 0.0);
    for (auto& x : b) x = U(rng);
    for (int q = 0; q < nPi; ++q) y2[q] = b[q];
    auto run = [&](const std::vector<GemvItem>& items) {
        // all items of one group read before any writes land (as on the GPU,
        // where no item of a group reads what another writes)
        std::vector<std::pair<int, double>> out;
        for (const GemvItem& it : items)
            for (int r = it.row0; r < it.row0 + it.nrows; ++r) {
                double acc = 0.0;
                for (int c = it.col0; c < it.col0 + it.ncols; ++c)
                    acc += W[it.moff + (size_t)r * it.ld + c] * y2[idx[it.iidx_off + c]];
                out.push_back({idx[it.oidx_off + r], acc});
            }
        for (auto& o : out) y2[o.first] += o.second;
    };
    for (auto& g : P.fwd) run(g);
    for (auto& g : P.bwd) run(g);
    // ---- dense reference
    std::vector<double> A = S, x = b;
    std::vector<int> pv(nPi);
    for (int p = 0; p < nPi; ++p) {
        int r = p;
        for (int i = p + 1; i < nPi; ++i)
            if (std::fabs(A[(size_t)i * nPi + p]) > std::fabs(A[(size_t)r * nPi + p])) r = i;
        if (r != p) {
            for (int j = 0; j < nPi; ++j) std::swap(A[(size_t)p * nPi + j], A[(size_t)r * nPi + j]);
            std::swap(x[p], x[r]);
        }
        for (int i = p + 1; i < nPi; ++i) {
            const double l = A[(size_t)i * nPi + p] / A[(size_t)p * nPi + p];
            for (int j = p; j < nPi; ++j) A[(size_t)i * nPi + j] -= l * A[(size_t)p * nPi + j];
            x[i] -= l * x[p];
        }
    }
    for (int p = nPi - 1; p >= 0; --p) {
        double a = x[p];
        for (int j = p + 1; j < nPi; ++j) a -= A[(size_t)p * nPi + j] * x[j];
        x[p] = a / A[(size_t)p * nPi + p];
    }
    double num = 0.0, den = 0.0;
    for (int q = 0; q < nPi; ++q) {
        num += (y2[nPi + q] - x[q]) * (y2[nPi + q] - x[q]);
        den += x[q] * x[q];
    }
    const double err = std::sqrt(num / den);
    printf("ok %.3e %zu %zu %d\n", err, P.fr.size(), P.by_height.size(), nPi);
    return err < 1e-9 ? 0 : 1;
}
