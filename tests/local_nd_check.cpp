// Host check of the local nested-dissection plan (no GPU).
//
// Builds the library's host mesh for a tensor partition and the plan of one level
// of nested dissection inside every subdomain (child boxes, the subdomain
// numbering [separators, interface], the child -> subdomain index maps), then
// checks it two ways:
//  * structure: the children tile every subdomain, each child's interface dof
//    maps to the subdomain-local index that holds the same global dof, every
//    subdomain-interior dof is a separator or interior to exactly one child;
//  * algebra: with a random dense matrix per child box (diagonally dominant,
//    non-symmetric) the subdomain matrix is their sum; its Schur complement onto
//    the interface by one dense elimination must equal the two-level result
//    (children's Schur complements extend-added over [separators, interface]
//    by the plan's maps, then the separators eliminated);
//  * condensation and recovery in the library's order: for a random load f and
//    interface values u_B, g = f_B - A_BI A_II^{-1} f_I and u_I = A_II^{-1}(f_I -
//    A_IB u_B) by one dense solve equal the two-level results (children
//    condensed into a copy of f, then the separators; separators recovered first,
//    then the children from the values on their boundaries).
//
// usage: local_nd_check nx ny nz m seed   (slabs of m elements; m < 0: random 1..|m|)
// prints "ok <largest relative difference> <children> <separators>" and exits 0, or exits 1.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <unordered_map>
#include <vector>

#include "../paper_2501_01676_gb300/csrc/bddc_internal.h"

void bddc_set_last_error(const char*, const char*, int) {}

typedef std::vector<double> Mat;   // row-major, n x n

// x <- M[0:k, 0:k]^{-1} x (partial pivoting; M row-major with n columns)
static bool solve_lead(const Mat& M, int n, int k, std::vector<double>& x) {
    Mat A((size_t)k * k);
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) A[(size_t)i * k + j] = M[(size_t)i * n + j];
    for (int p = 0; p < k; ++p) {
        int piv = p;
        for (int i = p + 1; i < k; ++i)
            if (std::fabs(A[(size_t)i * k + p]) > std::fabs(A[(size_t)piv * k + p])) piv = i;
        if (A[(size_t)piv * k + p] == 0.0) return false;
        if (piv != p) {
            for (int j = 0; j < k; ++j) std::swap(A[(size_t)p * k + j], A[(size_t)piv * k + j]);
            std::swap(x[p], x[piv]);
        }
        for (int i = p + 1; i < k; ++i) {
            const double l = A[(size_t)i * k + p] / A[(size_t)p * k + p];
            for (int j = p; j < k; ++j) A[(size_t)i * k + j] -= l * A[(size_t)p * k + j];
            x[i] -= l * x[p];
        }
    }
    for (int i = k - 1; i >= 0; --i) {
        double v = x[i];
        for (int j = i + 1; j < k; ++j) v -= A[(size_t)i * k + j] * x[j];
        x[i] = v / A[(size_t)i * k + i];
    }
    return true;
}

// Condensation of a box matrix M (n x n, [interior k, interface]): g = f_B - M_BI M_II^{-1} f_I
static bool condense(const Mat& M, int n, int k, const std::vector<double>& f, std::vector<double>& g) {
    std::vector<double> y(f.begin(), f.begin() + k);
    if (!solve_lead(M, n, k, y)) return false;
    g.assign(f.begin() + k, f.end());
    for (int i = k; i < n; ++i)
        for (int j = 0; j < k; ++j) g[i - k] -= M[(size_t)i * n + j] * y[j];
    return true;
}

// Recovery: u_I = M_II^{-1} (f_I - M_IB u_B)
static bool recover(const Mat& M, int n, int k, const std::vector<double>& f, const std::vector<double>& uB,
                    std::vector<double>& uI) {
    uI.assign(f.begin(), f.begin() + k);
    for (int i = 0; i < k; ++i)
        for (int j = k; j < n; ++j) uI[i] -= M[(size_t)i * n + j] * uB[j - k];
    return solve_lead(M, n, k, uI);
}

// S = M[keep, keep] - M[keep, el] M[el, el]^{-1} M[el, keep]; el = the first k indices,
// keep the rest (partial pivoting within el)
static bool schur_tail(const Mat& M, int n, int k, Mat& S) {
    Mat A = M;
    for (int p = 0; p < k; ++p) {
        int piv = p;
        for (int i = p + 1; i < k; ++i)
            if (std::fabs(A[(size_t)i * n + p]) > std::fabs(A[(size_t)piv * n + p])) piv = i;
        if (A[(size_t)piv * n + p] == 0.0) return false;
        if (piv != p)
            for (int j = 0; j < n; ++j) std::swap(A[(size_t)p * n + j], A[(size_t)piv * n + j]);
        for (int i = p + 1; i < n; ++i) {
            const double l = A[(size_t)i * n + p] / A[(size_t)p * n + p];
            if (l == 0.0) continue;
            for (int j = p; j < n; ++j) A[(size_t)i * n + j] -= l * A[(size_t)p * n + j];
        }
    }
    const int m = n - k;
    S.assign((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) S[(size_t)i * m + j] = A[(size_t)(k + i) * n + k + j];
    return true;
}

int main(int argc, char** argv) {
    if (argc < 6) return 2;
    const int ns[3] = {atoi(argv[1]), atoi(argv[2]), atoi(argv[3])};
    const int m = atoi(argv[4]);
    std::mt19937_64 rng((unsigned long long)atoll(argv[5]));
    std::uniform_real_distribution<double> U(-1.0, 1.0);
    std::vector<int> slabs[3];
    for (int d = 0; d < 3; ++d)
        for (int s = 0; s < ns[d]; ++s) slabs[d].push_back(m > 0 ? m : 1 + (int)(rng() % (unsigned)(-m)));
    bddc_partition part;
    for (int d = 0; d < 3; ++d) {
        part.nsub[d] = ns[d];
        part.elems_per_slab[d] = slabs[d].data();
    }
    HostMesh hm;
    if (build_host_boxes(nullptr, &part, hm) != BDDC_OK) return 1;
    const HostMesh orig = hm;
    LocalND nd;
    if (build_local_nd(hm, nd) != BDDC_OK) {
        printf("plan failed\n");
        return 1;
    }
    const HostMesh& ch = nd.child;
    int nsep = 0;
    double worst = 0.0;
    for (int s = 0; s < hm.nsd; ++s) {
        const SubInfo& S = hm.sub[s];
        const SubInfo& O = orig.sub[s];
        nsep += S.nI;
        if (S.nB != O.nB || S.n != S.nI + S.nB) return 1;
        for (int j = 0; j < S.nB; ++j)
            if (S.dofs[S.nI + j] != O.dofs[O.nI + j]) return 1;       // interface order kept
        // children of s; every interior dof of s is a separator or interior to one child
        std::vector<int> kids;
        for (int c = 0; c < ch.nsd; ++c)
            if (nd.parent[c] == s) kids.push_back(c);
        std::unordered_map<int, int> cnt;
        for (int c : kids)
            for (int q = 0; q < ch.sub[c].nI; ++q) cnt[ch.sub[c].dofs[q]]++;
        for (int q = 0; q < S.nI; ++q) cnt[S.dofs[q]]++;
        for (int q = 0; q < O.nI; ++q)
            if (cnt[O.dofs[q]] != 1) {
                printf("interior dof %d covered %d times\n", O.dofs[q], cnt[O.dofs[q]]);
                return 1;
            }
        size_t tot = 0;
        for (auto& kv : cnt) tot += kv.second;
        if (tot != (size_t)O.nI) return 1;
        // maps hold the same global dofs
        for (int c : kids) {
            const SubInfo& K = ch.sub[c];
            for (int j = 0; j < K.nB; ++j) {
                const int li = nd.map[c][j];
                if (li < 0 || li >= S.n || S.dofs[li] != K.dofs[K.nI + j]) {
                    printf("map mismatch child %d\n", c);
                    return 1;
                }
            }
        }
        // algebra: random child matrices; one elimination vs the two levels
        std::unordered_map<int, int> full;        // dof -> index in [original interior, interface]
        for (int q = 0; q < O.n; ++q) full[O.dofs[q]] = q;
        Mat Af((size_t)O.n * O.n, 0.0), P((size_t)S.n * S.n, 0.0);
        std::unordered_map<int, double> fd;       // a random load on the subdomain's dofs
        for (int q = 0; q < O.n; ++q) fd[O.dofs[q]] = U(rng);
        std::vector<double> uB(S.nB);
        for (auto& v : uB) v = U(rng);
        std::vector<double> fp(S.n);              // the load in [separators, interface] with the children's corrections
        for (int q = 0; q < S.n; ++q) fp[q] = fd[S.dofs[q]];
        std::vector<Mat> Akid;
        for (int c : kids) {
            const SubInfo& K = ch.sub[c];
            Mat Ac((size_t)K.n * K.n);
            for (int i = 0; i < K.n; ++i)
                for (int j = 0; j < K.n; ++j) Ac[(size_t)i * K.n + j] = U(rng) + (i == j ? 2.0 * K.n : 0.0);
            Akid.push_back(Ac);
            std::vector<double> fc(K.n, 0.0), gc;           // the child's interior load; its boundary gets 0
            for (int q = 0; q < K.nI; ++q) fc[q] = fd[K.dofs[q]];
            if (!condense(Ac, K.n, K.nI, fc, gc)) return 1;
            for (int j = 0; j < K.nB; ++j) fp[nd.map[c][j]] += gc[j];
            for (int i = 0; i < K.n; ++i)
                for (int j = 0; j < K.n; ++j)
                    Af[(size_t)full[K.dofs[i]] * O.n + full[K.dofs[j]]] += Ac[(size_t)i * K.n + j];
            Mat Sc;
            if (!schur_tail(Ac, K.n, K.nI, Sc)) return 1;
            for (int a = 0; a < K.nB; ++a)
                for (int b = 0; b < K.nB; ++b) P[(size_t)nd.map[c][a] * S.n + nd.map[c][b]] += Sc[(size_t)a * K.nB + b];
        }
        Mat S1, S2;
        if (!schur_tail(Af, O.n, O.nI, S1) || !schur_tail(P, S.n, S.nI, S2)) return 1;
        // condensation: one dense step vs children then separators
        std::vector<double> f1(O.n), g1, g2;
        for (int q = 0; q < O.n; ++q) f1[q] = fd[O.dofs[q]];
        if (!condense(Af, O.n, O.nI, f1, g1) || !condense(P, S.n, S.nI, fp, g2)) return 1;
        // recovery: one dense step vs separators then children
        std::vector<double> u1, uS;
        if (!recover(Af, O.n, O.nI, f1, uB, u1)) return 1;
        if (!recover(P, S.n, S.nI, fp, uB, uS)) return 1;
        std::unordered_map<int, double> u2;       // dof -> value
        for (int q = 0; q < S.nI; ++q) u2[S.dofs[q]] = uS[q];
        for (int q = 0; q < S.nB; ++q) u2[S.dofs[S.nI + q]] = uB[q];
        for (size_t t = 0; t < kids.size(); ++t) {
            const SubInfo& K = ch.sub[kids[t]];
            std::vector<double> fc(K.n, 0.0), ub(K.nB), ui;
            for (int q = 0; q < K.nI; ++q) fc[q] = fd[K.dofs[q]];
            for (int j = 0; j < K.nB; ++j) ub[j] = u2[K.dofs[K.nI + j]];
            if (!recover(Akid[t], K.n, K.nI, fc, ub, ui)) return 1;
            for (int q = 0; q < K.nI; ++q) u2[K.dofs[q]] = ui[q];
        }
        double gn = 0.0, gd = 0.0, un = 0.0, ud = 0.0;
        for (int q = 0; q < S.nB; ++q) {
            gn = std::fmax(gn, std::fabs(g1[q] - g2[q]));
            gd = std::fmax(gd, std::fabs(g1[q]));
        }
        for (int q = 0; q < O.nI; ++q) {
            un = std::fmax(un, std::fabs(u1[q] - u2[O.dofs[q]]));
            ud = std::fmax(ud, std::fabs(u1[q]));
        }
        worst = std::fmax(worst, gd > 0 ? gn / gd : gn);
        worst = std::fmax(worst, ud > 0 ? un / ud : un);
        double num = 0.0, den = 0.0;
        for (size_t q = 0; q < S1.size(); ++q) {
            num = std::fmax(num, std::fabs(S1[q] - S2[q]));
            den = std::fmax(den, std::fabs(S1[q]));
        }
        worst = std::fmax(worst, den > 0 ? num / den : num);
    }
    printf("ok %.3e %d %d\n", worst, ch.nsd, nsep);
    return worst < 1e-10 ? 0 : 1;
}
