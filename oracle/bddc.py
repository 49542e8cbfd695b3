"""Adaptive BDDC for the stabilised advection-diffusion system (Sect. 3).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Plain FP64 numpy/scipy, one subdomain, face or edge at a time, in the order
and notation of the paper.  Readings of passages that are silent, ambiguous
or garbled:

* g^(i) = f_B - A_BI A_II^{-1} f_I (the printed formula drops A_BI).
* Deluxe scaling: D_X^(k) = (sum_{l in n(X)} S_XX^(l))^{-1} S_XX^(k), from the
  principal blocks of the non-symmetric local Schur complements; vertices are
  primal and get 1/|n(V)|.
* Generalised eigenproblems X v = lambda Y v with X, Y symmetric positive
  semi-definite are solved through the pencil X v = sigma (X+Y) v: directions
  where X+Y vanishes (eigenvalue <= 1e-12 * max) carry no energy and are
  dropped; lambda = sigma/(1-sigma) (infinite when 1-sigma <= 1e-12).
  Eigenvalues with lambda >= Theta are selected, i.e. sigma >= Theta/(1+Theta)
  less a 1e-12 slack (ties are selected).
* Pseudo-inverses (parallel sum, the elimination of (w^_E, w^_H) in the edge
  GEP) drop eigenvalues <= 1e-12 * max.
* Constraint spans: Q = orthonormal basis of the span of the selected
  constraint vectors, by SVD with relative rank tolerance 1e-10.
* New edge GEP with |n(E)| = m subdomains (the paper writes m = 3): w_check
  has m-1 blocks, the first subdomain of the sorted n(E) is the reference.
  The prior-selected primal set H_k of subdomain k holds all vertices of k and
  all face primal coordinates Q_F^T w_F of the faces of k; a primal unknown
  shared by several subdomains of n(E) is one coordinate of w^_H.
* Conventional edge GEP: B_E = sum_i sum_{k != i} D^(k)^T B_E^(i) D^(k).
* Theta_F = 1 + ln(m), natural log, m = largest slab element count over the
  subdomains of the face; Theta_E = 10.
* M^{-1} = R~^T D~ S~^{-1} D~^T R~ is applied literally: residuals are split
  with D^T, solutions averaged with D.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla

from . import fem
from .mesh import Mesh

EIG_DROP = 1e-12
RANK_TOL = 1e-10


# ---------------------------------------------------------------------------
# small dense building blocks
# ---------------------------------------------------------------------------
def schur(M, keep):
    """M_kk - M_ke M_ee^{-1} M_ek, eliminating every index not in `keep`."""
    keep = np.asarray(keep, dtype=int)
    mask = np.ones(M.shape[0], dtype=bool)
    mask[keep] = False
    el = np.nonzero(mask)[0]
    if el.size == 0:
        return M[np.ix_(keep, keep)].copy()
    X = np.linalg.solve(M[np.ix_(el, el)], M[np.ix_(el, keep)])
    return M[np.ix_(keep, keep)] - M[np.ix_(keep, el)] @ X


def pinv_sym(A, drop=EIG_DROP):
    """Pseudo-inverse of a symmetric positive semi-definite matrix."""
    A = 0.5 * (A + A.T)
    if A.shape[0] == 0:
        return A.copy()
    lam, U = np.linalg.eigh(A)
    top = max(abs(lam).max(), 0.0)
    keep = lam > drop * top if top > 0 else np.zeros_like(lam, dtype=bool)
    return (U[:, keep] / lam[keep]) @ U[:, keep].T


def pinv_schur(M, w, r, drop=EIG_DROP):
    """M_ww - M_wr M_rr^+ M_rw (generalised Schur complement of a PSD matrix)."""
    w = np.asarray(w, dtype=int)
    r = np.asarray(r, dtype=int)
    return M[np.ix_(w, w)] - M[np.ix_(w, r)] @ pinv_sym(M[np.ix_(r, r)], drop) @ M[np.ix_(r, w)]


def parallel_sum(A, B, drop=EIG_DROP):
    """A : B = A (A + B)^+ B  (Anderson-Duffin parallel sum, Sect. 3)."""
    return A @ pinv_sym(A + B, drop) @ B


def sigma_pencil(X, Y, drop=EIG_DROP):
    """Eigenpairs of X v = lambda Y v through X v = sigma (X+Y) v.

    Returns (sigma, lambda, V), sorted by decreasing sigma, V normalised so that
    V^T (X+Y) V = I.  Directions in the kernel of X+Y are dropped.
    """
    X = 0.5 * (X + X.T)
    Y = 0.5 * (Y + Y.T)
    K = X + Y
    n = K.shape[0]
    if n == 0:
        return np.zeros(0), np.zeros(0), np.zeros((0, 0))
    kap, U = np.linalg.eigh(K)
    top = kap.max()
    if top <= 0:
        return np.zeros(0), np.zeros(0), np.zeros((n, 0))
    keep = kap > drop * top
    W = U[:, keep] / np.sqrt(kap[keep])
    C = W.T @ X @ W
    sig, Yv = np.linalg.eigh(0.5 * (C + C.T))
    order = np.argsort(-sig)
    sig = sig[order]
    V = W @ Yv[:, order]
    with np.errstate(divide='ignore'):
        lam = np.where(1.0 - sig <= 1e-12, np.inf, sig / np.maximum(1.0 - sig, 1e-300))
    return sig, lam, V


def select(sig, theta):
    """Indices with lambda >= theta (sigma >= theta/(1+theta) - 1e-12)."""
    return np.nonzero(sig >= theta / (1.0 + theta) - 1e-12)[0]


def orth(C, tol=RANK_TOL):
    """Orthonormal basis of range(C) by SVD, relative rank tolerance `tol`."""
    if C.shape[1] == 0:
        return np.zeros((C.shape[0], 0))
    U, s, _ = np.linalg.svd(C, full_matrices=False)
    if s.size == 0 or s[0] == 0.0:
        return np.zeros((C.shape[0], 0))
    r = int(np.sum(s > tol * s[0]))
    return U[:, :r]


def complement(Q):
    """Orthonormal basis of the orthogonal complement of range(Q)."""
    n = Q.shape[0]
    if Q.shape[1] == 0:
        return np.eye(n)
    if Q.shape[1] == n:
        return np.zeros((n, 0))
    return sla.null_space(Q.T)


# ---------------------------------------------------------------------------
# the solver
# ---------------------------------------------------------------------------
class BDDC:
    """Adaptive BDDC on a tensor partition; FP64 dense per subdomain.

    edge_gep: 'new' (this paper), 'old' (conventional edge GEP), 'none'
    (vertices and faces only).  face_gep=False gives vertex-only constraints
    on faces.  all_primal=True makes every interface dof primal.
    """

    def __init__(self, prob, edge_gep='new', face_gep=True, all_primal=False,
                 theta_E=None, theta_F=None, ref_choice=None):
        self.prob = prob
        self.mesh = Mesh(prob.slabs)
        mesh = self.mesh
        self.theta_E = prob.theta_E if theta_E is None else theta_E
        self.theta_F_fixed = prob.theta_F if theta_F is None else theta_F
        self.edge_mode = edge_gep
        self.use_face_gep = face_gep
        self.all_primal = all_primal
        self.ref_choice = ref_choice or {}
        f_node = prob.f_node if prob.f_node is not None else np.zeros(prob.beta_node.shape[0])
        Ae, Fe, nodes = fem.element_matrices(mesh, prob.nu_elem, prob.beta_node, f_node, prob.c,
                                             element=getattr(prob, 'element', 'q1'))
        Fe = fem.lift_dirichlet(mesh, Ae, Fe, nodes, getattr(prob, 'dirichlet_node', None))
        self.Ae, self.Fe, self.enodes = Ae, Fe, nodes
        self.A, F = fem.assemble_global(mesh, Ae, Fe, nodes)
        self.F = F if prob.load is None else np.asarray(prob.load, dtype=float)
        self._subdomains()
        self._deluxe()
        self._faces()
        self._edges()
        self._constraints()
        self._kkt()

    # ---- O4: subdomain matrices and Schur complements (Sect. 3) ----------
    def _subdomains(self):
        mesh = self.mesh
        self.Aloc, self.floc, self.S, self.B = [], [], [], []
        self.gidx = []            # global Gamma index of each local interface dof
        for s in range(mesh.nsd):
            A, f = fem.assemble_subdomain(mesh, s, self.Ae, self.Fe, self.enodes)
            nI = mesh.sub_nI[s]
            AII, AIB = A[:nI, :nI], A[:nI, nI:]
            ABI, ABB = A[nI:, :nI], A[nI:, nI:]
            S = ABB - ABI @ np.linalg.solve(AII, AIB) if nI else ABB.copy()
            self.Aloc.append(A)
            self.floc.append(f)
            self.S.append(S)
            self.B.append(0.5 * (S + S.T))
            self.gidx.append(np.array([mesh.gamma_index[int(d)] for d in mesh.interface_local(s)]))
        self.nG = len(mesh.gamma)

    def local_pos(self, s, dofs):
        return np.searchsorted(self.mesh.interface_local(s), dofs)

    def local_loads(self, F):
        """Per-subdomain loads f^(i): interior entries whole, interface split evenly."""
        mesh = self.mesh
        cnt = np.zeros(mesh.ndof)
        for s in range(mesh.nsd):
            cnt[mesh.sub_dofs[s]] += 1
        return [F[mesh.sub_dofs[s]] / cnt[mesh.sub_dofs[s]] for s in range(mesh.nsd)]

    def condense(self, F=None):
        """g = sum_i R_i^T g^(i), g^(i) = f_B - A_BI A_II^{-1} f_I."""
        mesh = self.mesh
        F = self.F if F is None else F
        fl = self.local_loads(F)
        g = np.zeros(self.nG)
        for s in range(mesh.nsd):
            nI = mesh.sub_nI[s]
            A = self.Aloc[s]
            gs = fl[s][nI:] - A[nI:, :nI] @ np.linalg.solve(A[:nI, :nI], fl[s][:nI])
            np.add.at(g, self.gidx[s], gs)
        return g

    def recover(self, uG, F=None):
        """Global solution: u_I = A_II^{-1}(f_I - A_IB u_B) per subdomain."""
        mesh = self.mesh
        F = self.F if F is None else F
        u = np.zeros(mesh.ndof)
        u[mesh.gamma] = uG
        for s in range(mesh.nsd):
            nI = mesh.sub_nI[s]
            A = self.Aloc[s]
            uB = uG[self.gidx[s]]
            fI = F[mesh.sub_dofs[s][:nI]]
            u[mesh.sub_dofs[s][:nI]] = np.linalg.solve(A[:nI, :nI], fI - A[:nI, nI:] @ uB)
        return u

    def apply_S(self, x):
        """y = sum_i R_i^T S^(i) R_i x (the Schur system operator)."""
        y = np.zeros(self.nG)
        for s in range(self.mesh.nsd):
            np.add.at(y, self.gidx[s], self.S[s] @ x[self.gidx[s]])
        return y

    # ---- O7: deluxe scaling ------------------------------------------------
    def _deluxe(self):
        self.D = {}               # (entity index, subdomain) -> D_X^(k)
        self.pos = {}             # (entity index, subdomain) -> local interface positions
        for ei, e in enumerate(self.mesh.entities):
            for k in e['subs']:
                self.pos[(ei, k)] = self.local_pos(k, e['dofs'])
            if e['kind'] == 'V':
                for k in e['subs']:
                    self.D[(ei, k)] = np.eye(1) / len(e['subs'])
                continue
            blocks = {k: self.S[k][np.ix_(self.pos[(ei, k)], self.pos[(ei, k)])] for k in e['subs']}
            tot = sum(blocks.values())
            for k in e['subs']:
                self.D[(ei, k)] = np.linalg.solve(tot, blocks[k])

    def theta_F_of(self, e):
        if self.theta_F_fixed is not None:
            return self.theta_F_fixed
        mesh = self.mesh
        m = 0
        for k in e['subs']:
            c = mesh.sub_coords(k)
            m = max(m, max(mesh.slabs[d][c[d]] for d in range(3)))
        return 1.0 + math.log(m)

    # ---- O8: face GEP (Sect. 3, adaptive face constraints) -----------------
    def face_gep(self, ei):
        e = self.mesh.entities[ei]
        i, j = e['subs']
        pi, pj = self.pos[(ei, i)], self.pos[(ei, j)]
        Di, Dj = self.D[(ei, i)], self.D[(ei, j)]
        BFi = self.B[i][np.ix_(pi, pi)]
        BFj = self.B[j][np.ix_(pj, pj)]
        BF = Dj.T @ BFi @ Dj + Di.T @ BFj @ Di
        Bti = schur(self.B[i], pi)
        Btj = schur(self.B[j], pj)
        Bt = parallel_sum(Bti, Btj)
        sig, lam, V = sigma_pencil(BF, Bt)
        sel = select(sig, self.theta_F_of(e))
        Q = orth(BF @ V[:, sel])
        return dict(BF=BF, Bt=Bt, Bti=Bti, Btj=Btj, sig=sig, lam=lam, V=V, sel=sel, Q=Q)

    def _faces(self):
        self.Q = {}
        self.face_info = {}
        for ei, e in enumerate(self.mesh.entities):
            if e['kind'] == 'V':
                self.Q[ei] = np.eye(1)
            elif e['kind'] == 'F':
                n = len(e['dofs'])
                if self.all_primal:
                    self.Q[ei] = np.eye(n)
                elif not self.use_face_gep:
                    self.Q[ei] = np.zeros((n, 0))
                else:
                    info = self.face_gep(ei)
                    self.face_info[ei] = info
                    self.Q[ei] = info['Q']

    # ---- O9/O10: new edge GEP on prior-selected primal constraints ---------
    def face_basis(self, s):
        """Orthogonal T_s acting on faces only: w_F = [Q_F, Q_F^perp] y_F.

        Returns T (nB x nB) and the list of H_k coordinate keys with their
        positions in the transformed coordinates."""
        mesh = self.mesh
        nB = len(mesh.interface_local(s))
        T = np.eye(nB)
        hkeys, hpos = [], []
        for ei in mesh.sub_entities[s]:
            e = mesh.entities[ei]
            p = self.pos[(ei, s)]
            if e['kind'] == 'V':
                hkeys.append(('V', ei, 0))
                hpos.append(int(p[0]))
            elif e['kind'] == 'F':
                Q = self.Q[ei]
                T[np.ix_(p, p)] = np.hstack([Q, complement(Q)])
                for l in range(Q.shape[1]):
                    hkeys.append(('F', ei, l))
                    hpos.append(int(p[l]))
        return T, hkeys, hpos

    def edge_gep_new(self, ei, ref=None):
        mesh = self.mesh
        e = mesh.entities[ei]
        subs = list(e['subs'])
        if ref is not None:
            subs.remove(ref)
            subs = [ref] + subs
        m = len(subs)
        n = len(e['dofs'])
        I = np.eye(n)
        D = {k: self.D[(ei, k)] for k in subs}
        BE = {k: self.B[k][np.ix_(self.pos[(ei, k)], self.pos[(ei, k)])] for k in subs}
        # T_E^(k): w_k,E = T^(k) (w_check_{k_2..k_m}; w^_E)   (eq. equ-trans)
        Tk = {}
        for k in subs:
            blocks = []
            for kl in subs[1:]:
                blocks.append(I - D[kl] if k == kl else -D[kl])
            blocks.append(I)
            Tk[k] = np.hstack(blocks)
        nw = (m - 1) * n
        Tbar = np.vstack([Tk[k][:, :nw] for k in subs])
        M_E = Tbar.T @ sla.block_diag(*[BE[k] for k in subs]) @ Tbar
        # B~^(k): Schur complement onto E and the prior primal set H_k
        Bt, hk = {}, {}
        for k in subs:
            T, hkeys, hpos = self.face_basis(k)
            Bp = T.T @ self.B[k] @ T
            keep = list(self.pos[(ei, k)]) + hpos
            Bt[k] = schur(Bp, keep)
            hk[k] = hkeys
        Hall = sorted(set(key for k in subs for key in hk[k]))
        hidx = {key: t for t, key in enumerate(Hall)}
        nz = nw + n + len(Hall)
        Bt_E = np.zeros((nz, nz))
        for k in subs:
            J = np.zeros((n + len(hk[k]), nz))
            J[:n, :nw + n] = Tk[k]
            for t, key in enumerate(hk[k]):
                J[n + t, nw + n + hidx[key]] = 1.0
            Bt_E += J.T @ Bt[k] @ J
        BB = pinv_schur(Bt_E, np.arange(nw), np.arange(nw, nz))
        sig, lam, V = sigma_pencil(M_E, BB)
        sel = select(sig, self.theta_E)
        Cm = M_E @ V[:, sel]
        cols = [Cm[b * n:(b + 1) * n, l] for l in range(Cm.shape[1]) for b in range(m - 1)]
        Q = orth(np.array(cols).T if cols else np.zeros((n, 0)))
        return dict(M_E=M_E, BB=BB, Bt_E=Bt_E, sig=sig, lam=lam, V=V, sel=sel, Q=Q,
                    subs=subs, Tk=Tk, Bt=Bt, H=Hall, hk=hk)

    def edge_gep_old(self, ei):
        """Conventional edge GEP B_E v = lambda B~_E v (comparison method)."""
        e = self.mesh.entities[ei]
        subs = list(e['subs'])
        D = {k: self.D[(ei, k)] for k in subs}
        BE = {k: self.B[k][np.ix_(self.pos[(ei, k)], self.pos[(ei, k)])] for k in subs}
        n = len(e['dofs'])
        BEs = np.zeros((n, n))
        for i in subs:
            for k in subs:
                if k != i:
                    BEs += D[k].T @ BE[i] @ D[k]
        Bt = None
        for k in subs:
            Btk = schur(self.B[k], self.pos[(ei, k)])
            Bt = Btk if Bt is None else parallel_sum(Bt, Btk)
        sig, lam, V = sigma_pencil(BEs, Bt)
        sel = select(sig, self.theta_E)
        Q = orth(BEs @ V[:, sel])
        return dict(BE=BEs, Bt=Bt, sig=sig, lam=lam, V=V, sel=sel, Q=Q)

    def _edges(self):
        self.edge_info = {}
        for ei, e in enumerate(self.mesh.entities):
            if e['kind'] != 'E':
                continue
            n = len(e['dofs'])
            if self.all_primal:
                self.Q[ei] = np.eye(n)
            elif self.edge_mode == 'new':
                info = self.edge_gep_new(ei, self.ref_choice.get(ei))
                self.edge_info[ei] = info
                self.Q[ei] = info['Q']
            elif self.edge_mode == 'old':
                info = self.edge_gep_old(ei)
                self.edge_info[ei] = info
                self.Q[ei] = info['Q']
            else:
                self.Q[ei] = np.zeros((n, 0))

    # ---- O12: primal constraints ------------------------------------------
    def _constraints(self):
        mesh = self.mesh
        self.prim_off = {}
        n = 0
        for kind in ('V', 'F', 'E'):
            for ei, e in enumerate(mesh.entities):
                if e['kind'] == kind:
                    self.prim_off[ei] = n
                    n += self.Q[ei].shape[1]
        self.nPi = n
        self.pnumF = sum(self.Q[ei].shape[1] for ei, e in enumerate(mesh.entities) if e['kind'] == 'F')
        self.pnumE = sum(self.Q[ei].shape[1] for ei, e in enumerate(mesh.entities) if e['kind'] == 'E')
        self.C, self.RPi, self.TPi, self.TDl, self.Dmat = [], [], [], [], []
        for s in range(mesh.nsd):
            nB = len(mesh.interface_local(s))
            rows, rpi, tdl = [], [], []
            Dm = np.zeros((nB, nB))
            for ei in mesh.sub_entities[s]:
                p = self.pos[(ei, s)]
                Q = self.Q[ei]
                for l in range(Q.shape[1]):
                    r = np.zeros(nB)
                    r[p] = Q[:, l]
                    rows.append(r)
                    rpi.append(self.prim_off[ei] + l)
                Qp = complement(Q)
                for l in range(Qp.shape[1]):
                    c = np.zeros(nB)
                    c[p] = Qp[:, l]
                    tdl.append(c)
                Dm[np.ix_(p, p)] = self.D[(ei, s)]
            C = np.array(rows) if rows else np.zeros((0, nB))
            self.C.append(C)
            self.RPi.append(np.array(rpi, dtype=int))
            self.TPi.append(C.T.copy())
            self.TDl.append(np.array(tdl).T if tdl else np.zeros((nB, 0)))
            self.Dmat.append(Dm)

    # ---- O13: S~^{-1} through the constrained (KKT) local problems ---------
    def _kkt(self):
        mesh = self.mesh
        self.Kf, self.Phi, self.Psi = [], [], []
        SPi = np.zeros((self.nPi, self.nPi))
        for s in range(mesh.nsd):
            S, C = self.S[s], self.C[s]
            nB, nc = S.shape[0], C.shape[0]
            K = np.block([[S, C.T], [C, np.zeros((nc, nc))]])
            Kt = np.block([[S.T, C.T], [C, np.zeros((nc, nc))]])
            rhs = np.vstack([np.zeros((nB, nc)), np.eye(nc)])
            Phi = np.linalg.solve(K, rhs)[:nB]
            Psi = np.linalg.solve(Kt, rhs)[:nB]
            self.Kf.append(sla.lu_factor(K))
            self.Phi.append(Phi)
            self.Psi.append(Psi)
            r = self.RPi[s]
            SPi[np.ix_(r, r)] += Psi.T @ S @ Phi
        self.SPi = SPi

    def G_apply(self, s, rho):
        nB = self.S[s].shape[0]
        nc = self.C[s].shape[0]
        return sla.lu_solve(self.Kf[s], np.concatenate([rho, np.zeros(nc)]))[:nB]

    def Stilde_inv(self, rhos):
        """Per-subdomain w_i of S~^{-1} applied to the local functionals rho_i."""
        rPi = np.zeros(self.nPi)
        for s, rho in enumerate(rhos):
            np.add.at(rPi, self.RPi[s], self.Psi[s].T @ rho)
        uPi = np.linalg.solve(self.SPi, rPi) if self.nPi else rPi
        return [self.G_apply(s, rho) + self.Phi[s] @ uPi[self.RPi[s]] for s, rho in enumerate(rhos)]

    def apply_M(self, r):
        """z = M^{-1} r = sum_i R_i^T D_i (S~^{-1} (D_j^T R_j r)_j)_i   (Sect. 3)."""
        rhos = [self.Dmat[s].T @ r[self.gidx[s]] for s in range(self.mesh.nsd)]
        ws = self.Stilde_inv(rhos)
        z = np.zeros(self.nG)
        for s in range(self.mesh.nsd):
            np.add.at(z, self.gidx[s], self.Dmat[s] @ ws[s])
        return z

    # ---- second route: S~ assembled on the partially coupled space W~ ------
    def wtilde_operator(self):
        """Dense S~ = sum R~^(i)T S^(i) R~^(i) and the maps R~^(i) (small cases)."""
        mesh = self.mesh
        offs, n = [], self.nPi
        for s in range(mesh.nsd):
            offs.append(n)
            n += self.TDl[s].shape[1]
        Rt = []
        St = np.zeros((n, n))
        for s in range(mesh.nsd):
            nB = self.S[s].shape[0]
            R = np.zeros((nB, n))
            R[:, self.RPi[s]] = self.TPi[s]
            R[:, offs[s]:offs[s] + self.TDl[s].shape[1]] = self.TDl[s]
            Rt.append(R)
            St += R.T @ self.S[s] @ R
        return St, Rt

    def apply_M_wtilde(self, r, St=None, Rt=None):
        if St is None:
            St, Rt = self.wtilde_operator()
        b = sum(Rt[s].T @ (self.Dmat[s].T @ r[self.gidx[s]]) for s in range(self.mesh.nsd))
        y = np.linalg.solve(St, b)
        z = np.zeros(self.nG)
        for s in range(self.mesh.nsd):
            np.add.at(z, self.gidx[s], self.Dmat[s] @ (Rt[s] @ y))
        return z

    # ---- dense global operators (tests) ------------------------------------
    def S_dense(self):
        Sg = np.zeros((self.nG, self.nG))
        for s in range(self.mesh.nsd):
            g = self.gidx[s]
            Sg[np.ix_(g, g)] += self.S[s]
        return Sg

    def M_dense(self):
        return np.array([self.apply_M(e) for e in np.eye(self.nG)]).T

    # ---- solve --------------------------------------------------------------
    def solve(self, rtol=None, restart=None, max_iter=None, precondition=True, F=None):
        from .krylov import gmres
        p = self.prob
        rtol = p.rtol if rtol is None else rtol
        restart = p.restart if restart is None else restart
        max_iter = p.max_iter if max_iter is None else max_iter
        Fv = self.F if F is None else F
        if Fv.ndim == 2:
            outs = [self.solve(rtol, restart, max_iter, precondition, Fv[:, c]) for c in range(Fv.shape[1])]
            return np.stack([o[0] for o in outs], axis=1), [o[1] for o in outs]
        g = self.condense(Fv)
        M = self.apply_M if precondition else (lambda v: v)
        uG, info = gmres(self.apply_S, g, M, rtol=rtol, restart=restart, max_iter=max_iter)
        u = self.recover(uG, Fv)
        info['pnumF'] = self.pnumF
        info['pnumE'] = self.pnumE
        info['nPi'] = self.nPi
        info['true_relres'] = float(np.linalg.norm(g - self.apply_S(uG)) / np.linalg.norm(g))
        return u, info
