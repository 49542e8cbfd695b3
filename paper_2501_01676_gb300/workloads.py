"""Seeded synthetic inputs for the advection-diffusion BDDC solver.

This module holds only input recipes (mesh slabs and coefficient fields).  It
contains none of the method's arithmetic, so both the FP64 CPU oracle (in the
tests) and the CUDA library may be fed from it.

Every problem lives on the unit cube with homogeneous Dirichlet conditions
(model problem of Sect. 2).  Fields are returned as plain numpy arrays:

* ``nu_elem``  (nelem,)     viscosity, constant per element, element id
                            ex + Ex*(ey + Ey*ez)
* ``beta_node`` (nnodes, 3) velocity at the nodes, node id ix + (Ex+1)*(iy + (Ey+1)*iz)
* ``f_node``   (nnodes,)    source at the nodes (None when ``load`` is given)
* ``load``     (ndof, nrhs) assembled nodal loads on the free dofs, or None

The five recipes follow the synthetic workloads of the benchmark suite:
unit cube, Q1 hexes, tensor partitions.  Seeds are 20250103 + recipe id.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np


@dataclass
class Problem:
    name: str
    slabs: List[List[int]]
    nu_elem: np.ndarray
    beta_node: np.ndarray
    f_node: Optional[np.ndarray]
    load: Optional[np.ndarray] = None
    c: float = 0.0
    theta_E: float = 10.0
    theta_F: Optional[float] = None      # None: 1 + ln(H/h)
    restart: int = 0                     # 0: full GMRES
    rtol: float = 1e-8
    max_iter: int = 300
    meta: dict = field(default_factory=dict)
    element: str = 'q1'                  # 'q1' bricks, 'p1' the six Kuhn tetrahedra of each brick
    dirichlet_node: Optional[np.ndarray] = None   # Dirichlet values at the nodes (None: zero)

    @property
    def ne(self):
        return [sum(s) for s in self.slabs]

    @property
    def nrhs(self):
        return 1 if self.load is None else self.load.shape[1]


def _grid(slabs):
    ne = [sum(s) for s in slabs]
    h = [1.0 / n for n in ne]
    ix = np.arange(ne[0] + 1) * h[0]
    iy = np.arange(ne[1] + 1) * h[1]
    iz = np.arange(ne[2] + 1) * h[2]
    Z, Y, X = np.meshgrid(iz, iy, ix, indexing='ij')           # x fastest in ravel
    return ne, h, X.ravel(), Y.ravel(), Z.ravel()


def _elem_centres(slabs):
    ne = [sum(s) for s in slabs]
    h = [1.0 / n for n in ne]
    cz, cy, cx = np.meshgrid((np.arange(ne[2]) + 0.5) * h[2], (np.arange(ne[1]) + 0.5) * h[1],
                             (np.arange(ne[0]) + 0.5) * h[0], indexing='ij')
    return cx.ravel(), cy.ravel(), cz.ravel()


def _elem_subdomain(slabs):
    """Subdomain id of every element."""
    ne = [sum(s) for s in slabs]
    owners = []
    for d in range(3):
        o = np.repeat(np.arange(len(slabs[d])), slabs[d])
        owners.append(o)
    ez, ey, ex = np.meshgrid(np.arange(ne[2]), np.arange(ne[1]), np.arange(ne[0]), indexing='ij')
    sx, sy, sz = owners[0][ex.ravel()], owners[1][ey.ravel()], owners[2][ez.ravel()]
    nx, ny = len(slabs[0]), len(slabs[1])
    return sx + nx * (sy + ny * sz)


def ndof_of(slabs):
    ne = [sum(s) for s in slabs]
    return (ne[0] - 1) * (ne[1] - 1) * (ne[2] - 1)


def uniform(nsub, m, nu=1.0, beta=(1.0, 1.0, 1.0), f=1.0, name='uniform', **kw):
    """Uniform tensor partition nsub^3 with H/h = m, constant nu, beta and f."""
    ns = nsub if isinstance(nsub, (list, tuple)) else (nsub, nsub, nsub)
    slabs = [[m] * ns[d] for d in range(3)]
    ne, h, X, Y, Z = _grid(slabs)
    nelem = ne[0] * ne[1] * ne[2]
    beta_node = np.tile(np.asarray(beta, dtype=float), (X.size, 1))
    return Problem(name, slabs, np.full(nelem, float(nu)), beta_node, np.full(X.size, float(f)), **kw)


def mms(nsub=2, m=4, nu=1.0, beta=(1.0, 1.0, 1.0)):
    """u = sin(pi x) sin(pi y) sin(pi z); f = -nu Lap u + beta.grad u at the nodes."""
    p = uniform(nsub, m, nu=nu, beta=beta, name='mms')
    _, _, X, Y, Z = _grid(p.slabs)
    pi = math.pi
    sx, sy, sz = np.sin(pi * X), np.sin(pi * Y), np.sin(pi * Z)
    cx, cy, cz = np.cos(pi * X), np.cos(pi * Y), np.cos(pi * Z)
    u = sx * sy * sz
    f = 3 * pi * pi * nu * u + pi * (beta[0] * cx * sy * sz + beta[1] * sx * cy * sz + beta[2] * sx * sy * cz)
    p.f_node = f
    p.meta['u_exact'] = lambda x, y, z: np.sin(pi * x) * np.sin(pi * y) * np.sin(pi * z)
    return p


def config1():
    """2x2x2 subdomains, H/h=4, nu=1, beta=(1,1,1), manufactured sin-sin-sin solution."""
    p = mms(2, 4, 1.0, (1.0, 1.0, 1.0))
    p.name = 'c1_2x2x2_m4_mms'
    return p


def config2():
    """4x4x4 subdomains, H/h=8, nu=0.01, beta=(1,0.5,0.25), f=1, GMRES(50)."""
    return uniform(4, 8, nu=0.01, beta=(1.0, 0.5, 0.25), f=1.0, name='c2_4x4x4_m8', restart=50)


def config3(seed_offset=3):
    """8x8x8 subdomains, H/h=8, nu per subdomain 10^U(-4,0), rotating beta, f=1."""
    rng = np.random.default_rng(20250103 + seed_offset)
    slabs = [[8] * 8 for _ in range(3)]
    ne, h, X, Y, Z = _grid(slabs)
    sub = _elem_subdomain(slabs)
    nu_sub = 10.0 ** rng.uniform(-4.0, 0.0, size=512)
    beta = np.stack([-(Y - 0.5), X - 0.5, np.full_like(X, 0.1)], axis=1)
    return Problem('c3_8x8x8_m8_jumps', slabs, nu_sub[sub], beta, np.ones(X.size))


def config3_layers(layers=2, seed_offset=3):
    """The first `layers` of the 8 subdomain layers (in z) of the 8x8x8 jump
    workload as a problem of its own on the unit cube: the same per-subdomain
    nu and H/h, 64 * layers subdomains.  A bounded timing sample of that
    workload (same per-subdomain work)."""
    rng = np.random.default_rng(20250103 + seed_offset)
    nu_all = 10.0 ** rng.uniform(-4.0, 0.0, size=512)
    slabs = [[8] * 8, [8] * 8, [8] * layers]
    ne, h, X, Y, Z = _grid(slabs)
    sub = _elem_subdomain(slabs)
    beta = np.stack([-(Y - 0.5), X - 0.5, np.full_like(X, 0.1)], axis=1)
    return Problem(f'c3_layers_{layers}', slabs, nu_all[:64 * layers][sub], beta, np.ones(X.size))


def config4(seed_offset=4, nrhs=64):
    """6x6x6 subdomains, per-slab H/h ~ U{6..10}, nu=1e-2, beta=(1,1,0), nrhs N(0,1) loads."""
    rng = np.random.default_rng(20250103 + seed_offset)
    slabs = [list(rng.integers(6, 11, size=6)) for _ in range(3)]
    ne, h, X, Y, Z = _grid(slabs)
    nelem = ne[0] * ne[1] * ne[2]
    beta = np.tile(np.array([1.0, 1.0, 0.0]), (X.size, 1))
    load = rng.standard_normal((ndof_of(slabs), nrhs))
    return Problem('c4_6x6x6_uneven_64rhs', slabs, np.full(nelem, 1e-2), beta, None, load=load)


def fourier_beta(rng, X, Y, Z, modes=4):
    """Divergence-free sum of sine modes, sum of amplitudes 1 (so |beta| <= 1)."""
    pts = np.stack([X, Y, Z], axis=1)
    ks, amps, phis = [], [], []
    for _ in range(modes):
        while True:
            k = rng.integers(0, 3, size=3)
            if k.any():
                break
        a = rng.standard_normal(3)
        a -= (a @ k) / (k @ k) * k                                   # a perpendicular to k
        ks.append(k.astype(float)); amps.append(a); phis.append(rng.uniform(0, 2 * math.pi))
    scale = 1.0 / sum(np.linalg.norm(a) for a in amps)
    beta = np.zeros_like(pts)
    for k, a, ph in zip(ks, amps, phis):
        beta += scale * np.outer(np.sin(2 * math.pi * pts @ k + ph), a)
    return beta


def channels(rng, slabs, count=12, nu_bg=1e-4, nu_ch=1.0):
    """nu_bg everywhere except `count` straight tubes, one element wide, of nu_ch."""
    ne = [sum(s) for s in slabs]
    nu = np.full(ne[0] * ne[1] * ne[2], nu_bg).reshape(ne[2], ne[1], ne[0])
    for _ in range(count):
        axis = int(rng.integers(0, 3))
        a, b = [d for d in range(3) if d != axis]
        pa, pb = int(rng.integers(0, ne[a])), int(rng.integers(0, ne[b]))
        idx = [slice(None)] * 3
        # array axes are (z, y, x): direction d lives on array axis 2-d
        idx[2 - a] = pa
        idx[2 - b] = pb
        nu[tuple(idx)] = nu_ch
    return nu.ravel()


def config5(seed_offset=5, nsub=8, m=8):
    """8x8x8 subdomains, H/h=8, nu=1e-4 with 12 channels of nu=1, 4-mode Fourier beta, f=1."""
    rng = np.random.default_rng(20250103 + seed_offset)
    slabs = [[m] * nsub for _ in range(3)]
    ne, h, X, Y, Z = _grid(slabs)
    nu = channels(rng, slabs, 12)
    beta = fourier_beta(rng, X, Y, Z)
    return Problem('c5_8x8x8_m8_channels', slabs, nu, beta, np.ones(X.size))


def random_small(seed, nsub=(2, 2, 2), m=3, nu_range=(-3.0, 0.0), rotate=True):
    """Small random-coefficient problem (per-element log-uniform nu) for tests."""
    rng = np.random.default_rng(seed)
    ns = nsub if isinstance(nsub, (list, tuple)) else (nsub,) * 3
    ms = m if isinstance(m, (list, tuple)) else (m,) * 3
    slabs = [[ms[d]] * ns[d] for d in range(3)]
    ne, h, X, Y, Z = _grid(slabs)
    nelem = ne[0] * ne[1] * ne[2]
    nu = 10.0 ** rng.uniform(nu_range[0], nu_range[1], size=nelem)
    if rotate:
        beta = np.stack([-(Y - 0.5), X - 0.5, np.full_like(X, 0.1)], axis=1)
    else:
        beta = np.tile(rng.standard_normal(3), (X.size, 1))
    return Problem(f'random_s{seed}', slabs, nu, beta, rng.standard_normal(X.size))


def rotating_checker(test=3, nsub=2, m=6, nu_hi=1.0, nu_lo=1e-7, c=1.0):
    """The coefficient patterns of the paper's uniform-partition tests (Sect. 4)
    moved to the unit cube: beta = (-2 pi (y-1/2), 2 pi (x-1/2), sin 2 pi (x-1/2)),
    reaction c, nu_hi / nu_lo on two subdomain classes -- test 1: halves in x,
    test 2: columns (x+y parity), test 3: checkerboard (x+y+z parity); f = 1 and
    homogeneous Dirichlet conditions instead of the paper's boundary data."""
    p = uniform(nsub, m, nu=1.0, beta=(0.0, 0.0, 0.0), f=1.0, name=f'rot_checker_t{test}')
    ne, h, X, Y, Z = _grid(p.slabs)
    p.beta_node = np.stack([-2 * math.pi * (Y - 0.5), 2 * math.pi * (X - 0.5), np.sin(2 * math.pi * (X - 0.5))], axis=1)
    p.c = c
    sub = _elem_subdomain(p.slabs)
    ns = nsub if isinstance(nsub, (list, tuple)) else (nsub,) * 3
    sx, sy, sz = sub % ns[0], (sub // ns[0]) % ns[1], sub // (ns[0] * ns[1])
    if test == 1:
        hi = sx < (ns[0] + 1) // 2
    elif test == 2:
        hi = (sx + sy) % 2 == 0
    else:
        hi = (sx + sy + sz) % 2 == 0
    p.nu_elem = np.where(hi, nu_hi, nu_lo)
    return p


CONFIGS = {1: config1, 2: config2, 3: config3, 4: config4, 5: config5}


# Example 4.1 of the paper (Sect. 4): Omega = (-1/2,1/2)^2 x (0,1), 2 x 2 x 2 cubic
# subdomains of m^3 cubes, each cube split into six tetrahedra (P1), c = 1,
# velocity (-2 pi y, 2 pi x, sin 2 pi x), f = 0, u = 1 on z = 0 and 0 on the rest
# of the boundary.  The domain is the unit cube shifted by (-1/2, -1/2, 0): the grid
# is the unit cube's and the velocity is evaluated at the shifted coordinates.
# Subdomain numbering (reading of "anticlockwise helicoidal"): Omega_1..Omega_4
# anticlockwise around the bottom layer from (x < 0, y < 0), Omega_5..Omega_8 the same
# in the top layer, the only order that gives Omega_8 = (-1/2,0) x (0,1/2) x (1/2,1)
# and Test 1's halves x < 0 / x > 0.  Tests 1-3 give nu_1 to the subdomains listed
# and nu_2 to the others.
EX41_HELIX = [(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0), (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)]
EX41_TESTS = {1: (1, 4, 5, 8), 2: (1, 5, 6, 8), 3: (1, 3, 6, 8)}


def example41(test=1, m=6, nu1=1.0, nu2=1e-7, theta_E=10.0):
    slabs = [[m, m], [m, m], [m, m]]
    ne, h, X, Y, Z = _grid(slabs)
    sub = _elem_subdomain(slabs)
    nu_sub = np.full(8, nu2)
    for k in EX41_TESTS[test]:
        sx, sy, sz = EX41_HELIX[k - 1]
        nu_sub[sx + 2 * (sy + 2 * sz)] = nu1
    x, y = X - 0.5, Y - 0.5
    beta = np.stack([-2 * np.pi * y, 2 * np.pi * x, np.sin(2 * np.pi * x)], axis=1)
    g = np.where(np.isclose(Z, 0.0), 1.0, 0.0)
    return Problem(f"example41_test{test}_m{m}", slabs, nu_sub[sub], beta, None, c=1.0, theta_E=theta_E,
                   element='p1', dirichlet_node=g, meta={"test": test, "m": m, "nu": (nu1, nu2)})


def example41_random(n=2, m=4, seed_offset=6, theta_E=10.0):
    """Example 4.1's domain, velocity, reaction and boundary data on n x n x n cubic
    subdomains of m^3 cubes (P1 tetrahedra) with a random viscosity per cube,
    nu = 10^r, r ~ U(-3, 3) (Sect. 4, the random-viscosity table, columns n(m))."""
    slabs = [[m] * n, [m] * n, [m] * n]
    ne, h, X, Y, Z = _grid(slabs)
    rng = np.random.default_rng([20250103 + seed_offset, n, m])
    nu = 10.0 ** rng.uniform(-3.0, 3.0, ne[0] * ne[1] * ne[2])
    x, y = X - 0.5, Y - 0.5
    beta = np.stack([-2 * np.pi * y, 2 * np.pi * x, np.sin(2 * np.pi * x)], axis=1)
    g = np.where(np.isclose(Z, 0.0), 1.0, 0.0)
    return Problem(f"example41_random_n{n}_m{m}", slabs, nu, beta, None, c=1.0, theta_E=theta_E,
                   element='p1', dirichlet_node=g, meta={"n": n, "m": m})
