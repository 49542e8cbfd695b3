"""Write q1_unit_cube.txt: exact element integrals of trilinear (Q1) shape functions
on the unit cube, from the tensor-product structure alone (no quadrature, no code of
the library or of the oracle).

1D, phi_0 = 1 - x, phi_1 = x on [0, 1]:
    mass       m[i][j] = int phi_j phi_i       = [[1/3, 1/6], [1/6, 1/3]]
    stiffness  k[i][j] = int phi_j' phi_i'     = [[1, -1], [-1, 1]]
    convection c[i][j] = int phi_j' phi_i      = [[-1/2, 1/2], [-1/2, 1/2]]
3D node a has coordinates (a & 1, (a >> 1) & 1, (a >> 2) & 1); row = test i, column =
trial j:
    M  = m (x) m (x) m
    Kx = k (x) m (x) m,  K0 = Kx + Ky + Kz  (int grad phi_j . grad phi_i)
    Cx = c (x) m (x) m                     (int d_x phi_j phi_i)
Run: python tests/golden/make_q1_unit_cube.py
"""
import os
from fractions import Fraction as Fr

m = [[Fr(1, 3), Fr(1, 6)], [Fr(1, 6), Fr(1, 3)]]
k = [[Fr(1), Fr(-1)], [Fr(-1), Fr(1)]]
c = [[Fr(-1, 2), Fr(1, 2)], [Fr(-1, 2), Fr(1, 2)]]


def bit(a, d):
    return (a >> d) & 1


def tensor(fx, fy, fz):
    return [[fx[bit(i, 0)][bit(j, 0)] * fy[bit(i, 1)][bit(j, 1)] * fz[bit(i, 2)][bit(j, 2)] for j in range(8)]
            for i in range(8)]


M = tensor(m, m, m)
Kx, Ky, Kz = tensor(k, m, m), tensor(m, k, m), tensor(m, m, k)
K0 = [[Kx[i][j] + Ky[i][j] + Kz[i][j] for j in range(8)] for i in range(8)]
Cx = tensor(c, m, m)

out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "q1_unit_cube.txt")
with open(out, "w") as f:
    f.write("# Q1 element integrals on the unit cube, exact fractions (row = test i, column = trial j).\n")
    f.write("# Node a at (a & 1, (a >> 1) & 1, (a >> 2) & 1).  Written by make_q1_unit_cube.py from the\n")
    f.write("# tensor-product 1D integrals; the terms are those of the bilinear form of Sect. 2\n")
    f.write("# (diffusion int grad phi_j . grad phi_i, mass, convection int beta . grad phi_j phi_i).\n")
    for name, A in (("K0", K0), ("M", M), ("Kx", Kx), ("Cx", Cx)):
        f.write(f"[{name}]\n")
        for row in A:
            f.write(" ".join(str(v) for v in row) + "\n")
