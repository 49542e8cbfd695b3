"""Write p1_unit_brick.txt: exact integrals of the P1 functions of the six Kuhn
tetrahedra of the unit cube, summed into the cube's 8 x 8 matrices (no quadrature,
no code of the library or of the oracle).

Node a of the cube has coordinates (a & 1, (a >> 1) & 1, (a >> 2) & 1).  For every
permutation p of the three axes the tetrahedron has the vertices 0, e_p0,
e_p0 + e_p1 and (1, 1, 1) (all six share the main diagonal and tile the cube).  On a
tetrahedron of volume V with barycentric coordinates lambda_a (affine, gradients
g_a from the inverse of the edge matrix, computed here in exact rationals):
    stiffness   int grad lambda_b . grad lambda_a  = V g_a . g_b
    mass        int lambda_b lambda_a              = V (1 + delta_ab) / 20
    convection  int (d_x lambda_b) lambda_a        = V (g_b)_x / 4
    Kx          int (d_x lambda_b)(d_x lambda_a)   = V (g_a)_x (g_b)_x
(row = test a, column = trial b).
Run: python tests/golden/make_p1_unit_brick.py
"""
import itertools
import os
from fractions import Fraction as Fr


def xyz(a):
    return [Fr((a >> d) & 1) for d in range(3)]


def inv3(M):
    """Exact inverse of a 3 x 3 rational matrix by cofactors."""
    det = (M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0])
           + M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]))
    cof = [[(M[(r + 1) % 3][(c + 1) % 3] * M[(r + 2) % 3][(c + 2) % 3]
             - M[(r + 1) % 3][(c + 2) % 3] * M[(r + 2) % 3][(c + 1) % 3]) for c in range(3)] for r in range(3)]
    return [[cof[c][r] / det for c in range(3)] for r in range(3)], det


K0 = [[Fr(0)] * 8 for _ in range(8)]
M = [[Fr(0)] * 8 for _ in range(8)]
Kx = [[Fr(0)] * 8 for _ in range(8)]
Cx = [[Fr(0)] * 8 for _ in range(8)]
for p in itertools.permutations(range(3)):
    v = [0, 1 << p[0], (1 << p[0]) | (1 << p[1]), 7]
    P = [xyz(a) for a in v]
    E = [[P[r + 1][d] - P[0][d] for d in range(3)] for r in range(3)]     # rows: edges from vertex 0
    Ei, det = inv3(E)
    V = abs(det) / 6
    # lambda_r (r = 1..3) = row r-1 of E^{-T} applied to (x - x_0): gradient = column r-1 of E^{-1}
    g = [[None] * 3 for _ in range(4)]
    for r in range(3):
        g[r + 1] = [Ei[d][r] for d in range(3)]
    g[0] = [-(g[1][d] + g[2][d] + g[3][d]) for d in range(3)]
    for a in range(4):
        for b in range(4):
            i, j = v[a], v[b]
            K0[i][j] += V * sum(g[a][d] * g[b][d] for d in range(3))
            M[i][j] += V * (2 if a == b else 1) / 20
            Kx[i][j] += V * g[a][0] * g[b][0]
            Cx[i][j] += V * g[b][0] / 4

out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "p1_unit_brick.txt")
with open(out, "w") as f:
    f.write("# P1 integrals on the six Kuhn tetrahedra of the unit cube, summed into the cube's nodes;\n")
    f.write("# exact fractions (row = test i, column = trial j).  Node a at (a & 1, (a >> 1) & 1, (a >> 2) & 1).\n")
    f.write("# Written by make_p1_unit_brick.py from the barycentric gradients of each tetrahedron; the terms\n")
    f.write("# are those of the bilinear form of Sect. 2 on the paper's element (Sect. 4).\n")
    for name, A in (("K0", K0), ("M", M), ("Kx", Kx), ("Cx", Cx)):
        f.write(f"[{name}]\n")
        for row in A:
            f.write(" ".join(str(x) for x in row) + "\n")
