"""Tensor hexahedral mesh of the unit cube and its tensor subdomain partition.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Definitions (Sect. 3, first paragraphs: non-overlapping decomposition into
subdomains that meet in faces, edges and vertices):

* The cube [0,1]^3 is split per direction d into slabs; slab s holds
  ``slabs[d][s]`` elements.  Elements are uniform per direction with spacing
  h_d = 1 / sum_s slabs[d][s].
* Node (ix,iy,iz) has id ix + (Ex+1)*(iy + (Ey+1)*iz).  Nodes on the boundary
  of the cube carry the homogeneous Dirichlet condition and are removed.
  Free node (ix,iy,iz) has dof id (ix-1) + (Ex-1)*((iy-1) + (Ey-1)*(iz-1)).
* Subdomain (sx,sy,sz) has id sx + Nx*(sy + Ny*sz) and owns the elements of
  slab sx x slab sy x slab sz.  Its local dofs are the free nodes of its
  closed box: interior dofs (strictly inside the box) first, in ascending
  dof id, then interface dofs, in ascending dof id.
* n(x) of an interface dof is the set of subdomains whose closed box holds it.
  Interface dofs with equal n(x) form one entity: a face when |n(x)| = 2, an
  edge when |n(x)| = 4, a vertex when |n(x)| = 8 (tensor partitions).
* The global interface Gamma lists all interface dofs in ascending dof id.
"""
from __future__ import annotations

import numpy as np


class Mesh:
    def __init__(self, slabs):
        self.slabs = [list(int(v) for v in s) for s in slabs]
        assert len(self.slabs) == 3
        for s in self.slabs:
            assert len(s) >= 1 and all(v >= 1 for v in s)
        self.nsub = [len(s) for s in self.slabs]
        self.ne = [sum(s) for s in self.slabs]
        self.h = [1.0 / n for n in self.ne]
        self.off = [np.concatenate([[0], np.cumsum(s)]).astype(int) for s in self.slabs]
        self.nnode = [n + 1 for n in self.ne]
        self.nfree = [n - 1 for n in self.ne]
        self.ndof = int(np.prod(self.nfree))
        self.nsd = int(np.prod(self.nsub))
        self.nelem = int(np.prod(self.ne))
        self._build()

    # ---- numbering -------------------------------------------------------
    def node_id(self, ix, iy, iz):
        return ix + self.nnode[0] * (iy + self.nnode[1] * iz)

    def dof_of_node(self, ix, iy, iz):
        """dof id of a node, or -1 for a Dirichlet node."""
        if min(ix, iy, iz) <= 0 or ix >= self.ne[0] or iy >= self.ne[1] or iz >= self.ne[2]:
            return -1
        return (ix - 1) + self.nfree[0] * ((iy - 1) + self.nfree[1] * (iz - 1))

    def dof_coords(self, dof):
        fx, fy = self.nfree[0], self.nfree[1]
        ix = dof % fx + 1
        iy = (dof // fx) % fy + 1
        iz = dof // (fx * fy) + 1
        return ix, iy, iz

    def elem_id(self, ex, ey, ez):
        return ex + self.ne[0] * (ey + self.ne[1] * ez)

    def sub_id(self, sx, sy, sz):
        return sx + self.nsub[0] * (sy + self.nsub[1] * sz)

    def sub_coords(self, s):
        nx, ny = self.nsub[0], self.nsub[1]
        return s % nx, (s // nx) % ny, s // (nx * ny)

    @staticmethod
    def elem_local_nodes(ex, ey, ez):
        """The 8 nodes of element (ex,ey,ez), local index a = dx + 2 dy + 4 dz."""
        return [(ex + (a & 1), ey + ((a >> 1) & 1), ez + ((a >> 2) & 1)) for a in range(8)]

    def slabs_of_index(self, d, i):
        """Slabs in direction d whose closed node range holds node index i."""
        o = self.off[d]
        return [s for s in range(self.nsub[d]) if o[s] <= i <= o[s + 1]]

    # ---- partition and classification -----------------------------------
    def _build(self):
        nx, ny, nz = self.nsub
        self.sub_dofs = []       # local dof list: interior then interface
        self.sub_nI = []
        self.sub_elems = []
        for s in range(self.nsd):
            sx, sy, sz = self.sub_coords(s)
            x0, x1 = self.off[0][sx], self.off[0][sx + 1]
            y0, y1 = self.off[1][sy], self.off[1][sy + 1]
            z0, z1 = self.off[2][sz], self.off[2][sz + 1]
            interior, interface = [], []
            for iz in range(z0, z1 + 1):
                for iy in range(y0, y1 + 1):
                    for ix in range(x0, x1 + 1):
                        d = self.dof_of_node(ix, iy, iz)
                        if d < 0:
                            continue
                        inside = x0 < ix < x1 and y0 < iy < y1 and z0 < iz < z1
                        (interior if inside else interface).append(d)
            interior.sort()
            interface.sort()
            self.sub_dofs.append(np.array(interior + interface, dtype=int))
            self.sub_nI.append(len(interior))
            elems = [self.elem_id(ex, ey, ez)
                     for ez in range(z0, z1) for ey in range(y0, y1) for ex in range(x0, x1)]
            self.sub_elems.append(np.array(elems, dtype=int))

        # n(x) for every free dof
        owners = {}
        for s in range(self.nsd):
            for d in self.sub_dofs[s][self.sub_nI[s]:]:
                owners.setdefault(int(d), []).append(s)
        self.gamma = np.array(sorted(owners.keys()), dtype=int)
        self.gamma_index = {int(d): k for k, d in enumerate(self.gamma)}
        groups = {}
        for d in self.gamma:
            key = tuple(sorted(owners[int(d)]))
            assert len(key) >= 2
            groups.setdefault(key, []).append(int(d))
        kind_of = {2: 'F', 4: 'E', 8: 'V'}
        ents = []
        for key, dofs in groups.items():
            k = kind_of.get(len(key))
            if k is None:
                raise ValueError("non-tensor interface class")
            ents.append({'kind': k, 'subs': key, 'dofs': np.array(sorted(dofs), dtype=int)})
        order = {'V': 0, 'E': 1, 'F': 2}
        ents.sort(key=lambda e: (order[e['kind']], int(e['dofs'][0])))
        self.entities = ents
        self.faces = [e for e in ents if e['kind'] == 'F']
        self.edges = [e for e in ents if e['kind'] == 'E']
        self.vertices = [e for e in ents if e['kind'] == 'V']
        # per subdomain: local positions of interface dofs, entity membership
        self.sub_entities = [[] for _ in range(self.nsd)]
        for ei, e in enumerate(ents):
            for s in e['subs']:
                self.sub_entities[s].append(ei)

    # ---- helpers ----------------------------------------------------------
    def local_index(self, s):
        """dict global dof -> local position in subdomain s (I then B)."""
        return {int(d): k for k, d in enumerate(self.sub_dofs[s])}

    def interface_local(self, s):
        """Interface dofs of s in local interface order (ascending dof id)."""
        return self.sub_dofs[s][self.sub_nI[s]:]

    def node_xyz(self, ix, iy, iz):
        return (self.off_coord(0, ix), self.off_coord(1, iy), self.off_coord(2, iz))

    def off_coord(self, d, i):
        return i * self.h[d]

    def all_node_xyz(self):
        """Coordinates of all nodes, shape (nnodes, 3), in node-id order."""
        X, Y, Z = np.meshgrid(np.arange(self.nnode[0]) * self.h[0],
                              np.arange(self.nnode[1]) * self.h[1],
                              np.arange(self.nnode[2]) * self.h[2], indexing='ij')
        # node id = ix + Nx1*(iy + Ny1*iz): x fastest -> transpose to (z,y,x) ravel
        pts = np.stack([X.transpose(2, 1, 0).ravel(), Y.transpose(2, 1, 0).ravel(),
                        Z.transpose(2, 1, 0).ravel()], axis=1)
        return pts

    def free_node_ids(self):
        """Node id of every dof, in dof order."""
        fx, fy, fz = self.nfree
        iz, iy, ix = np.meshgrid(np.arange(1, fz + 1), np.arange(1, fy + 1),
                                 np.arange(1, fx + 1), indexing='ij')
        return (ix + self.nnode[0] * (iy + self.nnode[1] * iz)).ravel()
