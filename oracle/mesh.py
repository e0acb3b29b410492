"""Cartesian quad mesh numbering (test infrastructure only).

The paper's assembly-free matvec (Alg. 3) uses four maps (thread -> edge,
edge -> (E1, E2), local dof indices on each element) without fixing a numbering.
This module fixes one, which the GPU library must reproduce exactly:

  element   e = i + nx * j                  (x fastest, like I = i + j(p+1), Sec. 4)
  vertical edges (normal along x) first:    id = i + (nx + 1) j,  i in [0, nx], j in [0, ny)
  horizontal edges next:                    id = nv + i + nx j,   i in [0, nx), j in [0, ny]
      with nv = (nx + 1) ny
  local faces of an element: 0 = W, 1 = E, 2 = S, 3 = N
  edge nodes ordered by increasing global coordinate (no orientation flips)
  trace dof = edge * (p + 1) + a
  edge_to_elem[edge] = (low-side element, high-side element), -1 off the domain
  edge_local_face[edge] = (face of the edge in the low element, in the high one)
"""
import numpy as np


class Mesh:
    def __init__(self, nx, ny, x0=0.0, y0=0.0, x1=1.0, y1=1.0):
        if nx < 1 or ny < 1:
            raise ValueError("nx, ny >= 1")
        self.nx, self.ny = int(nx), int(ny)
        self.x0, self.y0, self.x1, self.y1 = float(x0), float(y0), float(x1), float(y1)
        self.hx = (self.x1 - self.x0) / self.nx
        self.hy = (self.y1 - self.y0) / self.ny
        self.nel = self.nx * self.ny
        self.nv = (self.nx + 1) * self.ny          # vertical edges
        self.nh = self.nx * (self.ny + 1)          # horizontal edges
        self.n_edges = self.nv + self.nh

    def elem(self, i, j):
        return i + self.nx * j

    def vedge(self, i, j):
        return i + (self.nx + 1) * j

    def hedge(self, i, j):
        return self.nv + i + self.nx * j

    def elem_to_edge(self):
        """[nel, 4] edge ids of faces W, E, S, N."""
        out = np.zeros((self.nel, 4), dtype=np.int32)
        for j in range(self.ny):
            for i in range(self.nx):
                e = self.elem(i, j)
                out[e] = (self.vedge(i, j), self.vedge(i + 1, j),
                          self.hedge(i, j), self.hedge(i, j + 1))
        return out

    def edge_to_elem(self):
        """[n_edges, 2] (low-side element, high-side element); -1 off the domain."""
        out = -np.ones((self.n_edges, 2), dtype=np.int32)
        out_face = -np.ones((self.n_edges, 2), dtype=np.int32)
        e2e = self.elem_to_edge()
        for e in range(self.nel):
            for f in range(4):
                ed = e2e[e, f]
                side = 1 if f in (0, 2) else 0   # W/S face: element is the high side
                out[ed, side] = e
                out_face[ed, side] = f
        return out, out_face

    def boundary_edges(self):
        e2el, _ = self.edge_to_elem()
        return np.nonzero((e2el[:, 0] < 0) | (e2el[:, 1] < 0))[0]

    def interior_edges(self):
        e2el, _ = self.edge_to_elem()
        return np.nonzero((e2el[:, 0] >= 0) & (e2el[:, 1] >= 0))[0]

    def elem_origin(self, e):
        i, j = e % self.nx, e // self.nx
        return self.x0 + i * self.hx, self.y0 + j * self.hy

    def elem_centres(self):
        i = np.arange(self.nx)
        j = np.arange(self.ny)
        xc = self.x0 + (i + 0.5) * self.hx
        yc = self.y0 + (j + 0.5) * self.hy
        X, Y = np.meshgrid(xc, yc)        # [ny, nx], element e = i + nx j
        return X.ravel(), Y.ravel()
