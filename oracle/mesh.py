"""Structured hexahedral spectral-element mesh of a slab box.

Section 2.3 and Fig. CEF / Fig. APD: the domain Omega_p is periodic in x and y and
bounded in z.  The mesh has nx x ny x nz uniform cells of size h_d = L_d / n_d; each
cell carries (p+1)^3 GLL nodes.

Numbering (shared interface convention, not arithmetic):

* global node (gx, gy, gz) with gx in [0, nx p), gy in [0, ny p) (periodic wrap of the
  last node of each row onto the first) and gz in [0, nz p];
* electrostatic (phi) node id  = gx + NX (gy + NY gz), NX = nx p, NY = ny p;
* wavefunction (psi) nodes drop the z-face planes that carry a homogeneous Dirichlet
  condition: psi id = gx + NX (gy + NY (gz - gz_lo));
* cells are ordered with cx fastest; local node (i, j, k) has id i + (p+1)(j + (p+1) k).
"""
import numpy as np

from .basis import gll


class Mesh:
    def __init__(self, L, ncell, p, psi_dirichlet=(True, True)):
        self.L = np.asarray(L, dtype=np.float64)
        self.ncell = tuple(int(n) for n in ncell)
        self.p = int(p)
        self.h = self.L / np.asarray(self.ncell, dtype=np.float64)
        nx, ny, nz = self.ncell
        self.NX, self.NY, self.NZ = nx * p, ny * p, nz * p + 1
        self.n_phi = self.NX * self.NY * self.NZ
        self.gz_lo = 1 if psi_dirichlet[0] else 0
        self.gz_hi = nz * p - 1 if psi_dirichlet[1] else nz * p
        self.NZpsi = self.gz_hi - self.gz_lo + 1
        self.n_psi = self.NX * self.NY * self.NZpsi
        self.psi_dirichlet = tuple(bool(b) for b in psi_dirichlet)
        self.xi, self.w = gll(p)
        self.ne = (p + 1) ** 3
        self.n_cells = nx * ny * nz

    # -- 1D coordinates -------------------------------------------------------------
    def axis_coord(self, d, g):
        """Coordinate of global 1D index g along axis d (g may equal n_d p for z)."""
        g = np.asarray(g)
        c = g // self.p
        i = g % self.p
        return c * self.h[d] + (self.xi[i] + 1.0) * 0.5 * self.h[d]

    def phi_grid_indices(self):
        gz, gy, gx = np.meshgrid(np.arange(self.NZ), np.arange(self.NY), np.arange(self.NX),
                                 indexing="ij")
        return gx.ravel(), gy.ravel(), gz.ravel()

    def phi_coords(self):
        gx, gy, gz = self.phi_grid_indices()
        return np.column_stack([self.axis_coord(0, gx), self.axis_coord(1, gy),
                                self.axis_coord(2, gz)])

    def psi_to_phi(self):
        """phi id of every psi node, in psi order."""
        return np.arange(self.n_psi) + self.NX * self.NY * self.gz_lo

    def psi_coords(self):
        return self.phi_coords()[self.psi_to_phi()]

    # -- cell connectivity ----------------------------------------------------------
    def cell_nodes(self):
        """phi ids of the (p+1)^3 nodes of every cell, shape [n_cells, ne]."""
        p = self.p
        nx, ny, nz = self.ncell
        loc = np.arange(p + 1)
        k, j, i = np.meshgrid(loc, loc, loc, indexing="ij")
        i, j, k = i.ravel(), j.ravel(), k.ravel()
        cz, cy, cx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        cx, cy, cz = cx.ravel()[:, None], cy.ravel()[:, None], cz.ravel()[:, None]
        gx = (cx * p + i[None, :]) % self.NX
        gy = (cy * p + j[None, :]) % self.NY
        gz = cz * p + k[None, :]
        return gx + self.NX * (gy + self.NY * gz)

    def node_cells(self, gx, gy, gz):
        """[(cell id, local id)] of every cell touching global node (gx, gy, gz)."""
        p = self.p
        nx, ny, nz = self.ncell

        def axis(g, n, periodic):
            out = []
            if g % p == 0:
                c = g // p
                if periodic:
                    out.append(((c - 1) % n, p))
                    out.append((c % n, 0))
                else:
                    if c - 1 >= 0:
                        out.append((c - 1, p))
                    if c < n:
                        out.append((c, 0))
            else:
                out.append((g // p, g % p))
            return out

        res = []
        for cx, i in axis(gx, nx, True):
            for cy, j in axis(gy, ny, True):
                for cz, k in axis(gz, nz, False):
                    res.append((cx + nx * (cy + ny * cz), i + (p + 1) * (j + (p + 1) * k)))
        return res
