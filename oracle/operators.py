"""Brute-force sparse restatement of the discrete Yee operators (test
infrastructure only).

The curls are assembled here from geometry -- Stokes' theorem on each primal
face (boundary loop of four edges) and on each dual face around a primal edge
(loop of four faces) -- rather than from the finite-difference formulas the C
oracle uses, so that an index or sign slip in either one shows up as a
mismatch.  Positions use doubled integer coordinates: a primal node sits at
even coordinates, an edge along axis a is odd along a and even along the
others, a face with normal a is even along a and odd along the others, a cell
centre is odd along all three.

Vector ordering matches ``OracleSim``: E = [Ex, Ey, Ez] flattened in (k, j, i)
C order with the full staggered shapes, H = [Hx, Hy, Hz] likewise, cells in
(k, j, i) order.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


class YeeGeometry:
    def __init__(self, nx, ny, nz, dx, dy, dz):
        self.n = (nx, ny, nz)
        self.d = (dx, dy, dz)
        # shapes in (i, j, k) order for each staggered component
        self.edge_shape = [
            (nx, ny + 1, nz + 1),
            (nx + 1, ny, nz + 1),
            (nx + 1, ny + 1, nz),
        ]
        self.face_shape = [
            (nx + 1, ny, nz),
            (nx, ny + 1, nz),
            (nx, ny, nz + 1),
        ]
        self.edge_off = np.cumsum([0] + [int(np.prod(s)) for s in self.edge_shape])
        self.face_off = np.cumsum([0] + [int(np.prod(s)) for s in self.face_shape])
        self.n_edges = int(self.edge_off[-1])
        self.n_faces = int(self.face_off[-1])
        self.n_cells = nx * ny * nz

    @staticmethod
    def _flat(shape, ijk):
        i, j, k = ijk
        return i + shape[0] * (j + shape[1] * k)

    def edge_index(self, a, D):
        """Global index of the edge along axis a at doubled position D, or None."""
        n = self.n
        for ax in range(3):
            if ax == a:
                if not (D[ax] % 2 == 1 and 1 <= D[ax] <= 2 * n[ax] - 1):
                    return None
            elif not (D[ax] % 2 == 0 and 0 <= D[ax] <= 2 * n[ax]):
                return None
        ijk = tuple(x // 2 for x in D)
        return int(self.edge_off[a]) + self._flat(self.edge_shape[a], ijk)

    def face_index(self, a, D):
        """Global index of the face with normal a at doubled position D, or None."""
        n = self.n
        for ax in range(3):
            if ax == a:
                if not (D[ax] % 2 == 0 and 0 <= D[ax] <= 2 * n[ax]):
                    return None
            elif not (D[ax] % 2 == 1 and 1 <= D[ax] <= 2 * n[ax] - 1):
                return None
        ijk = tuple(x // 2 for x in D)
        return int(self.face_off[a]) + self._flat(self.face_shape[a], ijk)

    def edges(self):
        """Yield (axis, doubled position, global index) for every edge."""
        for a in range(3):
            sh = self.edge_shape[a]
            for k in range(sh[2]):
                for j in range(sh[1]):
                    for i in range(sh[0]):
                        D = [2 * i, 2 * j, 2 * k]
                        D[a] += 1
                        yield a, tuple(D), self.edge_index(a, D)

    def faces(self):
        for a in range(3):
            sh = self.face_shape[a]
            for k in range(sh[2]):
                for j in range(sh[1]):
                    for i in range(sh[0]):
                        D = [2 * i + 1, 2 * j + 1, 2 * k + 1]
                        D[a] -= 1
                        yield a, tuple(D), self.face_index(a, D)

    def is_wall_edge(self, a, D):
        n = self.n
        return any(D[ax] in (0, 2 * n[ax]) for ax in range(3) if ax != a)

    # ------------------------------------------------------------ operators
    def curl_on_faces(self):
        """(curl E) at faces from the circulation of E around each face's boundary,
        divided by the face area: rows faces, columns edges."""
        rows, cols, vals = [], [], []
        for a, D, f in self.faces():
            b, c = (a + 1) % 3, (a + 2) % 3
            # counter-clockwise about the normal a in the (b, c) plane:
            # +b edge at c-1, +c edge at b+1, -b edge at c+1, -c edge at b-1
            loop = [(b, c, -1, +1), (c, b, +1, +1), (b, c, +1, -1), (c, b, -1, -1)]
            area = self.d[b] * self.d[c]
            for axis, shift_ax, shift, sign in loop:
                P = list(D)
                P[shift_ax] += shift
                e = self.edge_index(axis, P)
                rows.append(f)
                cols.append(e)
                vals.append(sign * self.d[axis] / area)
        return sp.csr_matrix((vals, (rows, cols)), shape=(self.n_faces, self.n_edges))

    def curl_on_edges(self):
        """(curl H) at edges from the circulation of H (living on dual edges through
        primal faces) around the dual face pierced by each edge: rows edges,
        columns faces.  Edges in a wall (incomplete dual loop) get no row."""
        rows, cols, vals = [], [], []
        for a, D, e in self.edges():
            if self.is_wall_edge(a, D):
                continue
            b, c = (a + 1) % 3, (a + 2) % 3
            loop = [(b, c, -1, +1), (c, b, +1, +1), (b, c, +1, -1), (c, b, -1, -1)]
            area = self.d[b] * self.d[c]
            for axis, shift_ax, shift, sign in loop:
                P = list(D)
                P[shift_ax] += shift
                f = self.face_index(axis, P)
                rows.append(e)
                cols.append(f)
                vals.append(sign * self.d[axis] / area)
        return sp.csr_matrix((vals, (rows, cols)), shape=(self.n_edges, self.n_faces))

    def div_on_cells(self):
        """Outward flux through the six faces of each cell over its volume."""
        nx, ny, nz = self.n
        rows, cols, vals = [], [], []
        for k in range(nz):
            for j in range(ny):
                for i in range(nx):
                    cidx = i + nx * (j + ny * k)
                    D = [2 * i + 1, 2 * j + 1, 2 * k + 1]
                    for a in range(3):
                        for s in (-1, +1):
                            P = list(D)
                            P[a] += s
                            rows.append(cidx)
                            cols.append(self.face_index(a, P))
                            vals.append(s / self.d[a])
        return sp.csr_matrix((vals, (rows, cols)), shape=(self.n_cells, self.n_faces))

    def face_to_cell_mean(self):
        """A: 3*n_cells x n_faces, the mean of the two faces of each cell with the
        same normal (component blocks x, y, z)."""
        nx, ny, nz = self.n
        rows, cols, vals = [], [], []
        for k in range(nz):
            for j in range(ny):
                for i in range(nx):
                    cidx = i + nx * (j + ny * k)
                    D = [2 * i + 1, 2 * j + 1, 2 * k + 1]
                    for a in range(3):
                        for s in (-1, +1):
                            P = list(D)
                            P[a] += s
                            rows.append(a * self.n_cells + cidx)
                            cols.append(self.face_index(a, P))
                            vals.append(0.5)
        return sp.csr_matrix((vals, (rows, cols)), shape=(3 * self.n_cells, self.n_faces))

    def edge_cells(self, a, D):
        """Cells (i, j, k) sharing the edge along a at doubled position D."""
        b, c = (a + 1) % 3, (a + 2) % 3
        out = []
        for sb in (-1, +1):
            for sc in (-1, +1):
                P = list(D)
                P[b] += sb
                P[c] += sc
                ijk = [x // 2 for x in P]
                if all(0 <= ijk[ax] < self.n[ax] for ax in range(3)) and all(P[ax] % 2 == 1 for ax in range(3)):
                    out.append(tuple(ijk))
        return out

    # ----------------------------------------------------- vector packing
    def pack_E(self, Ex, Ey, Ez):
        """(k, j, i)-shaped arrays -> one vector."""
        return np.concatenate([Ex.ravel(), Ey.ravel(), Ez.ravel()])

    def pack_H(self, Hx, Hy, Hz):
        return np.concatenate([Hx.ravel(), Hy.ravel(), Hz.ravel()])

    def unpack_E(self, v):
        out = []
        for a in range(3):
            sh = self.edge_shape[a]
            out.append(v[self.edge_off[a]:self.edge_off[a + 1]].reshape(sh[2], sh[1], sh[0]))
        return out

    def unpack_H(self, v):
        out = []
        for a in range(3):
            sh = self.face_shape[a]
            out.append(v[self.face_off[a]:self.face_off[a + 1]].reshape(sh[2], sh[1], sh[0]))
        return out


def maxwell_step_matrices(geo: YeeGeometry, eps_cell, sig_cell, pec_cell, dt, mu0, eps0):
    """One leap-frog step with M = 0 written with the assembled operators:
    H1 = H - (dt/2mu0) C_E E;  E1 = (sig/2 + eps/dt)^-1 [C_H H1 - (sig/2 - eps/dt) E];
    H2 = H1 - (dt/2mu0) C_E E1; wall and PEC edges held at 0.
    eps_cell etc. are (k, j, i) arrays.  Returns a function (E, H) -> (E2, H2)."""
    CE = geo.curl_on_faces()
    CH = geo.curl_on_edges()
    eps = np.zeros(geo.n_edges)
    sig = np.zeros(geo.n_edges)
    frozen = np.zeros(geo.n_edges, dtype=bool)
    for a, D, e in geo.edges():
        if geo.is_wall_edge(a, D):
            frozen[e] = True
            continue
        cells = geo.edge_cells(a, D)
        eps[e] = eps0 * np.mean([eps_cell[k, j, i] for (i, j, k) in cells])
        sig[e] = np.mean([sig_cell[k, j, i] for (i, j, k) in cells])
        if any(pec_cell[k, j, i] for (i, j, k) in cells):
            frozen[e] = True

    def step(E, H):
        H1 = H - (0.5 * dt / mu0) * (CE @ E)
        E1 = np.where(frozen, 0.0, (CH @ H1 - (sig / 2 - eps / dt) * E) / np.where(frozen, 1.0, sig / 2 + eps / dt))
        H2 = H1 - (0.5 * dt / mu0) * (CE @ E1)
        return E1, H2

    return step, frozen, eps
