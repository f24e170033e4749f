"""FP64 reference gradients of a probe objective for the coupled Yee-Maxwell
+ LLG step (arxiv 2510.22221, section "Numerical Model", Eqs. Ampere,
Faraday, LLG, llg_tra4-6, iterate_H).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``.  The step is written a
second time here in plain PyTorch CPU tensor operations (FP64, whole-array
slices instead of the C oracle's loops) so that the library's automatic
differentiation yields the exact gradient of the discrete map; the tests pin
this restatement to the C oracle step by step and its gradient to central
finite differences.  The LLG solve takes a fixed number of Jacobi iterates
(``fixed_iter``) so that the map is a fixed composition of smooth operations.

Objective:  J = sum over probe rows n in [n0, N) of |E(probe)|^2, the three
native edge values Ex, Ey, Ez of each probe cell after step n.
Parameters: eps_r of every cell of a design box, and |H_bias| (A/m) along
its fixed direction h (M starts at Ms h, independent of |H_bias|).
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import Material, Source

MU0 = 4e-7 * math.pi
C0 = 299792458.0
EPS0 = 1.0 / (MU0 * C0 * C0)


class TorchStep:
    """The C oracle's step (half-push with curl E^n, E push at t_{n+1/2},
    half-push with curl E^{n+1}) on (E, H, M) at integer times, full staggered
    array shapes: Ex (nz+1, ny+1, nx), Ey (nz+1, ny, nx+1), Ez (nz, ny+1, nx+1),
    Hx (nz, ny, nx+1), Hy (nz, ny+1, nx), Hz (nz+1, ny, nx), M (3, nz, ny, nx)."""

    def __init__(self, nx, ny, nz, dx, dy, dz, dt, materials, mat_id, h_dir, sources=(), probes=(),
                 design_box=None, fixed_iter=3):
        self.nx, self.ny, self.nz = nx, ny, nz
        self.dx, self.dy, self.dz, self.dt = dx, dy, dz, dt
        self.mats = [m if isinstance(m, Material) else Material(**m) for m in materials]
        self.mid = np.asarray(mat_id, dtype=np.int64)
        self.h_dir = np.asarray(h_dir, dtype=np.float64)
        self.sources = [s if isinstance(s, Source) else Source(**s) for s in sources]
        self.probes = list(probes)
        self.box = design_box       # (i0, j0, k0, bx, by, bz) or None
        self.R = fixed_iter
        t = lambda a: torch.as_tensor(np.asarray(a, dtype=np.float64))
        self.eps_mat = t([m.eps_r for m in self.mats])[self.mid]
        self.sig_cell = t([m.sigma for m in self.mats])[self.mid]
        self.pec_cell = torch.as_tensor(np.array([m.pec for m in self.mats])[self.mid])
        self.Ms = t([m.Ms for m in self.mats])[self.mid]
        self.alpha = t([m.alpha for m in self.mats])[self.mid]
        self.kap = MU0 * t([m.gamma for m in self.mats])[self.mid] * (0.5 * dt) / 2.0
        self.mag = self.Ms > 0
        self.Ms_safe = torch.where(self.mag, self.Ms, torch.ones_like(self.Ms))
        self._frozen = [self._edge_frozen(c) for c in range(3)]
        self._sigma_e = [self._edge_mean(self.sig_cell, c) for c in range(3)]

    # ------------------------------------------------------- edge materials
    def _edge_stack(self, cell, comp):
        """The four cells sharing each edge, zero-padded outside the grid (R4);
        returns (sum over in-grid cells, count of in-grid cells)."""
        nz, ny, nx = self.nz, self.ny, self.nx
        ones = torch.ones(nz, ny, nx, dtype=torch.float64)
        if comp == 0:
            pad = lambda a: torch.nn.functional.pad(a, (0, 0, 1, 1, 1, 1))          # j, k
            A, N = pad(cell), pad(ones)
            s = A[1:, 1:] + A[1:, :-1] + A[:-1, 1:] + A[:-1, :-1]
            n = N[1:, 1:] + N[1:, :-1] + N[:-1, 1:] + N[:-1, :-1]
        elif comp == 1:
            pad = lambda a: torch.nn.functional.pad(a, (1, 1, 0, 0, 1, 1))          # i, k
            A, N = pad(cell), pad(ones)
            s = A[1:, :, 1:] + A[1:, :, :-1] + A[:-1, :, 1:] + A[:-1, :, :-1]
            n = N[1:, :, 1:] + N[1:, :, :-1] + N[:-1, :, 1:] + N[:-1, :, :-1]
        else:
            pad = lambda a: torch.nn.functional.pad(a, (1, 1, 1, 1, 0, 0))          # i, j
            A, N = pad(cell), pad(ones)
            s = A[:, 1:, 1:] + A[:, 1:, :-1] + A[:, :-1, 1:] + A[:, :-1, :-1]
            n = N[:, 1:, 1:] + N[:, 1:, :-1] + N[:, :-1, 1:] + N[:, :-1, :-1]
        return s, n

    def _edge_mean(self, cell, comp):
        s, n = self._edge_stack(cell, comp)
        return s / torch.clamp(n, min=1.0)

    def _edge_frozen(self, comp):
        s, _ = self._edge_stack(self.pec_cell.to(torch.float64), comp)
        fz = s > 0
        if comp == 0:
            fz[0] = fz[-1] = True
            fz[:, 0] = fz[:, -1] = True
        elif comp == 1:
            fz[0] = fz[-1] = True
            fz[:, :, 0] = fz[:, :, -1] = True
        else:
            fz[:, 0] = fz[:, -1] = True
            fz[:, :, 0] = fz[:, :, -1] = True
        return fz

    def eps_cell(self, eps_design):
        if self.box is None or eps_design is None:
            return self.eps_mat
        i0, j0, k0, bx, by, bz = self.box
        e = self.eps_mat.clone()
        e[k0:k0 + bz, j0:j0 + by, i0:i0 + bx] = eps_design
        return e

    # ---------------------------------------------------------------- curls
    def curl_e(self, Ex, Ey, Ez):
        cx = (Ez[:, 1:, :] - Ez[:, :-1, :]) / self.dy - (Ey[1:] - Ey[:-1]) / self.dz
        cy = (Ex[1:] - Ex[:-1]) / self.dz - (Ez[:, :, 1:] - Ez[:, :, :-1]) / self.dx
        cz = (Ey[:, :, 1:] - Ey[:, :, :-1]) / self.dx - (Ex[:, 1:, :] - Ex[:, :-1, :]) / self.dy
        return cx, cy, cz

    def curl_h(self, Hx, Hy, Hz):
        F = torch.nn.functional.pad
        Hzj, Hyk = F(Hz, (0, 0, 1, 1)), F(Hy, (0, 0, 0, 0, 1, 1))
        cx = (Hzj[:, 1:] - Hzj[:, :-1]) / self.dy - (Hyk[1:] - Hyk[:-1]) / self.dz
        Hxk, Hzi = F(Hx, (0, 0, 0, 0, 1, 1)), F(Hz, (1, 1))
        cy = (Hxk[1:] - Hxk[:-1]) / self.dz - (Hzi[:, :, 1:] - Hzi[:, :, :-1]) / self.dx
        Hyi, Hxj = F(Hy, (1, 1)), F(Hx, (0, 0, 1, 1))
        cz = (Hyi[:, :, 1:] - Hyi[:, :, :-1]) / self.dx - (Hxj[:, 1:] - Hxj[:, :-1]) / self.dy
        return cx, cy, cz

    # ----------------------------------------------------------- half-push
    @staticmethod
    def _faces_minus_half_dm(Hs, dM):
        """Face value H^* - (dM_low + dM_high)/2 per component (R3)."""
        F = torch.nn.functional.pad
        px, py, pz = F(dM[0], (1, 1)), F(dM[1], (0, 0, 1, 1)), F(dM[2], (0, 0, 0, 0, 1, 1))
        return (Hs[0] - 0.5 * (px[:, :, :-1] + px[:, :, 1:]),
                Hs[1] - 0.5 * (py[:, :-1] + py[:, 1:]),
                Hs[2] - 0.5 * (pz[:-1] + pz[1:]))

    @staticmethod
    def _cell_mean(Hx, Hy, Hz):
        return torch.stack([0.5 * (Hx[:, :, :-1] + Hx[:, :, 1:]), 0.5 * (Hy[:, :-1] + Hy[:, 1:]),
                            0.5 * (Hz[:-1] + Hz[1:])])

    def _scatter(self, vals, like):
        """Cell array equal to vals (3, n_magnetic) on magnetic cells, 0 elsewhere."""
        out = torch.zeros_like(like)
        out[:, self.mag] = vals
        return out

    def half_push(self, E, H, M, hbias):
        c = 0.5 * self.dt / MU0
        ce = self.curl_e(*E)
        Hs = tuple(H[q] - c * ce[q] for q in range(3))
        if not bool(self.mag.any()):
            return Hs, M
        hb = hbias.reshape(3, 1)
        mk = self.mag                                        # the LLG acts on magnetic cells only
        cross = lambda a, b: torch.stack([a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2],
                                          a[0] * b[1] - a[1] * b[0]])
        Mm = M[:, mk]
        Ms, kap, al = self.Ms[mk], self.kap[mk], self.alpha[mk]
        He_n = self._cell_mean(*H)[:, mk] + hb
        b = Mm - kap * cross(Mm, He_n)                       # Eq. llg_tra6
        a0 = -(al / Ms) * Mm
        dM = torch.zeros_like(M)
        for _ in range(self.R):
            faces = self._faces_minus_half_dm(Hs, dM)
            He = self._cell_mean(*faces)[:, mk] + hb
            a = -kap * He + a0                                # Eq. llg_tra5
            ab = (a * b).sum(0)
            aa = (a * a).sum(0)
            Mt = (b + ab * a - cross(a, b)) / (1.0 + aa)      # Eq. llg_tra4
            nrm = torch.sqrt((Mt * Mt).sum(0))
            dM = self._scatter(Ms * Mt / nrm - Mm, M)
        return self._faces_minus_half_dm(Hs, dM), M + dM

    # ----------------------------------------------------------------- step
    def e_push(self, E, H, eps_cell, t_half):
        ch = self.curl_h(*H)
        out = []
        for q in range(3):
            eps = EPS0 * self._edge_mean(eps_cell, q)
            sig = self._sigma_e[q]
            J = torch.zeros_like(E[q])
            for s in self.sources:
                if s.comp == q:
                    i, j, k = s.ijk
                    J[k, j, i] = J[k, j, i] + _source(s, t_half)
            new = (ch[q] - (sig / 2 - eps / self.dt) * E[q] - J) / (sig / 2 + eps / self.dt)
            out.append(torch.where(self._frozen[q], torch.zeros_like(new), new))
        return tuple(out)

    def step(self, E, H, M, eps_cell, hbias, n):
        H, M = self.half_push(E, H, M, hbias)
        E = self.e_push(E, H, eps_cell, (n + 0.5) * self.dt)
        H, M = self.half_push(E, H, M, hbias)
        return E, H, M

    def zero_state(self, hbias_norm):
        nx, ny, nz = self.nx, self.ny, self.nz
        z = lambda *s: torch.zeros(*s, dtype=torch.float64)
        E = (z(nz + 1, ny + 1, nx), z(nz + 1, ny, nx + 1), z(nz, ny + 1, nx + 1))
        H = (z(nz, ny, nx + 1), z(nz, ny + 1, nx), z(nz + 1, ny, nx))
        u = torch.as_tensor(self.h_dir / np.linalg.norm(self.h_dir))
        M = self.Ms * u.reshape(3, 1, 1, 1)
        return E, H, M

    def probe_e(self, E):
        return torch.stack([torch.stack([E[0][k, j, i], E[1][k, j, i], E[2][k, j, i]]) for (i, j, k) in self.probes])


def _source(s, t):
    """Eq. of section "Modeling Setup": J0 exp(-(t - tpk)^2 / (2 Tp^2)) cos(2 pi f0 t)."""
    Tp = s.Tp if s.Tp > 0 else 1.0 / s.f0
    tpk = s.tpk if s.tpk > 0 else 3.0 * Tp
    u = t - tpk
    return s.J0 * math.exp(-u * u / (2.0 * Tp * Tp)) * math.cos(2.0 * math.pi * s.f0 * t)


def run(model: TorchStep, nsteps: int, eps_design=None, h0=None, n0=0, segment=25, record=False):
    """Objective J (and, with record, the probe E rows) after nsteps steps.
    eps_design and h0 may require grad; steps are grouped into checkpointed
    segments so that memory stays bounded."""
    from torch.utils.checkpoint import checkpoint

    h_dir = torch.as_tensor(model.h_dir / np.linalg.norm(model.h_dir))
    if h0 is None:
        h0 = torch.tensor(float(np.linalg.norm(model.h_dir)), dtype=torch.float64)
    hbias = h0 * h_dir
    eps_cell = model.eps_cell(eps_design)
    E, H, M = model.zero_state(None)
    J = torch.zeros((), dtype=torch.float64)
    rows = []

    def seg(n_a, n_b, *state):
        E_, H_, M_ = state[0:3], state[3:6], state[6]
        eps_c, hb = state[7], state[8]
        acc = torch.zeros((), dtype=torch.float64)
        recs = []
        for n in range(n_a, n_b):
            E_, H_, M_ = model.step(E_, H_, M_, eps_c, hb, n)
            pe = model.probe_e(E_)
            recs.append(pe)
            if n >= n0:
                acc = acc + (pe * pe).sum()
        return (*E_, *H_, M_, acc, torch.stack(recs))

    for n_a in range(0, nsteps, segment):
        n_b = min(nsteps, n_a + segment)
        out = checkpoint(seg, n_a, n_b, *E, *H, M, eps_cell, hbias, use_reentrant=False)
        E, H, M, acc, rec = out[0:3], out[3:6], out[6], out[7], out[8]
        J = J + acc
        if record:
            rows.append(rec.detach())
    if record:
        return J, torch.cat(rows).numpy()
    return J


def gradients(model: TorchStep, nsteps: int, eps_design, h0: float, n0: int, segment=25):
    """(J, dJ/d eps_design, dJ/d |H_bias|) in FP64 by reverse-mode
    differentiation of the discrete step."""
    e = torch.as_tensor(np.asarray(eps_design, dtype=np.float64)).clone().requires_grad_(True)
    h = torch.tensor(float(h0), dtype=torch.float64, requires_grad=True)
    J = run(model, nsteps, e, h, n0=n0, segment=segment)
    J.backward()
    # without a magnetic cell |H_bias| enters no operation (it acts only
    # through H_eff in the LLG update of magnetic cells): its derivative is 0
    gh = 0.0 if h.grad is None else float(h.grad)
    return float(J.detach()), e.grad.numpy().copy(), gh
