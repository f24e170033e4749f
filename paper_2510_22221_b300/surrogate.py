"""The physics-informed sequence surrogate of the paper (Results, "HPC and ML
framework"; Methods "LEM Cell", "ML Training Implementation", "Physics
Loss"): an LEM encoder-decoder trained on this solver's own probe series
with a data loss and the trapezoidal-LLG physics loss.

``LemSurrogate`` marshals arguments into the CUDA entry points of
include/lem_surrogate.h (forward pass, losses, back-propagation, Adam: every
step runs in the library's kernels).  ``export_probe_series`` runs a solver
handle and returns the probe series in the bias frame; ``windows`` cuts
training sequences from them; ``curriculum`` is the staged schedule of the
paper's training (learning rate, prediction length, batch size and physics
weight raised or lowered stage by stage).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import _abi
from ._abi import check

MU0 = 4e-7 * np.pi


def bias_frame(u) -> np.ndarray:
    """Rows e1, e2, e3 of a right-handed orthonormal frame with e3 along u."""
    e3 = np.asarray(u, dtype=np.float64)
    e3 = e3 / np.linalg.norm(e3)
    a = np.array([1.0, 0.0, 0.0]) if abs(e3[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = np.cross(a, e3)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(e3, e1)
    return np.stack([e1, e2, e3])


def kappa_of(gamma: float, dt_ml: float) -> float:
    """kappa = mu0 |gamma| dt_ML / 4 of Eqs. llg_tra5-6 for the sampling step."""
    return MU0 * abs(gamma) * dt_ml / 4.0


def export_probe_series(sim, probes, steps: int, every: int, bias_dir, Ms: float) -> dict:
    """Run ``steps`` steps of a configured solver handle (its probe capacity
    at least ``steps``) and return, for the listed probe ids, every
    ``every``-th sample of the probe rows in the bias frame: ``m`` [nprobe,
    T, 2] (the transverse components of M / Ms) and ``h`` [nprobe, T, 3]
    (the probe's H in frame components, A/m), with ``dt_ml`` = every x dt."""
    sim.step(int(steps))
    R = bias_frame(bias_dir)
    ms, hs = [], []
    for p in probes:
        rows = sim.probe(int(p), cap_rows=steps)[every - 1::every]
        ms.append((rows[:, 6:9] @ R.T)[:, :2] / Ms)
        hs.append(rows[:, 3:6] @ R.T)
    return dict(m=np.stack(ms), h=np.stack(hs), dt_ml=float(sim.dt) * every)


def windows(m, h, t_in: int, t_out: int, starts) -> tuple:
    """Training sequences from series m [S, T, 2] and h [S, T, 3]: for each
    (series, start) pair the inputs m[start : start + t_in], the targets and
    the field over the next t_out samples, as arrays [t, batch, c] (the
    layout of include/lem_surrogate.h)."""
    u = np.stack([m[s, a:a + t_in] for s, a in starts], 1)
    tg = np.stack([m[s, a + t_in:a + t_in + t_out] for s, a in starts], 1)
    hh = np.stack([h[s, a + t_in:a + t_in + t_out] for s, a in starts], 1)
    return (np.ascontiguousarray(u, dtype=np.float32), np.ascontiguousarray(tg, dtype=np.float32),
            np.ascontiguousarray(hh, dtype=np.float32))


@dataclass
class Stage:
    epochs: int
    lr: float
    t_out: int
    batch: int
    lam: float


def curriculum(total_epochs: int = 1250, lr0: float = 1e-3, lr1: float = 1.25e-4, t_out0: int = 50,
               t_out1: int = 400, batch0: int = 64, batch1: int = 512, lam1: float = 2.5e6, stages: int = 4) -> list:
    """The staged schedule of "ML Training Implementation": the learning rate
    falls geometrically from lr0 to lr1, the prediction length and the batch
    grow from (t_out0, batch0) to (t_out1, batch1), and the physics weight
    starts at 0 and rises to lam1 (stage s of n uses lam1 s / (n - 1))."""
    out = []
    for s in range(stages):
        f = s / max(stages - 1, 1)
        out.append(Stage(epochs=total_epochs // stages, lr=float(lr0 * (lr1 / lr0) ** f),
                         t_out=int(round(t_out0 + (t_out1 - t_out0) * f)),
                         batch=int(round(batch0 * (batch1 / batch0) ** f)), lam=float(lam1 * f)))
    return out


def init_params(d: int, m: int, seed: int = 0) -> np.ndarray:
    """Uniform(-1/sqrt(d), 1/sqrt(d)) initial parameters (seeded), FP32."""
    n = _abi.load().fdtd_llg_lem_param_count(int(d), int(m))
    if n <= 0:
        raise ValueError("d must be 16, 32 or 64 and 1 <= m <= 4")
    r = 1.0 / np.sqrt(d)
    return np.random.default_rng(seed).uniform(-r, r, n).astype(np.float32)


class LemSurrogate:
    """Parameters, Adam moments and the work space on one GPU.  Sequences are
    torch CUDA float32 tensors [t, batch, c] (or arrays, copied to the
    device)."""

    def __init__(self, d: int = 64, m: int = 2, dt: float = 1.0, theta=None, seed: int = 0, device: int = 0):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("LemSurrogate needs a CUDA device: the surrogate has no CPU path")
        self.torch = torch
        self.dev = torch.device("cuda", device)
        self.d, self.m, self.dt = int(d), int(m), float(dt)
        lib = _abi.load()
        self.nparam = int(lib.fdtd_llg_lem_param_count(self.d, self.m))
        if self.nparam <= 0:
            raise ValueError("d must be 16, 32 or 64 and 1 <= m <= 4")
        th = init_params(d, m, seed) if theta is None else np.asarray(theta, dtype=np.float32)
        if th.size != self.nparam:
            raise ValueError(f"theta has {th.size} values, the layout {self.nparam}")
        self.theta = torch.tensor(th, device=self.dev)
        self.mom = torch.zeros_like(self.theta)
        self.vel = torch.zeros_like(self.theta)
        self.t = 0
        self._ws = torch.empty(0, dtype=torch.uint8, device=self.dev)

    # ------------------------------------------------------------- marshalling
    def _dev(self, x):
        t = self.torch
        if isinstance(x, t.Tensor):
            return x.to(self.dev, t.float32).contiguous()
        return t.tensor(np.ascontiguousarray(x, dtype=np.float32), device=self.dev)

    def _check(self, u, target=None, h=None):
        """Shapes against the layout of include/lem_surrogate.h (the library
        reads exactly that many values)."""
        if u.dim() != 3 or u.shape[2] != self.m:
            raise ValueError(f"u must be [t_in, batch, {self.m}], got {tuple(u.shape)}")
        if target is not None and (target.dim() != 3 or target.shape[1:] != u.shape[1:]):
            raise ValueError(f"target must be [t_out, {u.shape[1]}, {self.m}], got {tuple(target.shape)}")
        if h is not None and tuple(h.shape) != (target.shape[0], u.shape[1], 3):
            raise ValueError(f"h must be [{target.shape[0]}, {u.shape[1]}, 3], got {tuple(h.shape)}")

    def _shape(self, batch, t_in, t_out):
        s = _abi.LemShape()
        s.d, s.m, s.batch, s.t_in, s.t_out, s.dt = self.d, self.m, int(batch), int(t_in), int(t_out), self.dt
        return s

    def _work(self, s):
        n = C.c_size_t()
        check(_abi.load().fdtd_llg_lem_workspace_bytes(C.byref(s), C.byref(n)))
        if self._ws.numel() < n.value:
            self._ws = self.torch.empty(n.value, dtype=self.torch.uint8, device=self.dev)
        return self._ws

    def _views(self, s, ws):
        ptr = [C.c_void_p() for _ in range(4)]
        check(_abi.load().fdtd_llg_lem_views(C.byref(s), C.c_void_p(ws.data_ptr()), *[C.byref(p) for p in ptr]))
        base = ws.data_ptr()

        def view(p, n, dtype, esize):
            o = p.value - base
            return ws[o:o + n * esize].view(dtype)

        t = self.torch
        return dict(recon=view(ptr[0], s.t_in * s.batch * self.m, t.float32, 4).view(s.t_in, s.batch, self.m),
                    out=view(ptr[1], s.t_out * s.batch * self.m, t.float32, 4).view(s.t_out, s.batch, self.m),
                    grad=view(ptr[2], self.nparam, t.float32, 4), loss=view(ptr[3], 4, t.float64, 8))

    def _stream(self):
        return C.c_void_p(self.torch.cuda.current_stream(self.dev).cuda_stream)

    @staticmethod
    def _phys(lam, kappa, alpha, h0):
        p = _abi.LemPhysics()
        p.lam, p.kappa, p.alpha, p.h0 = float(lam), float(kappa), float(alpha), float(h0)
        return p

    # ------------------------------------------------------------------- calls
    def forward(self, u, t_out: int):
        """(reconstruction, prediction) for inputs u [t_in, batch, m]."""
        u = self._dev(u)
        self._check(u)
        s = self._shape(u.shape[1], u.shape[0], t_out)
        ws = self._work(s)
        check(_abi.load().fdtd_llg_lem_forward(C.byref(s), C.c_void_p(self.theta.data_ptr()), C.c_void_p(u.data_ptr()),
                                               C.c_void_p(ws.data_ptr()), self._stream()))
        v = self._views(s, ws)
        return v["recon"].clone(), v["out"].clone()

    def gradient(self, u, target, h, lam=0.0, kappa=0.0, alpha=0.0, h0=0.0):
        """(losses (total, L_rec, L_pred, L_phy), gradient) of the current
        parameters on one batch; nothing is updated."""
        u, target = self._dev(u), self._dev(target)
        h = self._dev(h) if h is not None else None
        self._check(u, target, h)
        s = self._shape(u.shape[1], u.shape[0], target.shape[0])
        ws = self._work(s)
        lib, st, w = _abi.load(), self._stream(), C.c_void_p(ws.data_ptr())
        ph = self._phys(lam, kappa, alpha, h0)
        check(lib.fdtd_llg_lem_forward(C.byref(s), C.c_void_p(self.theta.data_ptr()), C.c_void_p(u.data_ptr()), w, st))
        check(lib.fdtd_llg_lem_loss(C.byref(s), C.byref(ph), C.c_void_p(u.data_ptr()), C.c_void_p(target.data_ptr()),
                                    C.c_void_p(h.data_ptr() if h is not None else 0), w, st))
        check(lib.fdtd_llg_lem_backward(C.byref(s), C.c_void_p(self.theta.data_ptr()), C.c_void_p(u.data_ptr()), w, st))
        v = self._views(s, ws)
        return v["loss"].cpu().numpy().copy(), v["grad"].clone()

    def train_step(self, u, target, h, lr: float, lam=0.0, kappa=0.0, alpha=0.0, h0=0.0, read_loss=True):
        """One Adam step on one batch; returns the batch's losses before the
        update (one device-to-host read of 4 doubles) or None."""
        u, target = self._dev(u), self._dev(target)
        h = self._dev(h) if h is not None else None
        self._check(u, target, h)
        s = self._shape(u.shape[1], u.shape[0], target.shape[0])
        ws = self._work(s)
        self.t += 1
        ph = self._phys(lam, kappa, alpha, h0)
        check(_abi.load().fdtd_llg_lem_train_step(
            C.byref(s), C.byref(ph), C.c_void_p(self.theta.data_ptr()), C.c_void_p(u.data_ptr()),
            C.c_void_p(target.data_ptr()), C.c_void_p(h.data_ptr() if h is not None else 0),
            C.c_void_p(self.mom.data_ptr()), C.c_void_p(self.vel.data_ptr()), float(lr), int(self.t),
            C.c_void_p(ws.data_ptr()), self._stream()))
        if not read_loss:
            return None
        return self._views(s, ws)["loss"].cpu().numpy().copy()

    def adam(self, grad, lr: float):
        """One Adam step with a given gradient (device tensor)."""
        g = self._dev(grad)
        if g.numel() != self.nparam:
            raise ValueError(f"grad must hold {self.nparam} values")
        self.t += 1
        check(_abi.load().fdtd_llg_lem_adam(self.nparam, C.c_void_p(self.theta.data_ptr()), C.c_void_p(g.data_ptr()),
                                            C.c_void_p(self.mom.data_ptr()), C.c_void_p(self.vel.data_ptr()),
                                            float(lr), 0.9, 0.999, 1e-8, int(self.t), self._stream()))
