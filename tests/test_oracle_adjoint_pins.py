"""Pins of the FP64 reference gradients (oracle/adjoint.py): its PyTorch
restatement of the step equals the C oracle, and its reverse-mode gradients
of the probe objective J = sum |E(probe)|^2 equal central finite differences
of J (arxiv 2510.22221, section "Numerical Model"; the objective and the
parameters are those of the adjoint design case)."""
import numpy as np
import pytest
import torch

import oracle
from oracle import adjoint as A
from paper_2510_22221_b300 import workloads as W
from tests.helpers import oracle_from_workload


def _model(w, R=3):
    dt = oracle.courant_dt(w.dx, w.dy, w.dz, w.courant)
    src = [dict(comp=s["comp"], ijk=(s["i"], s["j"], s["k"]), J0=s["J0"], f0=s["f0"], Tp=s["Tp"], tpk=s["tpk"])
           for s in w.sources]
    return A.TorchStep(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, dt, w.materials, w.mat_id, w.hbias, sources=src,
                       probes=w.probes, design_box=w.design_box, fixed_iter=R)


def _J(m, steps, eps, h0, n0):
    with torch.no_grad():
        return float(A.run(m, steps, torch.as_tensor(eps), torch.tensor(h0, dtype=torch.float64), n0=n0))


@pytest.mark.parametrize("seed", [1, 2])
def test_torch_step_equals_c_oracle(seed):
    w = W.random_small(seed, nx=9, ny=8, nz=7, steps=30, design=True)
    m = _model(w)
    orc = oracle_from_workload(w, llg_fixed_iter=3)
    ref = orc.run(30)["probes"]
    J, rows = A.run(m, 30, torch.as_tensor(w.eps_design), None, n0=0, segment=7, record=True)
    np.testing.assert_allclose(rows, ref[:, :, :3], rtol=0, atol=1e-13 * np.abs(ref[:, :, :3]).max())
    E, H, M = m.zero_state(None)
    eps_c, hb = m.eps_cell(torch.as_tensor(w.eps_design)), torch.as_tensor(w.hbias)
    for n in range(30):
        E, H, M = m.step(E, H, M, eps_c, hb, n)
    for name, t in zip(("Ex", "Ey", "Ez", "Hx", "Hy", "Hz"), (*E, *H)):
        a = getattr(orc, name)
        np.testing.assert_allclose(t.numpy(), a, rtol=0, atol=1e-13 * np.abs(a).max())
    np.testing.assert_allclose(M.numpy(), orc.M, rtol=0, atol=1e-12 * 1.4e5)


def test_eps_gradient_equals_central_differences():
    w = W.adjoint_small(n=16, steps=260, design=(6, 6, 2), block=(4, 4, 2))
    m = _model(w)
    h0 = float(np.linalg.norm(w.hbias))
    J, ge, gh = A.gradients(m, 260, w.eps_design, h0, n0=160)
    assert J > 0
    rng = np.random.default_rng(5)
    for _ in range(4):
        idx = tuple(int(rng.integers(0, s)) for s in w.eps_design.shape)
        e1, e2 = w.eps_design.copy(), w.eps_design.copy()
        d = 1e-4 * e1[idx]
        e1[idx] += d
        e2[idx] -= d
        fd = (_J(m, 260, e1, h0, 160) - _J(m, 260, e2, h0, 160)) / (2 * d)
        assert ge[idx] == pytest.approx(fd, rel=1e-6)


def test_bias_gradient_equals_central_differences():
    """The bias enters only through H_eff of the LLG (M starts along the bias
    direction whatever its size), so this pins the differentiation of the
    trapezoidal LLG solve, its Jacobi iterates and the face coupling."""
    w = W.anticrossing_sweep(n_inst=1, b_lo=0.05, b_hi=0.05, steps=900, design=(4, 3, 1))[0]
    m = _model(w)
    h0 = float(np.linalg.norm(w.hbias))
    J, ge, gh = A.gradients(m, 900, w.eps_design, h0, n0=500)
    d = 1e-5 * h0
    fd = (_J(m, 900, w.eps_design, h0 + d, 500) - _J(m, 900, w.eps_design, h0 - d, 500)) / (2 * d)
    assert gh == pytest.approx(fd, rel=1e-6)
    idx = (0, 1, 2)
    e1, e2 = w.eps_design.copy(), w.eps_design.copy()
    de = 1e-4 * e1[idx]
    e1[idx] += de
    e2[idx] -= de
    fd = (_J(m, 900, e1, h0, 500) - _J(m, 900, e2, h0, 500)) / (2 * de)
    assert ge[idx] == pytest.approx(fd, rel=1e-6)
