"""Pins of the surrogate's FP64 oracle (oracle/lem.py) against closed forms,
an ODE solver, a direct linear solve, exact rotations and central
differences: the LEM cell of Eq. discrete_lem, the trapezoidal LLG map of
Eqs. llg_tra4-6 used by the physics loss (Eqs. ml_tra1-3), the gradients and
the Adam step."""
import numpy as np
import pytest
import torch
from scipy.integrate import solve_ivp

from oracle import lem

torch.set_default_dtype(torch.float64)


def _cell(d, m, rng, scale=0.5):
    W = torch.tensor(rng.normal(0, scale, (4, d, d)))
    V = torch.tensor(rng.normal(0, scale, (4, d, m)))
    b = torch.tensor(rng.normal(0, scale, (4, d)))
    return W, V, b


def test_layout_size():
    """The flat layout holds 4 cells of 4 (W, V, b) gate blocks and the head."""
    d, m = 5, 2
    theta = torch.zeros(lem.param_count(d, m))
    P = lem.unpack(theta, d, m)
    total = sum(t.numel() for c in lem.CELLS for t in P[c]) + P["Wo"].numel()
    assert total == lem.param_count(d, m) == 4 * (4 * d * d + 4 * d) + 4 * d * (m + d + m + d) + m * d


def test_zero_weights_follow_the_geometric_closed_form():
    """With every W and V zero the gates are constants a = dt sig(b1),
    abar = dt sig(b2), so from zero states z_n = (1 - (1-a)^n) tanh(bz) and
    y_n = (1 - (1-abar)^n) tanh(by) (a geometric series): the reconstruction
    is Wo y_n of the top encoder cell."""
    rng = np.random.default_rng(0)
    d, m, T, dt = 3, 2, 9, 0.7
    theta = torch.zeros(lem.param_count(d, m))
    P = lem.unpack(theta, d, m)
    with torch.no_grad():
        for c in lem.CELLS:
            P[c][2].copy_(torch.tensor(rng.normal(0, 1, (4, d))))
        P["Wo"].copy_(torch.tensor(rng.normal(0, 1, (m, d))))
    u = torch.tensor(rng.normal(0, 1, (T, 2, m)))
    rec, out = lem.forward(theta, u, 4, d, dt)
    b = P["enc1"][2]
    abar = dt / (1 + np.exp(-b[1].numpy()))
    n = np.arange(1, T + 1)[:, None]
    y = (1 - (1 - abar) ** n) * np.tanh(b[3].numpy())
    want = y @ P["Wo"].numpy().T
    assert np.allclose(rec.numpy(), want[:, None, :], rtol=0, atol=1e-14)
    # the decoder continues the same constant-gate series from the encoder's state
    bd = P["dec1"][2].numpy()
    ad = dt / (1 + np.exp(-bd[1]))
    yT = y[-1]
    yk = [yT]
    for _ in range(4):
        yk.append((1 - ad) * yk[-1] + ad * np.tanh(bd[3]))
    assert np.allclose(out.numpy(), (np.array(yk[1:]) @ P["Wo"].numpy().T)[:, None, :], atol=1e-14)


def test_small_step_limit_is_the_two_scale_ode():
    """As dt -> 0 the IMEX steps converge (first order) to Eq. lem with the
    gates as rates: dz/dt = s1 (tanh(Wz y + Vz u + bz) - z), dy/dt = s2
    (tanh(Wy z + Vy u + by) - y), s_i = sigmoid(W_i y + V_i u + b_i); the
    error against an accurate ODE solve halves with dt."""
    rng = np.random.default_rng(1)
    d, m = 4, 2
    Wc = _cell(d, m, rng, 0.8)
    u = torch.tensor(rng.normal(0, 1, (1, m)))
    y0 = torch.tensor(rng.normal(0, 0.5, (1, d)))
    z0 = torch.tensor(rng.normal(0, 0.5, (1, d)))
    W, V, bb = (t.numpy() for t in Wc)
    un = u.numpy()[0]

    def rhs(t, s):
        y, z = s[:d], s[d:]
        sg = lambda x: 1 / (1 + np.exp(-x))
        s1 = sg(W[0] @ y + V[0] @ un + bb[0])
        s2 = sg(W[1] @ y + V[1] @ un + bb[1])
        dz = s1 * (np.tanh(W[2] @ y + V[2] @ un + bb[2]) - z)
        dy = s2 * (np.tanh(W[3] @ z + V[3] @ un + bb[3]) - y)
        return np.concatenate([dy, dz])

    T = 1.0
    ref = solve_ivp(rhs, (0, T), np.concatenate([y0.numpy()[0], z0.numpy()[0]]), rtol=1e-12, atol=1e-12).y[:, -1]
    errs = []
    for nstep in (200, 400, 800):
        y, z = y0, z0
        for _ in range(nstep):
            y, z = lem.lem_cell(Wc, y, z, u, T / nstep)
        errs.append(np.abs(np.concatenate([y.numpy()[0], z.numpy()[0]]) - ref).max())
    assert errs[2] < 2e-3
    assert 1.7 < errs[0] / errs[1] < 2.3 and 1.7 < errs[1] / errs[2] < 2.3


def test_y_update_reads_the_new_z():
    """The y update uses z_n of the same step: from zero states with only Wy
    non-zero and by = 0, y_1 = abar tanh(Wy z_1) is non-zero (reading z_0 = 0
    would leave y_1 = 0)."""
    d, m, dt = 2, 1, 0.5
    W = torch.zeros(4, d, d)
    W[3] = torch.tensor([[1.0, -0.5], [0.3, 2.0]])
    V = torch.zeros(4, d, m)
    b = torch.zeros(4, d)
    b[2] = torch.tensor([0.8, -1.1])
    y, z = lem.lem_cell((W, V, b), torch.zeros(1, d), torch.zeros(1, d), torch.zeros(1, m), dt)
    z1 = 0.5 * dt * np.tanh([0.8, -1.1])
    assert np.allclose(z.numpy()[0], z1, atol=1e-15)
    assert np.allclose(y.numpy()[0], 0.5 * dt * np.tanh(W[3].numpy() @ z1), atol=1e-15)


def _rodrigues(v, axis, th):
    k = axis / np.linalg.norm(axis)
    return v * np.cos(th) + np.cross(k, v) * np.sin(th) + k * (k @ v) * (1 - np.cos(th))


@pytest.mark.parametrize("h", [(0.0, 0.0, 0.0), (350.0, -120.0, 80.0)])
def test_llg_map_is_the_cayley_rotation_without_damping(h):
    """With alpha = 0 and a constant field, x + a x x = b with a = -kappa H,
    b = m - kappa m x H is the Cayley transform: m rotated about H by
    2 atan(kappa |H|) in the sense of -m x H (exact for any step); |m| is kept."""
    h0, kappa = 1.4e4, 3.1e-5
    rng = np.random.default_rng(2)
    pq = rng.normal(0, 0.1, (5, 2))
    hv = torch.tensor(np.tile(h, (5, 1)), dtype=torch.float64)
    px, qx = lem.llg_next(torch.tensor(pq[:, 0]), torch.tensor(pq[:, 1]), hv, hv, kappa, 0.0, h0)
    H = np.array(h) + np.array([0, 0, h0])
    th = 2 * np.arctan(kappa * np.linalg.norm(H))
    for r in range(5):
        mv = np.array([pq[r, 0], pq[r, 1], 1.0])
        want = _rodrigues(mv, H, th)   # +theta about H: e1 -> e2 for H along e3, as -m x H
        assert px[r].item() == pytest.approx(want[0], abs=1e-14)
        assert qx[r].item() == pytest.approx(want[1], abs=1e-14)


def test_llg_map_solves_its_linear_system():
    """Eq. llg_tra4 is the closed-form solution of M~ + a x M~ = b: a direct
    3x3 solve with the a and b of Eqs. llg_tra5-6 (H^{k+1} in a, H^k in b)
    gives the same M~ (before N), here with damping and distinct fields."""
    rng = np.random.default_rng(3)
    kappa, alpha, h0 = 2e-5, 0.01, 1.2e4
    for _ in range(4):
        p, q = rng.normal(0, 0.2, 2)
        hk, hk1 = rng.normal(0, 800, 3), rng.normal(0, 800, 3)
        m = np.array([p, q, 1.0])
        Hk, Hk1 = hk + [0, 0, h0], hk1 + [0, 0, h0]
        b = m - kappa * np.cross(m, Hk)
        a = -(kappa * Hk1 + alpha * m)
        A = np.eye(3) + np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
        x = np.linalg.solve(A, b)
        x *= np.linalg.norm(m) / np.linalg.norm(x)
        px, qx = lem.llg_next(torch.tensor([p]), torch.tensor([q]), torch.tensor([hk]), torch.tensor([hk1]), kappa,
                              alpha, h0)
        assert px.item() == pytest.approx(x[0], abs=1e-14) and qx.item() == pytest.approx(x[1], abs=1e-14)


def test_damping_relaxes_towards_the_bias():
    """With alpha > 0 in a bias field alone the transverse amplitude falls every
    step while |m| is kept; with alpha = 0 it stays."""
    kappa, h0 = 4e-5, 1.5e4
    p, q = torch.tensor([0.2]), torch.tensor([0.0])
    h = torch.zeros(1, 3)
    amp = []
    for _ in range(20):
        p, q = lem.llg_next(p, q, h, h, kappa, 0.05, h0)
        amp.append(float(torch.hypot(p, q)))
    assert all(b < a for a, b in zip(amp, amp[1:]))
    p0, q0 = lem.llg_next(torch.tensor([0.2]), torch.tensor([0.0]), h, h, kappa, 0.0, h0)
    assert float(torch.hypot(p0, q0)) == pytest.approx(0.2, abs=1e-15)


def test_physics_loss_vanishes_on_an_exact_precession():
    """Predictions that precess exactly (alpha = 0, bias only) have zero
    physics residual; a perturbed sequence does not."""
    d, m, B, T = 3, 2, 2, 6
    kappa, h0 = 3e-5, 1.3e4
    th = 2 * np.arctan(kappa * h0)
    ph = np.arange(T)[:, None] * th + np.array([0.3, 1.1])[None, :]
    seq = np.stack([0.1 * np.cos(ph), 0.1 * np.sin(ph)], -1)
    out = torch.tensor(seq)
    h = torch.zeros(T, B, 3)
    px, qx = lem.llg_next(out[:-1, :, 0], out[:-1, :, 1], h[:-1], h[1:], kappa, 0.0, h0)
    assert torch.abs(px - out[1:, :, 0]).max() < 1e-15 and torch.abs(qx - out[1:, :, 1]).max() < 1e-15
    out2 = out.clone()
    out2[3, 0, 0] += 1e-3
    px, qx = lem.llg_next(out2[:-1, :, 0], out2[:-1, :, 1], h[:-1], h[1:], kappa, 0.0, h0)
    assert torch.abs(px - out2[1:, :, 0]).max() > 5e-4


def test_gradient_matches_central_differences():
    """torch.autograd's gradient of the total loss (data + lambda physics)
    equals central differences of the loss in float64."""
    rng = np.random.default_rng(4)
    d, m, B, T_in, T_out = 3, 2, 2, 5, 4
    theta = rng.normal(0, 0.4, lem.param_count(d, m))
    u = rng.normal(0, 0.3, (T_in, B, m))
    tgt = rng.normal(0, 0.3, (T_out, B, m))
    h = rng.normal(0, 300, (T_out, B, 3))
    args = dict(lam=0.7, kappa=4e-5, alpha=0.02, h0=1e4, d=d, dt=0.8)
    r = lem.train_grad(theta, u, tgt, h, **args)
    tt = lambda x: torch.tensor(x)
    f = lambda th: float(lem.losses(tt(th), tt(u), tt(tgt), tt(h), args["lam"], args["kappa"], args["alpha"],
                                    args["h0"], d, args["dt"])[0])
    eps = 1e-6
    idx = rng.choice(theta.size, 40, replace=False)
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = eps
        fd = (f(theta + e) - f(theta - e)) / (2 * eps)
        assert r["grad"][i] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_adam_first_step_moves_by_the_learning_rate():
    """From zero moments the bias-corrected first Adam step is
    -lr g / (|g| + eps) per parameter."""
    g = np.array([3.0, -0.2, 1e-3])
    th, mo, ve = lem.adam(np.zeros(3), g, np.zeros(3), np.zeros(3), 0.01, 1)
    assert np.allclose(th, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_decoder_is_the_encoder_fed_its_own_outputs():
    """With the decoder cells given the encoder cells' weights, the decoder
    (started from the encoder's final states, input 0 first and then the
    previous output) produces what the encoder reconstructs from the input
    sequence extended by 0, o_0, o_1, ...: the autoregressive wiring."""
    rng = np.random.default_rng(5)
    d, m, B, T_in, T_out, dt = 4, 2, 3, 6, 5, 0.9
    theta = torch.tensor(rng.normal(0, 0.6, lem.param_count(d, m)))
    P = lem.unpack(theta, d, m)
    with torch.no_grad():
        for src, dst in (("enc0", "dec0"), ("enc1", "dec1")):
            for a, b in zip(P[src], P[dst]):
                b.copy_(a)
    u = torch.tensor(rng.normal(0, 0.5, (T_in, B, m)))
    _, out = lem.forward(theta, u, T_out, d, dt)
    ext = torch.cat([u, torch.zeros(1, B, m), out[:-1]], 0)
    rec, _ = lem.forward(theta, ext, 1, d, dt)
    assert torch.allclose(rec[T_in:], out, atol=1e-14, rtol=0)
