"""The surrogate's CUDA path (include/lem_surrogate.h) against the FP64 oracle
(oracle/lem.py): forward pass, losses with the trapezoidal-LLG physics term,
the gradient, Adam, the fused training step, and training on the solver's
own probe series (Methods "LEM Cell", "ML Training Implementation", "Physics
Loss")."""
import numpy as np
import pytest

from oracle import lem as O

from tests.helpers import record

gpu = pytest.mark.gpu

# FP32 against FP64: the recurrences contract (gates in (0, dt), tanh), so the
# forward error stays at a few FP32 roundings of the state times the head's
# gain, at every length (measured on a B300: 6e-8 to 1.1e-7 up to 600 steps);
# the gradient's relative L2 error measured 1.2e-7 to 5.8e-7.  The bounds are
# about ten times the largest measured error.
TOL_OUT = 1e-6       # max abs error of reconstruction and prediction (values ~0.1)
TOL_LOSS = 2e-6      # relative error of each loss
TOL_GRAD = 5e-6      # relative L2 error of the gradient


def _case(d, m, B, T_in, T_out, seed, amp=0.1):
    rng = np.random.default_rng(seed)
    theta = rng.uniform(-1, 1, O.param_count(d, m)).astype(np.float32) / np.sqrt(d)
    t = np.arange(T_in + T_out)[:, None]
    w = rng.uniform(0.05, 0.3, B)[None, :]
    ph = rng.uniform(0, 2 * np.pi, B)[None, :]
    seq = amp * np.stack([np.cos(w * t + ph + c * np.pi / 2) for c in range(m)], -1)
    seq = (seq + rng.normal(0, 0.01 * amp, seq.shape)).astype(np.float32)
    h = rng.normal(0, 300.0, (T_out, B, 3)).astype(np.float32)
    return theta, seq[:T_in], seq[T_in:], h


PHYS = dict(lam=0.5, kappa=2.5e-5, alpha=0.01, h0=1.2e4)


def _surrogate(theta, d, m, dt=0.9):
    from paper_2510_22221_b300.surrogate import LemSurrogate

    return LemSurrogate(d=d, m=m, dt=dt, theta=theta)


@gpu
@pytest.mark.parametrize("d,B,T_in,T_out", [(16, 11, 13, 9), (32, 8, 40, 17), (64, 20, 50, 30)])
def test_forward_matches_oracle(d, B, T_in, T_out):
    m = 2
    theta, u, tg, h = _case(d, m, B, T_in, T_out, seed=d + B)
    S = _surrogate(theta, d, m)
    rec, out = S.forward(u, T_out)
    r = O.train_grad(theta, u, tg, h, d=d, dt=0.9, **PHYS)
    e_rec = np.abs(rec.cpu().numpy() - r["recon"]).max()
    e_out = np.abs(out.cpu().numpy() - r["out"]).max()
    record(f"lem_forward_d{d}_B{B}", max(e_rec, e_out), TOL_OUT)
    assert e_rec < TOL_OUT and e_out < TOL_OUT


@gpu
@pytest.mark.parametrize("d,m,B,T_in,T_out,lam", [(16, 2, 11, 13, 9, 0.5), (64, 2, 20, 50, 30, 0.5),
                                                   (32, 3, 9, 12, 7, 0.0), (16, 2, 5, 6, 1, 0.5)])
def test_losses_and_gradient_match_oracle(d, m, B, T_in, T_out, lam):
    theta, u, tg, h = _case(d, m, B, T_in, T_out, seed=7 * d + B)
    S = _surrogate(theta, d, m)
    phys = dict(PHYS, lam=lam)
    loss, g = S.gradient(u, tg, h if m == 2 else None, **phys)
    r = O.train_grad(theta, u, tg, h if m == 2 else np.zeros((T_out, B, 3)), d=d, dt=0.9, **phys)
    want = [r["total"], r["rec"], r["pred"], r["phy"] if m == 2 else 0.0]
    for a, b in zip(loss, want):
        assert a == pytest.approx(b, rel=TOL_LOSS, abs=1e-12)
    g = g.cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(g - r["grad"]) / np.linalg.norm(r["grad"])
    record(f"lem_gradient_d{d}_m{m}_B{B}_T{T_in}+{T_out}", rel, TOL_GRAD)
    assert rel < TOL_GRAD


@gpu
def test_physics_gradient_alone_matches_oracle():
    """The physics term's gradient (dual-number derivative of the LLG map and
    the residual's direct term) isolated: prediction target equal to the
    prediction makes L_pred's gradient vanish, lam large."""
    d, m, B, T_in, T_out = 16, 2, 9, 10, 12
    theta, u, _, h = _case(d, m, B, T_in, T_out, seed=3)
    S = _surrogate(theta, d, m)
    _, out = S.forward(u, T_out)
    tg = out.cpu().numpy()
    phys = dict(PHYS, lam=1e3)
    loss, g = S.gradient(u, tg, h, **phys)
    r = O.train_grad(theta, u, tg, h, d=d, dt=0.9, **phys)
    assert loss[3] == pytest.approx(r["phy"], rel=1e-4)
    g = g.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - r["grad"]) / np.linalg.norm(r["grad"]) < TOL_GRAD


@gpu
def test_adam_and_train_step_match_the_oracle_and_the_parts():
    import torch

    d, m, B, T_in, T_out = 16, 2, 10, 12, 8
    theta, u, tg, h = _case(d, m, B, T_in, T_out, seed=11)
    A = _surrogate(theta, d, m)
    Bm = _surrogate(theta, d, m)
    th, mo, ve = theta.astype(np.float64), np.zeros(theta.size), np.zeros(theta.size)
    for t in range(1, 4):
        loss = A.train_step(u, tg, h, lr=1e-3, **PHYS)
        # the parts, and the oracle's Adam on the GPU gradient
        l2, g = Bm.gradient(u, tg, h, **PHYS)
        Bm.adam(g, lr=1e-3)
        assert np.array_equal(loss, l2)
        th, mo, ve = O.adam(th, g.cpu().numpy().astype(np.float64), mo, ve, 1e-3, t)
        torch.cuda.synchronize()
        assert torch.equal(A.theta, Bm.theta)
        assert np.abs(A.theta.cpu().numpy() - th).max() < 1e-6
        # the next step starts from the oracle-updated parameters, rounded to FP32
        th = A.theta.cpu().numpy().astype(np.float64)


@gpu
def test_gradient_is_the_same_bits_every_run_and_for_a_padded_batch():
    """Fixed-order sums: two runs give the same bits; a batch that is not a
    multiple of a CTA's sequences pads without changing the values of the
    real sequences' outputs."""
    d, m, B, T_in, T_out = 32, 2, 13, 20, 10
    theta, u, tg, h = _case(d, m, B, T_in, T_out, seed=5)
    S = _surrogate(theta, d, m)
    l1, g1 = S.gradient(u, tg, h, **PHYS)
    l2, g2 = S.gradient(u, tg, h, **PHYS)
    assert np.array_equal(l1, l2) and bool((g1 == g2).all())
    _, o_all = S.forward(u, T_out)
    _, o_one = S.forward(u[:, 3:4], T_out)
    assert np.array_equal(o_all.cpu().numpy()[:, 3], o_one.cpu().numpy()[:, 0])


@gpu
def test_two_sequences_per_thread_give_the_same_bits():
    """A batch large enough for two sequences per thread (a CTA of 8 instead
    of 4) gives every sequence the same bits as a small batch, and matches
    the oracle on sampled sequences."""
    d, m, B, T_in, T_out = 16, 2, 1300, 24, 12
    theta, u, tg, h = _case(d, m, B, T_in, T_out, seed=9)
    S = _surrogate(theta, d, m)
    rec, out = S.forward(u, T_out)
    pick = [0, 5, 777, 1299]
    rec_s, out_s = S.forward(u[:, pick], T_out)
    assert np.array_equal(out.cpu().numpy()[:, pick], out_s.cpu().numpy())
    assert np.array_equal(rec.cpu().numpy()[:, pick], rec_s.cpu().numpy())
    r = O.train_grad(theta, u[:, pick], tg[:, pick], h[:, pick], d=d, dt=0.9, **PHYS)
    assert np.abs(out_s.cpu().numpy() - r["out"]).max() < TOL_OUT
    loss, g = S.gradient(u, tg, h, **PHYS)
    assert np.all(np.isfinite(g.cpu().numpy()))


@gpu
def test_full_size_forward_samples_and_gradient():
    """The paper's sizes: hidden width 64, 200 input samples, 400 predicted,
    batch 512 (the last curriculum stage).  Forward outputs of 4 sampled
    sequences against the oracle run on those sequences alone; the whole
    gradient against the oracle's."""
    d, m, B, T_in, T_out = 64, 2, 512, 200, 400
    theta, u, tg, h = _case(d, m, B, T_in, T_out, seed=21)
    S = _surrogate(theta, d, m)
    rec, out = S.forward(u, T_out)
    pick = [0, 137, 300, 511]
    r = O.train_grad(theta, u[:, pick], tg[:, pick], h[:, pick], d=d, dt=0.9, **PHYS)
    e = max(np.abs(rec.cpu().numpy()[:, pick] - r["recon"]).max(), np.abs(out.cpu().numpy()[:, pick] - r["out"]).max())
    record("lem_forward_full_d64_B512_T200+400_sampled", e, TOL_OUT)
    assert e < TOL_OUT
    loss, g = S.gradient(u, tg, h, **PHYS)
    rf = O.train_grad(theta, u, tg, h, d=d, dt=0.9, **PHYS)
    g = g.cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(g - rf["grad"]) / np.linalg.norm(rf["grad"])
    record("lem_gradient_full_d64_B512_T200+400", rel, TOL_GRAD)
    assert rel < TOL_GRAD
    assert loss[0] == pytest.approx(rf["total"], rel=TOL_LOSS)


@gpu
def test_training_on_the_solvers_probe_series_reduces_the_data_loss():
    """Training data exported from the solver (the YIG block of the 32^3
    cavity, nine probes in the block's mid-plane: its centre, corners and edge
    midpoints, as in the paper's film), scaled to unit amplitude: 300 Adam
    steps on the exported windows take the data loss down by 10x."""
    import paper_2510_22221_b300 as pkg
    from paper_2510_22221_b300 import surrogate as SG
    from paper_2510_22221_b300 import workloads as W

    w = W.cavity_block(steps=6000)
    sim = pkg.from_workload(w, probe_capacity=6000)
    probes = [sim.add_probe(i, j, 15) for i in (12, 15, 19) for j in (12, 15, 19)]
    Ms = max(mt["Ms"] for mt in w.materials)
    ser = SG.export_probe_series(sim, probes, 6000, 10, w.hbias, Ms)
    sim.destroy()
    scale = np.abs(ser["m"]).max()
    assert np.isfinite(scale) and scale > 0
    m, hh = ser["m"] / scale, ser["h"]
    T_in, T_out = 100, 50
    starts = [(s, a) for s in range(len(probes)) for a in range(0, 600 - T_in - T_out, 25)]
    u, tg, hw = SG.windows(m, hh, T_in, T_out, starts)
    S = SG.LemSurrogate(d=32, m=2, dt=1.0, seed=0)
    first = S.train_step(u, tg, hw, lr=3e-3)
    for _ in range(300):
        S.train_step(u, tg, hw, lr=3e-3, read_loss=False)
    last = S.train_step(u, tg, hw, lr=3e-3)
    record("lem_training_data_loss_cavity_block_9_probes", float(last[1] + last[2]), 0.1 * float(first[1] + first[2]))
    assert np.all(np.isfinite(last))
    assert last[1] + last[2] < 0.1 * (first[1] + first[2])
