"""Absorbing layers (convolutional PML, the oracle's reading R15) on the CUDA
path against the FP64 oracle, through the C ABI; tolerances as in
test_gpu_parity (the layers add one FP32 recursion per memory and step, of
the same rounding order as the curls they correct)."""
import ctypes as C

import numpy as np
import pytest

import paper_2510_22221_b300 as pkg
from paper_2510_22221_b300 import _abi
from paper_2510_22221_b300 import workloads as W
from tests.helpers import compact, oracle_from_workload, record
from tests.test_gpu_parity import FAMILIES, check_energy, check_probes, compare_fields, probe_errors, rel_err, run_pair, tol

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed,layers,kappa,alpha", [(0, (6, 5, 4), 1.0, 0.0), (1, (6, 0, 4), 3.0, 0.3),
                                                     (2, (3, 7, 5), 5.0, 0.05)])
def test_layers_match_oracle(seed, layers, kappa, alpha):
    w = W.pml_small(seed, layers=layers, kappa_max=kappa, alpha_max=alpha)
    sim, orc, out, M0 = run_pair(w, w.steps)
    t = tol(w.steps)
    for p, (i, j, k) in enumerate(w.probes):
        errs = probe_errors(sim.probe(p), out["probes"][:, p], M0[:, k, j, i], t, w.steps)
        check_probes(errs, t, w.steps, p)
    check_energy(sim.energy(), out["energy"], t, w.steps)
    compare_fields(sim, orc, M0, t)


def test_layers_match_oracle_over_many_steps():
    """400 steps: the drive's fields have entered the layers for hundreds of
    steps, so the memories have run long recursions."""
    w = W.pml_small(3, steps=400)
    sim, orc, out, M0 = run_pair(w, w.steps)
    t = tol(w.steps)
    for p, (i, j, k) in enumerate(w.probes):
        errs = probe_errors(sim.probe(p), out["probes"][:, p], M0[:, k, j, i], t, w.steps)
        check_probes(errs, t, w.steps, p)
    check_energy(sim.energy(), out["energy"], t, w.steps)
    compare_fields(sim, orc, M0, t)


def test_batch_members_with_and_without_layers():
    """One batch: a member lined on every face, a member without layers, a
    member lined on two axes; each equals its own oracle run (the members
    share spacings and Courant factor, hence dt)."""
    ws = [W.pml_small(4), W.random_small(4, steps=60), W.pml_small(5, layers=(4, 4, 0))]
    b = pkg.FdtdLlg.create_batch([(w.nx, w.ny, w.nz) for w in ws], [(w.dx, w.dy, w.dz) for w in ws],
                                 courant_factor=0.6, probe_capacity=60)
    for q, w in enumerate(ws):
        pkg.configure(b.batch_member(q), w)
    orcs = [oracle_from_workload(w) for w in ws]
    M0s = [o.M.copy() for o in orcs]
    b.step(60)
    t = tol(60)
    for q, (w, o) in enumerate(zip(ws, orcs)):
        m = b.batch_member(q)
        out = o.run(60)
        for p, (i, j, k) in enumerate(w.probes):
            errs = probe_errors(m.probe(p), out["probes"][:, p], M0s[q][:, k, j, i], t, 60)
            check_probes(errs, t, 60, p)
        check_energy(m.energy(), out["energy"], t, 60)
        compare_fields(m, o, M0s[q], t)
    b.destroy()


def test_save_and_load_carry_the_memories():
    w = W.pml_small(6, steps=80)
    a = pkg.from_workload(w, probe_capacity=80)
    a.step(30)
    blob = a.save_state()
    a.step(50)
    ref = {n: a.get_field(n) for n in FAMILIES["E"] + FAMILIES["H"]}
    b = pkg.from_workload(w, probe_capacity=80)
    b.load_state(blob)
    b.step(50)
    for n, v in ref.items():
        assert np.array_equal(b.get_field(n), v), n


def test_refusals():
    w = W.pml_small(7)
    sim = pkg.from_workload(w, probe_capacity=10)
    lib = _abi.load()
    bad = (C.c_int32 * 3)(13, 5, 4)   # magnetic block from x = 12: inside 13 layers
    assert lib.fdtd_llg_set_pml(sim._h, bad, 3.0, 1.0, 1.0, 0.0) == -1
    half = (C.c_int32 * 3)(16, 5, 4)  # more than half of nx = 30
    assert lib.fdtd_llg_set_pml(sim._h, half, 3.0, 1.0, 1.0, 0.0) == -1
    assert lib.fdtd_llg_run_checkpointed(sim._h, 10, 0) == -8
    buf = np.zeros(9 * w.nx * w.ny + w.nx + w.ny, np.float32)
    assert lib.fdtd_llg_planes(sim._h, 0, 1, buf.ctypes.data_as(C.POINTER(C.c_float)), buf.size, 1) == -8
    # the handle still steps after the refusals
    sim.step(5)
    sim.sync()


# ---------------------------------------------------------------- full size
FULL_STEPS = 20


def test_full_size_vanishing_layers_are_the_plain_run_bit_for_bit():
    """256x256x128 strip resonator as the benchmark launches it: layers with
    sigma = 0, kappa = 1, alpha = 0 on every face fold exact zeros into E and
    H, so every field equals the run without layers bit for bit."""
    w = W.strip_resonator(steps=FULL_STEPS)
    a = pkg.from_workload(w, probe_capacity=FULL_STEPS)
    b = pkg.from_workload(w, probe_capacity=FULL_STEPS)
    b.set_pml((10, 10, 8), 3.0, 0.0, 1.0, 0.0)
    a.step(FULL_STEPS)
    b.step(FULL_STEPS)
    for n in FAMILIES["E"] + FAMILIES["H"] + ("dMx", "dMy", "dMz"):
        assert np.array_equal(a.get_field(n), b.get_field(n)), n
    assert np.array_equal(a.energy(), b.energy())


def test_full_size_corner_window_equals_oracle():
    """256x256x128 strip resonator lined with layers (10, 10, 8): a seeded E
    patch in the low corner, reaching into the layers, evolves for 20 steps.
    An explicit step reaches one cell further per step, so the oracle run on
    the corner window alone (its cut faces as walls, the same layers at its
    low ends) must give the same fields, provided nothing active lies within
    N + 2 cells of the cut faces: the window extends that far past the patch
    and past the window's own high-end layers, which the oracle also places
    and which then see only zero fields.  Drive and films sit ~100 cells
    away, and M starts along the bias (no torque)."""
    layers = (10, 10, 8)
    w = W.strip_resonator_pml(steps=FULL_STEPS, layers=layers)
    lo_p, hi_p = np.array([2, 3, 2]), np.array([14, 22, 20])        # patch, (k, j, i) cells
    reach = FULL_STEPS + 2
    win = hi_p + reach + np.array(layers[::-1])                     # window extent (k, j, i)
    rng = np.random.default_rng(5)
    patch = [1e3 * rng.standard_normal(tuple(hi_p - lo_p)).astype(np.float32) for _ in range(3)]
    sim = pkg.from_workload(w, probe_capacity=FULL_STEPS)
    for q, n in enumerate(("Ex", "Ey", "Ez")):
        a = np.zeros((w.nz, w.ny, w.nx), np.float32)
        a[lo_p[0]:hi_p[0], lo_p[1]:hi_p[1], lo_p[2]:hi_p[2]] = patch[q]
        sim.set_field(n, a)
    sim.step(FULL_STEPS)
    # active cells of the full grid (sources, magnetised cells) stay out of reach
    ms = np.array([m["Ms"] for m in w.materials])[w.mat_id]
    mag = np.argwhere(ms > 0)
    assert np.all(np.any(mag >= win + reach, axis=1))
    for s_ in w.sources:
        assert np.any(np.array([s_["k"], s_["j"], s_["i"]]) >= win + reach)
    # the oracle on the window alone
    kz, jy, ix = (int(v) for v in win)
    ww = W.Workload("corner", ix, jy, kz, w.dx, w.dy, w.dz, w.courant, FULL_STEPS, w.materials,
                    np.ascontiguousarray(w.mat_id[:kz, :jy, :ix]), w.hbias, [], [], pml=w.pml)
    orc = oracle_from_workload(ww)
    sl = (slice(lo_p[0], hi_p[0]), slice(lo_p[1], hi_p[1]), slice(lo_p[2], hi_p[2]))
    for q, n in enumerate(("Ex", "Ey", "Ez")):
        a = np.zeros(getattr(orc, n).shape)
        a[sl] = patch[q]
        orc.set_fields(**{n: a})
    orc.run(FULL_STEPS)
    orc.half_push()
    ref = compact(orc)
    t = tol(FULL_STEPS)
    for fam in ("E", "H"):
        names = FAMILIES[fam][:3]
        scale = max(float(np.abs(ref[n]).max()) for n in names)
        for n in names:
            got = sim.get_field(n)[:kz, :jy, :ix].astype(np.float64)
            e = rel_err(got, ref[n], scale)
            record(f"field {n}", e, t, steps=FULL_STEPS)
            assert e < t, n
    # the layers took energy out of the patch's field
    assert np.abs(ref["Ex"][:, :, :layers[0]]).max() > 0


def test_cpw_device_window_equals_oracle():
    """The paper's CPW device at full size (120 x 250 x 1000, sigma = 1e11 S/m
    metal, layers on all six faces) for 20 steps from its drive beside the
    first feeding patch.  The oracle runs a window holding the whole x extent
    (its real layers), the low-y layers, the drive and 22 cells of reach in
    y and z; the window's own layers at its high-y end and both z cuts lie
    beyond that reach and see only zero fields."""
    w = W.cpw_device(steps=FULL_STEPS)
    reach = FULL_STEPS + 2
    s0 = w.sources[0]
    d = w.pml["layers"]
    j1 = s0["j"] + reach + d[1] + 1
    k0, k1 = s0["k"] - reach - d[2] - 1, s0["k"] + reach + d[2] + 2
    ms = np.array([m["Ms"] for m in w.materials])[w.mat_id]
    mag = np.argwhere(ms > 0)
    # the film starts along the bias (no torque): it stays still unless the
    # drive's field reaches it, which it does not within the window's steps
    assert np.all(mag[:, 1] > s0["j"] + reach)
    sim = pkg.from_workload(w, probe_capacity=FULL_STEPS)
    sim.step(FULL_STEPS)
    ww = W.Workload("cpw_window", w.nx, j1, k1 - k0, w.dx, w.dy, w.dz, w.courant, FULL_STEPS, w.materials,
                    np.ascontiguousarray(w.mat_id[k0:k1, :j1, :]), w.hbias,
                    [dict(s0, k=s0["k"] - k0)], [], pml=w.pml)
    orc = oracle_from_workload(ww)
    orc.run(FULL_STEPS)
    orc.half_push()
    ref = compact(orc)
    t = tol(FULL_STEPS)
    for fam in ("E", "H"):
        names = FAMILIES[fam][:3]
        scale = max(float(np.abs(ref[n]).max()) for n in names)
        assert scale > 0
        for n in names:
            got = sim.get_field(n)[k0:k1, :j1, :].astype(np.float64)
            e = rel_err(got, ref[n], scale)
            record(f"field {n}", e, t, steps=FULL_STEPS)
            assert e < t, n
