"""Parity at full size: the 256x256x128 strip resonator and the 512x512x256
eight-strip array, run as the benchmark runs them (whole grid, default
tiling, a stream of their own), against the FP64 oracle on outputs it can
compute one by one (arxiv 2510.22221, section "Numerical Model"); the
64-cube bias sweep and the 128x128x64 design grid, which the oracle runs
whole, cell by cell (at the end of this file).

An explicit Yee step reaches one cell further per step: E^{n+1} at a cell
uses H^{n+1/2} of that cell and its low neighbours, which use E^n of the cell
and its neighbours, and the stored H is half a step ahead.  A magnetic
region couples its own cells within a step (the LLG solve), so it counts as
one block.  After N steps every field in a window of the grid therefore
equals that of the oracle run on the window alone, with the window's cut
faces as walls, provided no cell that is active at the start (a magnetised
cell or a source edge) lies within N + 2 cells of a cut face inside the
window or of the window from outside it.  Each window below is checked for
that before the comparison, and the comparison covers every cell of it (E,
H and the change of M) and the probes inside it, with the tolerances of
test_gpu_parity.

The workloads' drive sits some 90 cells from the first film, beyond what a
few dozen steps reach, and M starts along the bias (no torque), so both
sides also start from the same seeded E patch around the first film: the
film window then holds real field and magnet dynamics from the first step."""
import numpy as np
import pytest

import paper_2510_22221_b300 as pkg
from paper_2510_22221_b300 import workloads as W
from tests.helpers import compact, oracle_from_workload, record
from tests.test_gpu_parity import check_probes, m_floor, probe_errors, rel_err, tol, tol_m

pytestmark = pytest.mark.gpu

STEPS = 20


def _film0(w):
    """(k, j, i) of the cells of the first magnetic region."""
    from scipy import ndimage

    ms = np.array([m["Ms"] for m in w.materials])
    lab, _ = ndimage.label(ms[w.mat_id] > 0)
    return np.argwhere(lab == 1)


def _patch(w):
    """Seeded initial E (three (nz, ny, nx) arrays, zero outside) on the first
    film's box grown by one cell, 1 kV/m scale."""
    cells = _film0(w)
    lo = np.maximum(cells.min(0) - 1, 0)
    hi = np.minimum(cells.max(0) + 2, [w.nz, w.ny, w.nx])
    rng = np.random.default_rng(11)
    out = []
    for _ in range(3):
        a = np.zeros((w.nz, w.ny, w.nx), dtype=np.float32)
        a[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]] = 1e3 * rng.standard_normal(tuple(hi - lo))
        out.append(a)
    return out, lo, hi


def _active_cells(w, plo, phi):
    """(k, j, i) of the magnetised cells, source edges and patch cells."""
    ms = np.array([m["Ms"] for m in w.materials])
    cells = np.argwhere(ms[w.mat_id] > 0)
    src = np.array([(s["k"], s["j"], s["i"]) for s in w.sources]).reshape(-1, 3)
    patch = np.stack(np.meshgrid(*[np.arange(a, b) for a, b in zip(plo, phi)], indexing="ij"), -1).reshape(-1, 3)
    return np.concatenate([cells, src, patch])


def _window(w, core_lo, core_hi, m):
    """Box (k, j, i) [lo, hi) around a core box, grown by m, clipped to the grid."""
    shape = np.array([w.nz, w.ny, w.nx])
    return np.maximum(np.array(core_lo) - m, 0), np.minimum(np.array(core_hi) + m, shape)


def _check_window(w, lo, hi, margin, plo, phi):
    """Every active cell inside is >= margin from each cut face (a face not on
    the grid boundary); every active cell outside is >= margin from the box."""
    shape = np.array([w.nz, w.ny, w.nx])
    act = _active_cells(w, plo, phi)
    inside = np.all((act >= lo) & (act < hi), axis=1)
    for d in range(3):
        if lo[d] > 0:
            assert np.all(act[inside, d] - lo[d] >= margin)
        if hi[d] < shape[d]:
            assert np.all(hi[d] - 1 - act[inside, d] >= margin)
    out = act[~inside]
    gap = np.max(np.maximum(np.maximum(lo - out, out - (hi - 1)), 0), axis=1)
    assert np.all(gap >= margin)


def _crop(w, lo, hi):
    """The workload restricted to box [lo, hi) (k, j, i); sources and probes
    outside are dropped.  Returns it and the kept probe indices."""
    (z0, y0, x0), (z1, y1, x1) = lo, hi
    inb = lambda i, j, k: x0 <= i < x1 and y0 <= j < y1 and z0 <= k < z1
    src = [dict(s, i=s["i"] - x0, j=s["j"] - y0, k=s["k"] - z0) for s in w.sources if inb(s["i"], s["j"], s["k"])]
    keep = [p for p, (i, j, k) in enumerate(w.probes) if inb(i, j, k)]
    probes = [(w.probes[p][0] - x0, w.probes[p][1] - y0, w.probes[p][2] - z0) for p in keep]
    mid = np.ascontiguousarray(w.mat_id[z0:z1, y0:y1, x0:x1])
    c = W.Workload(w.name + "_window", x1 - x0, y1 - y0, z1 - z0, w.dx, w.dy, w.dz, w.courant, w.steps, w.materials,
                   mid, w.hbias, src, probes)
    return c, keep


def _windows(w, margin, plo, phi):
    """One window around the first source, one around the first magnetic
    region with its patch and the probes, each grown by margin."""
    s = w.sources[0]
    ks = (s["k"], s["j"], s["i"])
    probes = np.array([(k, j, i) for (i, j, k) in w.probes])
    core = np.concatenate([_film0(w), probes, [plo, np.asarray(phi) - 1]])
    return [_window(w, ks, np.array(ks) + 1, margin), _window(w, core.min(0), core.max(0) + 1, margin)]


@pytest.fixture(scope="module", params=["strip_resonator", "multi_strip"])
def full_run(request):
    import torch

    w = W.strip_resonator(steps=STEPS) if request.param == "strip_resonator" else W.multi_strip(steps=STEPS)
    patch, plo, phi = _patch(w)
    with torch.cuda.stream(torch.cuda.Stream()):
        sim = pkg.from_workload(w, probe_capacity=STEPS)
        for n, a in zip(("Ex", "Ey", "Ez"), patch):
            sim.set_field(n, a)
        sim.step(STEPS)
        sim.sync()
        got = {n: sim.get_field(n) for n in ("Ex", "Ey", "Ez", "Hx", "Hy", "Hz", "dMx", "dMy", "dMz")}
        probes = [sim.probe(p) for p in range(len(w.probes))]
        sim.destroy()
    return w, got, probes, patch, plo, phi


@pytest.mark.parametrize("which", [0, 1])
def test_full_size_window_equals_oracle(full_run, which):
    w, got, probes, patch, plo, phi = full_run
    margin = STEPS + 3
    lo, hi = _windows(w, margin, plo, phi)[which]
    _check_window(w, lo, hi, STEPS + 2, plo, phi)
    c, keep = _crop(w, lo, hi)
    orc = oracle_from_workload(c)
    sl = tuple(slice(a, b) for a, b in zip(lo, hi))
    for name, a in zip(("Ex", "Ey", "Ez"), patch):
        getattr(orc, name)[: c.nz, : c.ny, : c.nx] = a[sl]
    M0 = orc.M.copy()
    out = orc.run(STEPS)
    t = tol(STEPS)
    for q, p in enumerate(keep):
        i, j, k = c.probes[q]
        errs = probe_errors(probes[p], out["probes"][:, q], M0[:, k, j, i], t, STEPS)
        check_probes(errs, t, STEPS, p)
    orc.half_push()
    ref = compact(orc)
    for fam in (("Ex", "Ey", "Ez"), ("Hx", "Hy", "Hz")):
        scale = max(float(np.abs(ref[n]).max()) for n in fam)
        assert scale > 0
        for n in fam:
            _chk(n, rel_err(got[n][sl], ref[n], scale), t, STEPS)
    dm = {n: ref[n] - M0[d] for d, n in enumerate(("Mx", "My", "Mz"))}
    tm = tol_m(STEPS)
    scale = max(max(float(np.abs(v).max()) for v in dm.values()), m_floor(float(np.abs(M0).max()), orc.step) / tm)
    for n, v in dm.items():
        _chk("d" + n, rel_err(got["d" + n][sl], v, scale), tm, STEPS)


# ------------------------------------------------ configs 2 and 3 in full

def _seed_patch(w, rng_seed):
    """Seeded E (three (nz, ny, nx) arrays) on the first magnetic region's box
    grown by two cells, 1 kV/m scale: real field and magnet dynamics from the
    first step (the drives start far below that within a few dozen steps)."""
    cells = _film0(w)
    lo = np.maximum(cells.min(0) - 2, 0)
    hi = np.minimum(cells.max(0) + 3, [w.nz, w.ny, w.nx])
    rng = np.random.default_rng(rng_seed)
    out = []
    for _ in range(3):
        a = np.zeros((w.nz, w.ny, w.nx), dtype=np.float32)
        a[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]] = 1e3 * rng.standard_normal(tuple(hi - lo))
        out.append(a)
    return out


def _compare_whole(got, probes, w, patch, dt, steps, llg_fixed_iter=0):
    """Every cell of E, H and the change of M, and the probes, against the
    FP64 oracle run of the whole workload from the same patch."""
    orc = oracle_from_workload(w, dt=dt, llg_fixed_iter=llg_fixed_iter)
    for name, a in zip(("Ex", "Ey", "Ez"), patch):
        getattr(orc, name)[: w.nz, : w.ny, : w.nx] = a
    M0 = orc.M.copy()
    out = orc.run(steps)
    t = tol(steps)
    for p, (i, j, k) in enumerate(w.probes):
        errs = probe_errors(probes[p], out["probes"][:, p], M0[:, k, j, i], t, steps)
        check_probes(errs, t, steps, p)
    orc.half_push()
    ref = compact(orc)
    for fam in (("Ex", "Ey", "Ez"), ("Hx", "Hy", "Hz")):
        scale = max(float(np.abs(ref[n]).max()) for n in fam)
        assert scale > 0
        for n in fam:
            _chk(n, rel_err(got[n], ref[n], scale), t, steps)
    dm = {n: ref[n] - M0[d] for d, n in enumerate(("Mx", "My", "Mz"))}
    tm = tol_m(steps)
    scale = max(max(float(np.abs(v).max()) for v in dm.values()), m_floor(float(np.abs(M0).max()), orc.step) / tm)
    assert max(float(np.abs(v).max()) for v in dm.values()) > 1e3 * m_floor(float(np.abs(M0).max()), orc.step)
    for n, v in dm.items():
        _chk("d" + n, rel_err(got["d" + n], v, scale), tm, steps)


_NAMES = ("Ex", "Ey", "Ez", "Hx", "Hy", "Hz", "dMx", "dMy", "dMz")


def _chk(name, err, t, steps):
    record(f"field {name}", err, t, steps=steps)
    assert err < t, name


def test_bias_sweep_batch_members_equal_oracle():
    """The 64-cube bias sweep as the benchmark builds it (one batch, its
    common time step): the smallest and the largest cube against the oracle
    run of that cube alone, every cell."""
    import torch

    steps = 30
    ws = W.bias_sweep(steps=steps)
    order = np.argsort([w.cells for w in ws])
    picks = [int(order[0]), int(order[-1])]
    with torch.cuda.stream(torch.cuda.Stream()):
        batch = pkg.FdtdLlg.create_batch([(w.nx, w.ny, w.nz) for w in ws], [(w.dx, w.dy, w.dz) for w in ws],
                                         courant_factor=0.5, probe_capacity=steps)
        for q, w in enumerate(ws):
            pkg.configure(batch.batch_member(q), w)
        patches = {q: _seed_patch(ws[q], 100 + q) for q in picks}
        for q in picks:
            for n, a in zip(("Ex", "Ey", "Ez"), patches[q]):
                batch.batch_member(q).set_field(n, a)
        batch.step(steps)
        batch.sync()
        dt = batch.dt
        res = {}
        for q in picks:
            m = batch.batch_member(q)
            res[q] = ({n: m.get_field(n) for n in _NAMES}, [m.probe(p) for p in range(len(ws[q].probes))])
        batch.destroy()
    for q in picks:
        _compare_whole(res[q][0], res[q][1], ws[q], patches[q], dt, steps)


def test_adjoint_design_grid_forward_equals_oracle():
    """The 128 x 128 x 64 design case's forward run (three fixed LLG iterates,
    as the adjoint uses) against the oracle, every cell."""
    import torch

    steps = 30
    w = W.adjoint_design(steps=steps)
    patch = _seed_patch(w, 7)
    with torch.cuda.stream(torch.cuda.Stream()):
        sim = pkg.from_workload(w, probe_capacity=steps, llg_fixed_iter=3)
        for n, a in zip(("Ex", "Ey", "Ez"), patch):
            sim.set_field(n, a)
        sim.step(steps)
        sim.sync()
        got = {n: sim.get_field(n) for n in _NAMES}
        probes = [sim.probe(p) for p in range(len(w.probes))]
        dt = sim.dt
        sim.destroy()
    _compare_whole(got, probes, w, patch, dt, steps, llg_fixed_iter=3)
