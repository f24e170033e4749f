"""FP32 CUDA path against stored FP64 oracle runs at the sizes the
benchmark configurations name (arxiv 2510.22221, section "Results": E_x
spectra of probe series over a bias sweep, ESPRIT polariton pairs, Eq.
omega_pm).  The stored values were written by
tests/golden/make_reference_runs.py, which calls only the oracle and the
seeded workload generators.

  * The 256 x 256 x 128 strip resonator, 20000 steps: the Hann-windowed |DFT|
    of E_x, E_z and H_y at both probes agrees to 1e-4 in relative L2 over
    0.05-1.5 THz and its peak frequency to 1e-4; every 100th probe row and
    energy agree within the parity tests' bounds TOL(N), TOL_W(N).
  * The 64-cube bias sweep (10000 steps, one batch at the common time
    step), every 4th cube (16 cubes over 0.05-0.15 T): each probe spectrum
    to 1e-4 in relative L2, the ESPRIT modes of each E_x trace (block means
    over 20 steps after the first fifth of the run) to 1e-4, and the splitting
    2g of Eq. omega_pm fitted over the cubes with a clear pair to 1e-4 of the
    FP64 fit."""
import json
import os

import numpy as np
import pytest

import paper_2510_22221_b300 as pkg
from paper_2510_22221_b300 import workloads as W
from tests.helpers import record
from tests.test_gpu_parity import tol, tol_w

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _peak(freqs, spec):
    k = int(np.argmax(spec))
    if 0 < k < len(spec) - 1:
        a, b, c = spec[k - 1], spec[k], spec[k + 1]
        return float(freqs[k] + 0.5 * (a - c) / (a - 2 * b + c) * (freqs[1] - freqs[0]))
    return float(freqs[k])


def test_strip_resonator_20000_steps_matches_fp64_spectra():
    ref = _load("strip_resonator_256x256x128_fp64.json")
    st = ref["settings"]
    N = ref["steps"]
    w = W.strip_resonator(steps=N)
    sim = pkg.from_workload(w, probe_capacity=N)
    assert sim.dt == pytest.approx(ref["dt"], rel=1e-14)
    sim.step(N)
    freqs = np.linspace(st["fmin"], st["fmax"], st["nfreq"])
    for key, ospec in ref["spectra"].items():
        p, c = (int(v) for v in key.split(":"))
        spec = sim.probe_spectrum(p, c, st["fmin"], st["fmax"], st["nfreq"], window="hann")
        ospec = np.asarray(ospec)
        e = float(np.linalg.norm(spec - ospec) / np.linalg.norm(ospec))
        record(f"spectrum {key}", e, 1e-4, steps=N)
        assert e < 1e-4, (key, e)
        fe = abs(_peak(freqs, spec) - ref["peaks"][key]) / ref["peaks"][key]
        record(f"peak {key}", fe, 1e-4, steps=N)
        assert fe < 1e-4, (key, fe)
    # sampled rows: E and H families at both probes, against the parity bound
    every = ref["rows_every"]
    orows = np.asarray(ref["rows"])                     # (N / every, nprobe, 9)
    t = tol(N)
    for p in range(orows.shape[1]):
        g = sim.probe(p)[every - 1::every]
        for fam, sl in (("E", slice(0, 3)), ("H", slice(3, 6))):
            scale = float(np.abs(orows[:, p, sl]).max())
            e = float(np.abs(g[:, sl] - orows[:, p, sl]).max()) / scale
            record(f"rows {p} {fam}", e, t, steps=N)
            assert e < t, (p, fam, e)
    oe = np.asarray(ref["energy_every"])
    ge = sim.energy()[every - 1::every]
    e = float(np.abs(ge - oe).max() / np.abs(oe).max())
    record("energy", e, tol_w(N), steps=N)
    assert e < tol_w(N)
    sim.destroy()


def test_bias_sweep_spectra_modes_and_splitting_match_fp64():
    ref = _load("bias_sweep_64_fp64.json")
    st = ref["settings"]
    N, skip = ref["steps"], ref["skip"]
    ws = W.bias_sweep(steps=N)
    batch = pkg.FdtdLlg.create_batch([(x.nx, x.ny, x.nz) for x in ws], [(x.dx, x.dy, x.dz) for x in ws],
                                     courant_factor=ws[0].courant, probe_capacity=N)
    for q, x in enumerate(ws):
        pkg.configure(batch.batch_member(q), x)
    dt = batch.dt
    assert dt == pytest.approx(ref["dt"], rel=1e-14)
    batch.step(N)
    gpu = {}
    for r in ref["per_instance"]:
        m = batch.batch_member(r["index"])
        spec = m.probe_spectrum(0, 0, st["fmin"], st["fmax"], st["nfreq"], window="hann")
        ospec = np.asarray(r["spectrum"])
        e = float(np.linalg.norm(spec - ospec) / np.linalg.norm(ospec))
        record(f"spectrum {r['name']}", e, 1e-4, steps=N)
        assert e < 1e-4, (r["name"], e)
        tr = m.probe(0)[skip:, 0]
        f, a, amp, Q = pkg.fit_modes(tr, dt, st["order"], pencil=st["pencil"], fmin=st["fmin"], fmax=st["fmax"],
                                     max_modes=2, decimate=st["decimate"])
        assert len(f) == len(r["modes_hz"]), (r["name"], f, r["modes_hz"])
        fe = float(np.max(np.abs(f - np.asarray(r["modes_hz"])) / np.asarray(r["modes_hz"])))
        record(f"modes {r['name']}", fe, 1e-4, steps=N)
        assert fe < 1e-4, (r["name"], f, r["modes_hz"])
        gpu[r["index"]] = f
    batch.destroy()
    pairs = [ref["per_instance"][q]["index"] for q in ref["pairs"]]
    fp, g = pkg.fit_coupling([gpu[i][1] for i in pairs], [gpu[i][0] for i in pairs])
    e2g = abs(2 * g - ref["fit"]["two_g_hz"]) / ref["fit"]["two_g_hz"]
    record("two_g", e2g, 1e-4, steps=N)
    assert e2g < 1e-4, (2 * g, ref["fit"]["two_g_hz"])
    assert fp == pytest.approx(ref["fit"]["f_p_hz"], rel=1e-5)
