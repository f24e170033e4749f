"""Spectra and the anti-crossing fit through the C ABI against the FP64
oracle (arxiv 2510.22221, section "Results": E_x spectra over a bias sweep,
ESPRIT polariton frequencies, Eq. omega_pm).

1. The GPU transform of the device probe ring equals the oracle's explicit
   DFT of the same samples (both FP64: rtol 1e-10 of the peak).
2. End to end: the bias sweep run as one batch on the GPU (FP32 fields)
   and instance by instance in the FP64 oracle; ESPRIT on each E_x trace
   after the pulse (library on the GPU run, oracle routine on the oracle
   run) and the (f_p, g) fit over the sweep.  The polariton frequencies agree
   to 1e-5 relative and the splitting 2g to 1e-4 relative: FP32 field errors
   (~1e-6 of the field, TOL(N) of the parity tests) move a frequency extracted
   from a few hundred periods of a clean trace by far less."""
import numpy as np
import pytest

import paper_2510_22221_b300 as pkg
from oracle import spectra as S
from paper_2510_22221_b300 import workloads as W
from tests.helpers import oracle_from_workload

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cap,steps,window", [(1024, 600, "hann"), (256, 600, "rect")])
def test_probe_spectrum_equals_oracle_dft_of_the_ring(cap, steps, window):
    w = W.cavity_block(steps=steps)
    sim = pkg.from_workload(w, probe_capacity=cap)
    sim.step(steps)
    x = sim.probe(0)                       # the rows the ring holds, oldest first
    assert x.shape[0] == min(cap, steps)
    for comp in (0, 4):
        got = sim.probe_spectrum(0, comp, 1e9, 40e9, 333, window=window)
        ref = S.dft_magnitude(x[:, comp], sim.dt, np.linspace(1e9, 40e9, 333), kind=window)
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-10 * ref.max())
    sim.destroy()


def test_anticrossing_sweep_spectra_polaritons_and_splitting_match_oracle():
    steps, skip, order, pencil, band = 16000, 1000, 40, 400, (3.0e9, 4.2e9)
    ws = W.anticrossing_sweep(n_inst=4, steps=steps)
    dims = [(x.nx, x.ny, x.nz) for x in ws]
    sp = [(x.dx, x.dy, x.dz) for x in ws]
    batch = pkg.FdtdLlg.create_batch(dims, sp, courant_factor=ws[0].courant, probe_capacity=steps)
    for q, x in enumerate(ws):
        pkg.configure(batch.batch_member(q), x)
    batch.step(steps)
    dt = batch.dt
    freqs = np.linspace(band[0], band[1], 241)
    gpu, orc = [], []
    for q, w in enumerate(ws):
        m = batch.batch_member(q)
        tr = m.probe(0)[:, 2]
        o = oracle_from_workload(w, dt=dt)
        otr = o.run(steps)["probes"][:, 0, 2]
        # spectra of the whole trace: GPU transform of the FP32 run vs the oracle transform of the FP64 run
        spec = m.probe_spectrum(0, 2, band[0], band[1], freqs.size)
        ospec = S.dft_magnitude(otr, dt, freqs)
        assert np.linalg.norm(spec - ospec) / np.linalg.norm(ospec) < 1e-4
        assert abs(freqs[np.argmax(spec)] - freqs[np.argmax(ospec)]) <= 1e-4 * freqs[np.argmax(ospec)]
        # ESPRIT after the pulse: library on the GPU trace, oracle routine on the oracle trace
        f, a, amp, Q = pkg.fit_modes(tr[skip:], dt, order, pencil=pencil, fmin=band[0], fmax=band[1], max_modes=2)
        of, oa, oamp, oQ = S.strongest_in_band(S.matrix_pencil(otr[skip:], dt, order, pencil), band[0], band[1], 2)
        assert len(f) == 2 and len(of) == 2
        np.testing.assert_allclose(f, of, rtol=1e-5)
        np.testing.assert_allclose(Q, oQ, rtol=5e-2)
        gpu.append(f)
        orc.append(of)
    batch.destroy()
    fp_g, g_g = pkg.fit_coupling([p[1] for p in gpu], [p[0] for p in gpu])
    fp_o, g_o = S.coupling_fit([p[1] for p in orc], [p[0] for p in orc])
    assert fp_g == pytest.approx(fp_o, rel=1e-5)
    assert 2 * g_g == pytest.approx(2 * g_o, rel=1e-4)
    assert 0.02 < g_o / fp_o < 0.1   # one anti-crossing of the cavity mode in the band
