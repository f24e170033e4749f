"""Write the stored FP64 reference values of the full-size spectral parity
tests.  Calls only the FP64 oracle (``oracle/``) and the seeded workload
generators; nothing here comes from the CUDA path.

    python tests/golden/make_reference_runs.py strip   [--steps N]
    python tests/golden/make_reference_runs.py sweep   [--steps N] [--stride S]

``strip``: the 256 x 256 x 128 strip resonator (8.39 M cells, the FP32
throughput configuration) for 20000 steps; stores every 100th probe row, the
Hann-windowed |DFT| of E_x, E_z and H_y at both probes over 0.05-1.5 THz and
the peak frequency of each (section "Results": the E_x spectra of probe
time series).

``sweep``: the 64-cube bias sweep (uneven cubes 48^3-96^3, bias 0.05-0.15 T)
for 10000 steps at the batch's common time step (0.5 x the Courant limit of
the finest cube), every 4th cube (16 cubes over the whole bias range); per
cube the |DFT| of the probe's E_x over 1.5-4.5 GHz, the block means of E_x
over 20 steps, and the ESPRIT modes of those block means after the first
fifth of the run (the polariton pair, section "Results"; the block means keep
the frequencies and put several periods in one pencil), then the fit of Eq.
omega_pm over the cubes whose two modes are both clearly present.

Each run uses every host core (the oracle's results do not depend on the
thread count).
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from oracle import spectra as S  # noqa: E402
from paper_2510_22221_b300 import workloads as W  # noqa: E402
from tests.helpers import oracle_from_workload  # noqa: E402

# spectral settings shared with the GPU tests that read these files
STRIP = dict(steps=20000, every=100, fmin=0.05e12, fmax=1.5e12, nfreq=291, comps=(0, 2, 4))
THREADS = [0]
SWEEP = dict(steps=10000, skip_frac=5, decimate=20, order=24, pencil=100, fmin=1.5e9, fmax=4.5e9, nfreq=61,
             amp_ratio=0.2)


def peak(freqs, spec):
    """Frequency of the largest sample, refined by the parabola through it and
    its two neighbours."""
    k = int(np.argmax(spec))
    if 0 < k < len(spec) - 1:
        a, b, c = spec[k - 1], spec[k], spec[k + 1]
        d = 0.5 * (a - c) / (a - 2 * b + c)
        return float(freqs[k] + d * (freqs[1] - freqs[0]))
    return float(freqs[k])


def strip(steps, out):
    w = W.strip_resonator(steps=steps)
    o = oracle_from_workload(w)
    dt = o.dt
    t0 = time.time()
    res = o.run(steps)
    wall = time.time() - t0
    pr = res["probes"]                      # (steps, nprobe, 9)
    freqs = np.linspace(STRIP["fmin"], STRIP["fmax"], STRIP["nfreq"])
    spectra, peaks = {}, {}
    for p in range(pr.shape[1]):
        for c in STRIP["comps"]:
            s = S.dft_magnitude(pr[:, p, c], dt, freqs, kind="hann")
            spectra[f"{p}:{c}"] = s.tolist()
            peaks[f"{p}:{c}"] = peak(freqs, s)
    every = STRIP["every"]
    doc = {
        "what": "FP64 oracle run of the 256x256x128 strip resonator (seeded workload strip_resonator)",
        "cite": "section 'Numerical Model' (the step), section 'Results' (E_x spectra of probe series)",
        "made_by": "python tests/golden/make_reference_runs.py strip",
        "workload": w.name, "steps": steps, "dt": dt, "probes": [list(p) for p in w.probes],
        "threads": THREADS[0], "wall_s": round(wall, 1),
        "settings": STRIP, "freqs": [freqs[0], freqs[-1], len(freqs)],
        "spectra": spectra, "peaks": peaks,
        "rows_every": every, "rows": pr[every - 1::every].tolist(),
        "energy_every": res["energy"][every - 1::every].tolist(),
        "noconv": bool(res["noconv"]),
    }
    with open(out, "w") as f:
        json.dump(doc, f)
    print(f"wrote {out}: {steps} steps in {wall:.0f} s")


def sweep(steps, stride, out):
    ws = W.bias_sweep(steps=steps)[::stride]
    dmin = min(min(w.dx, w.dy, w.dz) for w in W.bias_sweep(steps=steps))
    dt = oracle.courant_dt(dmin, dmin, dmin, ws[0].courant)
    freqs = np.linspace(SWEEP["fmin"], SWEEP["fmax"], SWEEP["nfreq"])
    skip = steps // SWEEP["skip_frac"]
    per = []
    t0 = time.time()
    for q, w in enumerate(ws):
        o = oracle_from_workload(w, dt=dt)
        tr = o.run(steps)["probes"][:, 0, 0]
        spec = S.dft_magnitude(tr, dt, freqs, kind="hann")
        D = SWEEP["decimate"]
        xd = S.block_means(tr[skip:], D)
        f, a, amp, Q = S.strongest_in_band(S.matrix_pencil(xd, dt * D, SWEEP["order"], SWEEP["pencil"]),
                                           SWEEP["fmin"], SWEEP["fmax"], 2)
        per.append({"name": w.name, "index": q * stride, "n": w.nx, "bias_T": float(w.hbias[2] * W.MU0),
                    "spectrum": spec.tolist(), "modes_hz": f.tolist(), "decay": a.tolist(), "amp": amp.tolist(),
                    "q": Q.tolist(), "ex_block_means": S.block_means(tr, D).tolist()})
        print(f"  {w.name}: modes {np.round(f / 1e9, 4)} amp {amp}", flush=True)
    wall = time.time() - t0
    pairs = [q for q, r in enumerate(per)
             if len(r["modes_hz"]) == 2 and min(r["amp"]) >= SWEEP["amp_ratio"] * max(r["amp"])]
    fit = None
    if len(pairs) >= 2:
        fp, g = S.coupling_fit([per[q]["modes_hz"][1] for q in pairs], [per[q]["modes_hz"][0] for q in pairs])
        fit = {"f_p_hz": fp, "two_g_hz": 2 * g}
    doc = {
        "what": "FP64 oracle runs of the 64-cube bias sweep (seeded workload bias_sweep), one cube at a time",
        "cite": "section 'Results' (E_x spectra vs bias, ESPRIT polariton pairs), Eq. omega_pm (the fit)",
        "made_by": "python tests/golden/make_reference_runs.py sweep",
        "steps": steps, "dt": dt, "instances": len(ws), "stride": stride, "threads": THREADS[0], "wall_s": round(wall, 1),
        "settings": SWEEP, "freqs": [freqs[0], freqs[-1], len(freqs)], "skip": skip,
        "per_instance": per, "pairs": pairs, "fit": fit,
    }
    with open(out, "w") as f:
        json.dump(doc, f)
    print(f"wrote {out}: {len(ws)} cubes x {steps} steps in {wall:.0f} s; pairs {pairs}; fit {fit}")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("which", choices=["strip", "sweep"])
    ap.add_argument("--steps", type=int, default=0)
    ap.add_argument("--stride", type=int, default=4, help="every stride-th cube of the 64 (4: 16 cubes over the whole bias range)")
    ap.add_argument("--out", default="")
    ap.add_argument("--threads", type=int, default=0, help="oracle threads (0: every host core)")
    a = ap.parse_args()
    THREADS[0] = oracle.set_threads(a.threads)
    if a.which == "strip":
        strip(a.steps or STRIP["steps"], a.out or os.path.join(HERE, "strip_resonator_256x256x128_fp64.json"))
    else:
        sweep(a.steps or SWEEP["steps"], a.stride, a.out or os.path.join(HERE, "bias_sweep_64_fp64.json"))


if __name__ == "__main__":
    main()
