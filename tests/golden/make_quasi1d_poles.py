"""Write the stored analytic polariton poles of the quasi-1-D resonator runs
(workloads.quasi1d_film: the supplement's film, Table S1, across a PEC
parallel-plate resonator at 1700, 1800 and 1900 Oe).  Calls only the
oracle's analytic model (``oracle/supplement.py``) and the seeded workload
generators; nothing here comes from the CUDA path.

    python tests/golden/make_quasi1d_poles.py

For each bias: the two complex poles of chi (Eq. S5b) with theta_zy(w) from
the cavity solve of Eqs. S7-S9 for the run's geometry (PEC walls, the
grid's transverse wavenumber (2/dy) sin(pi/(2 ny)), the film one cell
thick at i = nx/8 with the film-normal demagnetising factor 1/2 of a
one-cell film in the Yee scheme), as frequency Re w / 2 pi and decay rate
-Im w (amplitude ~ exp(-a t)).
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import supplement as S  # noqa: E402
from paper_2510_22221_b300 import workloads as W  # noqa: E402


def poles(w):
    i_f = w.probes[0][0]
    d1, L = i_f * w.dx, w.nx * w.dx
    kt = 2.0 / w.dy * np.sin(np.pi / (2 * w.ny))
    H = float(w.hbias[2])
    gam, ms = S.TABLE_S1["gamma"], S.TABLE_S1["Ms"]
    wm = gam * np.sqrt(H * (H + 0.5 * ms))
    wc = S.C0 * np.sqrt((np.pi / L) ** 2 + kt * kt)
    return S.cavity_poles(H, d1, d1 + w.dx, L, [wm, wc], kt=kt, walls="pec", demag=0.5)


def main():
    out = {"source": "oracle/supplement.py cavity_poles (Eqs. S5b, S7-S9), demag 1/2, PEC walls",
           "workload": "quasi1d_film", "runs": []}
    for w in W.quasi1d_film():
        z = poles(w)
        out["runs"].append({"name": w.name, "h_oe": round(float(w.hbias[2]) / S.OE, 6),
                            "freq_hz": [float(v) for v in z.real / (2 * np.pi)],
                            "decay_per_s": [float(v) for v in -z.imag]})
    path = os.path.join(HERE, "quasi1d_poles.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path)


if __name__ == "__main__":
    main()
