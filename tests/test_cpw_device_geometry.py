"""The CPW device workload against the sizes printed in the paper's section
"Modeling Setup" (CPU only): grid and cell sizes, time step at CFL 0.9,
substrate and metal thickness, ground, gap and centre-line widths, the
film's thickness, width and length, the feeding patches and gap capacitors,
and the materials."""
import numpy as np
import pytest

import oracle
from paper_2510_22221_b300 import workloads as W

UM = 1e-6


@pytest.fixture(scope="module")
def w():
    return W.cpw_device()


def _runs(a):
    """(value, start, length) runs of a 1-D integer array."""
    out, s = [], 0
    for i in range(1, len(a) + 1):
        if i == len(a) or a[i] != a[s]:
            out.append((int(a[s]), s, i - s))
            s = i
    return out


def test_grid_and_time_step(w):
    assert (w.nx, w.ny, w.nz) == (120, 250, 1000)
    assert np.isclose(w.nx * w.dx, 0.6e-3) and np.isclose(w.ny * w.dy, 4.75e-3) and np.isclose(w.nz * w.dz, 1e-3)
    dt = oracle.courant_dt(w.dx, w.dy, w.dz, w.courant)
    assert abs(dt - 2.94e-15) < 0.005e-15             # printed 2.94e-15 s at CFL 0.9


def test_layers_of_the_stack(w):
    m = w.mat_id
    eps = np.array([q["eps_r"] for q in w.materials])
    sig = np.array([q["sigma"] for q in w.materials])
    col = m[:, 5, 5]                                   # under the ground plane, away from the line
    runs = _runs(col)
    assert eps[runs[0][0]] == 11.4 and runs[0][2] * w.dz == 500 * UM      # silicon, 500 um
    assert sig[runs[1][0]] == 1e11 and runs[1][2] * w.dz == 2 * UM        # metal, 2 um, 1e11 S/m
    assert eps[runs[2][0]] == 1.0 and sig[runs[2][0]] == 0.0              # vacuum above


def test_coplanar_cross_section_and_film(w):
    sig = np.array([q["sigma"] for q in w.materials])
    ms = np.array([q["Ms"] for q in w.materials])
    metal = sig[w.mat_id[500, w.ny // 2 + 20]] > 0     # a cross-section of the metal layer (x)
    runs = _runs(metal.astype(int))
    widths = [(v, n) for v, _, n in runs]             # cells of 5 um
    assert widths == [(1, 50), (0, 5), (1, 10), (0, 5), (1, 50)]    # 250, 25, 50, 25, 250 um
    assert np.isclose(w.dx, 5 * UM)
    film = ms[w.mat_id] > 0
    k, j, i = np.nonzero(film)
    assert k.max() - k.min() + 1 == 5 and k.min() == 502                       # 5 um (1 um cells) on the metal
    assert i.max() - i.min() + 1 == 6                                          # 30 um (5 um cells) wide, centred
    assert i.min() - 55 == 65 - 1 - i.max()
    length = (j.max() - j.min() + 1) * w.dy
    assert abs(length - 2.82e-3) < w.dy                                        # 2.82 mm
    assert film.sum() == 6 * 148 * 5                                           # in one piece
    split = W.cpw_device(split=True)
    assert (ms[split.mat_id] > 0).sum() == 6 * 147 * 5                         # cut by one cell layer
    Ms = ms[ms > 0][0]
    assert np.isclose(4 * np.pi * Ms * 1e-3, 1.2e4)                            # 4 pi Ms = 1.2e4 G
    assert [q["alpha"] for q in w.materials if q["Ms"] > 0] == [3e-3]


def test_line_gaps_and_feeding_patches(w):
    sig = np.array([q["sigma"] for q in w.materials])
    along = (sig[w.mat_id[500, :, 60]] > 0).astype(int)   # down the centre of the line (y)
    runs = _runs(along)
    lens = [(v, n * w.dy) for v, _, n in runs]
    # feeding patch, gap capacitor, centre line, gap capacitor, feeding patch
    assert [v for v, _ in lens] == [1, 0, 1, 0, 1]
    assert abs(lens[0][1] - 300 * UM) < w.dy and abs(lens[1][1] - 200 * UM) < w.dy
    assert abs(lens[2][1] - 3.75e-3) < w.dy
    assert lens[0] == lens[4] and lens[1] == lens[3]
