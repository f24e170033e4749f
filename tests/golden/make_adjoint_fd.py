"""Write the stored FP64 central differences of the adjoint design objective
on 16 random design cells.  Calls only the FP64 oracle (``oracle/``) and the
seeded workload generators; nothing here comes from the CUDA path.

    python tests/golden/make_adjoint_fd.py [--threads T]

Workload: the 128 x 128 x 64 adjoint design case (4000 steps; design region
32 x 32 x 4 cells with eps_r ~ U[1, 12]; a YIG block; an x-current source and
an E probe).  Objective J = sum over steps n >= 3000 of |E(probe)|^2 (the three
native edge values at the probe cell).  The LLG solve uses three fixed
Jacobi iterates, the fixed map that the adjoint differentiates (section
"Numerical Model", Eqs. llg_tra4-6, iterate_H).  For each of 16 design cells
drawn with seed 3: (J(eps + h) - J(eps - h)) / 2h with h = 1e-3 eps of that
cell, in FP64; the truncation error is O(h^2) and the rounding error of the
difference ~1e-16 J / h, both far below the 1e-3 the GPU gradient is checked
to.
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
from paper_2510_22221_b300 import workloads as W  # noqa: E402
from tests.helpers import oracle_from_workload  # noqa: E402

STEPS, N0, NCELLS, SEED, REL_H = 4000, 3000, 16, 3, 1e-3


def objective(w):
    o = oracle_from_workload(w, llg_fixed_iter=3)
    rows = o.run(STEPS)["probes"][:, :, :3]
    return float((rows[N0:] ** 2).sum())


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--out", default=os.path.join(HERE, "adjoint_design_fd16_fp64.json"))
    a = ap.parse_args()
    threads = oracle.set_threads(a.threads)
    base = W.adjoint_design(steps=STEPS)
    shape = base.eps_design.shape
    rng = np.random.default_rng(SEED)
    flat = rng.choice(base.eps_design.size, size=NCELLS, replace=False)
    cells = [tuple(int(v) for v in np.unravel_index(int(q), shape)) for q in flat]
    t0 = time.time()
    # resumable: cells already differenced are kept in a side file until done
    part = a.out + ".part"
    done = {}
    if os.path.exists(part):
        with open(part) as f:
            for line in f:
                r = json.loads(line)
                done[tuple(r["cell_kji"])] = r
    J0 = done[("J",)]["J"] if ("J",) in done else objective(base)
    if ("J",) not in done:
        with open(part, "a") as f:
            f.write(json.dumps({"cell_kji": ["J"], "J": J0}) + "\n")
    out = []
    for idx in cells:
        if idx in done:
            out.append(done[idx])
            continue
        h = REL_H * float(base.eps_design[idx])
        Js = []
        for sgn in (1.0, -1.0):
            w = W.adjoint_design(steps=STEPS)
            w.eps_design = w.eps_design.copy()
            w.eps_design[idx] += sgn * h
            Js.append(objective(w))
        out.append({"cell_kji": list(idx), "eps": float(base.eps_design[idx]), "h": h,
                    "fd": (Js[0] - Js[1]) / (2 * h), "J_plus": Js[0], "J_minus": Js[1]})
        with open(part, "a") as f:
            f.write(json.dumps(out[-1]) + "\n")
        print(idx, out[-1]["fd"], flush=True)
    doc = {
        "what": "FP64 oracle central differences of the probe objective on 16 design cells of the 128x128x64 "
                "adjoint design case (seeded workload adjoint_design)",
        "cite": "section 'Numerical Model' (the step, with three fixed LLG iterates)",
        "made_by": "python tests/golden/make_adjoint_fd.py",
        "workload": base.name, "steps": STEPS, "n0": N0, "seed": SEED, "rel_h": REL_H, "llg_fixed_iter": 3,
        "J": J0, "threads": threads, "wall_s": round(time.time() - t0, 1), "cells": out,
    }
    with open(a.out, "w") as f:
        json.dump(doc, f, indent=1)
    os.remove(part)
    print(f"wrote {a.out}")


if __name__ == "__main__":
    main()
