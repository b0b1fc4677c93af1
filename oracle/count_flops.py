"""Algorithmic FLOPs of the face flux, counted by running the oracle's own code.

Writes tests/golden/face_flops.json, which the benchmark reads for its
roofline.  The count runs the oracle's face flux (Sec. 2.2: Roe average and
eigenvectors, characteristic projections, the Roe / local Lax-Friedrichs
switch, the reconstructions and F = R g) on the counting number type of
orc.cpp, over the 17 faces of one 16-cell block row along x with its 3-cell
stencil margins.  That type counts the add, subtract, multiply, divide and
square-root operations the outputs depend on, after merging repeated
expressions of the same operands (a cell's primitive variables and physical
flux count once per row, not once per face) and dropping operations with the
literal zeros and ones of the eigenvectors and the projections of fields that
are upwinded.

Which branch each face takes depends on the data, so each row below is built
so that every one of its faces takes the same pattern (checked by the test
that re-runs this script):

* all fields upwinded (subsonic flow, u = c/2);
* fields 1-3 (the entropy and shear waves, eigenvalue u) on the LLF split
  (u alternating in sign from cell to cell), fields 0 and 4 upwinded;
* field 0 (u - c) split (u - c alternating in sign), the others upwinded;
* field 4 (u + c) split.

The cost of a pattern beyond the all-upwinded row is stored as its extra, and
the bench combines them with the measured share of faces of each pattern.
Per cell and stage the flux differences (3 differences, 2 sums and the
division by the cell size per variable, leaf_rhs) and the TVD-RK3 update
(u + dt L, then a un + b t; at stage 0 only the first) add fixed counts.

Usage: python oracle/count_flops.py [--check]
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, ROOT)

import oracle  # noqa: E402

OUT = os.path.join(ROOT, "tests", "golden", "face_flops.json")
GAMMA = 1.4
RECON_WENO, RECON_LINEAR, RECON_TENO, RECON_WENOAO = 0, 2, 3, 4
FLUX_ROE = 0
NCELLS = 22            # cells -3 .. 18 of a row
PATTERNS = ("all_upwind", "split_123", "split_0", "split_4")


def row_states(pattern: str, d: int = 0) -> np.ndarray:
    """Conserved lab-frame states of the 22 cells of a row along d whose 17
    faces all take `pattern`: smooth density and pressure, velocity along d
    chosen against the local sound speed."""
    m = np.arange(NCELLS)
    rho = 1.0 + 0.3 * np.sin(0.7 * m)
    p = 1.0 + 0.2 * np.cos(0.5 * m)
    c = np.sqrt(GAMMA * p / rho)
    alt = np.where(m % 2 == 0, 1.0, -1.0)
    if pattern == "all_upwind":
        u = 0.5 * c
    elif pattern == "split_123":
        u = 0.1 * c * alt
    elif pattern == "split_0":
        u = c * (1.0 + 0.2 * alt)
    elif pattern == "split_4":
        u = -c * (1.0 + 0.2 * alt)
    else:
        raise ValueError(pattern)
    vt1, vt2 = 0.05 * np.cos(m), -0.03 * np.sin(1.3 * m)
    vel = np.zeros((NCELLS, 3))
    vel[:, d] = u
    vel[:, (d + 1) % 3] = vt1
    vel[:, (d + 2) % 3] = vt2
    U = np.zeros((NCELLS, 5))
    U[:, 0] = rho
    U[:, 1:4] = rho[:, None] * vel
    U[:, 4] = p / (GAMMA - 1.0) + 0.5 * rho * (vel ** 2).sum(axis=1)
    return U


def compute() -> dict:
    rows = {}
    for mode, name in ((RECON_WENO, "weno5"), (RECON_LINEAR, "linear5")):
        counts = {}
        for pat in PATTERNS:
            per_dir = [oracle.count_row_flops(row_states(pat, d), d, GAMMA, 0.0, mode, FLUX_ROE) for d in range(3)]
            assert all((c == per_dir[0]).all() for c in per_dir), (pat, per_dir)
            counts[pat] = [int(x) for x in per_dir[0]]
        rows[name] = counts
    recon = {name: [int(x) for x in oracle.count_recon_flops(mode)]
             for mode, name in ((RECON_WENO, "weno5"), (RECON_LINEAR, "linear5"), (RECON_TENO, "teno5"),
                                (RECON_WENOAO, "wenoao53"))}
    nv = 5
    return {
        "what": "FLOPs of the oracle's face flux (Roe flux with the per-field LLF fallback) over one block row "
                "of 16 cells and 17 faces; entries are [FLOPs, add/sub, mul, div, sqrt]",
        "command": "python oracle/count_flops.py",
        "row": {"faces": 17, "cells": 16, "weno5": rows["weno5"], "linear5": rows["linear5"]},
        "recon": recon,
        "cell": {"divergence": nv * (3 + 2 + 1), "update_rk3_mean": nv * (2 + 5 + 5) / 3.0},
    }


def main():
    table = compute()
    if "--check" in sys.argv:
        old = json.load(open(OUT))
        sys.exit(0 if old == table else 1)
    with open(OUT, "w") as f:
        json.dump(table, f, indent=1)
        f.write("\n")
    print(json.dumps(table, indent=1))


if __name__ == "__main__":
    main()
