"""The roofline's algorithmic FLOPs: the stored table is what the oracle's own
face flux counts, each counting row takes the branch pattern it is named for,
and the counting number type counts a formula as written by hand.
"""
import json
import os
import sys

import numpy as np

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.join(ROOT, "oracle"))

import count_flops  # noqa: E402


def test_stored_table_is_the_oracle_count():
    stored = json.load(open(count_flops.OUT))
    assert stored == count_flops.compute()


def _patterns(U, gamma=1.4):
    """Per face of the row (cells f+2, f+3) and per characteristic field:
    'u' upwinded (the two cells' and the Roe eigenvalue share a strict sign)
    or 's' split; the Roe average written out from its textbook definition."""
    rho = U[:, 0]
    vel = U[:, 1:4] / rho[:, None]
    p = (gamma - 1) * (U[:, 4] - 0.5 * rho * (vel ** 2).sum(1))
    c = np.sqrt(gamma * p / rho)
    H = (U[:, 4] + p) / rho
    out = []
    for f in range(17):
        i, j = f + 2, f + 3
        wl, wr = np.sqrt(rho[i]), np.sqrt(rho[j])
        ut = (wl * vel[i] + wr * vel[j]) / (wl + wr)
        Ht = (wl * H[i] + wr * H[j]) / (wl + wr)
        ct = np.sqrt((gamma - 1) * (Ht - 0.5 * (ut ** 2).sum()))
        lam = lambda un, cc: (un - cc, un, un, un, un + cc)
        la, lb, lt = lam(vel[i, 0], c[i]), lam(vel[j, 0], c[j]), lam(ut[0], ct)
        out.append("".join("u" if (min(x) > 0 or max(x) < 0) else "s" for x in zip(la, lb, lt)))
    return out


def test_each_row_takes_its_branch_pattern():
    want = {"all_upwind": "uuuuu", "split_123": "usssu", "split_0": "suuuu", "split_4": "uuuus"}
    for pat, code in want.items():
        got = _patterns(count_flops.row_states(pat, 0))
        assert got == [code] * 17, (pat, got)


def test_counting_type_counts_the_linear_scheme_by_hand():
    """linear5 = (0.1 q0 + 0.6 q1) + 0.3 q2 with q0 = ((2a - 7b) + 11c)/6 (3
    mul, 2 add/sub, 1 div), q1 = ((-b + 5c) + 2d)/6 (2 mul, 2 add, 1 div; the
    negation is free), q2 = ((2c + 5d) - e)/6 (2 mul, 2 add/sub, 1 div) and the
    combination (3 mul, 2 add): 21 = 8 add/sub + 10 mul + 3 div."""
    assert list(oracle.count_recon_flops(2)) == [21, 8, 10, 3, 0]


def test_count_depends_only_on_the_branches():
    """Another row with the same branch pattern (different values) gives the
    same count: the count is structural, apart from the branch decisions."""
    U = count_flops.row_states("all_upwind", 0).copy()
    U[:, 0] *= 1.7
    U[:, 1:] *= 1.7
    assert _patterns(U) == ["uuuuu"] * 17
    a = oracle.count_row_flops(U, 0, 1.4, 0.0, 0, 0)
    b = oracle.count_row_flops(count_flops.row_states("all_upwind", 0), 0, 1.4, 0.0, 0, 0)
    assert (a == b).all()


def test_split_costs_what_the_upwinded_row_leaves_out():
    """The split of fields 1-3 costs at least the three second
    reconstructions and the split halves (three operations per cell and
    half) per face, which the upwinded row does not compute: the projections
    v = L U of upwinded fields, computed by the oracle but unused, are left out
    of the upwinded count."""
    t = json.load(open(count_flops.OUT))
    row = t["row"]["weno5"]["all_upwind"][0]
    split = t["row"]["weno5"]["split_123"][0]
    rec = t["recon"]["weno5"][0]
    assert split - row > 17 * 3 * (rec + 6 * 3)
