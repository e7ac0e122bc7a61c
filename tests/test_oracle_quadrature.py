"""Pins of the oracle's quadrature (Sec. III C-D, Table I) against numbers the
paper prints."""
from decimal import Decimal

import numpy as np
import pytest

from conftest import read_golden
from oracle import groups as G
from oracle import quadrature as QD

G1_6 = [1, 2, 3, 4, 5, 6]


@pytest.fixture(scope="module")
def cache5():
    return QD.MomentCache(5)


def test_table_i_orbits_match_printed_counts_and_lengths():
    # Every generated full-symmetric orbit has the printed size; every printed
    # length matches the vectors except rows 17 and 18, whose printed lengths
    # are exchanged (sqrt(19) and sqrt(17) for (3,2,2) and (3,3,1)).
    for gid, (base, count, len2) in G.TABLE_I.items():
        orb = G.orbit(gid)
        assert len(orb) == count, gid
        assert all(sum(c * c for c in v) == G.length2(gid) for v in orb), gid
        if gid == 17:
            assert (G.length2(17), len2) == (17, 19)
        elif gid == 18:
            assert (G.length2(18), len2) == (19, 17)
        else:
            assert G.length2(gid) == len2, gid


def test_printed_stencil_cardinalities():
    with open("tests/golden/stencil_cardinalities.txt") as fh:
        rows = [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]
    for groups, count in rows:
        gids = [int(g) for g in groups.split(",")]
        assert sum(len(G.orbit(g)) for g in gids) == int(count)


def test_d3q19_is_g1_g2_g3():
    # Sec. III C: the D3Q19 model uses {G1, G2, G3}.
    assert sum(len(G.orbit(g)) for g in (1, 2, 3)) == 19


def test_printed_weights_m5(cache5):
    # T1: the six printed weights at mbar = 5, v0 = 0.398 (10 decimals).
    gold = read_golden("quadrature_m5_G1-G6.txt")
    w = QD.weights_dec(G1_6, 5, gold["v0"], cache5)
    for k in range(6):
        printed = Decimal(gold["w%d" % (k + 1)])
        assert abs(w[k] - printed) < Decimal("1e-10"), (k, w[k], printed)


def test_printed_pruning_points_m5(cache5):
    # T2: w2 = 0 at v0 = 0.3965826549..., w3 = 0 at 0.3984063950...
    gold = read_golden("quadrature_m5_G1-G6.txt")
    z2 = QD.zero_of_weight(G1_6, 5, 1, "0.3960", "0.3972", iters=80, cache=cache5)
    z3 = QD.zero_of_weight(G1_6, 5, 2, "0.3980", "0.3990", iters=80, cache=cache5)
    assert abs(z2 - Decimal(gold["v0_w2_zero"])) < Decimal("1e-10")
    assert abs(z3 - Decimal(gold["v0_w3_zero"])) < Decimal("1e-10")


def test_printed_positive_window_m5(cache5):
    # The positive-weight window (0.3966, 0.3984) printed to 4 decimals.
    gold = read_golden("quadrature_m5_G1-G6.txt")
    (lo, hi), = QD.positive_window(G1_6, 5, 0.390, 0.405, samples=61, cache=cache5)
    assert round(lo, 4) == float(gold["window_lo"])
    assert round(hi, 4) == float(gold["window_hi"])


def test_weights_sum_to_one(cache5):
    # T4: sum_i w_i = int omega d^3p/p0 = 1 (Eq. 40).
    st = QD.Stencil(G1_6, 5, 0.398)
    w3, _, _, _ = st.populations3d()
    assert abs(w3.sum() - 1.0) < 1e-14
    w2, _, _, _, _ = st.populations2d()
    assert abs(w2.sum() - 1.0) < 1e-14


def test_fold_counts():
    # The fold merges +-n_z pairs within a group: 57 -> 39 for G1..G6.
    st = QD.Stencil(G1_6, 5, 0.398)
    w2, p2, d2, gi, mult = st.populations2d()
    assert len(w2) == 39 and mult.sum() == 57
    assert set(mult.tolist()) <= {1, 2}


def test_weights_reproduce_moments_exactly(cache5):
    # The solved system reproduces the six rest-frame moments to ~1e-45.
    A, b = QD.system_dec(G1_6, 5, "0.398", cache5)
    w = QD.weights_dec(G1_6, 5, "0.398", cache5)
    for r in range(6):
        assert abs(sum(A[r][k] * w[k] for k in range(6)) - b[r]) < Decimal("1e-40") * abs(b[r])


def test_superluminal_v0_rejected(cache5):
    # Sec. III D: v0 < 1/sqrt(5) for G6, pseudo-particles may not exceed c.
    with pytest.raises(ValueError):
        QD.weights_dec(G1_6, 5, "0.4473", cache5)
