"""Fixtures under tests/golden/ (text, each citing the passage it evaluates)
checked against the oracle, the library's host entry points and the volume
model."""
import os

import pytest

import oracle
from paper_2603_21444_gb300 import volume

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_static_cannon_table_q4():
    rows = [tuple(map(int, r)) for r in _rows("static_cannon_q4.txt")]
    q = 4
    assert len(rows) == q ** 3
    for i, j, r, rp in rows:
        assert oracle.static_cannon_schedule(q, i, j)[r] == rp
    # the library's schedule: instance (i, j, k, r) multiplies A tile (i lam + k, r') by B tile (r', j)
    tsg = pytest.importorskip("paper_2603_21444_gb300")
    try:
        a_tile, b_tile, gp = tsg.trident_schedule(q, 1)
    except OSError:
        pytest.skip("library not built")
    want = {(i, j, r): rp for i, j, r, rp in rows}
    t = 0
    for i in range(q):
        for j in range(q):
            for r in range(q):
                rp = want[(i, j, r)]
                assert a_tile[t] == i * q + rp and b_tile[t] == rp * q + j
                t += 1


def test_prop1_at_p256_lambda4():
    vals = {k: float(v) for k, v in _rows("prop1_p256_lambda4.txt")}
    m = volume.prop1_volumes(1.0, 256, 4)
    assert m["q"] == 8
    for key in ("per_round_gi", "per_round_li", "total_gi", "total_li"):
        assert m[key] == pytest.approx(vals[key], rel=1e-15)
    assert m["total_gi_closed_form"] == pytest.approx(vals["total_gi"], rel=1e-15)
