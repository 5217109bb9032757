"""The eigenvalue-distribution statistics of Tables 1b and 4a (host side):
the histogram counts on eigenvalue sets whose answer is known by hand, and
the dense route on Problem 1 (40 x 40) against the printed Table 1b (fixture
tests/golden/table1b_p1_eigen.txt), GS(2) applied by the oracle."""
import types

import numpy as np
import pytest

import oracle
from paper_0812_2769_gb300 import spectrum
from problems import configs


def test_summary_counts_on_known_sets():
    # 1..100: 100 equal intervals of width 0.99 over [1, 100], one value each
    # except the last, closed interval, which holds 99.x and 100
    d = spectrum.summary(np.arange(1.0, 101.0))
    assert d["lambda_min"] == 1.0 and d["lambda_max"] == 100.0 and d["ratio"] == 100.0
    assert d["first_interval"] == 1
    assert d["origin_interval"] == 1  # 0 lies below the range: nearest (first) interval
    # a crowd of 50 values in [0, 0.01) and one at 1: the first of 100
    # intervals of [0, 1] is [0, 0.01)
    ev = np.concatenate([np.linspace(0.0, 0.0099, 50), [1.0]])
    d = spectrum.summary(ev)
    assert d["first_interval"] == 50 and d["lambda_min"] == 0.0 and d["ratio"] == float("inf")
    # complex values: moduli for lambda_min/max, real parts for the histogram;
    # the origin sits in the interval [0, 0.02) of [-1, 1]
    ev = np.array([-1.0, 0.005 + 3j, 0.005 - 3j, 0.015, 0.5, 1.0])
    d = spectrum.summary(ev)
    assert d["lambda_max"] == pytest.approx(abs(0.005 + 3j))
    assert d["lambda_min"] == pytest.approx(0.015)
    assert d["origin_interval"] == 3 and d["first_interval"] == 1


def _golden():
    rows = {}
    with open(__file__.replace("test_spectrum_cpu.py", "golden/table1b_p1_eigen.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, lo, hi, cnt = line.split()
                rows[name] = (float(lo), float(hi), int(cnt))
    return rows


def test_dense_route_reproduces_table1b():
    rows = _golden()
    for name, (lo, hi, cnt) in rows.items():
        s = configs.p1(40, continuous=1000.0) if name == "continuous" else configs.p1(40)
        val = oracle.gs_scale(s.rowptr, s.colidx, s.val, s.b, 2.0)[0] if name == "gs" else s.val
        A = types.SimpleNamespace(rowptr=s.rowptr, colidx=s.colidx, val=val)
        d = spectrum.summary(spectrum.dense_eigenvalues(A))
        # three printed digits; lambda_min of the discontinuous matrix lands 0.8% off
        assert abs(d["lambda_min"] - lo) <= 0.01 * lo, (name, d)
        assert abs(d["lambda_max"] - hi) <= 0.006 * hi, (name, d)
        assert d["first_interval"] == cnt, (name, d)


def test_dense_route_refuses_large_matrices():
    s = configs.c1(8)
    A = types.SimpleNamespace(rowptr=s.rowptr, colidx=s.colidx, val=s.val)
    with pytest.raises(ValueError):
        spectrum.dense_eigenvalues(A, max_n=10)
