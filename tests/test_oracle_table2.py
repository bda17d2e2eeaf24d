"""Pins the oracle's rate formulas against the numbers printed in Table 2.

For every row, kappa(X) inferred from the APC column through Theorem 1 must
reproduce the B-Cimmino column through the Cimmino rate of Sec. 4.5; both use
T = 1/(-log rho) (Table 2 caption)."""
import math
import os

import pytest

from oracle import apc_oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden", "table2_convergence_times.txt")


def _rows():
    out = []
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        name, *vals = line.split()
        out.append((name, [float(v) for v in vals]))
    return out


def _kappa_from_apc_time(T):
    # invert T = 1/(-log rho), rho = (sqrt(k)-1)/(sqrt(k)+1)
    rho = math.exp(-1.0 / T)
    return ((1.0 + rho) / (1.0 - rho)) ** 2


@pytest.mark.parametrize("name,vals", _rows())
def test_apc_and_cimmino_columns_agree(name, vals):
    T_cim, T_apc = vals[4], vals[5]
    kappa = _kappa_from_apc_time(T_apc)
    assert O.convergence_time(O.rate_apc(kappa)) == pytest.approx(T_apc, rel=1e-9)
    assert O.convergence_time(O.rate_cimmino(kappa)) == pytest.approx(T_cim, rel=1e-2)


def test_apc_beats_every_other_column():
    # boldface APC column: smallest convergence time in every row
    for name, vals in _rows():
        assert vals[5] == min(vals), name
