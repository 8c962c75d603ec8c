"""Closed-form fixtures (tests/golden) against the generators and the oracle."""
import os

import numpy as np

from paper_1810_04597_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLD, name)) as f:
        return [list(map(float, ln.split())) for ln in f if ln.strip() and not ln.startswith("#")]


def test_alfven_speed_closed_form():
    for rho, p, B0, eta, gam, u in _rows("alfven_speed.txt"):
        assert abs(inputs.alfven_speed(rho, p, B0, eta, gam) ** 2 - u) < 1e-15


def test_mp5_jump_values(orc):
    for row in _rows("mp5_steps.txt"):
        assert orc.mp5_face(row[:5]) == row[5]


def test_mp5_bound_values(orc):
    """The limited value where u_UL, u_LC and u_MD in turn bound the
    interval; the result is u_or + (bound - u_or), one rounding each."""
    for row in _rows("mp5_bounds.txt"):
        assert abs(orc.mp5_face(row[:5]) - row[5]) <= 4e-16 * max(1.0, abs(row[5]))
