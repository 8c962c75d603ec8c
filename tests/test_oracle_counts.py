"""Pins of the oracle's operation-counting build (op_count.cpp), whose
per-unit counts are the roofline numerator of bench.py: hand-counted
operations of single reconstructions, the trivial-operand rule, and the
subexpression rule (cse) on a small step."""
import numpy as np
import pytest


def test_unlimited_mp5_is_seventeen_operations(orc):
    """MP5 on smooth data (the limiter not reached): the interpolant
    (2 u_-2 - 13 u_-1 + 47 u_0 + 27 u_1 - 3 u_2) / 60 takes 5 products, 4 sums
    and a division; u_mp = u_0 + minmod(u_1 - u_0, 4 (u_0 - u_-1)) two
    differences, one product and a sum (minmod is a selection); the test
    (u_or - u_0)(u_or - u_mp) two differences and a product: 9 additions,
    7 multiplications, 1 division."""
    v, c = orc.count_mp5_face(np.array([1.5, 1.6, 1.75, 1.95, 2.2]))
    assert abs(v - orc.mp5_face([1.5, 1.6, 1.75, 1.95, 2.2])) == 0.0
    assert (c["add"], c["mul"], c["div"], c["sqrt"]) == (9, 7, 1, 0), c
    _, c2 = orc.count_mp5_face(np.array([1.5, 1.6, 1.75, 1.95, 2.2]), cse=True)
    assert c2["flops"] == 17     # no repeated operation inside one reconstruction


def test_trivial_operands_are_not_counted(orc):
    """A product with an exact 1 (here u_-2 = 1 in 2 u_-2) is not an
    operation a specialised code would perform: one multiplication fewer."""
    _, c = orc.count_mp5_face(np.array([1.0, 1.6, 1.75, 1.95, 2.2]))
    assert (c["add"], c["mul"], c["div"]) == (9, 6, 1), c


def test_limited_mp5_counts_more(orc):
    """At a jump the limiter runs: curvatures, the four bounds and the
    median add operations beyond the seventeen of the accepted value."""
    _, c = orc.count_mp5_face(np.array([0.5, 0.5, 0.5, 2.5, 2.5]))
    assert c["flops"] > 17, c


def test_step_counts_are_consistent(orc):
    """One step of a small box: every step has units; counting each distinct
    operation once per unit never counts more than counting them all, and
    removes something in the faces (the flux, the conserved vector and the
    speeds of one state share v^2, B^2, v.B); sampling every 4th unit gives
    per-unit figures within a few percent of counting every unit."""
    from paper_1810_04597_gb300 import inputs
    prob = inputs.sweep_box(12, seed=3)
    cfg = orc.make_cfg(prob)
    full, st = orc.count_steps(cfg, prob.prims, prob.bface, 1)
    cse, _ = orc.count_steps(cfg, prob.prims, prob.bface, 1, cse=True)
    samp, _ = orc.count_steps(cfg, prob.prims, prob.bface, 1, cse=True, sample_every=4)
    for step in ("c2p", "faces", "emf", "assemble", "ct", "rk"):
        assert full[step]["units"] > 0 and full[step]["flops"] > 0, step
        assert cse[step]["flops"] <= full[step]["flops"], step
        assert abs(samp[step]["per_unit"] / cse[step]["per_unit"] - 1.0) <= 0.05, step
    assert cse["faces"]["flops"] < 0.9 * full["faces"]["flops"]
    # flat space: the update of a cell is 5 flux differences over 3 directions
    # (3 differences, 3 divisions by dx, 2 sums, plus the source-free store)
    assert cse["assemble"]["per_unit"] == pytest.approx(40.0)
    assert st["calls"] == 3 * prob.ncells
