"""Pins of the minimum-ignition-energy search (Application examples: the
ensemble ignition studies): the bisection against classifiers whose threshold is
known, and the product driver's host logic (probe energies, bracket update)
against the oracle's statement of the same search on the same outcomes."""
import numpy as np
import pytest

from oracle import ignition as oig
from paper_2202_02319_b300 import ignition as gig


def _threshold(E_star):
    return lambda Es: [E >= E_star for E in Es]


@pytest.mark.parametrize("members,rounds", [(1, 12), (3, 5), (7, 3)])
def test_bisection_brackets_a_known_threshold(members, rounds):
    """A monotone response with threshold E*: the bracket holds E* (failed below,
    ignited at the top) and shrinks by members + 1 per round."""
    E_star = 0.3712
    (lo, hi), hist = oig.bisect(_threshold(E_star), 0.0, 1.0, members, rounds)
    assert lo < E_star <= hi
    assert hi - lo == pytest.approx((members + 1) ** -rounds, rel=1e-9)
    assert len(hist) == rounds


def test_bisection_follows_the_lowest_transition():
    """A non-monotone response (ignites in [0.2, 0.3) and from 0.6 on): the bracket
    closes on the lowest failed-to-ignited transition the probes meet."""
    f = lambda Es: [(0.2 <= E < 0.3) or E >= 0.6 for E in Es]
    (lo, hi), _ = oig.bisect(f, 0.0, 1.0, 9, 3)
    assert lo < 0.2 <= hi and hi - lo < 2e-3


def test_ignition_test_reads_both_criteria():
    assert oig.is_ignited(900.0, 1.0, 2.0)
    assert not oig.is_ignited(599.0, 1.0, 2.0)          # too cold: failure
    assert not oig.is_ignited(900.0, 2.0, 1.0)          # heat release decays
    assert not oig.is_ignited(900.0, -3.0, -1.0)        # net endothermic


@pytest.mark.parametrize("seed", range(4))
def test_driver_host_logic_matches_the_oracle_search(seed):
    """The product driver's probes and bracket updates equal the oracle's on the
    same outcomes (random responses, several rounds)."""
    rng = np.random.default_rng(seed)
    members = int(rng.integers(1, 9))
    lo, hi = 0.5e-3, 40e-3
    glo, ghi = lo, hi
    outcomes = []

    def f(Es):
        r = [bool(x) for x in rng.integers(0, 2, len(Es))]
        outcomes.append(r)
        return r
    (olo, ohi), hist = oig.bisect(f, lo, hi, members, 4)
    for (probes, res, _), r in zip(hist, outcomes):
        Es = gig.probe_energies(glo, ghi, members)
        assert np.allclose(Es, probes, rtol=1e-15, atol=0.0)
        glo, ghi = gig.next_bracket(Es, r, glo, ghi)
    assert (glo, ghi) == pytest.approx((olo, ohi), rel=1e-15)
    assert gig.ignited(900.0, 1.0, 2.0) and not gig.ignited(599.0, 1.0, 2.0)
