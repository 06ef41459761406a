"""Host checks of the parity helper: the near-tie exemption is counted and
bounded, and a difference outside it fails."""
import numpy as np
import pytest

from tests._util import TIE_REL, check_match_parity


def _rows(dx, dy, gap=None, status=None):
    n = len(dx)
    d = {"dx": np.array(dx), "dy": np.array(dy),
         "status": np.zeros(n, np.int32) if status is None else np.array(status),
         "sub_dx": np.array(dx, np.float64), "sub_dy": np.array(dy, np.float64),
         "ssd": np.ones(n), "E": np.full(n, 100.0)}
    d["gap_rel"] = np.full(n, 1.0) if gap is None else np.array(gap)
    return d


def test_equal_offsets_count_no_ties():
    o = _rows([1, 2, 3], [0, 0, 0])
    p = check_match_parity(_rows([1, 2, 3], [0, 0, 0]), o)
    assert p.n_ok == 3 and p.n_tie == 0 and p.n_inb == 3


def test_difference_at_near_tie_is_counted():
    o = _rows([1, 2, 3], [0, 0, 0], gap=[1.0, 0.1 * TIE_REL, 1.0])
    p = check_match_parity(_rows([1, 5, 3], [0, 0, 0]), o)
    assert p.n_tie == 1 and p.n_near == 1 and p.n_ok == 2


def test_difference_without_tie_fails():
    o = _rows([1, 2], [0, 0], gap=[1.0, 10 * TIE_REL])
    with pytest.raises(AssertionError, match="integer offsets differ"):
        check_match_parity(_rows([1, 4], [0, 0]), o)


def test_too_many_exemptions_fail():
    o = _rows([1, 2, 3], [0, 0, 0], gap=[0.0, 0.0, 0.0])
    with pytest.raises(AssertionError, match="near-tie exemption"):
        check_match_parity(_rows([2, 3, 4], [0, 0, 0]), o, max_tie=1)


def test_out_of_bounds_rows_are_not_compared():
    o = _rows([0, 2], [0, 0], status=[1, 0])
    p = check_match_parity(_rows([9, 2], [9, 0], status=[1, 0]), o)
    assert p.n_inb == 1 and p.n_ok == 1
