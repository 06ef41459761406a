"""Pins for the oracle's near-tie outputs: the second-best SSD, the energy
E(v*) = sum T^2 + sum_window(v*) ||D_sen||^2 and the relative top-2 gap
(S2 - S1) / E(v*) of Eq. 4 (Sec. III-G).

The GPU parity rule exempts a CP from exact integer agreement only when the
oracle's gap is below 1e-6, so a wrong second-best (one that can read the best
lag again) or a wrong energy (taken at another lag) would widen the exemption
silently.  These tests plant surfaces whose values are known exactly:

* a one-pixel, one-channel template makes S(v) = (a - b(v))^2 and
  E(v) = a^2 + b(v)^2, with dyadic values so every number is exact in FP64;
* on random volumes the surface is re-derived by plain numpy loops over the
  window (independent of the oracle's loop order), and the second-best,
  energy and gap are read off that surface.
"""
import numpy as np
import pytest


def _point_case(r, a, plants, q=(0, 0), base=0.0, pad=3):
    """One-channel, one-pixel template of value a at the centre; the sensed
    window holds `base` except at the planted lags {(dy, dx): b}."""
    side = 2 * (r + abs(q[0]) + abs(q[1]) + pad) + 1
    c = side // 2
    dref = np.zeros((1, side, side))
    dref[0, c, c] = a
    dsen = np.full((1, side, side), base)
    for (dy, dx), b in plants.items():
        dsen[0, c + q[1] + dy, c + q[0] + dx] = b
    return dref, dsen, c


def test_planted_runner_up_far_from_best(orc):
    # best at v = (1, -1): S = 0, E = 1 + 1 = 2; runner-up at (-2, 2):
    # S = (1 - 0.75)^2 = 0.0625; every other lag: S = 1, E = 1
    dref, dsen, c = _point_case(3, 1.0, {(1, -1): 1.0, (-2, 2): 0.75})
    res = orc.match_one(dref, dsen, c, c, 1, 3)
    assert (res["dy"], res["dx"]) == (1, -1)
    assert res["ssd"] == 0.0
    assert res["second"] == 0.0625
    assert res["E"] == 2.0                     # at v*, not at v = 0 (E(0) = 1)
    assert res["gap_rel"] == 0.0625 / 2.0


def test_planted_runner_up_next_to_best(orc):
    # the runner-up is a 4-neighbour of the minimum
    dref, dsen, c = _point_case(2, 2.0, {(0, 1): 2.0, (0, 0): 1.5, (-1, -1): 0.5})
    res = orc.match_one(dref, dsen, c, c, 1, 2)
    assert (res["dy"], res["dx"]) == (0, 1)
    assert res["second"] == 0.25               # (2 - 1.5)^2
    assert res["E"] == 8.0                     # 2^2 + 2^2
    assert res["gap_rel"] == 0.25 / 8.0


def test_exact_two_way_tie_has_zero_gap(orc):
    # two lags with S = 0: the smaller (dy, dx) wins, the runner-up equals it
    dref, dsen, c = _point_case(2, 1.0, {(1, 1): 1.0, (-1, 0): 1.0})
    res = orc.match_one(dref, dsen, c, c, 1, 2)
    assert (res["dy"], res["dx"]) == (-1, 0)
    assert res["ssd"] == 0.0 and res["second"] == 0.0
    assert res["gap_rel"] == 0.0
    assert res["E"] == 2.0


def test_gap_with_prior_offset_and_nonzero_minimum(orc):
    # prior q = (qx, qy) = (2, -1) moves the window; the best S is not zero
    q = (2, -1)
    dref, dsen, c = _point_case(2, 1.0, {(-1, 1): 0.5, (1, -1): 0.25}, q=q, base=-1.0)
    res = orc.match_one(dref, dsen, c, c, 1, 2, qx=q[0], qy=q[1])
    assert (res["dy"], res["dx"]) == (q[1] - 1, q[0] + 1)
    assert res["ssd"] == 0.25                  # (1 - 0.5)^2
    assert res["second"] == 0.5625             # (1 - 0.25)^2
    assert res["E"] == 1.25                    # 1 + 0.25
    assert res["gap_rel"] == (0.5625 - 0.25) / 1.25


def test_flat_surface_gap_zero(orc):
    # every lag equal: the first lag in (dy, dx) order, gap 0
    dref, dsen, c = _point_case(2, 1.0, {}, base=0.5)
    res = orc.match_one(dref, dsen, c, c, 1, 2)
    assert (res["dy"], res["dx"]) == (-2, -2)
    assert res["gap_rel"] == 0.0 and res["second"] == res["ssd"] == 0.25


def _numpy_surface(dref, dsen, px, py, N, r, qx, qy):
    """S(v) and E(v) by explicit window slices, one lag at a time."""
    t0 = N // 2
    T = dref[:, py - t0:py - t0 + N, px - t0:px - t0 + N]
    L = 2 * r + 1
    S = np.empty((L, L))
    E = np.empty((L, L))
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            y0, x0 = py + qy - t0 + dy, px + qx - t0 + dx
            Wv = dsen[:, y0:y0 + N, x0:x0 + N]
            S[dy + r, dx + r] = ((T - Wv) ** 2).sum()
            E[dy + r, dx + r] = (T ** 2).sum() + (Wv ** 2).sum()
    return S, E


@pytest.mark.parametrize("seed,N,r,qx,qy", [(1, 5, 3, 0, 0), (2, 6, 4, 1, -2), (3, 7, 2, -1, 1)])
def test_second_energy_gap_against_numpy_surface(orc, seed, N, r, qx, qy):
    rng = np.random.default_rng(seed)
    dref = rng.random((3, 30, 30))
    dsen = rng.random((3, 30, 30))
    # copy the template into the window at a lag so the minimum is clear
    px, py = 15, 14
    vy, vx = rng.integers(-r + 1, r, 2)
    t0 = N // 2
    dsen[:, py + qy - t0 + vy:py + qy - t0 + vy + N, px + qx - t0 + vx:px + qx - t0 + vx + N] = \
        dref[:, py - t0:py - t0 + N, px - t0:px - t0 + N] + 0.01 * rng.random((3, N, N))
    S, E = _numpy_surface(dref, dsen, px, py, N, r, qx, qy)
    res = orc.match_one(dref, dsen, px, py, N, r, qx=qx, qy=qy)
    flat = S.ravel()
    best = int(np.argmin(flat))
    second = np.sort(flat)[1]
    assert (res["dy"], res["dx"]) == (best // (2 * r + 1) - r + qy, best % (2 * r + 1) - r + qx)
    assert res["ssd"] == pytest.approx(flat[best], rel=1e-12, abs=1e-12)
    assert res["second"] == pytest.approx(second, rel=1e-12)
    assert res["second"] > res["ssd"]
    assert res["E"] == pytest.approx(E.ravel()[best], rel=1e-12)
    assert res["gap_rel"] == pytest.approx((second - flat[best]) / E.ravel()[best], rel=1e-9)
    # the energy at v = 0 differs from E(v*): a reading of E at the wrong lag fails
    assert abs(E[r, r] - E.ravel()[best]) > 1e-6 * E.ravel()[best] or best == r * (2 * r + 1) + r


def test_match_many_carries_the_same_tie_outputs(orc):
    dref, dsen, c = _point_case(3, 1.0, {(1, -1): 1.0, (-2, 2): 0.75})
    many = orc.match_many(dref, dsen, np.array([c], np.int32), np.array([c], np.int32),
                          np.array([1], np.int32), np.array([3], np.int32))
    assert many["second"][0] == 0.0625 and many["E"][0] == 2.0
    assert many["gap_rel"][0] == 0.03125
