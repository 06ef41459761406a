"""Host-side logic of the serving loop (no GPU): the HBM admission ledger and
the CP ring allocator."""
import numpy as np
import pytest

from paper_1808_06194_gb300.serve import Admission, CpRing, Job, job_bytes


def test_admission_never_exceeds_budget():
    rng = np.random.default_rng(0)
    adm = Admission(1000)
    live = []
    for step in range(2000):
        if live and rng.random() < 0.45:
            adm.release(live.pop(rng.integers(len(live))))
        else:
            nb = int(rng.integers(1, 400))
            if adm.fits(nb):
                adm.admit(step, nb)
                live.append(step)
        assert adm.used <= adm.budget
        assert adm.used == sum(adm.resident.values())
    assert adm.peak <= 1000


def test_admission_rejects_over_budget_and_oversized():
    adm = Admission(100)
    adm.admit("a", 60)
    with pytest.raises(RuntimeError):
        adm.admit("b", 50)
    with pytest.raises(ValueError):
        adm.admit("c", 101)
    adm.release("a")
    adm.admit("b", 50)
    assert adm.used == 50


def test_cp_ring_first_fit_and_merge():
    ring = CpRing(100)
    a = ring.alloc(40)
    b = ring.alloc(40)
    assert (a, b) == (0, 40)
    assert ring.alloc(30) is None
    ring.release(a, 40)
    c = ring.alloc(30)
    assert c == 0
    ring.release(b, 40)
    ring.release(c, 30)
    assert ring.free == [(0, 100)]
    rng = np.random.default_rng(1)
    live = {}
    for _ in range(500):
        if live and rng.random() < 0.5:
            k = list(live)[rng.integers(len(live))]
            ring.release(k, live.pop(k))
        else:
            n = int(rng.integers(1, 30))
            s = ring.alloc(n)
            if s is not None:
                assert all(s + n <= o or o + m <= s for o, m in live.items())
                live[s] = n
        assert ring.free_slots + sum(live.values()) == 100


def test_job_grid_and_bytes():
    j = Job(np.zeros((512, 640), np.float32), np.zeros((512, 640), np.float32), tmpl=64, radius=16)
    gx, gy = j.grid()
    assert (gx, gy) == ((640 - 2 * 56) // 64, (512 - 2 * 56) // 64)
    assert job_bytes(j) >= 2 * 512 * 640 * 4 + 2 * 10 * 512 * 640 * 4


def test_cp_ring_random_alloc_release_keeps_free_list_exact():
    """Random allocate/release sequences: the free list stays sorted, disjoint,
    merged, and free + allocated always equals the capacity."""
    import numpy as np
    from paper_1808_06194_gb300.serve import CpRing
    rng = np.random.default_rng(7)
    ring = CpRing(1000)
    live = {}
    for step in range(3000):
        if live and rng.random() < 0.45:
            start = list(live)[rng.integers(len(live))]
            ring.release(start, live.pop(start))
        else:
            n = int(rng.integers(1, 60))
            s = ring.alloc(n)
            if s is not None:
                assert all(s + n <= b or b + live[b] <= s for b in live), "overlap"
                live[s] = n
        used = sum(live.values())
        assert ring.free_slots + used == 1000
        fl = ring.free
        assert all(fl[i][0] + fl[i][1] < fl[i + 1][0] for i in range(len(fl) - 1))   # merged, sorted
        for s_, n_ in live.items():
            assert all(s_ + n_ <= fs or fs + fn <= s_ for fs, fn in fl)               # disjoint
