"""Pins of the schedulers (Sec. III-C, Algs. 1 and 2, Eqs. R_LPT and R_part)."""
import os

import numpy as np
import pytest

from oracle import sched


def test_lpt_classic_worst_case():
    # P = 2, tasks 3,3,2,2,2: LPT gives 7, the optimum is 6; ratio 4/3 - 1/(3P) = 7/6
    rows, F = sched.lpt([3, 3, 2, 2, 2], 2)
    assert F.max() == 7 and sched.brute_opt_sequential([3, 3, 2, 2, 2], 2) == 6


@pytest.mark.parametrize("seed", range(12))
def test_lpt_bound_vs_brute_force(seed):
    rng = np.random.default_rng(seed)
    P = int(rng.integers(2, 5))
    taus = np.sort(rng.uniform(1, 10, int(rng.integers(3, 8))))[::-1]
    _, F = sched.lpt(taus, P)
    opt = sched.brute_opt_sequential(taus, P)
    assert F.max() <= (4 / 3 - 1 / (3 * P)) * opt + 1e-12
    assert F.max() >= opt - 1e-12


@pytest.mark.parametrize("seed", range(8))
def test_part_schedule_bound_vs_brute_force(seed):
    rng = np.random.default_rng(100 + seed)
    P = int(rng.integers(2, 4))
    W = np.sort(rng.uniform(1, 20, int(rng.integers(2, 5))) ** 2)[::-1]
    Pi, rows, cmax = sched.part_schedule(W, P)
    opt = sched.brute_opt_moldable(list(W), P)
    assert cmax <= 2 / (1 - 1 / P) * opt + 1e-9
    assert cmax >= opt - 1e-9
    assert Pi[Pi > 1].sum() <= P


def test_part_schedule_single_task_uses_all_processors():
    Pi, rows, cmax = sched.part_schedule(np.array([100.0]), 7)
    # one task alone: the increments stop when sum P_i would exceed P
    assert Pi[0] == 7 and abs(cmax - 100 / 7) < 1e-12


def test_approximate_squares():
    seq = [1]
    for _ in range(12):
        seq.append(sched.next_approx_square(seq[-1]))
    assert seq == [1, 2, 4, 6, 9, 12, 16, 20, 25, 30, 36, 42, 49]


def test_modified_vs_original_on_interposer_shape():
    """Sec. III-C-2: one task carries ~53% of the internal work and 128 tasks 0.30-0.43% each;
    the modified Part_Schedule keeps P_i above P_cutoff = 20 on approximate squares and its
    schedule stays within 15% of the original's."""
    rng = np.random.default_rng(7)
    small = rng.uniform(0.30, 0.43, 128)
    W = np.concatenate([[small.sum() * 53 / 47], small])
    W = np.sort(W)[::-1]
    worst = 0.0
    for P in (20, 40, 80, 160, 320, 640, 1000):
        Pm, _, cm = sched.part_schedule(W, P, p_cutoff=20)
        Po, _, co = sched.part_schedule(W, P)
        assert all(sched.is_approx_square(int(p)) for p in Pm if p > 20)
        assert Pm[Pm > 1].sum() <= P
        worst = max(worst, cm / co - 1)
    assert worst < 0.15



def test_modified_vs_original_on_srr_array_shape():
    """Sec. III-C-2 and the schedule-length comparison of Sec. IV-C's split-ring array: 1,488
    objects of three element sizes (scale 1, 1/2, 1/4) and 1,281,975 edges in all. Reading: a
    third of the objects per size, edges in proportion to the element's scale (a ring meshed at
    a fixed number of elements per unit length), 2% seeded jitter. Both algorithms stay above
    the ideal length sum W / P (a lower bound) and within 15% of each other; with these many
    similar objects few get more than one process and the two schedules coincide."""
    rng = np.random.default_rng(11)
    per = 1281975 / (496 * 1.75)
    n = np.concatenate([np.full(496, per * f) for f in (1.0, 0.5, 0.25)])
    W = np.sort(np.round(n * rng.uniform(0.98, 1.02, 1488)) ** 2)[::-1]
    for P in (40, 160, 640, 1280):
        Pm, _, cm = sched.part_schedule(W, P, p_cutoff=20)
        Po, _, co = sched.part_schedule(W, P)
        ideal = W.sum() / P
        assert cm >= ideal * (1 - 1e-12) and co >= ideal * (1 - 1e-12)
        assert cm / co - 1 < 0.15
        assert all(sched.is_approx_square(int(p)) for p in Pm if p > 20)


def bus_rows():
    """The high-speed bus structures of Sec. IV-B (tests/golden/bus_processes_per_conductor.txt):
    (conductors, P, N_E) per row."""
    path = os.path.join(os.path.dirname(__file__), "golden", "bus_processes_per_conductor.txt")
    rows = []
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            pairs, P, ne = (int(v) for v in line.split())
            rows.append((2 * pairs, P, ne))
    return rows


def test_bus_two_processes_per_conductor():
    """Sec. IV-B: on the buses of identical conductors, the modified Part_Schedule (P_cutoff =
    20, Sec. III-C-2) with the printed P assigns two processes to every conductor. The table's
    N_E is the same per conductor in every row (identical conductors: W_i = N_E,i^2 equal)."""
    rows = bus_rows()
    assert len(rows) == 7
    per = {ne // nc for nc, _, ne in rows}
    assert per == {7026} and all(ne % nc == 0 for nc, _, ne in rows)
    for nc, P, ne in rows:
        W = np.full(nc, float(ne // nc) ** 2)
        Pi, sched_rows, cmax = sched.part_schedule(W, P, p_cutoff=20)
        assert np.all(Pi == 2), (nc, P)
        assert cmax == W[0] / 2
        assert all(len(r) == 1 for r in sched_rows)  # one conductor per process
