"""The C-ABI library loads, exports every symbol include/bem_aim.h declares, and its host-only
scheduler (Sec. III-C, Alg. 2) matches the oracle. No GPU needed."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import sched
from paper_2108_03991_gb300 import api, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return api.lib()


def test_header_symbols_exported(L):
    src = open(os.path.join(ROOT, "include", "bem_aim.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b([a-z_][a-z0-9_]*)\s*\(", src)) - {"if", "sizeof", "defined"}
    assert names, "no declarations parsed"
    for n in names:
        assert hasattr(L, n), n
    assert set(api.SYMBOLS) <= names


@pytest.mark.parametrize("cut", [None, 20])
def test_part_schedule_matches_oracle(L, cut):
    rng = np.random.default_rng(3)
    small = rng.uniform(0.30, 0.43, 128)
    W = np.sort(np.concatenate([[small.sum() * 53 / 47], small]))[::-1]
    for P in (20, 40, 80, 160, 320, 640, 1000):
        Pi, cm = api.part_schedule(W, P, cut if cut else 0)
        Po, _, co = sched.part_schedule(W, P, cut)
        assert np.array_equal(Pi, Po)
        assert cm == co


def test_part_schedule_bus_matches_oracle(L):
    """The library's Part_Schedule on the identical-conductor buses of Sec. IV-B: two processes
    per conductor, as the oracle."""
    path = os.path.join(os.path.dirname(__file__), "golden", "bus_processes_per_conductor.txt")
    rows = [tuple(int(v) for v in ln.split()) for ln in open(path) if ln.strip() and ln[0] != "#"]
    assert len(rows) == 7
    for pairs, P, ne in rows:
        nc = 2 * pairs
        W = np.full(nc, float(ne // nc) ** 2)
        Pi, cm = api.part_schedule(W, P, 20)
        assert np.all(Pi == 2) and cm == W[0] / 2


def test_part_schedule_rejects_unsorted(L):
    with pytest.raises(api.BemError):
        api.part_schedule(np.array([1.0, 2.0]), 4)


def test_last_error_empty_string(L):
    assert isinstance(L.bem_last_error(), bytes)
