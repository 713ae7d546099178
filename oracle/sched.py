"""Task scheduling for the internal workloads (Sec. III-C). Test infrastructure (oracle).

* LPT (Alg. 1): tasks sorted by decreasing duration; each goes to the processor with the
  earliest finish time F_p (Eq. F_comptime). Worst case R = 4/3 - 1/(3P) (Eq. R_LPT).
* Moldable tasks: task i runs on P_i processors for tau_i = W_i / P_i, W_i = N_E,i^2 (Sec. III-C-2).
  Parallel tasks (P_i > 1) are placed first, all starting together on dedicated processors,
  which needs sum_{P_i > 1} P_i <= P; sequential tasks then follow by LPT.
* Part_Schedule (Belkhale 1990) and the modified Part_Schedule (Alg. 2) that restricts
  P_i >= P_cutoff to approximate squares Q^2 or Q(Q + 1). Worst case R = 2/(1 - 1/P) (Eq. R_part).

Readings of Alg. 2 (the listing is terse): "P_i < P_cutoff" takes d = 1; otherwise d is the
distance to the next approximate square above P_i; ties in tau or in F_p go to the lowest
index; the comparison "C_max != h" is exact on identical floating-point arithmetic. An
increment is undone, and the algorithm ends, when the new schedule is longer than the current
one (the termination rule stated in Sec. III-C); the listing's "not shorter" test would stop
at the first tie, whereas Sec. IV-B reports two processes per conductor for its buses of
identical conductors with P = 2 per conductor, which only the strict test gives.
"""
from __future__ import annotations

import itertools

import numpy as np


def lpt(taus, P):
    """Alg. 1 on sequential tasks already sorted by decreasing tau. Returns (rows, F)."""
    F = np.zeros(P)
    rows = [[] for _ in range(P)]
    for i, t in enumerate(taus):
        p = int(np.argmin(F))
        rows[p].append(i)
        F[p] += t
    return rows, F


def lpt_moldable(W, Pi, P):
    """Mixed schedule: parallel tasks first on dedicated processors (all start at t = 0), then
    the sequential tasks by LPT over all P processors. Tasks are indexed as given (the caller
    keeps them sorted by decreasing tau at P_i = 1). Returns (rows, F)."""
    W = np.asarray(W, dtype=np.float64)
    Pi = np.asarray(Pi, dtype=np.int64)
    F = np.zeros(P)
    rows = [[] for _ in range(P)]
    nxt = 0
    for i in np.nonzero(Pi > 1)[0]:
        for p in range(nxt, nxt + Pi[i]):
            rows[p].append(int(i))
            F[p] = W[i] / Pi[i]
        nxt += Pi[i]
    seq = [int(i) for i in np.nonzero(Pi == 1)[0]]
    seq.sort(key=lambda i: (-W[i], i))
    for i in seq:
        p = int(np.argmin(F))
        rows[p].append(i)
        F[p] += W[i]
    return rows, F


def is_approx_square(n):
    q = int(np.floor(np.sqrt(n)))
    return q * q == n or q * (q + 1) == n


def next_approx_square(n):
    m = n + 1
    while not is_approx_square(m):
        m += 1
    return m


def part_schedule(W, P, p_cutoff=None):
    """Alg. 2 (modified Part_Schedule); p_cutoff=None gives the original Part_Schedule.

    W must be sorted in decreasing order. Returns (Pi, rows, C_max)."""
    W = np.asarray(W, dtype=np.float64)
    Pi = np.ones(W.size, dtype=np.int64)
    a = P
    rows, F = lpt_moldable(W, Pi, P)
    cmax = F.max()
    while a > 0:
        tau = W / Pi
        i = int(np.argmax(tau))
        h = tau[i]
        if p_cutoff is None or Pi[i] < p_cutoff:
            d = 1
        else:
            d = next_approx_square(int(Pi[i])) - int(Pi[i])
        a = a - d - 1 if Pi[i] == 1 else a - d
        if cmax != h or a < 0:
            break
        Pi[i] += d
        rows2, F2 = lpt_moldable(W, Pi, P)
        if F2.max() > cmax:
            Pi[i] -= d
            break
        rows, F, cmax = rows2, F2, F2.max()
    return Pi, rows, cmax


def brute_opt_sequential(taus, P):
    """Optimal makespan of sequential tasks on P processors by exhaustive assignment."""
    best = np.inf
    for assign in itertools.product(range(P), repeat=len(taus)):
        F = np.zeros(P)
        for t, p in zip(taus, assign):
            F[p] += t
        best = min(best, F.max())
    return best


def brute_opt_moldable(W, P):
    """Optimal makespan of moldable tasks (tau_i = W_i / P_i) on P processors.

    Every P_i vector and every task order is tried with the serial schedule-generation scheme
    (each task starts at the earliest time P_i processors are free for tau_i); the set of such
    schedules contains an optimal one."""
    n = len(W)
    best = np.inf
    for Pi in itertools.product(range(1, P + 1), repeat=n):
        for order in itertools.permutations(range(n)):
            busy = []  # (start, end, procs)
            for i in order:
                dur = W[i] / Pi[i]
                cands = sorted({0.0} | {e for (_, e, _) in busy})
                for s in cands:
                    ok = True
                    pts = sorted({s} | {b for (b, _, _) in busy if s < b < s + dur})
                    for tpt in pts:
                        used = sum(p for (b, e, p) in busy if b <= tpt < e)
                        if used + Pi[i] > P:
                            ok = False
                            break
                    if ok:
                        busy.append((s, s + dur, Pi[i]))
                        break
            best = min(best, max(e for (_, e, _) in busy))
    return best
