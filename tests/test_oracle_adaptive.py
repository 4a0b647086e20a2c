"""Pins of the oracle's adaptive walk counts (Sec. 5.1, Eq. lengthdelta), CPU
only: on a row whose walk lengths have a closed-form law the counts settle
where z^2 Var / (Delta^2 mean^2) puts them and scale as Delta^-2; the counts
replay, round by round, from the lengths of the factor walks that
build_factor runs with them (so the adaptive walks are the factor walks);
the bounds (min, max, rounds, rows without walks) hold; and a schedule that
runs walks past each decision point and replays the decisions in walk order
(the GPU's launch rounds) reaches the same counts in fewer rounds."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from workloads import assemble


def _forced_path():
    # Path 0-1-2 without excess at nodes 1 and 2: walks from row 1 have
    # lengths 1 + 2J with J geometric on 1, 2, ... (p = 1/4), so
    # mean 1 + 2/p = 9 and variance 4 (1 - p) / p^2 = 48.
    return assemble(3, np.array([0, 1]), np.array([1, 2]), np.array([1.0, 3.0]), np.array([1.0, 0.0, 0.0]))


def test_forced_row_settles_at_the_closed_form_count():
    A = _forced_path()
    z = 1.959963984540054            # two-sided 95 %
    means = {}
    for delta in (0.1, 0.05):
        target = z * z * 48.0 / (delta * delta * 81.0)
        got = []
        for seed in range(40):
            b, rounds = oracle.adaptive_budget(A, seed, delta, z, min_walks=20, max_walks=65535, max_rounds=16)
            assert b[2] == 0 and rounds <= 16
            got.append(int(b[1]))
        m = float(np.mean(got))
        # the stopping rule acts on sample estimates and overshoots a little:
        # the mean count sits slightly above the closed form, never below 0.9 of it
        assert 0.9 * target < m < 1.35 * target, (delta, m, target)
        means[delta] = m
    assert 3.2 < means[0.05] / means[0.1] < 4.8


def _replay(lengths, delta, z, min_walks, max_walks, max_rounds):
    """Rounds of Sec. 5.1 replayed from a row's recorded factor-walk lengths:
    returns the count at which they stop (None if more lengths are needed)."""
    d2, z2 = delta * delta, z * z
    m, inc = 0, min_walks
    for _ in range(max_rounds):
        if inc == 0:
            break
        m += inc
        inc = 0
        if m > len(lengths):
            return None
        if 1 < m < max_walks:
            L = lengths[:m].astype(np.uint64)
            s1, s2 = int(L.sum()), int((L * L).sum())
            mean = float(s1) / float(m)
            var = (float(s2) - float(s1) * mean) / (float(m) - 1.0)
            lhs, rhs = d2 * (mean * mean) * float(m), z2 * var
            if not lhs > rhs:
                need = rhs / (d2 * (mean * mean))
                target = max_walks if need >= max_walks else int(math.ceil(need))
                inc = max(target, m + 1) - m
    return m


@pytest.mark.parametrize("case", range(3))
def test_counts_replay_from_the_factor_walks(case):
    rng = np.random.default_rng(70 + case)
    A = [W.grid2d_5pt(9, 7), W.random_rmatrix(30, rng), W.rgg(200, rng)][case]
    delta, z, mn, mx, rounds = 0.15, 1.6448536269514722, 8, 3000, 6
    b, r = oracle.adaptive_budget(A, 5 + case, delta, z, min_walks=mn, max_walks=mx, max_rounds=rounds)
    wr = oracle.walk_rows(A)
    assert np.all(b[wr] >= mn) and np.all(b[wr] <= mx)
    assert np.all(np.delete(b, wr) == 0)
    assert 1 <= r <= rounds
    F = oracle.build_factor(A, b, 5 + case, 0.0, records=True)
    off = np.concatenate([[0], np.cumsum(b[wr].astype(np.int64))])
    more = 0
    for i, k in enumerate(wr):
        lens = F["rec_len"][off[i]:off[i + 1]]
        assert _replay(lens, delta, z, mn, mx, rounds) == b[k], k
        more += int(b[k] > mn)
    assert more > 0          # some rows did take further rounds


def test_single_round_and_caps():
    A = W.grid2d_5pt(6, 5)
    wr = oracle.walk_rows(A)
    b, r = oracle.adaptive_budget(A, 3, 0.01, 3.0, min_walks=17, max_walks=4000, max_rounds=1)
    assert r == 1 and np.all(b[wr] == 17)
    # a tiny Delta asks for far more than the cap on every row whose first
    # walks do not all have the same length (zero sample variance stops at once)
    b, r = oracle.adaptive_budget(A, 3, 1e-4, 3.0, min_walks=5, max_walks=40, max_rounds=8)
    assert r == 2 and set(b[wr].tolist()) <= {5, 40} and np.sum(b[wr] == 40) > len(wr) // 2
    F = oracle.build_factor(A, b, 3, 0.0, records=True)
    off = np.concatenate([[0], np.cumsum(b[wr].astype(np.int64))])
    for i, k in enumerate(wr):
        lens = F["rec_len"][off[i]:off[i + 1]]
        assert (b[k] == 5) == (np.ptp(lens[:5]) == 0), k
    # a huge Delta is met at once
    b, r = oracle.adaptive_budget(A, 3, 1e3, 1.0, min_walks=5, max_walks=40, max_rounds=8)
    assert np.all(b[wr] == 5) and r == 1


def test_rejects_bad_arguments():
    A = W.grid2d_5pt(4, 4)
    for kw in (dict(delta=0.0), dict(z=-1.0), dict(min_walks=1), dict(max_walks=3),
               dict(max_walks=70000), dict(max_rounds=0)):
        args = dict(delta=0.1, z=2.0, min_walks=4, max_walks=100, max_rounds=4)
        args.update(kw)
        with pytest.raises(oracle.OracleError):
            oracle.adaptive_budget(A, 1, **args)


def _run_ahead_schedule(lengths, min_walks, max_walks, max_rounds, d2, z2, ahead):
    """Host model of the GPU's launch rounds for one row (test only): each
    round runs the row's walks up to `ahead` percent past its next decision
    point and replays the decisions in walk order over the lengths run.
    Returns (count, decisions, launch rounds)."""
    a = s1 = s2 = d = 0
    t = min_walks
    launches = 0
    while True:
        a1 = min(max_walks, t + t * ahead // 100)
        launches += 1
        while True:
            if a == t:
                d += 1
                nt = 0
                if 1 < t < max_walks:
                    mean = s1 / t
                    var = (s2 - s1 * mean) / (t - 1.0)
                    lhs = d2 * (mean * mean) * t
                    rhs = z2 * var
                    if not lhs > rhs:
                        need = rhs / (d2 * (mean * mean))
                        nt = max_walks if need >= max_walks else math.ceil(need)
                        nt = max(nt, t + 1)
                if nt == 0 or d >= max_rounds:
                    return t, d, launches
                t = nt
                continue
            if a == a1:
                break
            e = min(t, a1)
            seg = lengths[a:e].astype(np.uint64)
            s1 += int(seg.sum())
            s2 += int((seg * seg).sum())
            a = e


@pytest.mark.parametrize("ahead", [0, 30, 100, 400])
def test_run_ahead_rounds_give_the_oracle_counts(ahead):
    """Running walks past a row's next decision point and replaying the
    decisions in walk order (the GPU's launch rounds) gives the counts and the
    decision count of one decision per round: the walk lengths come from the
    oracle's factor walks, the counts from the oracle's adaptive rule."""
    rng = np.random.default_rng(77)
    A = W.grid3d(5, 4, 4, 27, rng, excess_frac=1e-3)
    delta, z, mn, mx, rounds = 0.15, 2.576, 8, 300, 10
    ref, rr = oracle.adaptive_budget(A, 5, delta, z, min_walks=mn, max_walks=mx, max_rounds=rounds)
    F = oracle.build_factor(A, mx, 5, 0.0, records=True)
    wr = F["walk_rows"]
    dmax, launches = 0, 0
    for i, k in enumerate(wr):
        lengths = F["rec_len"][i * mx:(i + 1) * mx]
        cnt, dec, lr = _run_ahead_schedule(lengths, mn, mx, rounds, delta * delta, z * z, ahead)
        assert cnt == ref[k], (k, cnt, ref[k])
        dmax, launches = max(dmax, dec), max(launches, lr)
    assert dmax == rr
    assert launches <= rr
    if ahead == 0:
        assert launches == rr
