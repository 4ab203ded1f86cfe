"""Pins of the log-odds occupancy oracle (Sec. III-A): closed forms for runs of hits and
misses, the clamps, the threshold, and the reduction to the one-hit rule of a cleared map."""
import numpy as np

from oracle import logodds


def run(seq, **p):
    L = np.zeros(len(seq[0]), np.int8)
    occ = None
    for hit in seq:
        L, occ = logodds.update(L, hit, **p)
    return L, occ


P = dict(l_hit=9, l_miss=4, l_min=-20, l_max=40, threshold=15)


def test_runs_of_hits_and_misses_in_closed_form():
    for n in range(0, 8):
        L, occ = run([np.ones(1)] * max(n, 1) if n else [np.zeros(1)], **P)
        expect = min(9 * n, 40) if n else -4
        assert int(L[0]) == expect and int(occ[0]) == (expect >= 15)
    for n in range(1, 12):
        L, _ = run([np.zeros(1)] * n, **P)
        assert int(L[0]) == max(-4 * n, -20)


def test_threshold_needs_two_hits_and_decays_after_misses():
    p = dict(P, threshold=13)
    hits = [np.array([1, 1, 0]), np.array([1, 0, 0]), np.array([0, 0, 0]), np.array([0, 0, 0])]
    L = np.zeros(3, np.int8)
    occs = []
    for h in hits:
        L, occ = logodds.update(L, h, **p)
        occs.append(occ.tolist())
    # voxel 0: 9, 18, 14, 10 (occupied from the second hit, through one miss); voxel 1: 9, 5, 1, -3
    assert occs == [[0, 0, 0], [1, 0, 0], [1, 0, 0], [0, 0, 0]]


def test_clamps_hold_at_the_int8_ends():
    p = dict(l_hit=100, l_miss=100, l_min=-128, l_max=127, threshold=1)
    L, occ = run([np.ones(1)] * 5, **p)
    assert int(L[0]) == 127 and int(occ[0]) == 1
    L, occ = logodds.update(L, np.zeros(1), **p)
    L, occ = logodds.update(L, np.zeros(1), **p)
    L, occ = logodds.update(L, np.zeros(1), **p)
    assert int(L[0]) == -128 and int(occ[0]) == 0


def test_one_hit_rule_of_a_cleared_map():
    rng = np.random.default_rng(0)
    p = dict(l_hit=1, l_miss=1, l_min=0, l_max=1, threshold=1)
    L = np.zeros(1000, np.int8)
    for _ in range(5):
        hit = (rng.random(1000) < 0.3).astype(np.uint8)
        L, occ = logodds.update(L, hit, **p)
        assert np.array_equal(occ, hit)
