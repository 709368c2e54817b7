"""Pins of the oracle's random search (Sec. IV-A: a random 20% of the grid,
early stop on an NCC threshold) against facts outside its own code:

- SplitMix64 against the published test vectors of its reference
  implementation (Steele, Lea and Flood, OOPSLA 2014; the values printed by
  Vigna's splitmix64.c for seeds 0 and 1234567);
- the Fisher-Yates order is a permutation and is uniform over the n!
  orderings (chi-square on n = 4; a j = x mod i off-by-one makes some
  orderings impossible);
- with no threshold and the whole grid the search is the full sweep's argmax
  (brute force over every cell); a -inf threshold stops after one batch; a
  noise-free query at a cell's own pose is found with NCC 1 and stops the
  search in that cell's batch.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
import scenegen as sg


def test_splitmix64_published_vectors():
    assert [int(x) for x in oracle.splitmix64(0, 2)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4]
    assert [int(x) for x in oracle.splitmix64(1234567, 3)] == [6457827717110365317, 3203168211198807973,
                                                             9817491932198370423]


@pytest.mark.parametrize("n", [1, 2, 7, 100, 8100])
def test_search_order_is_a_permutation(n):
    for seed in (0, 1, 2**63 + 5):
        o = oracle.search_order(seed, n)
        assert sorted(o.tolist()) == list(range(n))


def test_search_order_uniform_over_orderings():
    n, trials = 4, 24000
    counts = {p: 0 for p in itertools.permutations(range(n))}
    for seed in range(trials):
        counts[tuple(oracle.search_order(seed, n).tolist())] += 1
    expect = trials / math.factorial(n)
    chi2 = sum((c - expect) ** 2 / expect for c in counts.values())
    assert min(counts.values()) > 0
    assert chi2 < 60.0          # 23 degrees of freedom: P(chi2 > 60) < 1e-4


def test_visit_count():
    assert oracle.visit_count(0.2, 8100) == 1620
    assert oracle.visit_count(1.0, 64) == 64
    assert oracle.visit_count(1e-9, 64) == 1


@pytest.fixture(scope="module")
def small():
    s = sg.tiny_scene()
    cells = oracle.grid_poses(s.seed_pose, 5, 5, 4, 0.25, 2.0)
    query = (oracle.render(s.gaussians, s.hidden_pose, s.camera)["rgb"] + s.query_noise).astype(np.float32)
    return s, cells, query


def test_full_visit_without_threshold_is_the_sweep(small):
    s, cells, query = small
    full = oracle.render_views(s.gaussians, cells, s.camera, query=query, images=False, flags=False)["scores"]
    order = oracle.search_order(3, len(cells))
    r = oracle.random_search(s.gaussians, cells, s.camera, query, order, 16, np.inf)
    assert r["best_index"] == oracle.argmax(full)
    assert r["n_scored"] == len(cells) and not r["stopped_early"]
    np.testing.assert_array_equal(r["scores"], full)


def test_minus_inf_threshold_stops_after_one_batch(small):
    s, cells, query = small
    order = oracle.search_order(4, len(cells))[:40]
    r = oracle.random_search(s.gaussians, cells, s.camera, query, order, 16, -np.inf)
    assert r["n_scored"] == 16 and r["stopped_early"]
    first = order[:16]
    sc = r["scores"][first]
    assert r["best_index"] == int(first[np.lexsort((first, -sc))[0]])
    assert np.isnan(np.delete(r["scores"], first)).all()


def test_exact_query_found_and_stops(small):
    s, cells, _ = small
    target = 37
    query = oracle.render(s.gaussians, cells[target], s.camera)["rgb"].astype(np.float32)
    order = oracle.search_order(5, len(cells))
    pos = int(np.nonzero(order == target)[0][0])
    r = oracle.random_search(s.gaussians, cells, s.camera, query, order, 10, 0.999)
    assert r["best_index"] == target
    assert abs(r["best_score"] - 1.0) < 1e-6
    assert r["n_scored"] == min(len(order), (pos // 10 + 1) * 10)
