"""Pins of the oracle's partition distances (Methods, Evaluation metrics):
Mirkin / Rand distance, split-join distance, variation of information."""
import json
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _m(X, Y):
    """Distances between partition X (as the consensus) and Y (as the one input partition)."""
    return {k: v[0] for k, v in oracle.metrics(np.asarray([Y], np.int32), np.asarray(X, np.int32)).items()}


def test_hand_worked_example():
    g = json.load(open(os.path.join(GOLDEN, "metrics_example.json")))
    m = _m(g["X"], g["Y"])
    assert m["mirkin"] == g["mirkin"]
    assert m["split_join"] == g["split_join"]
    assert m["rand_distance"] == pytest.approx(g["rand_distance"], abs=1e-15)
    assert m["vi"] == pytest.approx(g["vi"], abs=1e-12)


@pytest.mark.parametrize("case", range(2))
def test_hand_worked_tied_overlaps(case):
    """Split-join with tied largest overlaps (each tie counts its value once)."""
    g = json.load(open(os.path.join(GOLDEN, "metrics_ties.json")))["cases"][case]
    m = _m(g["X"], g["Y"])
    assert m["mirkin"] == g["mirkin"]
    assert m["split_join"] == g["split_join"]
    assert m["rand_distance"] == pytest.approx(g["rand_distance"], abs=1e-15)
    assert m["vi"] == pytest.approx(g["vi"], abs=1e-12)
    # the distances are symmetric in X and Y
    r = _m(g["Y"], g["X"])
    assert (r["mirkin"], r["split_join"]) == (g["mirkin"], g["split_join"])
    assert r["vi"] == pytest.approx(g["vi"], abs=1e-12)


def _random_partition(rng, n, parts):
    return rng.integers(0, parts, n).astype(np.int32)


@pytest.mark.parametrize("seed", range(6))
def test_mirkin_is_pair_count_and_sums_to_objective(seed):
    rng = np.random.default_rng(seed)
    n, k = 60, 4
    labels = np.stack([_random_partition(rng, n, rng.integers(2, 9)) for _ in range(k)])
    C = _random_partition(rng, n, 7)
    m = oracle.metrics(labels, C)
    for i in range(k):
        assert m["mirkin"][i] == oracle.mirkin_pairs(C, labels[i])
    assert int(m["mirkin"].sum()) == oracle.objective(labels, C)


@pytest.mark.parametrize("seed", range(6))
def test_rand_and_vi_against_library_definitions(seed):
    skm = pytest.importorskip("sklearn.metrics")
    from scipy.stats import entropy

    rng = np.random.default_rng(100 + seed)
    n = 200
    X = _random_partition(rng, n, rng.integers(1, 15))
    Y = _random_partition(rng, n, rng.integers(1, 15))
    m = _m(X, Y)
    assert m["rand_distance"] == pytest.approx(1.0 - skm.rand_score(X, Y), abs=1e-12)
    hx = entropy(np.unique(X, return_counts=True)[1])
    hy = entropy(np.unique(Y, return_counts=True)[1])
    vi = hx + hy - 2 * skm.mutual_info_score(X, Y)
    assert m["vi"] == pytest.approx(vi, abs=1e-10)


def test_split_join_closed_forms():
    n = 37
    singles = np.arange(n, dtype=np.int32)
    whole = np.zeros(n, np.int32)
    assert _m(singles, singles)["split_join"] == 0
    assert _m(singles, whole)["split_join"] == n - 1
    assert _m(whole, singles)["split_join"] == n - 1
    assert _m(whole, whole)["vi"] == 0.0
    assert _m(singles, whole)["vi"] == pytest.approx(np.log(n), abs=1e-12)
    assert _m(singles, whole)["mirkin"] == n * (n - 1)


@pytest.mark.parametrize("seed", range(8))
def test_metric_axioms(seed):
    """Symmetry, identity and the triangle inequality of all three distances,
    and invariance to relabelling."""
    rng = np.random.default_rng(200 + seed)
    n = 80
    X, Y, Z = (_random_partition(rng, n, rng.integers(1, 12)) for _ in range(3))
    xy, yx, yz, xz = _m(X, Y), _m(Y, X), _m(Y, Z), _m(X, Z)
    for key in ("mirkin", "split_join"):
        assert xy[key] == yx[key]
        assert xz[key] <= xy[key] + yz[key]
        assert _m(X, X)[key] == 0
    assert xy["vi"] == pytest.approx(yx["vi"], abs=1e-12)
    assert xz["vi"] <= xy["vi"] + yz["vi"] + 1e-12
    perm = rng.permutation(1000)
    Xr = perm[X].astype(np.int32)
    assert _m(Xr, Y)["split_join"] == xy["split_join"]
    assert _m(Xr, Y)["vi"] == pytest.approx(xy["vi"], abs=1e-12)
