"""The seeded input generators (workloads/) against the recipe they state:
CSR form, realised mean degree and mixing of the LFR-style graphs, the
resolutions of the graded kNN partitions, and the steps of the perturbation
that makes input partitions.  Host only."""
import numpy as np
import pytest

from workloads import csr_from_edges, lfr_like, make_config, perturb
from workloads.configs import graded_partitions
from workloads.graphs import sbm


def _check_csr(row_off, col, n):
    assert row_off.dtype == np.int64 and col.dtype == np.int32
    assert row_off[0] == 0 and row_off[-1] == len(col) and np.all(np.diff(row_off) >= 0)
    src = np.repeat(np.arange(n), np.diff(row_off))
    assert np.all(col >= 0) and np.all(col < n)
    assert not np.any(src == col)  # no self-loops
    for v in range(0, n, max(1, n // 200)):  # sorted, no repeats
        nb = col[row_off[v]:row_off[v + 1]]
        assert np.all(np.diff(nb) > 0)
    fwd = np.sort(src.astype(np.int64) * n + col)
    back = np.sort(col.astype(np.int64) * n + src)
    np.testing.assert_array_equal(fwd, back)  # symmetric


def test_csr_from_edges_matches_sets():
    rng = np.random.default_rng(5)
    n = 60
    u = rng.integers(0, n, 400)
    v = rng.integers(0, n, 400)
    row_off, col = csr_from_edges(n, u, v)
    _check_csr(row_off, col, n)
    want = [set() for _ in range(n)]
    for a, b in zip(u.tolist(), v.tolist()):
        if a != b:
            want[a].add(b)
            want[b].add(a)
    for x in range(n):
        assert col[row_off[x]:row_off[x + 1]].tolist() == sorted(want[x])


def test_lfr_like_mean_degree_and_mixing():
    """The LFR-style graph reaches its stated mean degree (the second draw
    makes up for the dropped repeats) and about a share mu of each vertex's
    edges leave its community."""
    n, avg, mu = 20000, 20.0, 0.3
    row_off, col, truth = lfr_like(n, avg, 500, 2.5, 1.5, 20, 1000, mu, np.random.default_rng(7))
    _check_csr(row_off, col, n)
    assert abs(len(col) / n - avg) < 0.05 * avg
    src = np.repeat(np.arange(n), np.diff(row_off))
    external = float(np.mean(truth[src] != truth[col]))
    assert abs(external - mu) < 0.05
    sizes = np.bincount(truth)
    assert sizes.min() >= 20


def test_lfr_like_deterministic():
    a = lfr_like(3000, 12.0, 200, 2.5, 1.5, 20, 300, 0.2, np.random.default_rng(3))
    b = lfr_like(3000, 12.0, 200, 2.5, 1.5, 20, 300, 0.2, np.random.default_rng(3))
    c = lfr_like(3000, 12.0, 200, 2.5, 1.5, 20, 300, 0.2, np.random.default_rng(4))
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
    assert not np.array_equal(a[1], c[1])


def test_sbm_config_shapes_and_seed():
    a = make_config("sbm")
    b = make_config("sbm")
    assert a["labels"].shape == (10, 1000) and a["labels"].dtype == np.int32
    _check_csr(a["row_off"], a["col"], 1000)
    np.testing.assert_array_equal(a["col"], b["col"])
    np.testing.assert_array_equal(a["labels"], b["labels"])
    assert a["seed"] == 0x5EED
    c = make_config("sbm", seed=1)
    assert not np.array_equal(a["col"], c["col"])


def test_sbm_block_densities():
    """Planted-partition densities: edges inside a block at rate p_in,
    between blocks at p_out."""
    rng = np.random.default_rng(11)
    sizes = [200] * 10
    row_off, col, truth = sbm(sizes, 0.1, 0.005, rng)
    n = sum(sizes)
    _check_csr(row_off, col, n)
    src = np.repeat(np.arange(n), np.diff(row_off))
    inside = np.sum(truth[src] == truth[col]) / 2
    between = np.sum(truth[src] != truth[col]) / 2
    pairs_in = 10 * 200 * 199 / 2
    pairs_out = n * (n - 1) / 2 - pairs_in
    assert abs(inside / pairs_in - 0.1) < 0.01
    assert abs(between / pairs_out - 0.005) < 0.001


def _mixture_graph(n=3000, comps=20, dim=8, knn=10, seed=2):
    pytest.importorskip("torch")
    from workloads.graphs import knn_mixture

    rng = np.random.default_rng(seed)
    pts = []
    row_off, col, truth = knn_mixture(n, comps, dim, knn, rng, device="cpu", points_out=pts)
    return row_off, col, truth, pts[0], rng


def test_knn_mixture_graph():
    """Symmetrised exact kNN: every vertex keeps its knn nearest points."""
    row_off, col, truth, x, _ = _mixture_graph(n=800, comps=5, dim=4, knn=6)
    n = len(truth)
    _check_csr(row_off, col, n)
    assert np.all(np.diff(row_off) >= 6)
    for v in range(0, n, 97):
        d = np.sum((x - x[v]) ** 2, axis=1)
        d[v] = np.inf
        near = np.argsort(d, kind="stable")[:6]
        nb = set(col[row_off[v]:row_off[v + 1]].tolist())
        # the k-th distance may tie only by accident in float32 data
        assert set(near.tolist()) <= nb


@pytest.mark.parametrize("K", [10, 30])
def test_graded_partitions_resolution(K):
    """Without the neighbour relabel, a partition at resolution K has exactly
    K labels: K <= components groups whole components; K > components (which
    no grouping of components can reach) cuts components by rank along a
    random projection, so every label stays inside one component."""
    row_off, col, truth, x, rng = _mixture_graph()
    comps = 20
    assert np.all(np.bincount(truth, minlength=comps) > 0)
    lab = graded_partitions(truth, x, comps, row_off, col, 3, rng, kmin=K, kmax=K, relabel=0.0)
    for i in range(3):
        assert len(np.unique(lab[i])) == K
        if K <= comps:  # a component is never split
            for c in range(comps):
                assert len(np.unique(lab[i][truth == c])) == 1
        else:  # each label stays inside one component
            for g in np.unique(lab[i]):
                assert len(np.unique(truth[lab[i] == g])) == 1


def test_perturb_steps():
    rng = np.random.default_rng(9)
    row_off, col, truth = sbm([50] * 8, 0.3, 0.01, rng)
    n = len(truth)
    same = perturb(truth, row_off, col, np.random.default_rng(1), p_merge=0.0, p_split=0.0, rho=(0.0, 0.0))
    np.testing.assert_array_equal(same, truth)
    merged = perturb(truth, row_off, col, np.random.default_rng(1), p_merge=1.0, p_split=0.0, rho=(0.0, 0.0))
    assert len(np.unique(merged)) < len(np.unique(truth))
    for c in range(8):  # a merge keeps communities whole
        assert len(np.unique(merged[truth == c])) == 1
    split = perturb(truth, row_off, col, np.random.default_rng(1), p_merge=0.0, p_split=1.0, rho=(0.0, 0.0))
    for c in range(8):  # every community cut into two halves
        assert sorted(np.bincount(split[truth == c]).tolist())[-2:] == [25, 25]
    relab = perturb(truth, row_off, col, np.random.default_rng(1), p_merge=0.0, p_split=0.0, rho=(0.5, 0.5))
    moved = np.nonzero(relab != truth)[0]
    assert 0 < len(moved) < n
    for v in moved:  # a relabelled vertex carries a neighbour's label
        assert relab[v] in set(truth[col[row_off[v]:row_off[v + 1]]].tolist())
