"""cc_renumber_noalloc: the output renumbering for callers that cannot
allocate device memory (for instance code running under a framework whose
memory pool already holds the GPU, or a latency-bound path that must not pay
for cudaMalloc).  It must give exactly what cc_consensus_labels gives, call
after call, although every call reuses the same built-in scratch array.

This file is collected last on purpose (its name sorts last)."""
import numpy as np
import pytest

import oracle

from workloads import make_config

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cc():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2408_11331_gb300 as m

    return m


def _converged_job(cc, c):
    job = cc.Consensus(c["row_off"], c["col"], c["labels"])
    job.run_until_converged(20)
    return job


def test_noalloc_matches_consensus_labels_two_calls_in_a_row(cc):
    torch = pytest.importorskip("torch")
    from paper_2408_11331_gb300 import _native

    # a larger job first, then a smaller one: the second call must not see
    # anything the first left in the shared scratch
    jobs = [make_config("lfr", n=20000, k=8, cmin=20, cmax=1000, max_deg=500, seed=11),
            make_config("sbm", n=1000, k=10)]
    stream = torch.cuda.Stream()
    for c in jobs:
        n = c["labels"].shape[1]
        job = _converged_job(cc, c)
        try:
            want = job.consensus_labels()            # the existing entry point
            ids_ptr = job.cluster_ids_dev()
            out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
            torch.cuda.synchronize()
            _native.cc_renumber_noalloc(n, ids_ptr, out.data_ptr(), stream.cuda_stream)
            got = out.cpu().numpy()
            np.testing.assert_array_equal(got, want)
            assert got.max() + 1 == len(np.unique(job.cluster_ids()))
        finally:
            job.close()


def test_noalloc_rejects_bad_sizes_and_ids(cc):
    torch = pytest.importorskip("torch")
    from paper_2408_11331_gb300 import _native

    buf = torch.zeros(16, dtype=torch.int32, device="cuda")
    for n in (0, _native.CC_NOALLOC_MAX_N + 1):
        with pytest.raises(cc.CCError) as e:
            _native.cc_renumber_noalloc(n, buf.data_ptr(), buf.data_ptr())
        assert e.value.status == 1
    assert str(_native.CC_NOALLOC_MAX_N) in _native.cc_last_error()
    ids = torch.tensor([0, 1, 16, 2], dtype=torch.int32, device="cuda")  # 16 is outside [0, 4)
    out = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(cc.CCError) as e:
        _native.cc_renumber_noalloc(4, ids.data_ptr(), out.data_ptr())
    assert e.value.status == 1
    # a valid call right after the rejected one
    ids = torch.tensor([3, 3, 1, 3], dtype=torch.int32, device="cuda")
    _native.cc_renumber_noalloc(4, ids.data_ptr(), out.data_ptr())
    assert out.cpu().tolist() == [0, 0, 1, 0]


def _first_appearance(ids):
    """First-appearance renumbering written out with numpy (the reference)."""
    _, first = np.unique(ids, return_index=True)
    order = np.argsort(first, kind="stable")
    rank = np.empty(len(first), np.int64)
    rank[order] = np.arange(len(first))
    _, inv = np.unique(ids, return_inverse=True)
    return rank[inv].astype(np.int32)


def test_noalloc_at_the_size_limit(cc):
    """n = CC_NOALLOC_MAX_N (more than 1024 blocks of 1024 ids, so the block
    counts are scanned several per thread) and n just above 2^20, with
    random ids in [0, n), against a numpy first-appearance renumbering and
    the oracle's renumbering."""
    torch = pytest.importorskip("torch")
    from paper_2408_11331_gb300 import _native

    rng = np.random.default_rng(7)
    for n in (_native.CC_NOALLOC_MAX_N, (1 << 20) + 1):
        ids = rng.integers(0, n, n).astype(np.int32)
        want = _first_appearance(ids)
        np.testing.assert_array_equal(want, oracle.renumber(ids))
        d_ids = torch.from_numpy(ids).cuda()
        out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        _native.cc_renumber_noalloc(n, d_ids.data_ptr(), out.data_ptr())
        np.testing.assert_array_equal(out.cpu().numpy(), want)


def test_noalloc_on_batch_union_ids(cc):
    """A batch's cluster ids are union ids: the renumbering numbers the
    clusters of all jobs together, job after job, so each job's slice is its
    own labels (cc_job_labels) shifted by the clusters of the earlier jobs."""
    torch = pytest.importorskip("torch")
    from paper_2408_11331_gb300 import _native

    cs = [make_config("sbm", n=1000, k=10), make_config("lfr", n=5000, k=6, cmin=20, cmax=500, max_deg=200, seed=5)]
    with cc.ConsensusBatch([(c["row_off"], c["col"], c["labels"]) for c in cs]) as b:
        b.run_until_converged(20)
        N = int(b.offsets[-1])
        ptr = _native.cc_cluster_ids_dev(b._ctx)
        out = torch.full((N,), -1, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        _native.cc_renumber_noalloc(N, ptr, out.data_ptr())
        got = out.cpu().numpy()
        shift = 0
        for j in range(len(cs)):
            lab = b.labels(j)
            np.testing.assert_array_equal(got[b.offsets[j]:b.offsets[j + 1]], lab + shift)
            shift += int(lab.max()) + 1
