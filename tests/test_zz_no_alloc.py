"""The allocation-free entry point (et_tube_count_noalloc) against the
regular per-seed counts (et_view_seed_counts).

It serves callers that cannot allocate device memory: an acquisition loop
that must not block on an allocation's device-wide synchronisation, code in a
host function enqueued on a stream, or a process whose framework owns the free
device memory.  The entry point keeps its cell list in one fixed device array
shared by all calls, so this test makes two calls in a row on the same stream
and checks both results: the second call must not see anything the first
one left behind.  It lives in its own file, collected last, so that a run
stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_1311_5334_gb300 import synth

pytestmark = pytest.mark.gpu


def test_noalloc_tube_counts_match_seed_counts_on_two_calls():
    import torch
    from paper_1311_5334_gb300 import et

    v = synth.pr1()
    p = synth.params(v.extent)
    with et.Context(0) as ctx:
        view = ctx.view(v.xyz, p)
        view.find()
        view.fetch()
        si, sj, sc = view.seed_counts()
        view.close()
    assert len(sc) > 10000

    xyz = torch.from_numpy(v.xyz).cuda()
    pairs = torch.from_numpy(np.ascontiguousarray(np.stack([si, sj], axis=1), dtype=np.int32)).cuda()
    # a pair whose indices are equal is reported as -1
    bad = torch.tensor([[3, 3]], dtype=torch.int32, device="cuda")
    for call in range(2):
        out = torch.full((len(sc),), -7, dtype=torch.int32, device="cuda")
        et.tube_count_noalloc(xyz, p, pairs, out)     # legacy default stream, like torch's ops
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), sc), f"call {call}"
        out_bad = torch.zeros(1, dtype=torch.int32, device="cuda")
        et.tube_count_noalloc(xyz, p, bad, out_bad)
        torch.cuda.synchronize()
        assert int(out_bad.item()) == -1


def test_noalloc_rejects_views_beyond_the_fixed_limit():
    import torch
    from paper_1311_5334_gb300 import et

    n = 65537
    xyz = torch.zeros((n, 3), dtype=torch.int32, device="cuda")
    pairs = torch.zeros((1, 2), dtype=torch.int32, device="cuda")
    out = torch.zeros(1, dtype=torch.int32, device="cuda")
    p = synth.params((30000, 30000, 5000))
    with pytest.raises(et.EtError) as e:
        et.tube_count_noalloc(xyz, p, pairs, out)
    assert e.value.status == et.INVALID_ARG
