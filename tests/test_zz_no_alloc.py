"""The allocation-free entry point (tpc_row_params_noalloc) against the
grid stage of the regular path.

Some callers cannot allocate device memory: code that lives inside a memory
budget owned by its host framework, an allocator callback, or a server that
forbids CUDA allocations once it runs.  For them the library offers one
entry point whose scratch is a fixed file-scope device array; this test
checks, through the C ABI, that its output equals the regular path's
records bit for bit on two calls in a row (the array is reused and must be
cleared by each call), and that it rejects what exceeds its limit.  It sits
in a file of its own, collected last, and passes alone or after the rest.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _reference(clusters, off):
    import paper_1709_00618_b300 as tpc
    with tpc.Tracker(device=0) as trk:
        trk.load(clusters, off)
        trk.find()
        return trk.stage("rs_params")


def _noalloc(clusters, off):
    import torch

    import paper_1709_00618_b300 as tpc
    dev = torch.from_numpy(clusters.view(np.uint8).copy()).cuda()
    nreq = len(off) - 1
    out = torch.full((nreq * 36 * 159 * 32,), 0xAB, dtype=torch.uint8, device="cuda")
    rc = tpc.row_params_noalloc(dev, off, out)
    return rc, out.cpu().numpy().view(tpc.RS_PARAMS_DTYPE)


def test_noalloc_matches_grid_stage_twice():
    ev = synth.central_event(seed=1, n_primaries=2000, n_secondaries=400)
    off = [0, len(ev.clusters)]
    ref = _reference(ev.clusters, off)
    for _ in range(2):
        rc, got = _noalloc(ev.clusters, off)
        assert rc == 0
        assert got.tobytes() == ref.tobytes()


def test_noalloc_batch_of_requests_twice():
    reqs = synth.batch_requests(seed=7, n_requests=3, max_tracks=1500)
    cl = np.concatenate([r.clusters for r in reqs])
    off = np.concatenate([[0], np.cumsum([len(r.clusters) for r in reqs])])
    ref = _reference(cl, off)
    for _ in range(2):
        rc, got = _noalloc(cl, off)
        assert rc == 0 and got.tobytes() == ref.tobytes()


def test_noalloc_rejects_beyond_its_limit():
    import torch

    import paper_1709_00618_b300 as tpc
    ev = synth.one_sector(seed=0)
    n = len(ev.clusters)
    dev = torch.from_numpy(ev.clusters.view(np.uint8).copy()).cuda()
    off = np.linspace(0, n, 10).astype(np.int64)  # 9 requests: above the 8 the array holds
    out = torch.empty(9 * 36 * 159 * 32, dtype=torch.uint8, device="cuda")
    assert tpc.row_params_noalloc(dev, off, out) == tpc.TPC_EINVAL
    bad = ev.clusters.copy()
    bad["row"][3] = 500
    dev = torch.from_numpy(bad.view(np.uint8).copy()).cuda()
    assert tpc.row_params_noalloc(dev, [0, n], out) == tpc.TPC_EINVAL
    # and the next valid call is unaffected by the previous one
    rc, got = _noalloc(ev.clusters, [0, n])
    assert rc == 0 and got.tobytes() == _reference(ev.clusters, [0, n]).tobytes()


def test_noalloc_wrapper_refuses_bad_buffers():
    """The binding checks what the C entry point cannot: the output's size,
    contiguity and device, before any launch."""
    import torch

    import paper_1709_00618_b300 as tpc
    ev = synth.one_sector(seed=0)
    n = len(ev.clusters)
    dev = torch.from_numpy(ev.clusters.view(np.uint8).copy()).cuda()
    short = torch.empty(36 * 159 * 32 - 1, dtype=torch.uint8, device="cuda")
    with pytest.raises(ValueError):
        tpc.row_params_noalloc(dev, [0, n], short)
    strided = torch.empty(2 * 36 * 159 * 32, dtype=torch.uint8, device="cuda")[::2]
    with pytest.raises(ValueError):
        tpc.row_params_noalloc(dev, [0, n], strided)
    with pytest.raises(ValueError):
        tpc.row_params_noalloc(dev, [0, n], torch.empty(36 * 159 * 32, dtype=torch.uint8))
