"""BatchStager (render.py): double-buffered host-to-device staging of training batches on a copy
stream.  The batch a step takes holds exactly its host data, a buffer set is refilled only after
the step that used it, and misuse is refused: staging a third batch before one is taken, staging
into a set whose batch was taken but not marked done, marking done with no batch taken."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

dvgo = pytest.importorskip("paper_2111_11215_gb300")


def _host_batches(n, shapes, seed=3):
    g = np.random.default_rng(seed)
    return [tuple(torch.from_numpy(g.standard_normal(s).astype(np.float32)).pin_memory() for s in shapes)
            for _ in range(n)]


def test_staged_batches_hold_their_host_data():
    shapes = [(4096, 3), (4096, 3), (4096,)]
    host = _host_batches(7, shapes)
    stager = dvgo.BatchStager(tuple(torch.empty(s, device="cuda") for s in shapes))
    out = torch.empty(7, device="cuda")
    stager.stage(host[0])
    for k in range(7):
        b = stager.take()
        if k + 1 < 7:
            stager.stage(host[k + 1])
        # a "step" that reads the whole batch after a delay, so that a refill racing it would show
        torch.cuda._sleep(200000)
        out[k] = sum(x.double().sum() for x in b).float()
        stager.done()
    torch.cuda.synchronize()
    ref = np.array([sum(float(x.double().sum()) for x in h) for h in host], dtype=np.float32)
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-6, atol=1e-3)


def test_third_stage_before_a_take_raises():
    like = (torch.empty(16, device="cuda"),)
    host = _host_batches(3, [(16,)])
    stager = dvgo.BatchStager(like)
    stager.stage(host[0])
    stager.stage(host[1])
    with pytest.raises(RuntimeError, match="both buffer sets"):
        stager.stage(host[2])
    torch.cuda.synchronize()


def test_restaging_a_set_in_use_and_done_without_take_raise():
    like = (torch.empty(16, device="cuda"),)
    host = _host_batches(4, [(16,)])
    stager = dvgo.BatchStager(like)
    with pytest.raises(RuntimeError, match="no taken batch"):
        stager.done()
    stager.stage(host[0])
    b0 = stager.take()
    stager.stage(host[1])
    b1 = stager.take()
    # set 0 still holds batch 0, whose step was never marked done
    with pytest.raises(RuntimeError, match="not marked done"):
        stager.stage(host[2])
    stager.done()                      # batch 0
    stager.stage(host[2])              # now set 0 may be refilled
    stager.done()                      # batch 1
    b2 = stager.take()
    torch.cuda.synchronize()
    assert b2[0].data_ptr() == b0[0].data_ptr() and b1[0].data_ptr() != b0[0].data_ptr()
    np.testing.assert_array_equal(b2[0].cpu().numpy(), host[2][0].numpy())
    np.testing.assert_array_equal(b1[0].cpu().numpy(), host[1][0].numpy())
