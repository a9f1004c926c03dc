"""Host logic of checkpoint / resume (render.py) that needs no GPU: a snapshot of another kind or
version is refused, and a restored tensor must match its destination's shape and dtype."""
import pytest
import torch

dvgo = pytest.importorskip("paper_2111_11215_gb300")
render = dvgo.render


def test_snapshot_kind_and_version_are_checked():
    good = {"kind": "Proposal", "version": render.STATE_VERSION}
    render._check_version(good, "Proposal")
    for bad in ({"kind": "FineModel", "version": render.STATE_VERSION},
                {"kind": "Proposal", "version": render.STATE_VERSION + 1}, {"kind": "Proposal"}, [1, 2]):
        with pytest.raises(ValueError, match="not a Proposal state"):
            render._check_version(bad, "Proposal")


def test_restore_copies_only_into_a_matching_tensor():
    dst = torch.zeros(4, 3)
    src = torch.arange(12, dtype=torch.float32).reshape(4, 3)
    render._copy_on(dst, src, None)
    assert torch.equal(dst, src)
    with pytest.raises(ValueError, match="does not fit"):
        render._copy_on(dst, torch.zeros(3, 4), None)
    with pytest.raises(ValueError, match="does not fit"):
        render._copy_on(dst, src.double(), None)
    clone = render._clone_on(src, None)
    assert torch.equal(clone, src) and clone.data_ptr() != src.data_ptr()
    assert render._clone_on(None, None) is None
