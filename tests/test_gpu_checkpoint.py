"""Checkpoint / resume of the training state (render.py: state_dict / load_state_dict of FineModel,
CoarseModel, Proposal and ProposalTrainer).

A snapshot written with torch.save and read back with torch.load into freshly built objects
(different initial values) must restore every tensor bit for bit, the step counts and the
schedule's position.  Its effect is checked bit for bit where the library is deterministic: the
per-ray forward colours of the restored model and the proposal's samples equal those of the
original.  Training then continues on both; the backward adds gradients with FP32 atomics, whose
order varies from run to run, so the continued runs are compared within a tolerance far above that
spread (1e-3 relative) and far below what a lost Adam moment or a wrong step count would cause (the
first Adam step after a reset moves touched elements by about the learning rate).
"""
import io

import numpy as np
import pytest
import torch

import synth
from test_gpu_parity import _fine_inputs, _mlp_flat, cuda

pytestmark = pytest.mark.gpu

dvgo = pytest.importorskip("paper_2111_11215_gb300")

RES, R = 32, 2048
TOL = 1e-3


def _rel_l2(a, b):
    a, b = a.double(), b.double()
    return float((a - b).norm() / max(float(b.norm()), 1e-30))


def _fine_params(res):
    return dvgo.Params(mode=dvgo.DVGO_MODE_FINE, step=0.5 * 2.0 / res, bg=(1.0, 1.0, 1.0),
                       mlp_prec=dvgo.DVGO_MLP_BF16, shift_b=dvgo.dvgo_shift_from_alpha_init(1e-2, 2.0 / res))


def _chosen(seed):
    """A chosen-form trainer (BF16 MLP and feature copy, the overlapped feature-grid Adam, the
    learned proposal) with initial values drawn from `seed`."""
    dens, feat, mlp, _, _, _, _ = _fine_inputs(RES, 8, seed=seed)
    p = _fine_params(RES)
    model = dvgo.FineModel(cuda(dens), cuda(feat), cuda(_mlp_flat(mlp)), p, R, bf16_feat=True, overlap_adam=True)
    prop = dvgo.Proposal(synth.proposal_weights(39, 64, seed=seed + 1), p, model.dd, R,
                         sample_precision=dvgo.DVGO_MLP_BF16, train_precision=dvgo.DVGO_MLP_BF16)
    return dvgo.ProposalTrainer(model, prop, n_samples=48, uniform_every=4, train_rays=1024)


def _batch(i):
    return tuple(cuda(x) for x in synth.fine_batch(R, seed=900 + i))


def _roundtrip(sd):
    buf = io.BytesIO()
    torch.save(sd, buf)
    buf.seek(0)
    return torch.load(buf, map_location="cuda")


def _trainer_tensors(tr):
    m, p = tr.model, tr.proposal
    out = {"density": m.density, "feat": m.feat, "feat_bf16": m.feat_bf16, "mlp": m.mlp_flat, "prop": p.flat,
           "prop_m": p.adam.m, "prop_v": p.adam.v}
    for k, a in m.adam.items():
        out[f"{k}_m"], out[f"{k}_v"] = a.m, a.v
    return out


def _assert_bitwise(a, b):
    for k in a:
        assert a[k].shape == b[k].shape and a[k].dtype == b[k].dtype, k
        assert torch.equal(a[k], b[k]), k


def test_chosen_trainer_resumes_from_a_checkpoint():
    a = _chosen(seed=910)
    for i in range(6):                                  # 2 uniform steps (0, 4) and 4 proposal steps
        a.step(*_batch(i))
    sd = _roundtrip(a.state_dict())
    b = _chosen(seed=920)                               # other initial values, all overwritten
    b.load_state_dict(sd)
    torch.cuda.synchronize()
    _assert_bitwise(_trainer_tensors(a), _trainer_tensors(b))
    assert (b.i, b.n_uniform, b.n_proposal) == (a.i, a.n_uniform, a.n_proposal) == (6, 2, 4)
    assert (b.model.step_count, b.model.grid_t0, b.proposal.step_count) == \
        (a.model.step_count, a.model.grid_t0, a.proposal.step_count)
    for g in (b.model.g_density, b.model.g_feat, b.model.g_mlp, b.proposal.grad):
        assert not torch.any(g)

    # deterministic effects: per-ray colours of the restored model, the proposal's samples
    o, d, jit, _ = _batch(50)
    ca = a.model.forward(o, d, jit)[0].clone()
    cb = b.model.forward(o, d, jit)[0].clone()
    ta = a.proposal.sample(o, d, jit, 48)[0].clone()
    tb = b.proposal.sample(o, d, jit, 48)[0].clone()
    torch.cuda.synchronize()
    assert torch.equal(ca, cb) and torch.equal(ta, tb)

    # continued training: steps 6-9, a uniform step (8) among them
    la, lb = [], []
    for i in range(6, 10):
        la.append(float(a.step(*_batch(i)).item()))
        lb.append(float(b.step(*_batch(i)).item()))
    np.testing.assert_allclose(lb, la, rtol=TOL)
    ta_, tb_ = _trainer_tensors(a), _trainer_tensors(b)
    torch.cuda.synchronize()
    for k in ("density", "feat", "mlp", "prop"):
        assert _rel_l2(tb_[k], ta_[k]) <= TOL, (k, _rel_l2(tb_[k], ta_[k]))
    assert (b.i, b.n_uniform) == (a.i, a.n_uniform) == (10, 3)


def test_fine_model_resumes_on_the_snapshot_lattice_after_progressive_scaling():
    """A snapshot taken after a rescale restores the larger lattice and its sampling step into a
    model built on the original one."""
    dens, feat, mlp, _, _, _, _ = _fine_inputs(16, 8, seed=930)
    p = _fine_params(16)
    a = dvgo.FineModel(cuda(dens), cuda(feat), cuda(_mlp_flat(mlp)), p, R, bf16_feat=True)
    for i in range(2):
        a.train_step(*_batch(i))
    a.rescale((24, 24, 24), 0.5 * 2.0 / 24)
    a.train_step(*_batch(2))
    sd = _roundtrip(a.state_dict())
    b = dvgo.FineModel(cuda(dens), cuda(feat), cuda(_mlp_flat(mlp)), p, R, bf16_feat=True)
    b.load_state_dict(sd)
    assert b.shape == (24, 24, 24) and b.params.step == a.params.step and b.grid_t0 == a.grid_t0 == 2
    o, d, jit, _ = _batch(51)
    ca = a.forward(o, d, jit)[0].clone()
    cb = b.forward(o, d, jit)[0].clone()
    torch.cuda.synchronize()
    assert torch.equal(ca, cb)
    la = float(a.train_step(*_batch(3)).item())
    lb = float(b.train_step(*_batch(3)).item())
    np.testing.assert_allclose(lb, la, rtol=TOL)
    assert _rel_l2(b.density, a.density) <= TOL and _rel_l2(b.feat, a.feat) <= TOL


def test_coarse_model_resumes_with_its_view_count_scale():
    res = 24
    g = np.random.default_rng(940)
    dens = cuda(g.normal(scale=0.1, size=(res,) * 3))
    rgb = cuda(g.normal(scale=0.1, size=(res,) * 3 + (3,)))
    p = dvgo.Params(mode=dvgo.DVGO_MODE_COARSE, step=0.5 * 2.0 / res, bg=(1.0, 1.0, 1.0),
                    shift_b=dvgo.dvgo_shift_from_alpha_init(1e-6, 2.0 / res))
    a = dvgo.CoarseModel(dens.clone(), rgb.clone(), p, R)
    rig = synth.hemisphere_rig(20, 941)
    a.set_view_counts(cuda(rig.c2w, torch.float64), rig.height, rig.width, rig.focal)
    for i in range(3):
        a.train_step(*_batch(i))
    sd = _roundtrip(a.state_dict())
    b = dvgo.CoarseModel(torch.zeros_like(dens), torch.zeros_like(rgb), p, R)
    b.load_state_dict(sd)
    torch.cuda.synchronize()
    for x, y in ((a.density, b.density), (a.rgb_grid, b.rgb_grid), (a.lr_scale, b.lr_scale),
                 (a.adam["density"].m, b.adam["density"].m), (a.adam["rgb"].v, b.adam["rgb"].v)):
        assert torch.equal(x, y)
    assert b.step_count == a.step_count == 3
    o, d, jit, _ = _batch(52)
    ca, cb = a.forward(o, d, jit)[0].clone(), b.forward(o, d, jit)[0].clone()
    torch.cuda.synchronize()
    assert torch.equal(ca, cb)
    la = float(a.train_step(*_batch(3)).item())
    lb = float(b.train_step(*_batch(3)).item())
    np.testing.assert_allclose(lb, la, rtol=TOL)
    assert _rel_l2(b.density, a.density) <= TOL and _rel_l2(b.rgb_grid, a.rgb_grid) <= TOL


def test_load_refuses_a_snapshot_of_another_model():
    a = _chosen(seed=950)
    sd = a.state_dict()
    with pytest.raises(ValueError, match="not a Proposal state"):
        a.proposal.load_state_dict(sd["model"])
    dens, feat, mlp, _, _, _, _ = _fine_inputs(RES, 8, seed=951)
    f32 = dvgo.FineModel(cuda(dens), cuda(feat), cuda(_mlp_flat(mlp)), _fine_params(RES), R, bf16_feat=False)
    with pytest.raises(ValueError, match="BF16 setting"):
        f32.load_state_dict(sd["model"])
