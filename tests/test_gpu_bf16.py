"""The chosen form (BF16 tensor-core colour MLP, FP32 accumulation; FP32 or BF16 feature storage)
against the FP64 oracle on the same seeded inputs.

BF16 keeps 8 significant bits (relative rounding 2^-9 = 2e-3) on the MLP inputs, weights, hidden
activations and backward operands; accumulation is FP32.  The bounds below are derived from that
(colour error a few 1e-3 after three layers and the sigmoid; gradient norms within a few 1e-2)
and the measured errors are printed for the record.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import oracle_params
from test_gpu_parity import _fine_inputs, _mlp_flat, _run_fine, cuda

pytestmark = pytest.mark.gpu

dvgo = pytest.importorskip("paper_2111_11215_gb300")

COLOUR_ABS_BOUND = 1e-2
GRAD_REL_L2_BOUND = 5e-2


def _rel_l2(got, ref):
    return float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-30))


@pytest.mark.parametrize("feat_dtype", [torch.float32, torch.bfloat16])
def test_bf16_mlp_against_oracle(feat_dtype, capsys):
    res, R = 24, 400
    dens, feat, mlp, o, d, jit, _ = _fine_inputs(res, R, seed=50)
    if feat_dtype == torch.bfloat16:
        feat = torch.as_tensor(feat).to(torch.bfloat16).float().numpy()
    step = 2.0 / res * 0.5
    p = dvgo.Params(mode=dvgo.DVGO_MODE_FINE, step=step, shift_b=dvgo.dvgo_shift_from_alpha_init(1e-2, 2.0 / res),
                    bg=(1.0, 1.0, 1.0), mlp_prec=dvgo.DVGO_MLP_BF16)
    g = np.random.default_rng(51)
    gC = g.normal(scale=1e-2, size=(R, 3))
    gT = g.normal(scale=1e-2, size=R)
    got = _run_fine(p, res, dens, feat, mlp, o, d, jit, gC, gT, feat_dtype)
    ref = oracle.render(oracle_params(p, (res,) * 3, 12), dens, feat, o, d, jitter=jit, mlp=mlp, grad_rgb=gC,
                        grad_tfinal=gT)
    np.testing.assert_array_equal(got["counts"], ref.n_samples)
    col_err = float(np.abs(got["rgb"] - ref.rgb).max())
    ref_m = np.concatenate([ref.grads[k].reshape(-1) for k in ("w1", "b1", "w2", "b2", "w3", "b3")])
    errs = {"rgb_max_abs": col_err, "tfinal_max_abs": float(np.abs(got["tfinal"] - ref.tfinal).max()),
            "grad_density_rel_l2": _rel_l2(got["g_d"], ref.grads["density"]),
            "grad_feat_rel_l2": _rel_l2(got["g_f"], ref.grads["cgrid"]),
            "grad_mlp_rel_l2": _rel_l2(got["g_m"], ref_m)}
    off = 0
    for k in ("w1", "b1", "w2", "b2", "w3", "b3"):
        n = mlp[k].size
        errs[f"grad_{k}_rel_l2"] = _rel_l2(got["g_m"][off:off + n], ref_m[off:off + n])
        off += n
    with capsys.disabled():
        print(f"\nBF16 MLP ({feat_dtype}) vs FP64 oracle:", {k: f"{v:.3g}" for k, v in errs.items()})
    assert col_err < COLOUR_ABS_BOUND
    assert errs["tfinal_max_abs"] < 1e-6       # transmittance does not depend on the MLP
    for k, v in errs.items():
        if k.endswith("rel_l2"):
            assert v < GRAD_REL_L2_BOUND, (k, v)


def test_bf16_full_size_colours_sampled():
    """160^3 scene, 8192 rays, the launch the benchmark times: colours on sampled rays."""
    res, R = 160, 8192
    dens, feat = synth.fine_scene(seed=0, res=res)
    mlp = synth.mlp_weights(39, 128, 3, seed=3)
    o, d, jit, _ = synth.fine_batch(R, seed=1)
    featb = torch.as_tensor(feat).to(torch.bfloat16)
    step = 2.0 / res * 0.5
    p = dvgo.Params(mode=dvgo.DVGO_MODE_FINE, step=step, shift_b=dvgo.dvgo_shift_from_alpha_init(1e-6, 2.0 / res),
                    bg=(1.0, 1.0, 1.0), mlp_prec=dvgo.DVGO_MLP_BF16)
    got = _run_fine(p, res, dens, featb.float().numpy(), mlp, o, d, jit, None, None, torch.bfloat16, bwd=False)
    idx = np.random.default_rng(9).choice(R, 96, replace=False)
    ref = oracle.render(oracle_params(p, (res,) * 3, 12), dens, featb.float().numpy(), o[idx], d[idx],
                        jitter=jit[idx], mlp=mlp)
    assert np.abs(got["rgb"][idx] - ref.rgb).max() < COLOUR_ABS_BOUND


def _train_chosen(overlap, steps=9, res=48, R=2048):
    dens, feat, mlp, _, _, _, _ = _fine_inputs(res, 8, seed=140)
    p = dvgo.Params(mode=dvgo.DVGO_MODE_FINE, step=0.5 * 2.0 / res, bg=(1.0, 1.0, 1.0), mlp_prec=dvgo.DVGO_MLP_BF16,
                    shift_b=dvgo.dvgo_shift_from_alpha_init(1e-2, 2.0 / res))
    model = dvgo.FineModel(cuda(dens), cuda(feat), cuda(_mlp_flat(mlp)), p, R, bf16_feat=True, overlap_adam=overlap)
    prop = dvgo.Proposal(synth.proposal_weights(39, 64, seed=141), p, model.dd, R,
                         sample_precision=dvgo.DVGO_MLP_BF16, train_precision=dvgo.DVGO_MLP_BF16)
    trainer = dvgo.ProposalTrainer(model, prop, n_samples=48, uniform_every=4, train_rays=1024)
    losses = []
    for i in range(steps):
        o, d, jit, tgt = (cuda(x) for x in synth.fine_batch(R, seed=150 + i))
        losses.append(trainer.step(o, d, jit, tgt).clone())
    model.wait_params()
    torch.cuda.synchronize()
    return (np.array([float(x.item()) for x in losses]),
            {k: t.detach().float().cpu().numpy() for k, t in (("density", model.density), ("feat", model.feat),
                                                                ("feat_bf16", model.feat_bf16), ("mlp", model.mlp_flat),
                                                                ("proposal", prop.flat))})


def test_overlapped_feature_adam_matches_serial():
    """The feature-grid Adam on the side stream (overlap_adam), and with it the proposal's training
    step of the uniform steps on a stream of its own, give the same training as the serial order:
    the differences stay within the run-to-run spread of two serial runs (the atomic summation
    order), scaled by 10, plus 1e-6; the proposal network's weights included."""
    l_ref, p_ref = _train_chosen(False)
    l_ref2, p_ref2 = _train_chosen(False)
    l_ov, p_ov = _train_chosen(True)
    assert np.all(np.isfinite(l_ov))
    spread = np.abs(l_ref2 - l_ref).max()
    assert np.abs(l_ov - l_ref).max() <= 10 * spread + 1e-6 * np.abs(l_ref).max(), (l_ov, l_ref, spread)
    for k in p_ref:
        base = _rel_l2(p_ref2[k], p_ref[k])
        got = _rel_l2(p_ov[k], p_ref[k])
        # the proposal backward adds its weight gradients with per-CTA FP32 atomics; their order moves
        # the trained weights between two outcomes 3.4e-5 apart (relative L2 after three proposal
        # steps; two serial runs land on either), so its floor is 1e-4 -- a wrong label or a step
        # missed would move them by orders of magnitude more
        floor = 1e-4 if k == "proposal" else 1e-6
        assert got <= 10 * base + floor, (k, got, base)
