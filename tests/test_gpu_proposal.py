"""GPU parity of the learned sample proposal against the FP64 oracle: weight-histogram labels,
proposal MLP forward (softmax, cross-entropy) and backward, inverse-CDF sampling, and a render
with the sampled explicit samples."""
import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import RTOL_COLOUR, RTOL_GRAD, assert_close, oracle_params
from test_gpu_parity import _fine_inputs, _mlp_flat, cuda

pytestmark = pytest.mark.gpu

dvgo = pytest.importorskip("paper_2111_11215_gb300")

NB, NFQ, PW = 64, 6, 64


def _proposal_weights(seed):
    w = synth.proposal_weights(3 + 6 * NFQ, PW, seed)
    w["b3"] = np.array([0.1], np.float32)
    return w


def _setup(res=24, R=160, seed=70):
    dens, feat, mlp, o, d, jit, _ = _fine_inputs(res, R, seed=seed)
    # a few rays that miss the box
    o[:3] = np.array([[0.0, 3.0, 0.0], [3.0, 3.0, 0.0], [0.0, 0.0, 5.0]], np.float32)
    d[:3] = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 1.0], [1.0, 0.0, 0.0]], np.float32)
    step = 2.0 / res * 0.5
    p = dvgo.Params(mode=dvgo.DVGO_MODE_FINE, step=step, shift_b=dvgo.dvgo_shift_from_alpha_init(1e-2, 2.0 / res),
                    bg=(1.0, 1.0, 1.0))
    return dens, feat, mlp, o, d, jit, p


def test_weight_bins_labels_match_oracle():
    res = 24
    dens, feat, mlp, o, d, jit, p = _setup(res)
    R = o.shape[0]
    dd, cd = dvgo.GridDesc((res,) * 3, 1), dvgo.GridDesc((res,) * 3, 12)
    r = dvgo.Renderer(p, dd, cd, R)
    views = dvgo.render.mlp_views(cuda(_mlp_flat(mlp)))
    r.forward(cuda(dens), cuda(feat), views, cuda(o), cuda(d), cuda(jit))
    labels = torch.empty((R, NB), device="cuda")
    dvgo.dvgo_weight_bins(p, dd, R, NB, r.workspace, labels)
    torch.cuda.synchronize()
    ref = oracle.render(oracle_params(p, (res,) * 3, 12), dens, feat, o, d, jitter=jit, mlp=mlp, n_bins=NB)
    got = labels.cpu().numpy()
    np.testing.assert_allclose(got.sum(axis=1), 1.0, rtol=1e-5)
    np.testing.assert_allclose(got[:3], 1.0 / NB)              # misses: uniform
    assert_close(got, ref.wbins, RTOL_COLOUR, "labels")


def test_proposal_forward_backward_match_oracle():
    res = 24
    dens, feat, mlp, o, d, jit, p = _setup(res, R=157)        # odd: a half tile
    R = o.shape[0]
    dd = dvgo.GridDesc((res,) * 3, 1)
    w = _proposal_weights(71)
    labels = np.random.default_rng(72).dirichlet(np.full(NB, 0.3), size=R).astype(np.float32)
    wd = {k: cuda(v) for k, v in w.items()}
    probs = torch.empty((R, NB), device="cuda")
    loss = torch.empty(1, device="cuda")
    dvgo.dvgo_proposal_fwd(p, dd, NB, NFQ, PW, wd, cuda(o), cuda(d), cuda(labels), probs, loss)
    flat = torch.zeros(sum(v.size for v in w.values()), device="cuda")
    dvgo.dvgo_proposal_bwd(p, dd, NB, NFQ, PW, wd, cuda(o), cuda(d), cuda(labels), flat)
    torch.cuda.synchronize()
    P = oracle_params(p, (res,) * 3, 12)
    ref_p, ref_loss, ref_g = oracle.proposal(P, w, NB, NFQ, o, d, labels=labels, want_grads=True)
    assert_close(probs.cpu().numpy(), ref_p, RTOL_COLOUR, "probs")
    assert float(loss.item()) == pytest.approx(ref_loss, rel=1e-5)
    g = flat.cpu().numpy()
    off = 0
    for k in oracle.PROP_KEYS:
        n = w[k].size
        if k == "b3":
            # d loss / d b3 = (1/R) sum_r sum_b (p_rb - h_rb) = 0 exactly: both sum to 1 per ray, so
            # only rounding noise (terms of order 1/R) remains on either side
            assert abs(g[off]) < 1e-6 and abs(ref_g[k][0]) < 1e-9
        else:
            assert_close(g[off:off + n], ref_g[k].reshape(-1), RTOL_GRAD, f"grad_{k}")
        off += n


def _bf16(a):
    return torch.as_tensor(np.asarray(a, np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


def _bf16_chain_fwd(P, w, o, d):
    """The proposal forward with BF16 rounding at exactly the points where the tensor-core kernel
    rounds (inputs, weights, hidden activations), in FP64 otherwise."""
    R = o.shape[0]
    X = np.zeros((R, NB, 64))
    hit = np.zeros(R, bool)
    for r in range(R):
        _, t0, t1, dn, _ = oracle.ray_bounds(P, o[r], d[r])
        if not t1 > t0:
            continue
        hit[r] = True
        tb = t0 + (np.arange(NB) + 0.5) * (t1 - t0) / NB
        x = (o[r].astype(np.float64)[None, :] + tb[:, None] * np.asarray(dn)[None, :]).astype(np.float32)
        x = x.astype(np.float64)
        X[r, :, :3] = x
        for a in range(3):
            for k in range(NFQ):
                X[r, :, 3 + a * NFQ + k] = np.sin(2.0 ** k * x[:, a])
                X[r, :, 3 + 3 * NFQ + a * NFQ + k] = np.cos(2.0 ** k * x[:, a])
        X[r, :, 3 + 6 * NFQ] = 1.0
    X = X.reshape(R * NB, 64)
    W0 = np.zeros((64, PW))
    W0[:3 + 6 * NFQ] = w["w0"]
    W0[3 + 6 * NFQ] = w["b0"]
    Xb, W0b, W1b, W2b = _bf16(X), _bf16(W0), _bf16(w["w1"]), _bf16(w["w2"])
    H0 = np.maximum(Xb @ W0b, 0)
    H1 = np.maximum(_bf16(H0) @ W1b + w["b1"], 0)
    H2 = np.maximum(_bf16(H1) @ W2b + w["b2"], 0)
    logit = (H2 @ w["w3"].reshape(PW, 1)).reshape(R, NB) + float(w["b3"][0])
    p = np.exp(logit - logit.max(axis=1, keepdims=True))
    p /= p.sum(axis=1, keepdims=True)
    p[~hit] = 1.0 / NB
    return {"Xb": Xb, "W1b": W1b, "W2b": W2b, "H0": H0, "H1": H1, "H2": H2, "p": p, "hit": hit}


def _bf16_chain_grads(P, w, o, d, labels):
    """The proposal backward with BF16 rounding at exactly the points where the tensor-core kernel
    rounds (inputs, weights, hidden activations, dlogit, the dZ of each layer), in FP64 otherwise:
    separates kernel bugs from BF16 rounding."""
    R = o.shape[0]
    f = _bf16_chain_fwd(P, w, o, d)
    Xb, W1b, W2b, H0, H1, H2, p, hit = (f[k] for k in ("Xb", "W1b", "W2b", "H0", "H1", "H2", "p", "hit"))
    dl = np.where(hit[:, None], p - labels, 0.0).reshape(-1)
    dlb = _bf16(dl)
    dZ2 = _bf16(dl[:, None] * w["w3"].reshape(1, PW) * (H2 > 0))
    dZ1 = _bf16((dZ2 @ W2b.T) * (H1 > 0))
    dZ0 = _bf16((dZ1 @ W1b.T) * (H0 > 0))
    G0 = Xb.T @ dZ0 / R
    return {"w0": G0[:3 + 6 * NFQ], "b0": G0[3 + 6 * NFQ], "w1": _bf16(H0).T @ dZ1 / R, "b1": dZ1.sum(0) / R,
            "w2": _bf16(H1).T @ dZ2 / R, "b2": dZ2.sum(0) / R, "w3": _bf16(H2).T @ dlb / R,
            "b3": np.array([dlb.sum() / R])}


@pytest.mark.parametrize("R", [157, 1001, 60000])
def test_proposal_bf16_forward(R):
    """BF16 tensor-core proposal forward (probabilities and cross-entropy) against the same chain
    rounded to BF16 at the kernel's rounding points.  Differences come only from values near a
    BF16 rounding midpoint that FP32 accumulation rounds the other way (each moves a logit by about
    one BF16 ulp of one hidden unit); a wrong operand layout or index moves probabilities by their
    own size.  R = 60000 gives every CTA more than 64 tiles, so the per-CTA clip pass runs twice;
    R = 157 ends on a tile with one ray; rays 0-2 miss the box (uniform PDF)."""
    res = 24
    dens, feat, mlp, o, d, jit, p = _setup(res, R=R, seed=83)
    dd = dvgo.GridDesc((res,) * 3, 1)
    w = _proposal_weights(85)
    labels = np.random.default_rng(86).dirichlet(np.full(NB, 0.3), size=R).astype(np.float32)
    wd = {k: cuda(v) for k, v in w.items()}
    probs, loss = torch.empty((R, NB), device="cuda"), torch.zeros(1, device="cuda")
    dvgo.dvgo_proposal_fwd(p, dd, NB, NFQ, PW, wd, cuda(o), cuda(d), cuda(labels), probs, loss,
                           precision=dvgo.DVGO_MLP_BF16)
    torch.cuda.synchronize()
    P = oracle_params(p, (res,) * 3, 12)
    parts = [_bf16_chain_fwd(P, w, o[i:i + 4096], d[i:i + 4096]) for i in range(0, R, 4096)]
    f = {k: np.concatenate([q[k] for q in parts]) for k in ("p", "hit")}
    pg = probs.cpu().numpy().astype(np.float64)
    assert f["hit"][3:].mean() > 0.5 and not f["hit"][:3].any()
    np.testing.assert_allclose(pg.sum(axis=1), 1.0, rtol=1e-5)
    np.testing.assert_array_equal(pg[:3], 1.0 / NB)
    err = np.abs(pg - f["p"])
    rel2 = float(np.linalg.norm(pg - f["p"]) / np.linalg.norm(f["p"]))
    ref_loss = -np.sum(np.where(f["hit"][:, None] & (labels > 0), labels * np.log(f["p"]), 0.0)) / R
    print(f"\nBF16 proposal forward R={R}: max |dp| {err.max():.2e} (max p {f['p'].max():.3f}), rel L2 {rel2:.2e}, "
          f"loss {float(loss.item()):.6f} vs {ref_loss:.6f}")
    assert rel2 < 2e-3 and err.max() < 2e-3 * f["p"].max()
    assert abs(float(loss.item()) - ref_loss) < 1e-3 * abs(ref_loss)


@pytest.mark.parametrize("R", [157, 1001, 20000])
def test_proposal_bf16_backward(R):
    """BF16 tensor-core proposal backward (BF16 operands, FP32 accumulation).  Gate: agreement with
    the same chain rounded to BF16 at the kernel's rounding points (relative L2 <= 3e-2 per tensor;
    measured 1e-3 at R = 1001 and 1e-2 at R = 157, where values that sit near a BF16 rounding
    boundary round differently after FP32 instead of FP64 arithmetic; a wrong operand layout or
    index gives errors of order 1).
    Reported (and bounded at 0.2): the relative L2 error against the FP64 oracle, which is the
    BF16 operand rounding amplified by the cancellation in the row sums of the weight gradients
    (the rounded chain itself is 6-10 % from the oracle on these random labels).
    R = 1001 gives the persistent CTAs several tiles each (the gradients accumulate in TMEM);
    R = 20000 more than 64 each (the per-CTA clip pass runs twice)."""
    res = 24
    dens, feat, mlp, o, d, jit, p = _setup(res, R=R, seed=73)
    dd = dvgo.GridDesc((res,) * 3, 1)
    w = _proposal_weights(74)
    labels = np.random.default_rng(75).dirichlet(np.full(NB, 0.3), size=R).astype(np.float32)
    wd = {k: cuda(v) for k, v in w.items()}
    flat = torch.zeros(sum(v.size for v in w.values()), device="cuda")
    dvgo.dvgo_proposal_bwd(p, dd, NB, NFQ, PW, wd, cuda(o), cuda(d), cuda(labels), flat,
                           precision=dvgo.DVGO_MLP_BF16)
    torch.cuda.synchronize()
    P = oracle_params(p, (res,) * 3, 12)
    _, _, ref_g = oracle.proposal(P, w, NB, NFQ, o, d, labels=labels, want_grads=True)
    emu = _bf16_chain_grads(P, w, o, d, labels)
    assert np.mean([oracle.ray_bounds(P, o[r], d[r])[2] > oracle.ray_bounds(P, o[r], d[r])[1]
                    for r in range(0, R, max(1, R // 500))]) > 0.5
    g = flat.cpu().numpy()
    assert np.all(np.isfinite(g))
    off, e_emu, e_ora = 0, {}, {}
    for k in oracle.PROP_KEYS:
        n = w[k].size
        gk = g[off:off + n].astype(np.float64)
        off += n
        if k == "b3":
            # exact value 0 (softmax and labels both sum to 1 per ray); BF16 dlogit leaves a residue
            e_emu[k] = abs(gk[0] - emu[k][0])
            e_ora[k] = abs(gk[0])
            continue
        e_emu[k] = float(np.linalg.norm(gk - emu[k].reshape(-1)) / np.linalg.norm(emu[k]))
        e_ora[k] = float(np.linalg.norm(gk - ref_g[k].reshape(-1)) / np.linalg.norm(ref_g[k]))
    print(f"\nBF16 proposal backward R={R}: rel L2 vs BF16-rounded chain",
          {k: f"{v:.1e}" for k, v in e_emu.items()}, "| vs FP64 oracle", {k: f"{v:.1e}" for k, v in e_ora.items()})
    for k in oracle.PROP_KEYS:
        if k == "b3":
            # worst case of the BF16 residue: 2^-8 (1/R) sum |dlogit| <= 2^-8 * 2
            assert e_emu[k] < 1e-6 and e_ora[k] < 2.0 ** -7, (k, e_emu[k], e_ora[k])
        else:
            assert e_emu[k] < 3e-2, (k, e_emu[k])
            assert e_ora[k] < 0.2, (k, e_ora[k])


def test_sample_pdf_matches_oracle_and_renders():
    res = 24
    dens, feat, mlp, o, d, jit, p = _setup(res, R=96)
    R = o.shape[0]
    dd, cd = dvgo.GridDesc((res,) * 3, 1), dvgo.GridDesc((res,) * 3, 12)
    g = np.random.default_rng(80)
    probs = g.dirichlet(np.full(NB, 0.2), size=R).astype(np.float32)
    probs[5] = 0.0
    probs[5, 17] = 1.0                                         # one-hot PDF
    ts, dts = torch.empty((R, 48), device="cuda"), torch.empty((R, 48), device="cuda")
    pj = synth.jitter(R, 81)
    dvgo.dvgo_sample_pdf(p, dd, cuda(o), cuda(d), cuda(probs), 48, cuda(pj), 1e-3, ts, dts)
    torch.cuda.synchronize()
    t_gpu, dt_gpu = ts.cpu().numpy(), dts.cpu().numpy()
    P = oracle_params(p, (res,) * 3, 12)
    for r in range(R):
        rc, t0, t1, dn, n = oracle.ray_bounds(P, o[r], d[r])
        if not t1 > t0:
            assert np.all(t_gpu[r] == 0)
            continue
        t, dt = oracle.sample_pdf(probs[r].astype(np.float64), t0, t1, 48, jit=float(pj[r]),
                                  eta=float(np.float32(1e-3)))
        np.testing.assert_allclose(t_gpu[r], t, rtol=2e-7, atol=1e-7)
        np.testing.assert_allclose(dt_gpu[r], dt, rtol=2e-6, atol=1e-7)
        assert np.all(np.diff(t_gpu[r]) >= 0)
    # the explicit samples drive a render that matches the oracle on the same samples
    rend = dvgo.Renderer(p, dd, cd, R, samples_per_ray=48)
    views = dvgo.render.mlp_views(cuda(_mlp_flat(mlp)))
    rgb, _, _ = rend.forward(cuda(dens), cuda(feat), views, cuda(o), cuda(d), None, (ts, dts))
    ref = oracle.render(P, dens, feat, o, d, mlp=mlp, explicit_t=t_gpu, explicit_dt=dt_gpu)
    assert_close(rgb.cpu().numpy(), ref.rgb, RTOL_COLOUR, "rgb_explicit")


@pytest.mark.parametrize("nb,ns,eta", [(50, 100, 0.0), (64, 48, 0.05), (7, 3, 0.3), (128, 200, 0.01), (64, 1, 0.05)])
def test_sample_pdf_shapes_and_zero_bins(nb, ns, eta):
    """Inverse-CDF sampling against the oracle for bin counts that are not a multiple of the warp
    width, the largest bin count (128), more samples than bins (outputs staged in several chunks of
    32), a single sample, eta = 0 with zero-mass bins, a one-hot PDF, and a ray count that leaves a
    partial block of 32 rays."""
    res, R = 24, 77
    _, _, _, o, d, _, p = _setup(res, R=R, seed=76)
    dd = dvgo.GridDesc((res,) * 3, 1)
    rng = np.random.default_rng(77)
    probs = rng.dirichlet(np.full(nb, 0.5), size=R)
    probs[rng.random((R, nb)) < 0.3] = 0.0                    # zero-mass bins
    probs[5] = 0.0
    probs[5, nb // 2] = 1.0                                   # one-hot
    probs = (probs / probs.sum(axis=1, keepdims=True)).astype(np.float32)
    jit = synth.jitter(R, 78)
    ts, dts = torch.empty((R, ns), device="cuda"), torch.empty((R, ns), device="cuda")
    dvgo.dvgo_sample_pdf(p, dd, cuda(o), cuda(d), cuda(probs), ns, cuda(jit), eta, ts, dts)
    torch.cuda.synchronize()
    t_gpu, dt_gpu = ts.cpu().numpy(), dts.cpu().numpy()
    P = oracle_params(p, (res,) * 3, 12)
    for r in range(R):
        _, t0, t1, _, _ = oracle.ray_bounds(P, o[r], d[r])
        if not t1 > t0:
            assert np.all(t_gpu[r] == 0) and np.all(dt_gpu[r] == 0)
            continue
        t, dt = oracle.sample_pdf(probs[r].astype(np.float64), t0, t1, ns, jit=float(jit[r]),
                                  eta=float(np.float32(eta)))
        np.testing.assert_allclose(t_gpu[r], t, rtol=2e-7, atol=1e-7)
        np.testing.assert_allclose(dt_gpu[r], dt, rtol=2e-6, atol=1e-7)
        if r == 5 and eta == 0.0:
            w = (t1 - t0) / nb
            assert np.all((t_gpu[r] >= t0 + (nb // 2) * w - 1e-6) & (t_gpu[r] <= t0 + (nb // 2 + 1) * w + 1e-6))


def test_trained_proposal_beats_uniform_48_samples():
    """Gain test: after training on labels from uniform renders, 48 proposal samples per ray give a
    clearly smaller colour error against the oracle's uniform 0.5-voxel render than 48 uniform
    samples.  The proposal backward accumulates its weight gradients with atomics, so the trained
    weights (and the error ratio) vary a little from run to run; the bound leaves room for that."""
    res, R = 128, 2048
    c, rad = synth.random_spheres(6, 90, rmin=0.15, rmax=0.35)
    dens = synth.sphere_density(res, c, rad, 50.0)
    feat = synth.smooth_features(res, 12, 91)
    mlp = synth.mlp_weights(39, 128, 3, 92)
    step = 2.0 / res * 0.5
    p = dvgo.Params(mode=dvgo.DVGO_MODE_FINE, step=step, shift_b=dvgo.dvgo_shift_from_alpha_init(1e-6, 2.0 / res),
                    bg=(1.0, 1.0, 1.0))
    model = dvgo.FineModel(cuda(dens), cuda(feat), cuda(_mlp_flat(mlp)), p, R)
    prop = dvgo.Proposal(_proposal_weights(93), p, model.dd, R)
    losses = []
    for i in range(300):
        o, d, _, _ = (cuda(x) for x in synth.fine_batch(R, seed=400 + i))
        model.forward(o, d, None)
        losses.append(prop.train_step(model.renderer.workspace, o, d).clone())
    losses = [float(x.item()) for x in losses]
    # cross-entropy is bounded below by the labels' entropy; it must still drop clearly
    assert np.mean(losses[-20:]) < np.mean(losses[:5]) - 0.1
    o_np, d_np, _, _ = synth.fine_batch(256, seed=777)
    o, d = cuda(o_np), cuda(d_np)
    ts, dts = prop.sample(o, d, None, 48)
    uni = torch.full((256, 64), 1.0 / 64, device="cuda")
    tu, dtu = torch.empty_like(ts), torch.empty_like(dts)
    dvgo.dvgo_sample_pdf(p, model.dd, o, d, uni, 48, None, 1e-3, tu, dtu)
    rend = dvgo.Renderer(p, model.dd, model.cd, 256, samples_per_ray=48)
    c_prop = rend.forward(model.density, model.cgrid, model.mlp, o, d, None, (ts, dts))[0].cpu().numpy()
    c_uni = rend.forward(model.density, model.cgrid, model.mlp, o, d, None, (tu, dtu))[0].cpu().numpy()
    ref = oracle.render(oracle_params(p, (res,) * 3, 12), dens, feat, o_np, d_np, mlp=mlp)
    e_prop, e_uni = np.abs(c_prop - ref.rgb).mean(), np.abs(c_uni - ref.rgb).mean()
    print(f"\nproposal-48 mean |err| {e_prop:.4g}, uniform-48 mean |err| {e_uni:.4g}")
    assert e_prop < 0.6 * e_uni
    # the BF16 tensor-core proposal forward gives (nearly) the same PDFs as the FP32 one
    pf, pb = torch.empty((256, 64), device="cuda"), torch.empty((256, 64), device="cuda")
    dvgo.dvgo_proposal_fwd(p, model.dd, 64, 6, 64, prop.w, o, d, None, pf, None)
    dvgo.dvgo_proposal_fwd(p, model.dd, 64, 6, 64, prop.w, o, d, None, pb, None,
                           precision=dvgo.DVGO_MLP_BF16)
    torch.cuda.synchronize()
    np.testing.assert_allclose(pb.sum(dim=1).cpu().numpy(), 1.0, rtol=1e-5)
    assert float((pb - pf).abs().max().item()) < 0.05 * float(pf.max().item())
