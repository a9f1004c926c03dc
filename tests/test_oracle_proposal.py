"""Pins of the oracle's sample-proposal pieces (CPU only).

The paper leaves hierarchical / importance sampling to future work (Supp. B, step-size
ablation); the 64-bin proposal PDF and 48 inverse-CDF samples are this library's addition.
These tests fix the oracle's versions against closed forms, brute force and finite differences.
"""
import math

import numpy as np
import pytest

import oracle
import synth


def test_uniform_pdf_gives_evenly_spaced_samples():
    t, dt = oracle.sample_pdf(np.full(64, 1 / 64), 2.0, 5.0, 48, jit=0.5, eta=1e-3)
    np.testing.assert_allclose(t, 2.0 + (np.arange(48) + 0.5) / 48 * 3.0, rtol=1e-13)
    np.testing.assert_allclose(dt, 3.0 / 48, rtol=1e-12)


def test_one_hot_pdf_puts_every_sample_in_its_bin():
    p = np.zeros(64); p[37] = 1.0
    t, dt = oracle.sample_pdf(p, 0.0, 64.0, 48, jit=0.5, eta=0.0)
    assert np.all((t >= 37.0) & (t < 38.0))
    np.testing.assert_allclose(t, 37.0 + (np.arange(48) + 0.5) / 48, rtol=1e-13)
    assert np.all(np.diff(t) > 0)


def test_sample_pdf_inverse_cdf_brute_force():
    g = np.random.default_rng(3)
    p = g.dirichlet(np.full(16, 0.5))
    eta = 1e-3
    t, dt = oracle.sample_pdf(p, 1.0, 3.0, 40, jit=0.3, eta=eta)
    q = (1 - eta) * p + eta / 16
    # brute-force CDF of the mixed PDF on a fine grid, evaluated at the returned samples
    edges = 1.0 + np.arange(17) * (2.0 / 16)
    for j, tj in enumerate(t):
        b = min(int((tj - 1.0) / (2.0 / 16)), 15)
        cdf = q[:b].sum() + q[b] * (tj - edges[b]) / (2.0 / 16)
        assert cdf == pytest.approx((j + 0.3) / 40, abs=1e-12)
    np.testing.assert_allclose(dt[:-1], np.diff(t), rtol=1e-13)
    assert dt[-1] == pytest.approx((2.0 / 16) / (40 * q[b]), rel=1e-12)


def _tiny_prop(seed=5):
    F, W, B = 2, 6, 8
    prop = {k: v.astype(np.float64) for k, v in synth.proposal_weights(3 + 6 * F, W, seed).items()}
    prop["b3"] = np.array([0.1])
    P = oracle.Params(grid_shape=(4, 4, 4))
    o, d = synth.sphere_rays(4, seed=seed + 1, radius=3.0, jitter_sd=0.1)
    labels = np.random.default_rng(seed + 2).dirichlet(np.ones(B), size=4)
    return P, prop, F, B, o, d, labels


def test_proposal_softmax_and_cross_entropy():
    P, prop, F, B, o, d, labels = _tiny_prop()
    probs, loss, _ = oracle.proposal(P, prop, B, F, o, d, labels=labels)
    np.testing.assert_allclose(probs.sum(axis=1), 1.0, rtol=1e-14)
    assert loss == pytest.approx(-np.mean(np.sum(labels * np.log(probs), axis=1)), rel=1e-13)


def test_proposal_gradient_matches_central_differences():
    P, prop, F, B, o, d, labels = _tiny_prop()
    _, _, grads = oracle.proposal(P, prop, B, F, o, d, labels=labels, want_grads=True)
    h = 1e-6
    for k, arr in prop.items():
        flat = arr.reshape(-1)
        num = np.zeros_like(flat)
        for i in range(flat.size):
            old = flat[i]
            flat[i] = old + h
            lp = oracle.proposal(P, prop, B, F, o, d, labels=labels)[1]
            flat[i] = old - h
            lm = oracle.proposal(P, prop, B, F, o, d, labels=labels)[1]
            flat[i] = old
            num[i] = (lp - lm) / (2 * h)
        scale = max(np.abs(num).max(), 1e-4)
        np.testing.assert_allclose(grads[k].reshape(-1), num, rtol=0, atol=3e-7 * scale, err_msg=k)


def test_proposal_logit_gradient_is_p_minus_h():
    # With every weight zero except the output bias row, d loss / d b3 = mean_r sum_b (p - h) = 0,
    # and d loss / d w3 = mean over rays of sum_b (p_b - h_b) h2_b: check the bias case exactly.
    P, prop, F, B, o, d, labels = _tiny_prop()
    probs, _, grads = oracle.proposal(P, prop, B, F, o, d, labels=labels, want_grads=True)
    assert grads["b3"][0] == pytest.approx(np.mean(np.sum(probs - labels, axis=1)), abs=1e-14)


def test_weight_histogram_constant_density_brute_force():
    """Per-ray histogram of compositing weights (labels for the proposal), constant density."""
    res, delta, nb = 5, 0.05, 8
    x0 = 1.0
    P = oracle.Params(grid_shape=(res,) * 3, shift_b=0.0, delta=delta)
    dens = np.full((res,) * 3, x0)
    rgb = np.zeros((res, res, res, 3))
    o, d = np.array([[-3.0, 0.1, 0.0]]), np.array([[1.0, 0.0, 0.0]])
    r = oracle.render(P, dens, rgb, o, d, jitter=[0.25], n_bins=nb)
    alpha = 1 - (1 + math.exp(x0)) ** (-delta)
    K = r.n_samples[0]
    t0, t1 = r.t_enter[0], r.t_exit[0]
    h = np.zeros(nb)
    for k in range(K):
        t = t0 + (k + 0.25) * delta
        h[min(int((t - t0) / (t1 - t0) * nb), nb - 1)] += (1 - alpha) ** k * alpha
    np.testing.assert_allclose(r.wbins[0], h / h.sum(), rtol=1e-12)
