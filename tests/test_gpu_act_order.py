"""GPU parity of the pre- and in-activation orders (Sec. 3 Eq. pre_in_post) against the FP64
oracle, coarse and fine, forward and backward, at the FP32 tolerances."""
import numpy as np
import pytest

import oracle
import synth
from helpers import BOUND_FP32, RTOL_COLOUR, RTOL_GRAD, assert_close, assert_within_bound, oracle_params
from test_gpu_parity import _fine_inputs, _run_coarse, _run_fine

pytestmark = pytest.mark.gpu

dvgo = pytest.importorskip("paper_2111_11215_gb300")


@pytest.mark.parametrize("order", [1, 2])
def test_coarse_orders(order):
    case = synth.coarse_case(seed=1, n_rays=1500)
    p = dvgo.Params(mode=dvgo.DVGO_MODE_COARSE, step=0.03125, shift_b=0.5, bg=(0.3, 0.6, 0.9), act_order=order)
    got, ref, refb = _run_coarse(case, p)
    np.testing.assert_array_equal(got["counts"], ref.n_samples)
    assert_close(got["rgb"], ref.rgb, RTOL_COLOUR, "rgb")
    assert_close(got["tfinal"], ref.tfinal, RTOL_COLOUR, "tfinal")
    assert_close(got["g_d"], refb.grads["density"], RTOL_GRAD, "grad_density")
    assert_close(got["g_c"], refb.grads["cgrid"], RTOL_GRAD, "grad_rgb")
    # the order matters on this input
    post = oracle.render(oracle_params(dvgo.Params(mode=dvgo.DVGO_MODE_COARSE, step=0.03125, shift_b=0.5,
                                                   bg=(0.3, 0.6, 0.9)), (32,) * 3, 3),
                         case["density"], case["rgb"], case["rays_o"], case["rays_d"])
    assert np.abs(post.tfinal - ref.tfinal).max() > 1e-4


@pytest.mark.parametrize("order", [1, 2])
def test_fine_orders_fp32(order):
    res, R = 24, 300
    dens, feat, mlp, o, d, jit, _ = _fine_inputs(res, R, seed=60)
    p = dvgo.Params(mode=dvgo.DVGO_MODE_FINE, step=2.0 / res * 0.5, bg=(1.0, 1.0, 1.0), act_order=order,
                    shift_b=dvgo.dvgo_shift_from_alpha_init(1e-2, 2.0 / res))
    g = np.random.default_rng(61)
    gC = g.normal(scale=1e-2, size=(R, 3))
    gT = g.normal(scale=1e-2, size=R)
    got = _run_fine(p, res, dens, feat, mlp, o, d, jit, gC, gT)
    ref = oracle.render(oracle_params(p, (res,) * 3, 12), dens, feat, o, d, jitter=jit, mlp=mlp, grad_rgb=gC,
                        grad_tfinal=gT, error_bound=BOUND_FP32)
    assert_close(got["rgb"], ref.rgb, RTOL_COLOUR, "rgb")
    assert_close(got["tfinal"], ref.tfinal, RTOL_COLOUR, "tfinal")
    assert_within_bound(got["g_d"], ref.grads["density"], ref.bounds["density"], "grad_density")
    assert_within_bound(got["g_f"], ref.grads["cgrid"], ref.bounds["cgrid"], "grad_feat")


def test_pre_order_saturated_corners_stay_finite():
    """Corners dense enough that every alpha rounds to 1 in FP32: transmittance 0 behind them,
    finite gradients, and agreement with the oracle."""
    case = synth.coarse_case(seed=2, n_rays=512)
    case["density"] = case["density"] * 0.0 + 400.0
    case["density"][:, :, :16] = -5.0                      # an empty half in front of the wall
    p = dvgo.Params(mode=dvgo.DVGO_MODE_COARSE, step=0.03125, shift_b=0.0, bg=(0.3, 0.6, 0.9), act_order=1)
    got, ref, refb = _run_coarse(case, p)
    assert np.all(np.isfinite(got["rgb"])) and np.all(np.isfinite(got["g_d"])) and np.all(np.isfinite(got["g_c"]))
    assert_close(got["rgb"], ref.rgb, RTOL_COLOUR, "rgb")
    assert got["tfinal"].min() < 1e-6
