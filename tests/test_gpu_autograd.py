"""The torch.autograd.Function over dvgo_render_fwd / dvgo_render_bwd (render.RenderFunction).

A scalar loss L = sum(A * rgb) + sum(b * T_final) with seeded A, b is back-propagated with
torch.autograd.backward through RenderFunction on a small fine-stage case (8^3 grids, the
12-channel feature grid and the 39-128-128-3 colour MLP the library supports, FP32 MLP, tau_f = 0
so that sample positions do not depend on any parameter).  Its gradients are checked

  * against the FP64 oracle's hand-derived gradient (the chain rule of Sec. 2 Eq. volume_rendering
    and Eq. photo_loss through Eq. interp, the post-activation and the MLP), element by element at
    the FP32 tolerances, and
  * against central finite differences of the GPU forward itself on the entries with the largest
    gradients of every parameter tensor (the wiring: which input each returned gradient belongs to,
    its sign and scale).

A second forward on the same renderer before the backward must raise, because the backward reads
the per-sample state that the forward left in the renderer's workspace.
"""
import numpy as np
import pytest
import torch

import oracle
from helpers import NORM_RTOL_GRAD, RTOL_GRAD, assert_close, oracle_params
from test_gpu_parity import _fine_inputs, _mlp_flat, cuda

pytestmark = pytest.mark.gpu

dvgo = pytest.importorskip("paper_2111_11215_gb300")

RES, R = 8, 160
MLP_KEYS = ("w1", "b1", "w2", "b2", "w3", "b3")


def _case():
    dens, feat, mlp, o, d, jit, _ = _fine_inputs(RES, R, seed=70, value=6.0, n_spheres=3)
    p = dvgo.Params(mode=dvgo.DVGO_MODE_FINE, step=2.0 / RES * 0.5, bg=(1.0, 1.0, 1.0),
                    shift_b=dvgo.dvgo_shift_from_alpha_init(1e-2, 2.0 / RES))
    # loss weights of one sign, so that the rays' contributions add up and the gradients stand well
    # above the FP32 rounding of the forward that the finite differences see
    g = np.random.default_rng(71)
    A = g.uniform(0.5, 1.5, size=(R, 3))
    b = g.uniform(0.5, 1.5, size=R)
    return p, dens, feat, mlp, o, d, jit, A, b


def _renderer(p):
    return dvgo.Renderer(p, dvgo.GridDesc((RES,) * 3, 1), dvgo.GridDesc((RES,) * 3, 12), R)


def _loss(rgb, tf, A, b):
    return (rgb.double() * A).sum() + (tf.double() * b).sum()


def test_render_function_backward_matches_oracle_and_finite_differences():
    p, dens, feat, mlp, o, d, jit, A, b = _case()
    rend = _renderer(p)
    D = cuda(dens).requires_grad_(True)
    F = cuda(feat).requires_grad_(True)
    Mf = cuda(_mlp_flat(mlp)).requires_grad_(True)
    ro, rd, jt = cuda(o), cuda(d), cuda(jit)
    At, bt = torch.as_tensor(A, device="cuda"), torch.as_tensor(b, device="cuda")
    rgb, tf = dvgo.RenderFunction.apply(rend, D, F, Mf, ro, rd, jt, None, None)
    torch.autograd.backward(_loss(rgb, tf, At, bt))
    torch.cuda.synchronize()
    got = {"density": D.grad.cpu().numpy(), "cgrid": F.grad.cpu().numpy(), "mlp": Mf.grad.cpu().numpy()}

    # (1) the oracle's gradient of the same scalar
    ref = oracle.render(oracle_params(p, (RES,) * 3, 12), dens, feat, o, d, jitter=jit, mlp=mlp, grad_rgb=A,
                        grad_tfinal=b)
    assert np.abs(ref.n_samples).sum() > 0
    ref_m = np.concatenate([ref.grads[k].reshape(-1) for k in MLP_KEYS])
    for name, g_, r_ in (("grad_density", got["density"], ref.grads["density"]),
                         ("grad_feat", got["cgrid"], ref.grads["cgrid"]), ("grad_mlp", got["mlp"], ref_m)):
        _, rel2 = assert_close(g_, r_, RTOL_GRAD, name)
        assert rel2 <= NORM_RTOL_GRAD, (name, rel2)

    # (2) central finite differences of the GPU forward (FP32 outputs, FP64 loss)
    def loss_at(Dv, Fv, Mv):
        with torch.no_grad():
            out = dvgo.RenderFunction.apply(rend, Dv, Fv, Mv, ro, rd, jt, None, None)
        return float(_loss(out[0], out[1], At, bt).item())

    D0, F0, M0 = D.detach().clone(), F.detach().clone(), Mf.detach().clone()
    checks = [("density", D0, 0, D0.numel(), 1e-2)]
    checks.append(("cgrid", F0, 0, F0.numel(), 1e-2))
    off = 0
    for k in MLP_KEYS:
        n = mlp[k].size
        checks.append((k, M0, off, n, 3e-3))
        off += n
    flat_grad = {"density": got["density"].reshape(-1), "cgrid": got["cgrid"].reshape(-1), "mlp": got["mlp"]}
    for name, base, start, n, h in checks:
        key = name if name in flat_grad else "mlp"
        g_seg = flat_grad[key][start:start + n]
        top = start + np.argsort(-np.abs(g_seg))[:4]
        scale = np.abs(g_seg).max()
        assert scale > 0, name
        for i in top:
            plus, minus = base.clone(), base.clone()
            plus.view(-1)[i] += h
            minus.view(-1)[i] -= h
            args_p = [D0, F0, M0]
            args_m = [D0, F0, M0]
            slot = {"density": 0, "cgrid": 1}.get(name, 2)
            args_p[slot], args_m[slot] = plus, minus
            fd = (loss_at(*args_p) - loss_at(*args_m)) / (2 * h)
            an = flat_grad[key][i]
            # central differences of an FP32 forward: truncation O(h^2) and the FP32 rounding of
            # the loss (~1e-7 of it) over 2h; a wrong tensor, sign or scale is off by far more
            assert abs(fd - an) <= 2e-2 * abs(an) + 2e-3 * scale, (name, int(i), fd, an)


def test_render_function_second_forward_before_backward_raises():
    p, dens, feat, mlp, o, d, jit, A, b = _case()
    rend = _renderer(p)
    D = cuda(dens).requires_grad_(True)
    F = cuda(feat).requires_grad_(True)
    Mf = cuda(_mlp_flat(mlp)).requires_grad_(True)
    ro, rd = cuda(o), cuda(d)
    At, bt = torch.as_tensor(A, device="cuda"), torch.as_tensor(b, device="cuda")
    first = dvgo.RenderFunction.apply(rend, D, F, Mf, ro, rd, None, None, None)
    dvgo.RenderFunction.apply(rend, D, F, Mf, ro, rd, None, None, None)      # reuses the workspace
    with pytest.raises(RuntimeError, match="reused by another forward"):
        torch.autograd.backward(_loss(first[0], first[1], At, bt))
