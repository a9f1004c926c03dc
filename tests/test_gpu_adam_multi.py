"""dvgo_adam_step_multi: several tensors updated in one launch give exactly the bits of one
dvgo_adam_step per tensor (same element arithmetic), with each tensor's own rate, step count,
learning-rate scale, BF16 copy, gradient clearing and lazy flag; sizes with a scalar tail."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

dvgo = pytest.importorskip("paper_2111_11215_gb300")


def _tensors(seed):
    g = torch.Generator().manual_seed(seed)
    specs = [dict(n=4 * 100003 + 3, lr=0.1, step=5, scale=True, bf16=True, zero=True, lazy=False),
             dict(n=22915, lr=1e-3, step=7, scale=False, bf16=False, zero=True, lazy=False),
             dict(n=1001, lr=0.05, step=2, scale=False, bf16=False, zero=False, lazy=True)]
    out = []
    for sp in specs:
        n = sp["n"]
        t = {k: torch.randn(n, generator=g).cuda() for k in ("param", "grad", "m")}
        t["v"] = torch.rand(n, generator=g).cuda()
        if sp["lazy"]:
            t["grad"][torch.rand(n, generator=g).cuda() < 0.5] = 0.0
        t["lr_scale"] = torch.rand(n, generator=g).cuda() if sp["scale"] else None
        t["param_bf16_out"] = torch.empty(n, dtype=torch.bfloat16, device="cuda") if sp["bf16"] else None
        t.update(lr=sp["lr"], step=sp["step"], zero_grad=sp["zero"], skip_zero_grad=sp["lazy"])
        out.append(t)
    return out


def _clone(ts):
    return [{k: (v.clone() if isinstance(v, torch.Tensor) else v) for k, v in t.items()} for t in ts]


def test_multi_equals_separate_steps_bit_for_bit():
    a = _tensors(11)
    b = _clone(a)
    for t in a:
        dvgo.dvgo_adam_step(t["param"], t["grad"], t["m"], t["v"], t["lr"], t["step"], lr_scale=t["lr_scale"],
                            param_bf16_out=t["param_bf16_out"], zero_grad=t["zero_grad"],
                            skip_zero_grad=t["skip_zero_grad"])
    dvgo.dvgo_adam_step_multi(b)
    torch.cuda.synchronize()
    for ta, tb in zip(a, b):
        for k in ("param", "grad", "m", "v", "param_bf16_out"):
            if ta[k] is None:
                continue
            assert torch.equal(ta[k], tb[k]), k
    # the update did something: the first tensor's parameters moved and its gradient was cleared
    assert float(b[0]["grad"].abs().max()) == 0.0
    assert not torch.equal(b[0]["param"], _tensors(11)[0]["param"])
