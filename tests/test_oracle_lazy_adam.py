"""Pins of the oracle's lazy Adam variant (this library's option; the paper's Adam is dense):
elements whose gradient is exactly 0 keep parameter and moments; every other element takes exactly
the dense step (Adam is elementwise, so the dense oracle on those elements alone is the reference)."""
import numpy as np

import oracle


def test_lazy_adam_skips_zero_gradients_and_matches_dense_elsewhere():
    g = np.random.default_rng(230)
    n = 101
    p, m, v = g.normal(size=n), g.normal(size=n) * 0.1, np.abs(g.normal(size=n)) * 0.01
    grad = g.normal(size=n)
    grad[g.uniform(size=n) < 0.4] = 0.0
    zero = grad == 0.0
    assert 20 < zero.sum() < 70
    pl, ml, vl = p.copy(), m.copy(), v.copy()
    oracle.adam(pl, grad.copy(), ml, vl, 0.05, 7, skip_zero_grad=True)
    pd, md, vd = p.copy(), m.copy(), v.copy()
    oracle.adam(pd, grad.copy(), md, vd, 0.05, 7)
    for lazy, dense, orig in ((pl, pd, p), (ml, md, m), (vl, vd, v)):
        np.testing.assert_array_equal(lazy[zero], orig[zero])
        np.testing.assert_array_equal(lazy[~zero], dense[~zero])
    # the dense step does move the zero-gradient elements (momentum) -- the two variants differ
    assert np.abs(pd[zero] - p[zero]).min() > 0
