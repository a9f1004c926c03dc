"""Double-float arithmetic of the GPU's inverse-CDF sampling, emulated on the CPU (numpy float32
operations, each rounded to nearest like the kernel's _rn intrinsics).

* The error-free transformations are exact: TwoSum and Fast2Sum give s + e = a + b, the FMA form
  of Dekker's product gives p + e = a * b, checked in rational arithmetic.
* The sampler's steps in the kernel's order (CDF summed once for its total and again merged with
  the sorted quantiles u_j = ((j + p)/n) Q, the in-bin fraction in FP32, t = t0 + (b + f) w in
  double-float) reproduce the FP64 oracle (Sec. 4.2 sampling reading) within the GPU test's
  tolerances: t to 2e-7 relative + 1e-7, dt to 2e-6 relative + 1e-7."""
from fractions import Fraction

import numpy as np
import pytest

import oracle

f32 = np.float32


def fadd(a, b):
    return f32(f32(a) + f32(b))


def fsub(a, b):
    return f32(f32(a) - f32(b))


def fmul(a, b):
    return f32(f32(a) * f32(b))


def fdiv(a, b):
    return f32(f32(a) / f32(b))


def fma_exact_result(a, b, c):
    # used only where the exact result is an FP32 number (the rounding error of a product or of a
    # quotient): the FP64 product of two FP32 numbers is exact, so one FP64 add then is too
    return f32(float(a) * float(b) + float(c))


def two_sum(a, b):
    s = fadd(a, b)
    bb = fsub(s, a)
    return s, fadd(fsub(a, fsub(s, bb)), fsub(b, bb))


def fast_two_sum(a, b):
    s = fadd(a, b)
    return s, fsub(b, fsub(s, a))


def dadd(a, b):
    s = two_sum(a[0], b[0])
    t = two_sum(a[1], b[1])
    s = fast_two_sum(s[0], fadd(s[1], t[0]))
    return fast_two_sum(s[0], fadd(s[1], t[1]))


def dneg(a):
    return f32(-a[0]), f32(-a[1])


def dmul(a, b):
    p = fmul(a[0], b[0])
    e = fma_exact_result(a[0], b[0], -p)
    return fast_two_sum(p, fadd(e, fadd(fmul(a[0], b[1]), fmul(a[1], b[0]))))


def dmul_f(a, b):
    p = fmul(a[0], b)
    e = fma_exact_result(a[0], b, -p)
    return fast_two_sum(p, fadd(e, fmul(a[1], b)))


def ddiv_n(a, n):
    q1 = fdiv(a[0], n)
    r = fma_exact_result(-q1, n, a[0])
    return fast_two_sum(q1, fdiv(fadd(r, a[1]), n))


def dfrom(x):
    hi = f32(x)
    return hi, f32(x - float(hi))


def dle(a, b):
    return a[0] < b[0] or (a[0] == b[0] and a[1] <= b[1])


def sample(p, t0d, t1d, ns, jit, eta):
    """The kernel's steps, in its order."""
    nb = len(p)
    t0, w = dfrom(t0d), dfrom((t1d - t0d) / nb)
    ome, enb = two_sum(f32(1), f32(-eta)), ddiv_n((f32(eta), f32(0)), f32(nb))

    def q_at(b):
        return dadd(dmul_f(ome, f32(p[b])), enb)
    Q = (f32(0), f32(0))
    for b in range(nb):
        Q = dadd(Q, q_at(b))
    b, Qb, qb, tprev = 0, (f32(0), f32(0)), q_at(0), None
    t, dt = np.zeros(ns, np.float32), np.zeros(ns, np.float32)
    for j in range(ns):
        u = dmul(ddiv_n(two_sum(f32(j), f32(jit)), f32(ns)), Q)
        while b < nb - 1:
            Qn = dadd(Qb, qb)
            if not dle(Qn, u):
                break
            Qb, b = Qn, b + 1
            qb = q_at(b)
        frac = fdiv(dadd(u, dneg(Qb))[0], qb[0])
        tt = dadd(t0, dmul(two_sum(f32(b), frac), w))
        t[j] = tt[0]
        if j > 0:
            dt[j - 1] = dadd(tt, dneg(tprev))[0]
        tprev = tt
    dt[ns - 1] = fdiv(w[0], fdiv(fmul(f32(ns), qb[0]), Q[0]))
    return t, dt


def test_error_free_transformations_are_exact():
    rng = np.random.default_rng(0)
    for _ in range(2000):
        a, b = (f32(x) for x in rng.normal(size=2) * 10.0 ** rng.integers(-6, 6, size=2))
        s, e = two_sum(a, b)
        assert Fraction(float(s)) + Fraction(float(e)) == Fraction(float(a)) + Fraction(float(b))
        big, small = (a, b) if abs(a) >= abs(b) else (b, a)
        s, e = fast_two_sum(big, small)
        assert Fraction(float(s)) + Fraction(float(e)) == Fraction(float(a)) + Fraction(float(b))
        p, e = dmul_f((a, f32(0)), b)
        assert Fraction(float(p)) + Fraction(float(e)) == Fraction(float(a)) * Fraction(float(b))


def test_double_float_division_and_split_are_accurate():
    rng = np.random.default_rng(1)
    for _ in range(500):
        x = float(rng.uniform(1e-3, 1e3))
        n = int(rng.integers(1, 200))
        hi, lo = dfrom(x)
        assert abs(Fraction(float(hi)) + Fraction(float(lo)) - Fraction(x)) <= Fraction(x) * Fraction(1, 2 ** 47)
        q = ddiv_n((hi, lo), f32(n))
        assert abs(Fraction(float(q[0])) + Fraction(float(q[1])) - Fraction(x) / n) <= Fraction(x) / n / 2 ** 44


@pytest.mark.parametrize("nb,ns,eta", [(64, 48, 0.05), (50, 100, 0.0), (7, 3, 0.3), (128, 200, 0.01)])
def test_emulated_sampler_matches_the_oracle(nb, ns, eta):
    rng = np.random.default_rng(nb * 1000 + ns)
    for trial in range(12):
        p = rng.dirichlet(np.full(nb, 0.3)).astype(np.float32)
        if trial % 3 == 0:
            p[rng.random(nb) < 0.3] = 0                      # zero-mass bins
        if trial == 1:
            p[:] = 0
            p[nb // 2] = 1                                   # one-hot
        p = (p / p.sum()).astype(np.float32)
        t0 = float(rng.uniform(0.5, 3.0))
        t1 = t0 + float(rng.uniform(0.01, 3.5))
        jit, e = float(f32(rng.random())), float(f32(eta))
        tg, dtg = sample(p, t0, t1, ns, jit, e)
        tr, dtr = oracle.sample_pdf(p.astype(np.float64), t0, t1, ns, jit=jit, eta=e)
        np.testing.assert_allclose(tg, tr, rtol=2e-7, atol=1e-7)
        np.testing.assert_allclose(dtg, dtr, rtol=2e-6, atol=1e-7)
