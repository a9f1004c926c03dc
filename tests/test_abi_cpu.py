"""CPU checks of the C ABI: the library loads and exports every declared entry point, and the
host-side helpers that need no GPU agree with the oracle."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^[A-Za-z_][\w \*]*?\b(dvgo_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import paper_2111_11215_gb300 as dvgo
    from paper_2111_11215_gb300 import build_lib
    build_lib.build()
    return dvgo.lib()


def test_library_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), f"libdvgo.so does not export {n}"
    import paper_2111_11215_gb300 as dvgo
    assert set(names) == set(dvgo.EXPORTED_SYMBOLS)


def test_abi_version_and_strings(lib):
    import paper_2111_11215_gb300 as dvgo
    assert dvgo.dvgo_abi_version() == 10
    assert dvgo.dvgo_status_string(0) == "ok"
    assert "workspace" in dvgo.dvgo_status_string(-2)


def test_host_helpers_match_oracle(lib):
    import oracle
    import paper_2111_11215_gb300 as dvgo
    for a, s in [(1e-6, 0.0625), (1e-2, 2 / 160), (1e-6, 2 / 160)]:
        assert dvgo.dvgo_shift_from_alpha_init(a, s) == pytest.approx(oracle.shift_from_alpha_init(a, s), rel=1e-6)
    for step in (0, 1, 777, 20000):
        assert dvgo.dvgo_lr_at(0.1, step) == pytest.approx(oracle.lr_decay(0.1, step), rel=1e-6)


def test_workspace_size_bounds_longest_ray(lib):
    import paper_2111_11215_gb300 as dvgo
    p = dvgo.Params(mode=dvgo.DVGO_MODE_FINE, step=2 / 160 * 0.5)
    g = dvgo.GridDesc((160, 160, 160), 1)
    n1 = dvgo.dvgo_workspace_size(p, g, 1)
    n2 = dvgo.dvgo_workspace_size(p, g, 8192)
    # ~555 samples of 40 bytes per ray in the fine mode
    assert n2 > 8192 * 555 * 40 and n2 < 8192 * 600 * 48
    assert n1 > 0
    assert dvgo.dvgo_workspace_size(dvgo.Params(step=0.0), g, 10) == 0


def test_grid_elements_per_layout(lib):
    """Canonical: nx ny nz C; packed: whole 4^3 bricks of 64 points per brick (no GPU needed)."""
    import paper_2111_11215_gb300 as dvgo
    for shape, C in (((160, 160, 160), 12), ((13, 6, 9), 1), ((4, 4, 4), 3), ((2, 5, 17), 2)):
        g = dvgo.GridDesc(shape, C)
        assert dvgo.dvgo_grid_elements(g) == shape[0] * shape[1] * shape[2] * C
        bricks = 1
        for n in shape:
            bricks *= -(-n // 4)
        assert dvgo.dvgo_grid_elements(g.with_(layout=dvgo.DVGO_LAYOUT_PACKED)) == bricks * 64 * C
    assert dvgo.dvgo_grid_elements(dvgo.GridDesc((8, 8, 8), 1, layout=7)) == 0      # invalid layout


def test_sample_pdf_rejects_bins_and_samples_out_of_range(lib):
    """dvgo_sample_pdf checks its sizes before any device work: 1 <= n_bins <= 128 (the staged PDF
    rows), 1 <= n_samples <= 2^24 (sample indices exact in FP32), 0 <= eta <= 1."""
    import ctypes as C
    import paper_2111_11215_gb300 as dvgo
    from paper_2111_11215_gb300 import binding
    p, g = dvgo.Params(mode=dvgo.DVGO_MODE_FINE, step=0.01).c(), dvgo.GridDesc((8, 8, 8), 1).c()
    buf = (C.c_float * 16)()
    ptr = C.cast(buf, C.c_void_p)

    def call(nb, ns, eta):
        return lib.dvgo_sample_pdf(C.byref(p), C.byref(g), 1, ptr, ptr, ptr, nb, ns, None, C.c_float(eta), ptr, ptr,
                                   None)
    for nb, ns, eta in ((0, 8, 0.1), (129, 8, 0.1), (64, 0, 0.1), (64, (1 << 24) + 1, 0.1), (64, 8, -0.5),
                        (64, 8, 1.5)):
        assert call(nb, ns, eta) == binding.DVGO_ERR_INVALID_ARG, (nb, ns, eta)


def test_profile_trace_without_records(lib):
    """Tracing needs no GPU while nothing was recorded: no records, no error; bad arguments are
    rejected."""
    import ctypes as C
    import paper_2111_11215_gb300 as dvgo
    from paper_2111_11215_gb300 import binding
    assert dvgo.binding.dvgo_profile_trace(16) == []
    n = C.c_int(7)
    assert lib.dvgo_profile_trace(-1, None, None, None, C.byref(n)) == binding.DVGO_ERR_INVALID_ARG
    assert lib.dvgo_profile_trace(4, None, None, None, C.byref(n)) == binding.DVGO_ERR_INVALID_ARG


def test_adam_step_multi_checks_before_launching(lib):
    """dvgo_adam_step_multi validates the tensor count and every tensor before enqueueing anything
    (so these calls need no GPU): more than DVGO_ADAM_MAX_TENSORS, a null array with a count, and a
    tensor with a null parameter or a step count of 0 are refused; an empty list is a no-op."""
    import ctypes as C
    from paper_2111_11215_gb300 import binding as B
    L = lib
    assert L.dvgo_adam_step_multi(None, 0, None) == 0
    assert L.dvgo_adam_step_multi(None, 1, None) == -1
    arr = (B._AdamTensor * 5)()
    assert L.dvgo_adam_step_multi(arr, 5, None) == -1
    assert L.dvgo_adam_step_multi(arr, -1, None) == -1
    arr[0].n = 16
    arr[0].h.step = 1
    arr[0].h.beta1, arr[0].h.beta2, arr[0].h.lr = 0.9, 0.999, 0.1
    assert L.dvgo_adam_step_multi(arr, 1, None) == -1      # null pointers with n > 0
    arr[0].n = 0
    arr[0].h.step = 0
    assert L.dvgo_adam_step_multi(arr, 1, None) == -1      # step count 0
    arr[0].h.step = 1
    assert L.dvgo_adam_step_multi(arr, 1, None) == 0       # an empty tensor: nothing to do
