"""Host-side checks of the C-ABI library (no GPU compute): it loads, exports
every function include/lb.h declares, and rejects invalid parameters before
touching the device."""
import ctypes

import pytest


@pytest.fixture(scope="module")
def lbmod():
    from paper_1806_06943_gb300 import build
    build.build()
    from paper_1806_06943_gb300 import lb
    return lb


def test_every_declared_symbol_is_exported(lbmod):
    names = lbmod.header_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lbmod.LIB, n), n
        assert n in lbmod.SIGNATURES, f"{n} has no binding"
    assert set(lbmod.SIGNATURES) == set(names)


def test_struct_layouts_match_header(lbmod):
    # lb_params: 2 ints, 2 doubles, 3 doubles, 2 doubles, 2 ints, 2 doubles, 2 ints, pointer
    assert ctypes.sizeof(lbmod.lb_params) == 8 + 16 + 24 + 16 + 8 + 16 + 8 + 8
    assert ctypes.sizeof(lbmod.lb_obs) == 8 + 16 + 32 + 8 * 5 + 8


@pytest.mark.parametrize("kw,needle", [
    (dict(nx=4, ny=16), "nx=4"),
    (dict(nx=16, ny=3), "ny=3"),
    (dict(nx=16, ny=16, tau=(0.5, 1.0)), "tau[0]"),
    (dict(nx=16, ny=16, tau=(1.0, float("nan"))), "tau[1]"),
    (dict(nx=16, ny=16, G1=float("inf")), "non-finite"),
    (dict(nx=16, ny=16, walls=2), "walls"),
    (dict(nx=16, ny=16, precision=7), "precision"),
    (dict(nx=16, ny=16, forcing=2), "forcing"),
    (dict(nx=16, ny=16, forcing=1, precision=1), "LB_FP64"),     # the velocity shift is FP64 only
])
def test_invalid_parameters_rejected(lbmod, kw, needle):
    p = lbmod.make_params(**kw)
    h = ctypes.c_void_p()
    rc = lbmod.LIB.lb_create(ctypes.byref(p), ctypes.byref(h))
    assert rc == lbmod.LB_EINVAL
    assert not h.value
    assert needle in lbmod.LIB.lb_last_error().decode()


def test_null_handles_rejected(lbmod):
    assert lbmod.LIB.lb_step(None, 1) == lbmod.LB_EINVAL
    assert lbmod.LIB.lb_observables(None, None) == lbmod.LB_EINVAL
    assert lbmod.LIB.lb_batch_step(None, 1) == lbmod.LB_EINVAL
    assert lbmod.LIB.lb_time(None) == -1
    lbmod.LIB.lb_destroy(None)
    lbmod.LIB.lb_batch_destroy(None)


def test_batch_rejects_mixed_precision(lbmod):
    arr = (lbmod.lb_params * 2)()
    arr[0] = lbmod.make_params(16, 16, precision=0)
    arr[1] = lbmod.make_params(16, 16, precision=1)
    b = ctypes.c_void_p()
    assert lbmod.LIB.lb_batch_create(arr, 2, ctypes.byref(b)) == lbmod.LB_EINVAL
    assert lbmod.LIB.lb_batch_create(arr, 0, ctypes.byref(b)) == lbmod.LB_EINVAL


@pytest.mark.parametrize("kw,needle", [
    (dict(nx=4, ny=8, nz=8), "nz must be >= 5"),
    (dict(nx=8, ny=8, nz=8, tau=(0.5, 1.0)), "tau"),
    (dict(nx=8, ny=8, nz=8, G1=float("nan")), "non-finite"),
    (dict(nx=8, ny=8, nz=8, precision=3), "precision"),
])
def test_3d_parameters_rejected_before_any_cuda_call(lbmod, kw, needle):
    with pytest.raises(lbmod.LBError) as ei:
        lbmod.Lattice3(**kw)
    assert ei.value.code == lbmod.LB_EINVAL and needle in str(ei.value)
