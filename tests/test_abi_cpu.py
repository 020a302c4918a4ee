"""Host-side checks of the C ABI that need no GPU: the library builds, loads and
exports every function include/ep_tv.h declares, and argument checking returns
synchronously before any device work."""
import ctypes
import os
import re

import pytest

from paper_2110_01585_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "ep_tv.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ep_tv_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def test_header_declares_the_boundary_calls():
    names = _declared_functions()
    for required in ("ep_tv_init", "ep_tv_sweep", "ep_tv_em_beta", "ep_tv_posterior"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert names
    for name in names:
        assert hasattr(lib, name), name
    # the binding wraps exactly what the header declares
    assert set(_lib.SIGNATURES) == set(names)


def test_default_params(lib):
    p = _lib.Params()
    assert lib.ep_tv_default_params(ctypes.byref(p)) == 0
    assert p.damping == 0.5 and p.var_cap == 1e8 and p.periodic == 1
    assert p.rbmc_samples == 32 and p.order_mode == 0 and p.precision == 0
    assert p.prior == _lib.PRIOR_L1
    assert lib.ep_tv_default_params(None) == 1


def _op(h=8, w=8, op=0, m=None):
    o = _lib.Operator()
    o.op, o.height, o.width, o.m = op, h, w, h * w if m is None else m
    return o


@pytest.mark.parametrize("mutate", [
    lambda o, p: setattr(p, "xi", 0.0),
    lambda o, p: setattr(p, "xi", float("nan")),
    lambda o, p: setattr(p, "beta", -1.0),
    lambda o, p: setattr(p, "damping", 0.0),
    lambda o, p: setattr(p, "damping", 1.5),
    lambda o, p: setattr(p, "var_cap", -1.0),
    lambda o, p: setattr(o, "width", 7),           # periodic needs even sizes
    lambda o, p: setattr(o, "m", 3),               # identity needs m == N
    lambda o, p: setattr(o, "op", 9),
    lambda o, p: (setattr(o, "op", 1)),            # convolution without a kernel
    lambda o, p: setattr(p, "order_mode", 3),
    lambda o, p: setattr(p, "prior", 3),
    # mixture priors (Sec. II-B): omega in (0, 1), positive component variances
    lambda o, p: (setattr(p, "prior", 1), setattr(p, "omega", 0.5), setattr(p, "s1_sq", 1.0)),
    lambda o, p: (setattr(p, "prior", 1), setattr(p, "omega", 1.0), setattr(p, "s1_sq", 1.0),
                  setattr(p, "s2_sq", 0.1)),
    lambda o, p: (setattr(p, "prior", 2), setattr(p, "omega", 0.0), setattr(p, "s1_sq", 1.0)),
    lambda o, p: (setattr(p, "prior", 2), setattr(p, "omega", 0.5), setattr(p, "s1_sq", -1.0)),
])
def test_invalid_arguments_are_rejected_on_the_host(lib, mutate):
    o = _op()
    p = _lib.Params()
    lib.ep_tv_default_params(ctypes.byref(p))
    p.xi, p.beta = 0.01, 1.0
    mutate(o, p)
    ctx = ctypes.c_void_p()
    y = ctypes.c_void_p(16)  # never dereferenced: argument checks come first
    assert lib.ep_tv_init(ctypes.byref(o), y, ctypes.byref(p), None, ctypes.byref(ctx)) == 1
    assert not ctx.value


def _hadamard_op(h, w, patterns):
    o = _op(h, w, op=_lib.OP_HADAMARD, m=len(patterns))
    keep = (ctypes.c_int32 * max(len(patterns), 1))(*patterns)
    o.patterns = ctypes.cast(keep, ctypes.POINTER(ctypes.c_int32))
    return o, keep


@pytest.mark.parametrize("h,w,patterns", [
    (8, 12, [0, 1, 2]),          # sides must be powers of two
    (6, 8, [0, 1, 2]),
    (8, 8, [0, 1, 1]),           # patterns must be distinct
    (8, 8, [0, 64]),             # and inside [0, N)
    (8, 8, [-1, 3]),
    (2, 2, [0, 1, 2, 3, 0]),     # M > N
])
def test_invalid_hadamard_operator_is_rejected_on_the_host(lib, h, w, patterns):
    o, keep = _hadamard_op(h, w, patterns)
    p = _lib.Params()
    lib.ep_tv_default_params(ctypes.byref(p))
    p.xi, p.beta = 0.01, 1.0
    ctx = ctypes.c_void_p()
    assert lib.ep_tv_init(ctypes.byref(o), ctypes.c_void_p(16), ctypes.byref(p), None,
                          ctypes.byref(ctx)) == 1
    assert not ctx.value
    o.patterns = None  # no pattern list
    assert lib.ep_tv_init(ctypes.byref(o), ctypes.c_void_p(16), ctypes.byref(p), None,
                          ctypes.byref(ctx)) == 1


def test_null_context_calls_return_arg_error(lib):
    assert lib.ep_tv_sweep(None, 1, None, 0) == 1
    assert lib.ep_tv_em_beta(None, None, None) == 1
    assert lib.ep_tv_posterior(None, None, None) == 1
    lib.ep_tv_destroy(None)


def test_status_strings(lib):
    for code in range(9):
        s = lib.ep_tv_status_str(code)
        assert isinstance(s, bytes) and s
