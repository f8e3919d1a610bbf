"""CPU-side checks of the boundary: the shared library builds/loads and
exports every entry point include/rtn.h declares (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "rtn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rtn_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("rtn_create", "rtn_linearize", "rtn_rti_step", "rtn_closed_loop", "rtn_destroy",
              "rtn_last_error", "rtn_mlp_eval", "rtn_qp_solve", "rtn_plant_step"):
        assert s in syms


def test_library_exports_every_declared_symbol():
    import paper_2203_07747_b300 as rtn
    path = rtn._build.build()
    lib = ctypes.CDLL(path)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing
    assert sorted(rtn.EXPORTS) == sorted(declared_symbols())


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_2203_07747_b300 as rtn
    monkeypatch.setattr(rtn, "_lib", None)
    monkeypatch.setattr(rtn._build, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(rtn.RtnError):
        rtn.load()


# ------------------------------------------------ argument checks (host only)
# rtn_create validates every size and option before its first CUDA call, so
# the rejections run without a GPU.

def _create(lib, nx=13, nu=4, N=(5,), dt=(0.05,), widths=(17, 16, 3), opt=None, mlp=True, quad=True):
    import paper_2203_07747_b300 as rtn
    C = ctypes
    B = len(N)
    Na = (C.c_int * max(B, 1))(*N)
    dta = (C.c_double * max(B, 1))(*dt)
    Q = (C.c_double * 13)(*([1.0] * 13))
    R = (C.c_double * 4)(*([0.1] * 4))
    q = rtn._Quad(0.75, 2.5e-3, 2.1e-3, 4.3e-3, 0.14, 0.05, 8.5, 9.81)
    keep = []
    mp = None
    if mlp:
        w = (C.c_int * len(widths))(*widths)
        Ws = [(C.c_float * (widths[l] * widths[l + 1]))() for l in range(len(widths) - 1)]
        bs = [(C.c_float * widths[l + 1])() for l in range(len(widths) - 1)]
        Wp = (C.POINTER(C.c_float) * len(Ws))(*[C.cast(a, C.POINTER(C.c_float)) for a in Ws])
        bp = (C.POINTER(C.c_float) * len(bs))(*[C.cast(a, C.POINTER(C.c_float)) for a in bs])
        keep += [w, Ws, bs, Wp, bp]
        m = rtn._MLP(len(widths) - 1, w, Wp, bp)
        keep.append(m)
        mp = C.byref(m)
    h = C.c_void_p()
    o = rtn._Opt(*(opt or (0, 0, 1, 0, 0, 0)))
    st = lib.rtn_create(C.byref(h), nx, nu, B, Na, dta, Q, R, None, C.byref(q) if quad else None, mp,
                        C.byref(o), None)
    assert not h.value  # no context on a rejected call
    return st, lib.rtn_last_error(None).decode()


@pytest.mark.parametrize("kw,status,msg", [
    (dict(N=()), 1, "bad batch"),                       # empty batch
    (dict(N=(5, 0), dt=(0.05, 0.05)), 1, "N[b] >= 1"),   # an empty horizon
    (dict(dt=(0.0,)), 1, "dt[b] > 0"),
    (dict(dt=(float("nan"),)), 1, "dt[b] > 0"),
    (dict(nx=12), 1, "nx, nu"),
    (dict(widths=(16, 8, 3)), 1, "17 inputs"),
    (dict(widths=(17, 8, 4)), 1, "17 inputs"),
    (dict(widths=(17, 5000, 3)), 1, "hidden width"),
    (dict(widths=(17, 3)), 1, "17 inputs"),             # no hidden layer
    (dict(quad=False), 1, "bad batch"),
    (dict(widths=(17, 8, 6), opt=(2, 0, 1, 0, 0, 0)), 7, "FP32 path"),   # 6 outputs on BF16 kernels
    (dict(mlp=False, opt=(0, 0, 1, 0, 0, 1)), 7, "second_order"),       # second order, no network
    (dict(opt=(1, 0, 1, 0, 0, 1)), 7, "second_order"),                  # second order, BF16
    (dict(opt=(5, 0, 1, 0, 0, 0)), 1, "precision"),
    (dict(opt=(0, 0, 1, 1, -1, 0)), 1, "box_max_iter"),
    (dict(nx=2, nu=1, widths=(3, 8, 1), opt=(0, 0, 1, 1, 0, 0)), 7, "double-integrator"),
    (dict(nx=2, nu=1, widths=(17, 8, 3)), 1, "double-integrator network"),
])
def test_create_rejects_bad_arguments(kw, status, msg):
    import paper_2203_07747_b300 as rtn
    lib = rtn.load(build_if_missing=True)
    st, err = _create(lib, **kw)
    assert st == status, (st, err)
    assert msg in err, err


def test_create_rejects_oversized_batch():
    # more than 2^28 states and nodes: rejected before any allocation
    import paper_2203_07747_b300 as rtn
    lib = rtn.load(build_if_missing=True)
    n = 1 << 20
    st, err = _create(lib, N=(300,) * n, dt=(0.05,) * n)
    assert st == 1 and "too large" in err


def test_rti_step_host_rejects_null_context_and_device_tensors():
    # no GPU needed: a NULL context is an argument error, and the binding
    # only takes contiguous host tensors of the right dtype and shape
    import torch
    import paper_2203_07747_b300 as rtn
    lib = rtn.load(build_if_missing=True)
    assert lib.rtn_rti_step_host(None, None, None, None, None, None) == 1
    with pytest.raises(rtn.RtnError):
        rtn._hptr(torch.zeros((4, 13), dtype=torch.float64), torch.float32, (4, 13), "x0")
    with pytest.raises(rtn.RtnError):
        rtn._hptr(torch.zeros((4, 12), dtype=torch.float32), torch.float32, (4, 13), "x0")
    with pytest.raises(rtn.RtnError):
        rtn._hptr(torch.zeros((13, 4), dtype=torch.float32).t(), torch.float32, (4, 13), "x0")
    assert rtn._hptr(torch.zeros((4, 13), dtype=torch.float32), torch.float32, (4, 13), "x0") is not None



def test_round_e4m3_grid():
    import numpy as np
    # the e4m3 grid of the FP8 workloads' weight quantisation: 3 mantissa
    # bits, exponent bias 7, subnormal spacing 2^-9, largest 448, ties to even
    import workload as W
    assert W.round_e4m3(448.0) == 448.0 and W.round_e4m3(1000.0) == 448.0 and W.round_e4m3(-500.0) == -448.0
    assert W.round_e4m3(2.0 ** -9) == 2.0 ** -9 and W.round_e4m3(2.0 ** -10) == 0.0  # tie -> even (0)
    assert W.round_e4m3(3 * 2.0 ** -10) == 2.0 ** -8                                 # tie -> even (2 x 2^-9)
    assert W.round_e4m3(1.0625) == 1.0 and W.round_e4m3(1.1875) == 1.25              # ties at 1 + 1/16, 1 + 3/16
    assert W.round_e4m3(1.07) == 1.125 and W.round_e4m3(-0.3) == -0.3125
    # every value between the grid points rounds to one of its two neighbours
    grid = sorted({W.round_e4m3(float(k) * 2.0 ** -9) for k in range(0, 1 << 18)})
    assert len(grid) == 127  # 0 and the 126 finite positive codes below 480 (7 subnormal, 119 normal + 448)
    x = np.random.default_rng(0).uniform(-448, 448, 10000)
    r = W.round_e4m3(x)
    assert np.all(np.isin(np.abs(r), grid))
    g = np.array(grid)
    lo = g[np.searchsorted(g, np.abs(x), side="right") - 1]
    hi = g[np.minimum(np.searchsorted(g, np.abs(x), side="left"), len(g) - 1)]
    assert np.all((np.abs(r) == lo) | (np.abs(r) == hi))
    assert np.all(np.abs(np.abs(r) - np.abs(x)) <= np.minimum(np.abs(x) - lo, hi - np.abs(x)) + 1e-12)


def test_quantize_e4m3_per_layer_scale():
    import numpy as np
    import workload as W
    layers = W.xavier_mlp([17, 64, 32, 3], 1)
    for (Wq, bq), (W0, b0) in zip(W.quantize_e4m3(layers), layers):
        s = np.float32(np.abs(np.float32(W0)).max()) / np.float32(448.0)
        codes = Wq / np.float64(s)
        amax = float(np.float32(np.abs(np.float32(W0)).max()))
        assert abs(np.abs(Wq).max() - amax) <= 2.0 ** -23 * amax           # amax maps to the code 448
        assert np.allclose(W.round_e4m3(codes), codes, rtol=1e-6, atol=0)    # every weight on the e4m3 grid
        assert np.abs(Wq - W0).max() <= 2.0 ** -4 * np.abs(W0).max()          # half a unit in the last place at most
        assert np.array_equal(bq, b0)
