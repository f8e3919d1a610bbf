"""The allocation-free FP32 network entry point, called through the C ABI.

rtn_mlp_eval_f32_noalloc serves callers that may not call cudaMalloc (for
example a real-time loop or a host that owns all device memory); it keeps
its activations in a fixed array inside the library.  Its result must equal
that of the FP64 oracle within the 1e-5 relative FP32 tolerance of the
other parity tests, and that of rtn_mlp_eval on an FP32 context (the entry
point that allocates, another FP32 path within 1e-5 of the oracle) within
2e-5, on two calls in a row with different inputs (the array
keeps the previous call's contents, which must not leak into the next
result), with hidden widths on and off the kernels' tile sizes and a node
count just under the array's limit.  This file is named to be collected
last."""
import ctypes as C

import numpy as np
import pytest

import workload as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel_rows(a, b, floor=1e-30):
    a = a.reshape(a.shape[0], -1); b = b.reshape(b.shape[0], -1)
    return float((np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), floor)).max())


@pytest.mark.parametrize("widths,N", [
    ([17, 128, 128, 128, 3], [5, 9, 1, 12]),
    # hidden widths that are not multiples of the hidden kernel's 128-row tile
    # or 16-wide K slice, and 582 nodes: 2 x 200 x 18 x 582 x 4 B = 16.76 MB,
    # just under the 16 MiB array
    ([17, 200, 72, 3], [100] * 5 + [82]),
])
def test_noalloc_matches_allocating_entry_point_and_oracle_twice(orc, widths, N):
    import paper_2203_07747_b300 as rtn
    lib = rtn.load(build_if_missing=True)
    layers = [(np.float32(Wl).astype(np.float64), np.float32(np.random.default_rng(i).normal(0, 0.1, bl.shape)).astype(np.float64))
              for i, (Wl, bl) in enumerate(W.xavier_mlp(widths, 4))]
    Wd = torch.as_tensor(np.concatenate([Wl.ravel() for Wl, _ in layers]), dtype=torch.float32, device="cuda")
    bd = torch.as_tensor(np.concatenate([bl.ravel() for _, bl in layers]), dtype=torch.float32, device="cuda")
    w = (C.c_int * len(widths))(*widths)
    N = np.array(N, np.int32)
    dt = np.full(len(N), 0.05)
    ctl = rtn.Controller(N, dt, W.Q_DIAG, W.R_DIAG, quad=W.QUAD, layers=layers)
    assert 2 * max(widths[1:-1]) * 18 * ctl.n_nodes * 4 <= 16 << 20
    rows = np.concatenate([np.arange(o, o + n) for o, n in zip(np.concatenate([[0], np.cumsum(N + 1)])[:-1], N)])
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for seed in (1, 2):
        X, U = W.random_nodes(ctl.n_states, seed)
        X = np.float32(X).astype(np.float64)
        U = np.float32(U[:ctl.n_nodes]).astype(np.float64)
        xd = torch.as_tensor(X, dtype=torch.float32, device="cuda")
        ud = torch.as_tensor(U, dtype=torch.float32, device="cuda")
        f_ref, J_ref = ctl.mlp_eval(xd, ud)
        xn = xd[torch.as_tensor(rows, device="cuda")].contiguous()
        fD = torch.full((ctl.n_nodes, 3), float("nan"), device="cuda")
        JD = torch.full((ctl.n_nodes, 3, 17), float("nan"), device="cuda")
        err = C.create_string_buffer(256)
        st = lib.rtn_mlp_eval_f32_noalloc(len(layers), w, C.c_void_p(Wd.data_ptr()), C.c_void_p(bd.data_ptr()),
                                          ctl.n_nodes, C.c_void_p(xn.data_ptr()), C.c_void_p(ud.data_ptr()),
                                          C.c_void_p(fD.data_ptr()), C.c_void_p(JD.data_ptr()), stream,
                                          err, 256)
        assert st == 0, err.value
        torch.cuda.synchronize()
        fD, JD = fD.double().cpu().numpy(), JD.double().cpu().numpy()
        # against the FP64 oracle at the FP32 bar of 1e-5, and against the
        # allocating entry point (another FP32 path, itself within 1e-5 of
        # the oracle) at twice that; f_D rows relative to max(|row|, 1e-3)
        # as in the FP32 network parity test
        fr, Jr, *_ = orc.linearize(W.QUAD, layers, N, dt, X, U)
        for Jb, fb, tol in ((Jr, fr, 1e-5), (J_ref.double().cpu().numpy(), f_ref.double().cpu().numpy(), 2e-5)):
            assert _rel_rows(JD, Jb) < tol
            assert _rel_rows(fD, fb, 1e-3) < tol


def test_noalloc_rejects_oversized_problem():
    import paper_2203_07747_b300 as rtn
    lib = rtn.load(build_if_missing=True)
    widths = (C.c_int * 3)(17, 512, 3)
    err = C.create_string_buffer(256)
    dummy = torch.zeros(16, device="cuda")
    p = C.c_void_p(dummy.data_ptr())
    # 2 * 512 * 18 * 1000 floats = 73.7 MB > 16 MiB: rejected before any launch
    st = lib.rtn_mlp_eval_f32_noalloc(2, widths, p, p, 1000, p, p, p, p, None, err, 256)
    assert st == 1 and b"bytes of activation scratch" in err.value
