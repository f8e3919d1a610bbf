"""GPU parity of the second-order local model (Eq. 4 to second order): the
network Hessian H_D by forward-over-forward differentiation, the RK4
linearisation with the quadratic term, the RTI step and the graph-captured
closed loop, through the C ABI, against the FP64 oracle.

Tolerances (per node, relative Frobenius norm, FP32 path): 1e-5 on f_D, J_D,
H_D, A, B, phi, u0 and the updated iterate -- the same bar as the first-order
path.  Each linearisation test also checks that the first-order oracle misses
the second-order one by far more than that bar, so that a dropped Hessian
term cannot pass."""
import numpy as np
import pytest

import workload as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

QUAD = W.QUAD


@pytest.fixture(scope="module")
def rtn():
    import paper_2203_07747_b300 as rtn
    rtn.load(build_if_missing=True)
    return rtn


def _dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _np(t):
    return t.detach().double().cpu().numpy()


def rel_rows(a, b, floor=1e-30):
    a = a.reshape(a.shape[0], -1); b = b.reshape(b.shape[0], -1)
    return float((np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), floor)).max())


def f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def _layers(widths, seed, bias=0.1):
    g = np.random.default_rng(seed + 100)
    return [(f32(Wl), f32(g.normal(0, bias, bl.shape))) for Wl, bl in W.xavier_mlp(widths, seed)]


def _points(N, seed):
    ns, nn = int(N.sum()) + len(N), int(N.sum())
    X, U = W.random_nodes(ns, seed)
    return f32(X), f32(U[:nn])


def _node_z(N, X, U):
    """z = [x_k; u_k] of every node in the node-packed order."""
    rows = np.concatenate([np.arange(n) + o for n, o in zip(N, np.concatenate([[0], np.cumsum(N + 1)])[:-1])])
    return np.concatenate([X[rows], U], 1)


def _ragged(seed, B):
    g = np.random.default_rng(seed)
    return g.integers(1, 23, B).astype(np.int32), f32(g.uniform(0.02, 0.1, B))


# widths cover one and several 64-row GEMM tiles, ragged hidden widths and a
# column count (171 per node) that ends inside a 64-column tile
@pytest.mark.parametrize("widths", [[17, 32, 32, 3], [17, 100, 200, 3], [17, 256, 256, 256, 256, 256, 3],
                                    [17, 64, 3]])
def test_mlp_hessian_matches_oracle(rtn, orc, widths):
    N, dt = _ragged(1, 7)
    layers = _layers(widths, 2)
    X, U = _points(N, 3)
    ctl = rtn.Controller(N, dt, W.Q_DIAG, W.R_DIAG, quad=QUAD, layers=layers, second_order=True)
    fD, JD, HD = ctl.mlp_hess(_dev(X), _dev(U))
    fD, JD, HD = _np(fD), _np(JD), _np(HD)
    Z = _node_z(N, X, U)
    ref = [orc.mlp_fwd_hess(layers, z) for z in Z]
    fr = np.stack([r[0] for r in ref]); Jr = np.stack([r[1] for r in ref]); Hr = np.stack([r[2] for r in ref])
    assert rel_rows(fD, fr, 1e-3) < 1e-5
    assert rel_rows(JD, Jr) < 1e-5
    assert rel_rows(HD, Hr) < 1e-5
    # both triangles are written from the same column: exactly symmetric
    assert np.array_equal(HD, np.swapaxes(HD, 2, 3))
    # f_D and J_D equal the first-order FP32 path's to rounding
    f1, J1 = rtn.Controller(N, dt, W.Q_DIAG, W.R_DIAG, quad=QUAD, layers=layers).mlp_eval(_dev(X), _dev(U))
    assert rel_rows(JD, _np(J1)) < 1e-5
    ctl.close()


@pytest.mark.parametrize("scale", [1.0, 3.0])
def test_linearize_second_order_matches_oracle(rtn, orc, scale):
    N, dt = _ragged(4, 9)
    layers = _layers([17, 64, 64, 3], 5)
    layers[0] = (f32(layers[0][0] * scale), layers[0][1])  # larger curvature
    X, U = _points(N, 6)
    ctl = rtn.Controller(N, dt, W.Q_DIAG, W.R_DIAG, quad=QUAD, layers=layers, second_order=True)
    fD, JD, A, Bm, c = ctl.linearize(_dev(X), _dev(U))
    fr, Jr, Hr, Ar, Br, cr = orc.linearize2(QUAD, layers, N, dt, X, U)
    xo = np.concatenate([[0], np.cumsum(N + 1)])[:-1]
    xn = np.concatenate([X[xo[b] + 1: xo[b] + 1 + N[b]] for b in range(len(N))])
    assert rel_rows(_np(JD), Jr) < 1e-5
    assert rel_rows(_np(A), Ar) < 1e-5
    assert rel_rows(_np(Bm), Br) < 1e-5
    assert rel_rows(_np(c) + xn, cr + xn) < 1e-5
    # the first-order model is far from this result
    _, _, A1, B1, c1 = orc.linearize(QUAD, layers, N, dt, X, U)
    assert rel_rows(A1, Ar) > 1e-3 and rel_rows(c1 + xn, cr + xn) > 1e-3
    ctl.close()


def test_rti_step_second_order_matches_oracle(rtn, orc):
    prob = W.make_problem("cfg2_fp32_batch", seed=1, B=6)
    N, dt = prob["N"], f32(prob["dt"])
    layers = _layers([17, 64, 64, 64, 3], 11)
    X, U = _points(N, 12)
    xref, uref = W.node_refs(prob)
    xref, uref = f32(xref), f32(uref)
    xo = np.concatenate([[0], np.cumsum(N + 1)])[:-1]
    x0 = f32(X[xo] + 0.03)
    ctl = rtn.Controller(N, dt, prob["Q"], prob["R"], quad=QUAD, layers=layers, riccati_f64=True,
                         second_order=True)
    ctl.set_iterate(_dev(X), _dev(U))
    u0, st = ctl.rti_step(_dev(x0), _dev(xref), _dev(uref))
    xn, un = ctl.get_iterate()
    u0r, xr, ur, str_ = orc.rti_step2(QUAD, layers, N, dt, prob["Q"], prob["R"], prob["QN"], X, U,
                                      xref, uref, x0)
    assert (st.cpu().numpy() == 0).all() and (str_ == 0).all()
    assert rel_rows(_np(u0), u0r) < 1e-5
    assert rel_rows(_np(xn), xr) < 1e-5
    assert rel_rows(_np(un), ur) < 1e-5
    u01, *_ = orc.rti_step(QUAD, layers, N, dt, prob["Q"], prob["R"], prob["QN"], X, U, xref, uref, x0)
    assert rel_rows(u01, u0r) > 1e-4


def test_closed_loop_second_order_matches_oracle(rtn, orc):
    # the graph-captured closed loop runs the forward-over-forward kernels
    # inside the graph; single instance on the circle, 60 steps, drag plant
    prob = W.make_problem("cfg1_single_fp64", seed=0)
    steps = 60
    N, dt = prob["N"], prob["dt"]
    layers = [(Wl, bl) for Wl, bl in _layers([17, 32, 32, 3], 3, bias=0.01)]
    xrt, urt = W.trajectory_refs(prob, steps)
    xrt, urt = f32(xrt), f32(urt)
    x0 = xrt[:, 0].copy()
    ctl = rtn.Controller(N, dt, prob["Q"], prob["R"], quad=QUAD, layers=layers, riccati_f64=True,
                         second_order=True)
    ctl.reset(_dev(x0))
    xp = _dev(x0, torch.float64)
    traj, uh = ctl.closed_loop(steps, _dev(xrt), _dev(urt), xp, plant="drag")
    torch.cuda.synchronize()
    tr, uhr = orc.closed_loop(QUAD, layers, 1, None, N, f32(dt), prob["Q"], prob["R"], prob["QN"],
                              x0, xrt, urt, steps, second=True)
    pos_err = np.linalg.norm(_np(traj)[:, 0, :3] - tr[:, 0, :3], axis=1)
    assert pos_err.max() < 1e-4, pos_err.max()
    assert np.allclose(_np(uh), uhr, atol=1e-3)


def test_second_order_option_checks(rtn):
    N, dt = np.array([5], np.int32), np.array([0.05])
    layers = _layers([17, 16, 3], 1)
    with pytest.raises(rtn.RtnError, match="UNSUPPORTED"):
        rtn.Controller(N, dt, W.Q_DIAG, W.R_DIAG, quad=QUAD, layers=layers, precision="bf16x2",
                       second_order=True)
    with pytest.raises(rtn.RtnError, match="UNSUPPORTED"):
        rtn.Controller(N, dt, W.Q_DIAG, W.R_DIAG, quad=QUAD, layers=None, second_order=True)
    ctl = rtn.Controller(N, dt, W.Q_DIAG, W.R_DIAG, quad=QUAD, layers=layers)
    X, U = _points(N, 2)
    with pytest.raises(rtn.RtnError, match="UNSUPPORTED"):
        ctl.mlp_hess(_dev(X), _dev(U))
    ctl.close()
