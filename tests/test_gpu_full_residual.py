"""GPU parity of the full residual model of Eq. 7, f_D = [0; 0; f_theta;
f_psi]: a 6-output network whose rows 0-2 (linear acceleration) add to dv/dt
and rows 3-5 (body angular acceleration) to domega/dt, through the C ABI, on
the FP32 path (first- and second-order local models), the RTI step, the
plant, the graph-captured closed loop and the training gradient, against the
FP64 oracle.  Tolerances as for the 3-output path: 1e-5 per node (relative
Frobenius norm)."""
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
    g = np.random.default_rng(seed + 200)
    return [(f32(Wl), f32(g.normal(0, bias, bl.shape))) for Wl, bl in W.xavier_mlp(widths, seed)]


def _stack(theta, psi):
    """theta and psi networks side by side as one 6-output network."""
    out = []
    for l, ((Wt, bt), (Wp, bp)) in enumerate(zip(theta, psi)):
        if l == 0:
            Wl = np.vstack([Wt, Wp])
        else:
            Wl = np.zeros((Wt.shape[0] + Wp.shape[0], Wt.shape[1] + Wp.shape[1]))
            Wl[:Wt.shape[0], :Wt.shape[1]] = Wt
            Wl[Wt.shape[0]:, Wt.shape[1]:] = Wp
        out.append((Wl, np.concatenate([bt, bp])))
    return out


def _ragged(seed, B):
    g = np.random.default_rng(seed)
    return g.integers(1, 23, B).astype(np.int32), f32(g.uniform(0.02, 0.1, B))


def _points(N, seed):
    ns, nn = int(N.sum()) + len(N), int(N.sum())
    X, U = W.random_nodes(ns, seed)
    return f32(X), f32(U[:nn])


def _xnext(N, X):
    xo = np.concatenate([[0], np.cumsum(N + 1)])[:-1]
    return np.concatenate([X[xo[b] + 1: xo[b] + 1 + N[b]] for b in range(len(N))])


@pytest.mark.parametrize("widths", [[17, 64, 64, 6], [17, 100, 200, 6], [17, 256, 256, 256, 6]])
def test_full_residual_network_matches_oracle(rtn, orc, widths):
    N, dt = _ragged(1, 7)
    layers = _layers(widths, 2)
    X, U = _points(N, 3)
    ctl = rtn.Controller(N, dt, W.Q_DIAG, W.R_DIAG, quad=QUAD, layers=layers)
    fD, JD = ctl.mlp_eval(_dev(X), _dev(U))
    assert fD.shape == (ctl.n_nodes, 6) and JD.shape == (ctl.n_nodes, 6, 17)
    fr, Jr, *_ = orc.linearize(QUAD, layers, N, dt, X, U)
    assert rel_rows(_np(fD), fr, 1e-3) < 1e-5
    assert rel_rows(_np(JD), Jr) < 1e-5
    ctl.close()


@pytest.mark.parametrize("second", [False, True])
def test_full_residual_linearize_matches_oracle(rtn, orc, second):
    N, dt = _ragged(4, 9)
    layers = _stack(_layers([17, 32, 32, 3], 5), _layers([17, 48, 24, 3], 6))
    X, U = _points(N, 6)
    ctl = rtn.Controller(N, dt, W.Q_DIAG, W.R_DIAG, quad=QUAD, layers=layers, second_order=second)
    fD, JD, A, Bm, c = ctl.linearize(_dev(X), _dev(U))
    if second:
        fr, Jr, Hr, Ar, Br, cr = orc.linearize2(QUAD, layers, N, dt, X, U)
        _, _, HD = ctl.mlp_hess(_dev(X), _dev(U))
        assert rel_rows(_np(HD), Hr) < 1e-5
    else:
        fr, Jr, Ar, Br, cr = orc.linearize(QUAD, layers, N, dt, X, U)
    xn = _xnext(N, X)
    assert rel_rows(_np(JD), Jr) < 1e-5
    assert rel_rows(_np(A), Ar) < 1e-5
    assert rel_rows(_np(Bm), Br) < 1e-5
    assert rel_rows(_np(c) + xn, cr + xn) < 1e-5
    # the angular rows matter: the 3-output truncation is far from this
    trunc = [(Wl, bl) for Wl, bl in _layers([17, 32, 32, 3], 5)]
    _, _, A3, _, c3 = orc.linearize(QUAD, trunc, N, dt, X, U)
    assert rel_rows(c3 + xn, cr + xn) > 1e-3
    ctl.close()


def test_full_residual_rti_step_matches_oracle(rtn, orc):
    prob = W.make_problem("cfg2_fp32_batch", seed=1, B=6)
    N, dt = prob["N"], f32(prob["dt"])
    layers = _layers([17, 64, 64, 6], 11)
    X, U = _points(N, 12)
    xref, uref = W.node_refs(prob)
    xref, uref = f32(xref), f32(uref)
    xo = np.concatenate([[0], np.cumsum(N + 1)])[:-1]
    x0 = f32(X[xo] + 0.03)
    ctl = rtn.Controller(N, dt, prob["Q"], prob["R"], quad=QUAD, layers=layers, riccati_f64=True)
    ctl.set_iterate(_dev(X), _dev(U))
    u0, st = ctl.rti_step(_dev(x0), _dev(xref), _dev(uref))
    xn, un = ctl.get_iterate()
    u0r, xr, ur, str_ = orc.rti_step(QUAD, layers, N, dt, prob["Q"], prob["R"], prob["QN"], X, U,
                                     xref, uref, x0)
    assert (st.cpu().numpy() == 0).all() and (str_ == 0).all()
    assert rel_rows(_np(u0), u0r) < 1e-5
    assert rel_rows(_np(xn), xr) < 1e-5
    assert rel_rows(_np(un), ur) < 1e-5


def test_full_residual_plant_matches_oracle(rtn, orc):
    layers = _layers([17, 32, 32, 6], 13)
    B = 5
    N, dt = np.full(B, 4, np.int32), np.full(B, 0.05)
    ctl = rtn.Controller(N, dt, W.Q_DIAG, W.R_DIAG, quad=QUAD, layers=layers)
    X, U = W.random_nodes(B, 14)
    X = X.astype(np.float64); X[:, 3:7] /= np.linalg.norm(X[:, 3:7], axis=1, keepdims=True)
    U = f32(U)
    xn = _np(ctl.plant_step(_dev(X, torch.float64), _dev(U), kind="mlp"))
    for b in range(B):
        ref = orc.plant_step(QUAD, X[b], U[b], 0.05, kind=2, layers=layers)
        assert np.abs(xn[b] - ref).max() / np.abs(ref).max() < 1e-9
    # the angular rows move omega: the truncated network's plant differs
    trunc = [layers[0], layers[1], (layers[2][0][:3], layers[2][1][:3])]
    ref3 = orc.plant_step(QUAD, X[0], U[0], 0.05, kind=2, layers=trunc)
    assert np.abs(ref3[10:13] - xn[0, 10:13]).max() > 1e-4


def test_full_residual_closed_loop_matches_oracle(rtn, orc):
    # graph-captured closed loop: controller and plant share the 6-output
    # network (the model is exact up to the local model), 60 steps
    prob = W.make_problem("cfg1_single_fp64", seed=0)
    steps = 60
    N, dt = prob["N"], prob["dt"]
    layers = _layers([17, 32, 32, 6], 15, bias=0.02)
    xrt, urt = W.trajectory_refs(prob, steps)
    xrt, urt = f32(xrt), f32(urt)
    x0 = xrt[:, 0].copy()
    ctl = rtn.Controller(N, dt, prob["Q"], prob["R"], quad=QUAD, layers=layers, riccati_f64=True)
    ctl.reset(_dev(x0))
    xp = _dev(x0, torch.float64)
    traj, uh = ctl.closed_loop(steps, _dev(xrt), _dev(urt), xp, plant="mlp")
    torch.cuda.synchronize()
    tr, uhr = orc.closed_loop(QUAD, layers, 2, layers, N, f32(dt), prob["Q"], prob["R"], prob["QN"],
                              x0, xrt, urt, steps)
    pos_err = np.linalg.norm(_np(traj)[:, 0, :3] - tr[:, 0, :3], axis=1)
    assert pos_err.max() < 1e-4, pos_err.max()
    assert np.allclose(_np(uh), uhr, atol=1e-3)


def test_full_residual_mse_gradient_matches_oracle(rtn, orc):
    layers = _layers([17, 48, 48, 6], 16)
    X, U = W.training_samples(300, 17)
    X, U = f32(X), f32(U)
    Y = f32(np.random.default_rng(18).normal(0, 1.0, (300, 6)))
    Z = np.concatenate([X, U], 1)
    loss_r, G_r = orc.mse_grad(layers, Z, Y)
    ctl = rtn.Controller(np.array([4], np.int32), np.array([0.05]), W.Q_DIAG, W.R_DIAG, quad=QUAD,
                         layers=layers)
    loss, g = ctl.mse_grad(_dev(X), _dev(U), _dev(Y))
    g = g.double().cpu().numpy()
    assert abs(loss - loss_r) / loss_r < 1e-5
    nw = sum(w.size for w, _ in layers)
    ow, ob = 0, nw
    for (Wr, br) in G_r:
        gw = g[ow:ow + Wr.size].reshape(Wr.shape)
        gb = g[ob:ob + br.size]
        assert np.linalg.norm(gw - Wr) / np.linalg.norm(Wr) < 1e-5
        assert np.linalg.norm(gb - br) / np.linalg.norm(br) < 1e-5
        ow += Wr.size
        ob += br.size


def test_full_residual_needs_fp32(rtn):
    layers = _layers([17, 16, 6], 1)
    for prec in ("bf16", "bf16x2"):
        with pytest.raises(rtn.RtnError, match="UNSUPPORTED"):
            rtn.Controller(np.array([5], np.int32), np.array([0.05]), W.Q_DIAG, W.R_DIAG, quad=QUAD,
                           layers=layers, precision=prec)
