"""GPU parity: every step of the CUDA path against the FP64 oracle on the
same seeded inputs, called through the C ABI.

Tolerances (per node, relative Frobenius norm against the oracle):
  FP32 path: 1e-5 (network value/Jacobian, A, B, phi, u0, updated iterate)
  FP64 steps: plant integration + quaternion renormalisation 1e-9; the FP64
  Riccati sweep writes FP32 outputs, so it must equal the oracle's result
  rounded to FP32 (relative 2^-23 per element).
The FP32 Riccati sweep is held to the same 1e-5 relative
bar on the QP step (measured about 3e-6 at N <= 22)."""
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
    """max over rows of |a - b| / |b| (Frobenius over the trailing axes)."""
    a = a.reshape(a.shape[0], -1); b = b.reshape(b.shape[0], -1)
    return float((np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), floor)).max())


def f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def layers32(layers):
    return [(f32(W_), f32(b)) for W_, b in layers]


def ragged(seed, B):
    g = np.random.default_rng(seed)
    return g.integers(1, 23, B).astype(np.int32), g.uniform(0.02, 0.1, B)


def points(N, seed):
    ns, nn = int(N.sum()) + len(N), int(N.sum())
    X, U = W.random_nodes(ns, seed)
    return f32(X), f32(U[:nn])


def first_rows(N):
    return np.concatenate([[0], np.cumsum(N + 1)])[:-1]


# ---------------------------------------------------------------- a1: network

@pytest.mark.parametrize("widths", [[17, 256, 256, 256, 256, 256, 3], [17, 32, 32, 3],
                                    [17, 100, 200, 3]])
def test_mlp_fp32_matches_oracle(rtn, orc, widths):
    N, dt = ragged(1, 7)
    layers = layers32(W.xavier_mlp(widths, 2))
    # non-zero biases exercise the bias path
    layers = [(Wl, f32(np.random.default_rng(i).normal(0, 0.1, bl.shape))) for i, (Wl, bl) in enumerate(layers)]
    X, U = points(N, 3)
    ctl = rtn.Controller(N, dt, W.Q_DIAG, W.R_DIAG, quad=QUAD, layers=layers)
    fD, JD = ctl.mlp_eval(_dev(X), _dev(U))
    fr, Jr, *_ = orc.linearize(QUAD, layers, N, dt, X, U)
    assert rel_rows(_np(JD), Jr) < 1e-5
    assert rel_rows(_np(fD), fr, 1e-3) < 1e-5


# ------------------------------------------------------------ a2: RK4 + sens.

@pytest.mark.parametrize("with_net", [True, False])
def test_linearize_matches_oracle(rtn, orc, with_net):
    N, dt = ragged(4, 9)
    layers = layers32(W.xavier_mlp([17, 64, 64, 3], 5)) if with_net else None
    X, U = points(N, 6)
    ctl = rtn.Controller(N, dt, W.Q_DIAG, W.R_DIAG, quad=QUAD, layers=layers)
    fD, JD, A, Bm, c = ctl.linearize(_dev(X), _dev(U))
    fr, Jr, Ar, Br, cr = orc.linearize(QUAD, layers, N, f32(dt), X, U)
    assert rel_rows(_np(A), Ar) < 1e-5
    assert rel_rows(_np(Bm), Br) < 1e-5
    # c = phi - x_{k+1}: compare phi
    xo = first_rows(N)
    xn = np.concatenate([X[xo[b] + 1: xo[b] + 1 + N[b]] for b in range(len(N))])
    assert rel_rows(_np(c) + xn, cr + xn) < 1e-5


# --------------------------------------------------------- a3 + a4: QP solve

def _qp_inputs(orc, seed, N, dt, layers=None):
    x, u = points(N, seed)
    fr, Jr, A, Bm, c = orc.linearize(QUAD, layers, N, dt, x, u)
    g = np.random.default_rng(seed)
    xref = f32(x + g.normal(0, 0.2, x.shape))
    uref = f32(np.full_like(u, W.hover_thrust()))
    x0 = f32(x[first_rows(N)] + g.normal(0, 0.05, (len(N), 13)))
    return f32(A), f32(Bm), f32(c), x, u, xref, uref, x0


def _oracle_qp(orc, N, A, Bm, c, x, u, xref, uref, x0):
    dxs, dus = [], []
    xo, uo = 0, 0
    for b, n in enumerate(N):
        st, dx, du = orc.riccati(A[uo:uo + n], Bm[uo:uo + n], c[uo:uo + n], x[xo:xo + n + 1],
                                 u[uo:uo + n], xref[xo:xo + n + 1], uref[uo:uo + n], W.Q_DIAG,
                                 W.R_DIAG, W.Q_DIAG, x0[b])
        assert st == 0
        dxs.append(dx); dus.append(du)
        xo += n + 1; uo += n
    return np.concatenate(dxs), np.concatenate(dus)


def test_qp_solve_fp64_sweep_matches_oracle(rtn, orc):
    N, dt = ragged(7, 11)
    N[0] = 1
    A, Bm, c, x, u, xref, uref, x0 = _qp_inputs(orc, 8, N, dt)
    ctl = rtn.Controller(N, dt, W.Q_DIAG, W.R_DIAG, quad=QUAD, riccati_f64=True)
    dx, du, st = ctl.qp_solve(*[_dev(a) for a in (A, Bm, c, x, u, xref, uref, x0)])
    assert (st.cpu().numpy() == 0).all()
    rdx, rdu = _oracle_qp(orc, N, A, Bm, c, x, u, xref, uref, x0)
    for got, ref in ((_np(dx), rdx), (_np(du), rdu)):
        # equal to the FP64 result up to the final rounding to FP32 (plus a
        # 1e-9 relative allowance for the FP64 arithmetic itself)
        assert np.all(np.abs(got - ref) <= 2.0 ** -23 * np.abs(ref) + 1e-9 * np.abs(ref).max())


def test_qp_solve_fp32_sweep_matches_oracle(rtn, orc):
    N, dt = ragged(7, 11)
    N[0] = 1
    A, Bm, c, x, u, xref, uref, x0 = _qp_inputs(orc, 8, N, dt)
    ctl = rtn.Controller(N, dt, W.Q_DIAG, W.R_DIAG, quad=QUAD)
    dx, du, st = ctl.qp_solve(*[_dev(a) for a in (A, Bm, c, x, u, xref, uref, x0)])
    assert (st.cpu().numpy() == 0).all()
    rdx, rdu = _oracle_qp(orc, N, A, Bm, c, x, u, xref, uref, x0)
    dx, du = _np(dx), _np(du)
    xo, uo = 0, 0
    for b, n in enumerate(N):
        ex = np.abs(dx[xo:xo + n + 1] - rdx[xo:xo + n + 1]).max() / np.abs(rdx[xo:xo + n + 1]).max()
        eu = np.abs(du[uo:uo + n] - rdu[uo:uo + n]).max() / np.abs(rdu[uo:uo + n]).max()
        assert ex < 1e-5 and eu < 1e-5, (b, n, ex, eu)
        xo += n + 1; uo += n


def test_qp_status_nonfinite_and_not_pd(rtn, orc):
    N = np.array([3, 3, 3], np.int32); dt = np.full(3, 0.05)
    A, Bm, c, x, u, xref, uref, x0 = _qp_inputs(orc, 9, N, dt)
    x0 = x0.copy(); x0[1, 4] = np.nan
    ctl = rtn.Controller(N, dt, W.Q_DIAG, W.R_DIAG, quad=QUAD)
    dx, du, st = ctl.qp_solve(*[_dev(a) for a in (A, Bm, c, x, u, xref, uref, x0)])
    assert list(st.cpu().numpy()) == [0, 3, 0]
    assert not _np(dx)[4:8].any() and not _np(du)[3:6].any()
    ctl2 = rtn.Controller(N, dt, W.Q_DIAG, -np.ones(4), quad=QUAD)
    Bz = np.zeros_like(Bm)
    _, _, st2 = ctl2.qp_solve(*[_dev(a) for a in (A, Bz, c, x, u, xref, uref, f32(np.nan_to_num(x0)))])
    assert (st2.cpu().numpy() == 4).all()


# ---------------------------------------------------------------- RTI step

@pytest.mark.parametrize("name,B", [("cfg1_single_fp64", 1), ("cfg2_fp32_batch", 6)])
def test_rti_step_matches_oracle(rtn, orc, name, B):
    prob = W.make_problem(name, seed=1, B=B)
    N, dt = prob["N"], f32(prob["dt"])
    layers = layers32(prob["layers"])
    X, U = points(N, 12)
    xref, uref = W.node_refs(prob)
    xref, uref = f32(xref), f32(uref)
    x0 = f32(X[first_rows(N)] + 0.03)
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


# ------------------------------------------------------------------ plant

@pytest.mark.parametrize("kind,kname", [(0, "nominal"), (1, "drag"), (2, "mlp")])
def test_plant_fp64_matches_oracle(rtn, orc, kind, kname):
    B = 5
    N = np.full(B, 3, np.int32); dt = np.random.default_rng(0).uniform(0.02, 0.1, B)
    layers = layers32(W.xavier_mlp([17, 32, 32, 3], 7))
    X, U = W.random_nodes(B, 13)
    X[:, 3:7] /= np.linalg.norm(X[:, 3:7], axis=1, keepdims=True)
    U = f32(U)
    ctl = rtn.Controller(N, dt, W.Q_DIAG, W.R_DIAG, quad=QUAD, layers=layers)
    xn = _np(ctl.plant_step(_dev(X, torch.float64), _dev(U), kind=kname, nsub=4))
    for b in range(B):
        ref = orc.plant_step(QUAD, X[b], U[b], dt[b], kind=kind, layers=layers, nsub=4)
        assert np.abs(xn[b] - ref).max() / np.abs(ref).max() < 1e-9
        assert abs(np.linalg.norm(xn[b, 3:7]) - 1) < 1e-15


# ------------------------------------------------------------ closed loop

def test_closed_loop_cfg1_matches_oracle(rtn, orc):
    # single instance, 17-32-32-3 residual, circle r = 2 m at 3 m/s, 100 steps
    prob = W.make_problem("cfg1_single_fp64", seed=0)
    steps = 100
    N, dt = prob["N"], prob["dt"]
    layers = layers32(prob["layers"])
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
    traj = _np(traj)
    pos_err = np.linalg.norm(traj[:, 0, :3] - tr[:, 0, :3], axis=1)
    # FP32 linearisation vs FP64 oracle on a stable closed loop: the
    # trajectories stay within 1e-4 m of each other over 100 steps
    assert pos_err.max() < 1e-4, pos_err.max()
    rmse_gpu = np.sqrt(np.mean(np.sum((traj[:, 0, :3] - xrt[0, 1:steps + 1, :3]) ** 2, 1)))
    rmse_orc = np.sqrt(np.mean(np.sum((tr[:, 0, :3] - xrt[0, 1:steps + 1, :3]) ** 2, 1)))
    assert abs(rmse_gpu - rmse_orc) < 1e-4 * max(1.0, rmse_orc)
    assert np.allclose(_np(uh), uhr, atol=1e-3)


def test_reset_and_hover_stationary(rtn):
    B = 4
    N = np.array([1, 2, 5, 3], np.int32); dt = np.full(B, 0.05)
    ctl = rtn.Controller(N, dt, W.Q_DIAG, W.R_DIAG, quad=QUAD)
    x0 = np.zeros((B, 13)); x0[:, 3] = 1; x0[:, :3] = np.arange(B)[:, None]
    ctl.reset(_dev(x0))
    x, u = ctl.get_iterate()
    u0, st = ctl.rti_step(_dev(x0), x.clone(), u.clone())
    assert (st.cpu().numpy() == 0).all()
    assert np.allclose(_np(u0), W.hover_thrust(), atol=2e-5)
