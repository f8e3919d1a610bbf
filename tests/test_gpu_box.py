"""GPU parity of the box-constrained QP (the thrust bounds of Sec. V inside
the QP; primal-dual active set on the Riccati structure) against the FP64
oracle.  The QP data (A, B, c) are the oracle's linearisation of the nominal
model rounded to FP32 and fed to both sides, so the comparison is the solver
alone.  The optimum is unique (R > 0), so the step agrees wherever both
sides converge, whatever sequence of active sets each took; the tolerance is
the FP32 path's 1e-5 per instance."""
import numpy as np
import pytest

import workload as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
QUAD = W.QUAD
Q, R = W.Q_DIAG, W.R_DIAG


@pytest.fixture(scope="module")
def rtn():
    import paper_2203_07747_b300 as rtn
    rtn.load(build_if_missing=True)
    return rtn


def f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def batch_qp(orc, B, N, seed, scale):
    """B instances of the nominal model linearised along perturbed hover
    trajectories with distant references (bounds become active)."""
    rng = np.random.default_rng(seed)
    xs, us, xrs, urs, x0s = [], [], [], [], []
    for b in range(B):
        x = np.zeros((N + 1, 13)); x[:, 3] = 1.0
        x[:, 7:10] += rng.normal(0, 2 * scale, 3)
        u = np.clip(np.full((N, 4), W.hover_thrust()) + rng.uniform(-1.5, 1.5, (N, 4)) * scale,
                    0, QUAD["u_max"])
        xr = np.zeros((N + 1, 13)); xr[:, 3] = 1.0
        xr[:, :3] += rng.normal(0, 3 * scale, 3)
        xs.append(x); us.append(u); xrs.append(xr); urs.append(np.full((N, 4), W.hover_thrust()))
        x0s.append(x[0] + rng.normal(0, 0.5 * scale, 13))
    x, u = f32(np.concatenate(xs)), f32(np.concatenate(us))
    xr, ur, x0 = f32(np.concatenate(xrs)), f32(np.concatenate(urs)), f32(np.array(x0s))
    Ns = np.full(B, N, np.int32)
    _, _, A, Bm, c = orc.linearize(QUAD, [], Ns, np.full(B, 0.05), x, u)
    return Ns, f32(A), f32(Bm), f32(c), x, u, xr, ur, x0


@pytest.mark.parametrize("scale", [0.5, 1.0])
def test_box_qp_matches_oracle(rtn, orc, scale):
    B, N = 24, 10
    Ns, A, Bm, c, x, u, xr, ur, x0 = batch_qp(orc, B, N, 3, scale)
    ctl = rtn.Controller(Ns, np.full(B, 0.05), Q, R, QN=Q, quad=QUAD, box_qp=True, box_max_iter=40)
    dx, du, st = ctl.qp_solve(dev(A), dev(Bm), dev(c), dev(x), dev(u), dev(xr), dev(ur), dev(x0))
    du, dx, st = du.double().cpu().numpy(), dx.double().cpu().numpy(), st.cpu().numpy()
    its = ctl.box_iterations()
    active_instances = 0
    for b in range(B):
        s_, e_ = b * N, (b + 1) * N
        lb, ub = -u[s_:e_], QUAD["u_max"] - u[s_:e_]
        sto, dxo, duo, ito = orc.box_qp(A[s_:e_], Bm[s_:e_], c[s_:e_], x[b * (N + 1):(b + 1) * (N + 1)],
                                        u[s_:e_], xr[b * (N + 1):(b + 1) * (N + 1)], ur[s_:e_], Q, R, Q,
                                        x0[b], lb, ub, max_iter=40)
        assert sto == 0 and st[b] == 0, (b, sto, st[b])
        g = du[s_:e_]
        err = np.linalg.norm(g - duo) / max(np.linalg.norm(duo), 1e-12)
        assert err < 1e-5, (b, err, its[b], ito)
        # the step keeps every thrust in [0, u_max] (up to FP32 rounding)
        assert (g >= lb - 1e-5).all() and (g <= ub + 1e-5).all()
        if ito > 1:
            active_instances += 1
        xs = dx[b * (N + 1):(b + 1) * (N + 1)]
        xo = dxo
        assert np.linalg.norm(xs - xo) / max(np.linalg.norm(xo), 1e-12) < 1e-5
    assert active_instances >= B // 3  # the bounds are exercised


def test_box_qp_inactive_bounds_equal_unconstrained(rtn, orc):
    B, N = 16, 10
    Ns, A, Bm, c, x, u, xr, ur, x0 = batch_qp(orc, B, N, 5, 0.05)
    args = [dev(v) for v in (A, Bm, c, x, u, xr, ur, x0)]
    cb = rtn.Controller(Ns, np.full(B, 0.05), Q, R, QN=Q, quad=QUAD, box_qp=True)
    cu = rtn.Controller(Ns, np.full(B, 0.05), Q, R, QN=Q, quad=QUAD)
    dxb, dub, stb = cb.qp_solve(*args)
    dxu, duu, stu = cu.qp_solve(*args)
    assert (cb.box_iterations() == 1).all()
    assert (stb.cpu().numpy() == 0).all() and (stu.cpu().numpy() == 0).all()
    assert torch.equal(dub, duu)  # the same sweep
    assert (dxb - dxu).abs().max().item() <= 1e-5 * max(1.0, dxu.abs().max().item())


def test_box_qp_iteration_cap_reports_and_stays_feasible(rtn, orc):
    B, N = 24, 10
    Ns, A, Bm, c, x, u, xr, ur, x0 = batch_qp(orc, B, N, 3, 1.0)
    ctl = rtn.Controller(Ns, np.full(B, 0.05), Q, R, QN=Q, quad=QUAD, box_qp=True, box_max_iter=1)
    _, du, st = ctl.qp_solve(dev(A), dev(Bm), dev(c), dev(x), dev(u), dev(xr), dev(ur), dev(x0))
    st, du = st.cpu().numpy(), du.double().cpu().numpy()
    assert set(np.unique(st)) <= {0, 8} and (st == 8).any()
    lb, ub = -u, QUAD["u_max"] - u
    assert (du >= lb - 1e-5).all() and (du <= ub + 1e-5).all()


def test_rti_step_box_matches_oracle(rtn, orc):
    # a full RTI step (a1..a4) with the small residual network and the box QP
    prob = W.make_problem("cfg2_fp32_batch", seed=3, B=6)
    layers = [(f32(w), f32(b)) for w, b in W.xavier_mlp([17, 32, 32, 3], 1)]
    N, dt = prob["N"], f32(prob["dt"])
    X, U = W.random_nodes(int(N.sum()) + len(N), 21)
    X, U = f32(X), f32(U[:int(N.sum())])
    xref, uref = W.node_refs(prob)
    xref, uref = f32(xref), f32(uref)
    x0 = f32(X[np.concatenate([[0], np.cumsum(N + 1)])[:-1]] + 0.5)
    ctl = rtn.Controller(N, dt, prob["Q"], prob["R"], QN=prob["QN"], quad=QUAD, layers=layers,
                         box_qp=True, box_max_iter=40, shift=False)
    ctl.set_iterate(dev(X), dev(U))
    u0, st = ctl.rti_step(dev(x0), dev(xref), dev(uref))
    xn, un = ctl.get_iterate()
    u0r, xr_, ur_, str_, itr = orc.rti_step_box(QUAD, layers, N, dt, prob["Q"], prob["R"], prob["QN"],
                                                X, U, xref, uref, x0, shift=False, max_iter=40)
    assert (str_ == 0).all() and (st.cpu().numpy() == 0).all()
    assert (itr > 1).any()  # some instance hit its bounds
    assert np.abs(u0.double().cpu().numpy() - u0r).max() / np.abs(u0r).max() < 1e-5
    un = un.double().cpu().numpy()
    assert np.abs(un - ur_).max() / np.abs(ur_).max() < 1e-5
    assert (un >= -1e-5).all() and (un <= QUAD["u_max"] + 1e-5).all()
