"""Pins of the FP64 oracle against facts that do not come from the oracle
itself: finite differences, closed-form trajectories, invariants, a dense
KKT solve, a textbook scalar Riccati fixed point and an independent rotation
library.  CPU only."""
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import workload as W

QUAD = W.QUAD
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# ------------------------------------------------------------------ MLP (Eq. 4)

@pytest.mark.parametrize("widths", [[17, 32, 32, 3], [17, 64, 64, 64, 3], [17, 8, 3]])
def test_mlp_jacobian_vs_central_fd(orc, widths):
    layers = W.xavier_mlp(widths, 3)
    rng = np.random.default_rng(1)
    for _ in range(3):
        z = rng.normal(0, 1, 17)
        f, J = orc.mlp_fwd_jac(layers, z)
        assert np.allclose(f, orc.mlp_forward(layers, z), rtol=0, atol=1e-15)
        Jfd = np.zeros_like(J)
        for j in range(17):
            h = 1e-6 * max(1.0, abs(z[j]))
            zp, zm = z.copy(), z.copy()
            zp[j] += h; zm[j] -= h
            Jfd[:, j] = (orc.mlp_forward(layers, zp) - orc.mlp_forward(layers, zm)) / (2 * h)
        assert _rel(J, Jfd) < 1e-8


def test_mlp_forward_vs_reverse_mode(orc):
    layers = W.xavier_mlp([17, 128, 128, 128, 3], 5)
    z = np.random.default_rng(2).normal(0, 2, 17)
    _, J = orc.mlp_fwd_jac(layers, z)
    assert _rel(J, orc.mlp_rev_jac(layers, z)) < 1e-13


def test_mlp_single_unit_closed_form(orc):
    # f = w2 tanh(w1 . z + b1) + b2 ; J = w2 (1 - tanh^2) w1
    rng = np.random.default_rng(3)
    w1, b1, w2, b2 = rng.normal(size=(1, 17)), rng.normal(size=1), rng.normal(size=(3, 1)), rng.normal(size=3)
    z = rng.normal(size=17)
    s = float((w1 @ z)[0] + b1[0])
    f, J = orc.mlp_fwd_jac([(w1, b1), (w2, b2)], z)
    assert np.allclose(f, w2[:, 0] * np.tanh(s) + b2, rtol=1e-15, atol=1e-15)
    assert np.allclose(J, np.outer(w2[:, 0], w1[0]) * (1 - np.tanh(s) ** 2), rtol=1e-14, atol=1e-16)


def test_mlp_zero_output_network(orc):
    # the runtime-analysis network of Sec. IV is forced to output zero
    layers = [(W_ * 0, b * 0) for W_, b in W.xavier_mlp([17, 16, 16, 3], 0)]
    f, J = orc.mlp_fwd_jac(layers, np.ones(17))
    assert not f.any() and not J.any()


# ---------------------------------------------------------- nominal model (Eq. 6)

def test_qrot_matches_rotation_library(orc):
    rng = np.random.default_rng(4)
    for _ in range(5):
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        v = rng.normal(size=3)
        ref = Rotation.from_quat([q[1], q[2], q[3], q[0]]).apply(v)
        assert np.allclose(orc.qrot(q, v), ref, atol=1e-14)
    # literal q v q^*: scales by |q|^2 for a non-unit quaternion
    q = np.array([2.0, 0, 0, 0])
    assert np.allclose(orc.qrot(q, [1.0, 2.0, 3.0]), [4.0, 8.0, 12.0])


def test_rotor_torques_from_fig3_geometry(orc):
    # torque of each single rotor = r_i x (0,0,T) with the X-layout positions,
    # yaw reaction -c_tau T for CCW rotors (0, 2), +c_tau T for CW (1, 3)
    d = QUAD["arm"] / np.sqrt(2)
    pos = np.array([[d, -d, 0], [-d, -d, 0], [-d, d, 0], [d, d, 0]])
    spin = np.array([-1, 1, -1, 1])
    J = np.array([QUAD["Jx"], QUAD["Jy"], QUAD["Jz"]])
    x = np.zeros(13); x[3] = 1.0
    for i in range(4):
        u = np.zeros(4); u[i] = 2.0
        tau = np.cross(pos[i], [0, 0, 2.0]) + [0, 0, spin[i] * QUAD["c_tau"] * 2.0]
        assert np.allclose(orc.quad_f(QUAD, x, u)[10:], tau / J, atol=1e-12)


def test_hover_is_equilibrium(orc):
    x = np.zeros(13); x[3] = 1.0
    u = np.full(4, W.hover_thrust())
    assert np.abs(orc.quad_f(QUAD, x, u)).max() < 1e-14


def test_free_fall_rk4_exact(orc):
    # T = 0, omega = 0: p(t) = p0 + v0 t + 1/2 g t^2, exact for RK4
    x = np.zeros(13)
    x[0:3] = [0.3, -0.2, 1.0]
    q = np.array([0.9, 0.1, -0.3, 0.2]); x[3:7] = q / np.linalg.norm(q)
    x[7:10] = [1.0, -2.0, 0.5]
    dt = 0.05
    phi, A, B = orc.rk4_lin(QUAD, x, np.zeros(4), dt)
    p = x[0:3] + x[7:10] * dt + 0.5 * np.array([0, 0, -QUAD["g"]]) * dt ** 2
    assert np.allclose(phi[0:3], p, atol=1e-14)
    assert np.allclose(phi[7:10], x[7:10] + np.array([0, 0, -QUAD["g"]]) * dt, atol=1e-14)
    # the p-v block of A is dt * I exactly
    assert np.allclose(A[0:3, 7:10], dt * np.eye(3), atol=1e-15)


def test_torque_free_principal_spin(orc):
    # omega along a principal axis with no torque stays constant; the
    # attitude is q(t) = (cos(wt/2), 0, 0, sin(wt/2))
    wz, dt = 2.0, 0.01
    x = np.zeros(13); x[3] = 1.0; x[12] = wz
    for _ in range(50):
        x = orc.rk4_true(QUAD, x, np.zeros(4), dt)
    t = 50 * dt
    assert abs(x[12] - wz) < 1e-15
    assert np.allclose(x[3:7], [np.cos(wz * t / 2), 0, 0, np.sin(wz * t / 2)], atol=1e-11)


def test_dfdz_vs_central_fd(orc):
    rng = np.random.default_rng(6)
    X, U = W.random_nodes(4, 1)
    for x, u in zip(X, U):
        D = orc.quad_dfdz(QUAD, x, u)
        z = np.concatenate([x, u])
        Dfd = np.zeros_like(D)
        for j in range(17):
            h = 1e-6 * max(1.0, abs(z[j]))
            zp, zm = z.copy(), z.copy()
            zp[j] += h; zm[j] -= h
            Dfd[:, j] = (orc.quad_f(QUAD, zp[:13], zp[13:]) - orc.quad_f(QUAD, zm[:13], zm[13:])) / (2 * h)
        assert _rel(D, Dfd) < 1e-8


# ------------------------------------------------- RK4 sensitivities (Eq. 2)

def test_rk4_sensitivities_vs_fd(orc):
    layers = W.xavier_mlp([17, 32, 32, 3], 1)
    X, U = W.random_nodes(3, 2)
    for x, u in zip(X, U):
        fbar, J = orc.mlp_fwd_jac(layers, np.concatenate([x, u]))
        phi, A, B = orc.rk4_lin(QUAD, x, u, 0.05, fbar, J)
        z = np.concatenate([x, u])
        G = np.zeros((13, 17))
        for j in range(17):
            h = 1e-6 * max(1.0, abs(z[j]))
            zp, zm = z.copy(), z.copy()
            zp[j] += h; zm[j] -= h
            # the local model stays anchored at (x, u) while the stage moves
            def ph(zz):
                xx, uu = zz[:13], zz[13:]
                f2 = fbar + J @ (zz - z)
                return orc.rk4_lin(QUAD, xx, uu, 0.05, f2, J)[0]
            G[:, j] = (ph(zp) - ph(zm)) / (2 * h)
        assert _rel(np.hstack([A, B]), G) < 1e-8


def test_local_model_error_is_third_order(orc):
    # |phi(f_F + f_D*) - phi(f_F + f_D)| = O(dt^3): halving dt divides it by ~8
    # (asymptotic regime: the thrust-driven stage offsets must be small)
    layers = W.xavier_mlp([17, 32, 32, 3], 2)
    X, U = W.random_nodes(6, 3)
    for x, u in zip(X, U):
        fbar, J = orc.mlp_fwd_jac(layers, np.concatenate([x, u]))
        err = []
        for dt in (0.002, 0.001, 0.0005):
            loc = orc.rk4_lin(QUAD, x, u, dt, fbar, J)[0]
            tru = orc.rk4_true(QUAD, x, u, dt, kind=2, layers=layers)
            err.append(np.linalg.norm(loc - tru))
        r1, r2 = err[0] / err[1], err[1] / err[2]
        assert 7.5 < r1 < 8.5 and 7.5 < r2 < 8.5, (err, r1, r2)


def test_zero_network_local_model_exact(orc):
    layers = [(W_ * 0, b * 0) for W_, b in W.xavier_mlp([17, 16, 3], 0)]
    x, u = W.random_nodes(1, 4)
    fbar, J = orc.mlp_fwd_jac(layers, np.concatenate([x[0], u[0]]))
    loc = orc.rk4_lin(QUAD, x[0], u[0], 0.05, fbar, J)[0]
    assert np.array_equal(loc, orc.rk4_true(QUAD, x[0], u[0], 0.05, kind=2, layers=layers))
    assert np.array_equal(loc, orc.rk4_true(QUAD, x[0], u[0], 0.05, kind=0))


# --------------------------------------------------------- quaternion norm

def test_plant_renormalises_quaternion(orc):
    X, U = W.random_nodes(5, 5)
    for x, u in zip(X, U):
        x = x.copy(); x[3:7] /= np.linalg.norm(x[3:7])
        xn = orc.plant_step(QUAD, x, u, 0.05, kind=1)
        assert abs(np.linalg.norm(xn[3:7]) - 1.0) <= 4e-16


@pytest.mark.parametrize("wz", [1.0, 5.0, 20.0])
def test_rk4_quaternion_norm_drift_closed_form(orc, wz):
    # constant spin about a principal axis with zero torque: the exact flow
    # keeps |q| = 1, one RK4 step is the 4th-order Taylor polynomial of the
    # rotation, whose modulus is sqrt(1 - th^6/72 + th^8/576), th = |w| dt / 2
    dt = 0.05
    x = np.zeros(13); x[3:7] = [0.8, 0.0, 0.0, 0.6]; x[12] = wz
    u = np.full(4, 1.0)
    xn = orc.rk4_true(QUAD, x, u, dt)
    th = wz * dt / 2
    assert abs(np.linalg.norm(xn[3:7]) - np.sqrt(1 - th ** 6 / 72 + th ** 8 / 576)) < 1e-15


def test_drag_matches_rotation_library(orc):
    rng = np.random.default_rng(7)
    for _ in range(4):
        q = rng.normal(size=4); q /= np.linalg.norm(q)
        v = rng.normal(0, 5, 3)
        x = np.zeros(13); x[3:7] = q; x[7:10] = v
        R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        ref = -R @ np.diag([0.3, 0.3, 0.1]) @ R.T @ v - 0.01 * np.linalg.norm(v) * v
        assert np.allclose(orc.drag(x), ref, atol=1e-13)


# ---------------------------------------------------------------- Riccati/QP

def _random_qp(rng, N, nx=13, nu=4):
    A = np.eye(nx) + 0.1 * rng.normal(size=(N, nx, nx))
    B = 0.1 * rng.normal(size=(N, nx, nu))
    c = 0.01 * rng.normal(size=(N, nx))
    x = rng.normal(size=(N + 1, nx)); u = rng.normal(size=(N, nu))
    xr = rng.normal(size=(N + 1, nx)); ur = rng.normal(size=(N, nu))
    Q = rng.uniform(0.1, 10, nx); R = rng.uniform(0.05, 1, nu); QN = rng.uniform(0.1, 10, nx)
    x0m = x[0] + 0.1 * rng.normal(size=nx)
    return A, B, c, x, u, xr, ur, Q, R, QN, x0m


@pytest.mark.parametrize("N", [1, 2, 3, 5])
def test_riccati_matches_dense_kkt(orc, N):
    rng = np.random.default_rng(10 + N)
    qp = _random_qp(rng, N)
    st, dx, du = orc.riccati(*qp)
    st2, dx2, du2 = orc.kkt_dense(*qp)
    assert st == 0 and st2 == 0
    assert _rel(dx, dx2) < 1e-10 and _rel(du, du2) < 1e-10


def test_riccati_kkt_residual(orc):
    # stationarity of the Lagrangian and primal feasibility at the solution
    rng = np.random.default_rng(20)
    N = 8
    A, B, c, x, u, xr, ur, Q, R, QN, x0m = _random_qp(rng, N)
    st, dx, du = orc.riccati(A, B, c, x, u, xr, ur, Q, R, QN, x0m)
    assert st == 0
    assert np.allclose(dx[0], x0m - x[0], atol=1e-12)
    for k in range(N):
        assert np.abs(dx[k + 1] - (A[k] @ dx[k] + B[k] @ du[k] + c[k])).max() < 1e-10
    # adjoint recursion: lam_N = QN(x_N + dx_N - xr_N); lam_k = Q(...) + A' lam_{k+1}
    lam = QN * (x[N] + dx[N] - xr[N])
    for k in range(N - 1, -1, -1):
        gu = R * (u[k] + du[k] - ur[k]) + B[k].T @ lam
        assert np.abs(gu).max() < 1e-10
        lam = Q * (x[k] + dx[k] - xr[k]) + A[k].T @ lam


def test_scalar_riccati_golden_ratio(orc):
    vals = dict(l.split() for l in open(os.path.join(GOLD, "scalar_lqr.txt")) if l[0] != "#")
    N = 60
    one = np.ones((N, 1, 1))
    z = np.zeros
    st, dx, du, K, k = orc.riccati(one, one, z((N, 1)), z((N + 1, 1)), z((N, 1)), z((N + 1, 1)),
                                   z((N, 1)), np.ones(1), np.ones(1), np.ones(1), np.ones(1),
                                   nx=1, nu=1, return_gains=True)
    assert st == 0
    assert abs(K[0, 0, 0] - float(vals["K_inf"])) < 1e-12
    # the scalar recursion P <- q + a^2 P - (abP)^2/(r + b^2 P) from P_N = 1
    P = 1.0
    for _ in range(N):
        P = 1 + P - P * P / (1 + P)
    assert abs(P - float(vals["P_inf"])) < 1e-12
    # closed loop from x0 = 1 decays by (1 + K) per step
    assert abs(dx[1, 0] - (1 + K[0, 0, 0])) < 1e-12


def test_riccati_reports_not_pd(orc):
    rng = np.random.default_rng(21)
    qp = list(_random_qp(rng, 3))
    qp[8] = -np.ones(4)  # R negative definite, Q_N small
    qp[9] = np.full(13, 1e-6)
    qp[1] = qp[1] * 0
    st, _, _ = orc.riccati(*qp)
    assert st == 4


# ------------------------------------------------------------------ RTI step

def test_rti_step_on_reference_is_stationary(orc):
    # hover at the reference point with the nominal model: the QP step is zero,
    # u0 = hover, and the shifted iterate is unchanged
    N = np.array([5], np.int32); dt = np.array([0.05])
    x = np.zeros((6, 13)); x[:, 3] = 1.0; x[:, 0:3] = [0.5, -0.5, 1.0]
    u = np.full((5, 4), W.hover_thrust())
    u0, xn, un, st = orc.rti_step(QUAD, [], N, dt, W.Q_DIAG, W.R_DIAG, W.Q_DIAG, x, u, x.copy(),
                                  u.copy(), x[:1].copy())
    assert st[0] == 0
    assert np.allclose(u0, W.hover_thrust(), atol=1e-12)
    assert np.allclose(xn, x, atol=1e-12) and np.allclose(un, u, atol=1e-12)


def test_rti_step_composition(orc):
    # one RTI step equals linearise -> Riccati -> update -> clamp -> shift
    prob = W.make_problem("cfg1_single_fp64", seed=3)
    N, dt = prob["N"], prob["dt"]
    X, U = W.random_nodes(int(N.sum()) + 1, 9)
    x, u = X, U[:-1]
    xref, uref = W.node_refs(prob)
    x0m = x[:1] + 0.05
    fD, JD, A, B, c = orc.linearize(QUAD, prob["layers"], N, dt, x, u)
    st, dx, du = orc.riccati(A, B, c, x, u, xref, uref, prob["Q"], prob["R"], prob["QN"], x0m[0])
    u0, xn, un, st2 = orc.rti_step(QUAD, prob["layers"], N, dt, prob["Q"], prob["R"], prob["QN"],
                                   x, u, xref, uref, x0m)
    xs, us = x + dx, u + du
    assert np.allclose(u0[0], np.clip(us[0], 0, QUAD["u_max"]), atol=1e-13)
    assert np.allclose(xn[:-1], xs[1:], atol=1e-13) and np.allclose(xn[-1], xs[-1], atol=1e-13)
    assert np.allclose(un[:-1], us[1:], atol=1e-13) and np.allclose(un[-1], us[-1], atol=1e-13)


def test_closed_loop_tracks_reference(orc):
    # cfg1: single instance, circle r = 2 m at 3 m/s, 100 steps; the plant is
    # the nominal model plus the same network, so the controller's model is
    # exact up to the local approximation: the position error settles
    prob = W.make_problem("cfg1_single_fp64", seed=0)
    steps = 100
    xrt, urt = W.trajectory_refs(prob, steps)
    x0 = xrt[:, 0].copy()
    traj, uh = orc.closed_loop(QUAD, prob["layers"], 2, prob["layers"], prob["N"], prob["dt"],
                               prob["Q"], prob["R"], prob["QN"], x0, xrt, urt, steps)
    err = np.linalg.norm(traj[:, 0, 0:3] - xrt[0, 1:steps + 1, 0:3], axis=1)
    assert np.all(np.isfinite(traj))
    assert err[-40:].mean() < 0.3
    assert np.all(uh >= 0) and np.all(uh <= QUAD["u_max"])


# ------------------------------------------------------------------ training

def test_mse_gradient_vs_fd(orc):
    layers = W.xavier_mlp([17, 16, 16, 3], 4)
    X, U = W.training_samples(8, 0)
    Z = np.concatenate([X, U], 1)
    Y = orc.drag_targets(X)
    loss, G = orc.mse_grad(layers, Z, Y)
    rng = np.random.default_rng(0)
    for l in range(len(layers)):
        for _ in range(4):
            i, j = rng.integers(layers[l][0].shape[0]), rng.integers(layers[l][0].shape[1])
            h = 1e-6
            Lp = [(w.copy(), b.copy()) for w, b in layers]; Lm = [(w.copy(), b.copy()) for w, b in layers]
            Lp[l][0][i, j] += h; Lm[l][0][i, j] -= h
            fd = (orc.mse_grad(Lp, Z, Y)[0] - orc.mse_grad(Lm, Z, Y)[0]) / (2 * h)
            assert abs(fd - G[l][0][i, j]) < 1e-6 * max(1.0, abs(fd))
        i = rng.integers(layers[l][1].shape[0])
        Lp = [(w.copy(), b.copy()) for w, b in layers]; Lm = [(w.copy(), b.copy()) for w, b in layers]
        Lp[l][1][i] += 1e-6; Lm[l][1][i] -= 1e-6
        fd = (orc.mse_grad(Lp, Z, Y)[0] - orc.mse_grad(Lm, Z, Y)[0]) / 2e-6
        assert abs(fd - G[l][1][i]) < 1e-6 * max(1.0, abs(fd))
    # loss is the mean of squared errors over samples and outputs
    pred = np.stack([orc.mlp_forward(layers, z) for z in Z])
    assert abs(loss - ((pred - Y) ** 2).mean()) < 1e-13


def test_adam_first_step_closed_form(orc):
    # from zero moments, the bias-corrected first step is lr * g / (|g| + eps)
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    p = np.array([1.0, 2.0, 3.0, 4.0]); p0 = p.copy()
    m = np.zeros(4); v = np.zeros(4)
    orc.adam(p, g, m, v, 1, 1e-3)
    assert np.allclose(p, p0 - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    # second step with the same gradient: m_hat = g, v_hat = g^2 again
    orc.adam(p, g, m, v, 2, 1e-3)
    assert np.allclose(p, p0 - 2e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-14)


# ---------------------------------------------------------------- box QP ---
# The thrust bounds 0 <= u_k + du_k <= u_max of Sec. V inside the QP.  Pins:
# the exact solution of the same bound-constrained problem by an independent
# solver (bounded-variable least squares on the condensed problem, built
# here from the dynamics), its KKT conditions, and the unconstrained Riccati
# solution when no bound is active.

def _linearised_qp(orc, seed, N=10, scale=1.0):
    """QP data of the nominal quadrotor linearised along a perturbed hover
    trajectory, with references far enough away that bounds become active."""
    rng = np.random.default_rng(seed)
    x = np.zeros((N + 1, 13)); x[:, 3] = 1.0
    x[:, 7:10] += rng.normal(0, 2 * scale, 3)
    u = np.clip(np.full((N, 4), W.hover_thrust()) + rng.uniform(-1.5, 1.5, (N, 4)) * scale,
                0, W.QUAD["u_max"])
    _, _, A, B, c = orc.linearize(W.QUAD, [], np.array([N]), np.array([0.05]), x, u)
    xr = np.zeros((N + 1, 13)); xr[:, 3] = 1.0
    xr[:, :3] += rng.normal(0, 3 * scale, 3)
    ur = np.full((N, 4), W.hover_thrust())
    x0m = x[0] + rng.normal(0, 0.5 * scale, 13)
    lb, ub = -u, W.QUAD["u_max"] - u
    return A, B, c, x, u, xr, ur, x0m, lb, ub


def _condensed(A, B, c, x, u, xr, ur, x0m, Q, R, QN):
    """Eliminate the dynamics: dx_k = Phi_k dx_0 + Gam_k du + e_k, so the cost
    is 1/2 du'H du + g'du + const."""
    N, nx, nu = A.shape[0], A.shape[1], B.shape[2]
    Phi, Gam, e = [np.eye(nx)], [np.zeros((nx, N * nu))], [np.zeros(nx)]
    for k in range(N):
        Phi.append(A[k] @ Phi[-1])
        Gk = A[k] @ Gam[-1]
        Gk[:, k * nu:(k + 1) * nu] += B[k]
        Gam.append(Gk)
        e.append(A[k] @ e[-1] + c[k])
    dx0 = x0m - x[0]
    H = np.diag(np.tile(R, N)).astype(float)
    g = np.concatenate([R * (u[k] - ur[k]) for k in range(N)])
    for k in range(N + 1):
        W_ = np.diag(QN if k == N else Q)
        off = x[k] + Phi[k] @ dx0 + e[k] - xr[k]
        H += Gam[k].T @ W_ @ Gam[k]
        g += Gam[k].T @ W_ @ off
    return H, g


@pytest.mark.parametrize("seed", range(6))
def test_box_qp_matches_bounded_least_squares(orc, seed):
    from scipy.optimize import lsq_linear
    A, B, c, x, u, xr, ur, x0m, lb, ub = _linearised_qp(orc, seed)
    Q, R = W.Q_DIAG, W.R_DIAG
    st, dx, du, its = orc.box_qp(A, B, c, x, u, xr, ur, Q, R, Q, x0m, lb, ub, max_iter=40)
    assert st == 0
    H, g = _condensed(A, B, c, x, u, xr, ur, x0m, Q, R, Q)
    L = np.linalg.cholesky(H)
    # min 1/2 v'Hv + g'v  ==  min 1/2 |L'v + L^-1 g|^2 under the same bounds
    ref = lsq_linear(L.T, -np.linalg.solve(L, g), bounds=(lb.ravel(), ub.ravel()), method="bvls",
                     tol=1e-14).x
    assert np.abs(du.ravel() - ref).max() < 1e-8 * max(1.0, np.abs(ref).max())
    at_bound = (np.abs(ref - lb.ravel()) < 1e-9) | (np.abs(ref - ub.ravel()) < 1e-9)
    # KKT with the condensed gradient: zero on free inputs, sign at the bounds
    G = H @ du.ravel() + g
    free = ~at_bound
    assert np.abs(G[free]).max() < 1e-6 * np.abs(g).max()
    assert (G[np.abs(ref - lb.ravel()) < 1e-9] > -1e-6 * np.abs(g).max()).all()
    assert (G[np.abs(ref - ub.ravel()) < 1e-9] < 1e-6 * np.abs(g).max()).all()
    # dx is the roll-out of du
    for k in range(A.shape[0]):
        assert np.allclose(dx[k + 1], A[k] @ dx[k] + B[k] @ du[k] + c[k], atol=1e-9)


def test_box_qp_inactive_bounds_is_riccati(orc):
    A, B, c, x, u, xr, ur, x0m, lb, ub = _linearised_qp(orc, 11, scale=0.3)
    Q, R = W.Q_DIAG, W.R_DIAG
    st0, dx0, du0 = orc.riccati(A, B, c, x, u, xr, ur, Q, R, Q, x0m)
    big = np.full_like(lb, 1e9)
    st, dx, du, its = orc.box_qp(A, B, c, x, u, xr, ur, Q, R, Q, x0m, -big, big)
    assert st == st0 == 0 and its == 1
    assert np.array_equal(du, du0) and np.array_equal(dx, dx0)


def test_box_qp_iteration_cap(orc):
    A, B, c, x, u, xr, ur, x0m, lb, ub = _linearised_qp(orc, 0)
    Q, R = W.Q_DIAG, W.R_DIAG
    st, dx, du, its = orc.box_qp(A, B, c, x, u, xr, ur, Q, R, Q, x0m, lb, ub, max_iter=1)
    assert st == 8 and its == 1
    assert (du >= lb).all() and (du <= ub).all()
    for k in range(A.shape[0]):
        assert np.allclose(dx[k + 1], A[k] @ dx[k] + B[k] @ du[k] + c[k], atol=1e-9)


def test_rti_step_box_keeps_thrust_in_bounds(orc):
    prob = W.make_problem("cfg2_fp32_batch", seed=3, B=6)
    N, dt = prob["N"], prob["dt"]
    X, U = W.random_nodes(int(N.sum()) + len(N), 21)
    U = U[:int(N.sum())]
    xref, uref = W.node_refs(prob)
    x0 = X[np.concatenate([[0], np.cumsum(N + 1)])[:-1]] + 0.5
    u0, xn, un, st, its = orc.rti_step_box(W.QUAD, [], N, dt, prob["Q"], prob["R"], prob["QN"], X, U,
                                           xref, uref, x0, shift=False, max_iter=40)
    assert (st == 0).all()
    assert (un >= -1e-12).all() and (un <= W.QUAD["u_max"] + 1e-12).all()
    assert np.allclose(u0, un[np.concatenate([[0], np.cumsum(N)])[:-1]])
    # without bounds the same step leaves the box somewhere (the bounds matter)
    _, _, un_free, _ = orc.rti_step(W.QUAD, [], N, dt, prob["Q"], prob["R"], prob["QN"], X, U, xref,
                                    uref, x0, shift=False)
    assert ((un_free < 0) | (un_free > W.QUAD["u_max"])).any()


def test_box_qp_pins_exercise_the_bounds(orc):
    # the seeds above are cases where bounds are active at the solution
    active = 0
    for seed in range(6):
        A, B, c, x, u, xr, ur, x0m, lb, ub = _linearised_qp(orc, seed)
        _, _, du, its = orc.box_qp(A, B, c, x, u, xr, ur, W.Q_DIAG, W.R_DIAG, W.Q_DIAG, x0m, lb, ub,
                                   max_iter=40)
        if ((np.abs(du - lb) < 1e-12) | (np.abs(du - ub) < 1e-12)).sum() >= 2 and its > 1:
            active += 1
    assert active >= 4, active


# ------------------------------------ double integrator (Sec. IV runtime model)

def _di_net(widths, seed, zero_out=False):
    layers = W.xavier_mlp(widths, seed)
    if zero_out:  # Sec. IV: weights set so that the network outputs zero
        Wl, bl = layers[-1]
        layers[-1] = (np.zeros_like(Wl), np.zeros_like(bl))
    return layers


def test_di_rk4_nominal_is_exact(orc):
    # the double integrator's trajectory is quadratic in t: RK4 reproduces it
    rng = np.random.default_rng(4)
    for _ in range(5):
        x, u, dt = rng.normal(0, 2, 2), rng.normal(0, 3), rng.uniform(0.01, 0.3)
        phi, A, B = orc.di_rk4_lin(x, u, dt)
        assert np.allclose(phi, [x[0] + x[1] * dt + u * dt * dt / 2, x[1] + u * dt], rtol=0, atol=1e-14)
        assert np.allclose(A, [[1, dt], [0, 1]], rtol=0, atol=1e-15)
        assert np.allclose(B, [dt * dt / 2, dt], rtol=0, atol=1e-15)


def test_di_rk4_constant_residual_closed_form(orc):
    # f_D* = constant c (zero Jacobian): the residual adds to the acceleration
    x, u, dt, c = np.array([0.3, -1.2]), 0.7, 0.05, -2.5
    phi, A, B = orc.di_rk4_lin(x, u, dt, fbar=c, J=np.zeros(3))
    assert np.allclose(phi, [x[0] + x[1] * dt + (u + c) * dt * dt / 2, x[1] + (u + c) * dt], rtol=0, atol=1e-14)


def test_di_rk4_sensitivities_vs_fd_and_order(orc):
    # A, B against central differences of the RK4 map (the local model held
    # fixed), and phi against the exact flow of the affine ODE (matrix
    # exponential): the error falls as dt^5
    from scipy.linalg import expm
    rng = np.random.default_rng(5)
    x, u = rng.normal(0, 1, 2), 0.4
    fbar, J = 0.3, np.array([-1.5, -0.7, 0.2])
    dt = 0.1
    phi, A, B = orc.di_rk4_lin(x, u, dt, fbar=fbar, J=J)
    h = 1e-6
    for j in range(3):
        xp, xm, up, um = x.copy(), x.copy(), u, u
        if j < 2:
            xp[j] += h; xm[j] -= h
        else:
            up += h; um -= h
        # the local model's expansion point stays at (x, u)
        def step(xx, uu):
            ff = fbar + J[0] * (xx[0] - x[0]) + J[1] * (xx[1] - x[1]) + J[2] * (uu - u)
            return orc.di_rk4_lin(xx, uu, dt, fbar=ff, J=J)[0]
        col = (step(xp, up) - step(xm, um)) / (2 * h)
        ref = A[:, j] if j < 2 else B
        assert np.allclose(col, ref, rtol=0, atol=1e-8)
    # exact flow of d/dt [p, v, 1] = M [p, v, 1]
    M = np.array([[0.0, 1.0, 0.0],
                  [J[0], J[1], u + fbar - J[0] * x[0] - J[1] * x[1]],
                  [0.0, 0.0, 0.0]])
    errs = []
    for d in (0.2, 0.1, 0.05):
        ex = (expm(M * d) @ np.array([x[0], x[1], 1.0]))[:2]
        errs.append(np.abs(orc.di_rk4_lin(x, u, d, fbar=fbar, J=J)[0] - ex).max())
    assert 24 < errs[0] / errs[1] < 40 and 24 < errs[1] / errs[2] < 40


def test_di_zero_output_network_is_nominal(orc):
    # Sec. IV: a network forced to output zero changes nothing
    layers = _di_net([3, 32, 32, 1], 6, zero_out=True)
    N = np.array([10, 7], np.int32); dt = np.array([0.05, 0.08])
    rng = np.random.default_rng(7)
    x = rng.normal(0, 1, (int(N.sum()) + len(N), 2)); u = rng.normal(0, 1, int(N.sum()))
    fD, JD, A, B, c = orc.di_linearize(layers, N, dt, x, u)
    assert np.all(fD == 0) and np.all(JD == 0)
    _, _, A0, B0, c0 = orc.di_linearize(None, N, dt, x, u)
    assert np.array_equal(A, A0) and np.array_equal(B, B0) and np.array_equal(c, c0)


def test_di_network_jacobian_vs_fd(orc):
    layers = _di_net([3, 16, 16, 1], 8)
    z = np.array([0.4, -0.9, 1.3])
    f, J = orc.mlp_fwd_jac(layers, z)
    for j in range(3):
        zp, zm = z.copy(), z.copy()
        zp[j] += 1e-6; zm[j] -= 1e-6
        assert abs((orc.mlp_forward(layers, zp) - orc.mlp_forward(layers, zm))[0] / 2e-6 - J[0, j]) < 1e-8


def test_di_rti_step_is_the_kkt_solution(orc):
    # the RTI update equals a dense KKT solve of the same linearised QP
    layers = _di_net([3, 16, 16, 1], 9)
    N = np.array([10, 6], np.int32); dt = np.array([0.05, 0.1])
    rng = np.random.default_rng(10)
    ns, nn = int(N.sum()) + len(N), int(N.sum())
    x = rng.normal(0, 1, (ns, 2)); u = rng.normal(0, 1, nn)
    xref = rng.normal(0, 1, (ns, 2)); uref = rng.normal(0, 0.5, nn)
    x0m = rng.normal(0, 1, (len(N), 2))
    Q, R, QN = np.array([10.0, 1.0]), np.array([0.1]), np.array([20.0, 2.0])
    u0, xn, un, st = orc.di_rti_step(layers, N, dt, Q, R, QN, x, u, xref, uref, x0m, shift=False)
    assert np.all(st == 0)
    _, _, A, B, c = orc.di_linearize(layers, N, dt, x, u)
    xs = us = 0
    for b, Nb in enumerate(N):
        s2, dx, du = orc.kkt_dense(A[us:us + Nb], B[us:us + Nb].reshape(Nb, 2, 1), c[us:us + Nb],
                                   x[xs:xs + Nb + 1], u[us:us + Nb].reshape(Nb, 1), xref[xs:xs + Nb + 1],
                                   uref[us:us + Nb].reshape(Nb, 1), Q, R, QN, x0m[b], nx=2, nu=1)
        assert s2 == 0
        assert np.allclose(xn[xs:xs + Nb + 1], x[xs:xs + Nb + 1] + dx, rtol=0, atol=1e-10)
        assert np.allclose(un[us:us + Nb], u[us:us + Nb] + du[:, 0], rtol=0, atol=1e-10)
        assert abs(u0[b] - un[us]) < 1e-15
        xs += Nb + 1; us += Nb


def test_di_long_horizon_gain_is_the_lqr_gain(orc):
    # far from the end of a long horizon the Riccati gain is the
    # infinite-horizon LQR gain of the discrete double integrator
    from scipy.linalg import solve_discrete_are
    dt, Nh = 0.1, 300
    Ad = np.array([[1, dt], [0, 1]]); Bd = np.array([[dt * dt / 2], [dt]])
    Q, R = np.array([4.0, 0.5]), np.array([0.2])
    P = solve_discrete_are(Ad, Bd, np.diag(Q), np.diag(R))
    K_lqr = -np.linalg.solve(np.diag(R) + Bd.T @ P @ Bd, Bd.T @ P @ Ad)
    A = np.repeat(Ad[None], Nh, 0); B = np.repeat(Bd[None], Nh, 0); c = np.zeros((Nh, 2))
    x = np.zeros((Nh + 1, 2)); u = np.zeros((Nh, 1))
    st, dx, du, K, k = orc.riccati(A, B, c, x, u, x, u, Q, R, Q, np.array([1.0, 0.0]), nx=2, nu=1,
                                   return_gains=True)
    assert st == 0 and np.allclose(K[0], K_lqr, rtol=1e-9, atol=1e-12)


# --------------------------------------- second-order local model (Eq. 4, H_D)

@pytest.mark.parametrize("widths", [[17, 16, 16, 3], [17, 24, 3]])
def test_mlp_hessian_vs_fd_of_jacobian(orc, widths):
    layers = W.xavier_mlp(widths, 11)
    z = np.random.default_rng(12).normal(0, 0.8, 17)
    f, J, H = orc.mlp_fwd_hess(layers, z)
    f1, J1 = orc.mlp_fwd_jac(layers, z)
    assert np.array_equal(f, f1) or np.allclose(f, f1, rtol=0, atol=1e-15)
    assert np.allclose(J, J1, rtol=0, atol=1e-15)
    assert np.allclose(H, np.transpose(H, (0, 2, 1)), rtol=0, atol=1e-14)
    Hfd = np.zeros_like(H)
    for j in range(17):
        zp, zm = z.copy(), z.copy()
        zp[j] += 1e-5; zm[j] -= 1e-5
        Hfd[:, :, j] = (orc.mlp_fwd_jac(layers, zp)[1] - orc.mlp_fwd_jac(layers, zm)[1]) / 2e-5
    assert _rel(H, Hfd) < 1e-7


def test_rk4_second_order_sensitivities_vs_fd(orc):
    # A, B of the second-order local model against central differences of
    # the RK4 map (expansion point held fixed)
    layers = W.xavier_mlp([17, 16, 16, 3], 13)
    rng = np.random.default_rng(14)
    x = W.random_nodes(1, 15)[0][0].astype(np.float64)
    u = np.full(4, 1.9)
    z0 = np.concatenate([x, u])
    f, J, H = orc.mlp_fwd_hess(layers, z0)
    H = H * 50.0  # a strong curvature so that the term matters
    dt = 0.05
    phi, A, B = orc.rk4_lin(QUAD, x, u, dt, f, J, H)
    def step(xx, uu):
        dz = np.concatenate([xx - x, uu - u])
        ff = f + J @ dz + 0.5 * np.einsum('j,rjm,m->r', dz, H, dz)
        JJ = J + H @ dz
        return orc.rk4_lin(QUAD, xx, uu, dt, ff, JJ, H)[0]
    h = 1e-6
    for j in range(17):
        xp, xm, up, um = x.copy(), x.copy(), u.copy(), u.copy()
        if j < 13:
            xp[j] += h; xm[j] -= h
        else:
            up[j - 13] += h; um[j - 13] -= h
        col = (step(xp, up) - step(xm, um)) / (2 * h)
        ref = A[:, j] if j < 13 else B[:, j - 13]
        assert np.allclose(col, ref, rtol=0, atol=1e-7), j
    phi1 = orc.rk4_lin(QUAD, x, u, dt, f, J)[0]
    assert np.abs(phi - phi1).max() > 1e-9  # the second-order term changes the step


def test_local_model_error_orders(orc):
    # Sec. III: replacing the network by its local model costs O(dz^2) per
    # evaluation for the first-order model and O(dz^3) for the second-order
    # one; over one RK4 step (dz = O(dt)) the step errors fall as dt^3 and
    # dt^4 when dt halves
    layers = W.xavier_mlp([17, 16, 16, 3], 16)
    x = W.random_nodes(1, 17)[0][0].astype(np.float64)
    x[7:10] = [3.0, -2.0, 1.5]  # velocity so that the stage points move
    u = np.array([2.3, 1.5, 2.0, 1.7])
    f, J, H = orc.mlp_fwd_hess(layers, np.concatenate([x, u]))
    e1, e2 = [], []
    for dt in (0.08, 0.04, 0.02):
        true = orc.rk4_true(QUAD, x, u, dt, kind=2, layers=layers)
        e1.append(np.abs(orc.rk4_lin(QUAD, x, u, dt, f, J)[0] - true).max())
        e2.append(np.abs(orc.rk4_lin(QUAD, x, u, dt, f, J, H)[0] - true).max())
    r1 = [e1[0] / e1[1], e1[1] / e1[2]]
    r2 = [e2[0] / e2[1], e2[1] / e2[2]]
    assert all(6 < r < 10 for r in r1), r1
    assert all(12 < r < 20 for r in r2), r2
    assert e2[-1] < e1[-1]


def test_rti_step2_is_the_kkt_solution(orc):
    layers = W.xavier_mlp([17, 16, 16, 3], 18)
    N = np.array([6, 4], np.int32); dt = np.array([0.05, 0.04])
    ns, nn = int(N.sum()) + len(N), int(N.sum())
    X, U = W.random_nodes(ns, 19)
    x = X.astype(np.float64); u = U[:nn].astype(np.float64)
    rng = np.random.default_rng(20)
    xref = x + rng.normal(0, 0.1, x.shape); uref = u + rng.normal(0, 0.1, u.shape)
    x0m = x[[0, N[0] + 1]] + rng.normal(0, 0.05, (2, 13))
    Q = np.full(13, 2.0); R = np.full(4, 0.5)
    u0, xn, un, st = orc.rti_step2(QUAD, layers, N, dt, Q, R, Q, x, u, xref, uref, x0m, shift=False)
    assert np.all(st == 0)
    _, _, _, A, B, c = orc.linearize2(QUAD, layers, N, dt, x, u)
    _, _, A1, B1, c1 = orc.linearize(QUAD, layers, N, dt, x, u)
    assert np.abs(A - A1).max() > 1e-12  # second order differs from first order
    xs = us = 0
    for b, Nb in enumerate(N):
        s2, dx, du = orc.kkt_dense(A[us:us + Nb], B[us:us + Nb], c[us:us + Nb], x[xs:xs + Nb + 1],
                                   u[us:us + Nb], xref[xs:xs + Nb + 1], uref[us:us + Nb], Q, R, Q, x0m[b])
        assert s2 == 0
        assert np.allclose(xn[xs:xs + Nb + 1], x[xs:xs + Nb + 1] + dx, rtol=0, atol=1e-9)
        assert np.allclose(un[us:us + Nb], u[us:us + Nb] + du, rtol=0, atol=1e-9)
        xs += Nb + 1; us += Nb


# ------------------------------ full residual of Eq. 7: [0; 0; f_theta; f_psi]

def stack_residual(theta, psi):
    """One 6-output network equal to the two networks of Eq. 7 side by side:
    the first layer stacks their rows, deeper layers are block-diagonal."""
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


def test_full_residual_constant_closed_form(orc):
    # zero weights, output bias [b; a e_i]: with zero thrust the nominal model
    # has no torque and no thrust, so v(t) = (b - g e_z) t, p(t) = v t / 2 and,
    # the angular residual acting on one principal axis (w x J w = 0),
    # w(t) = a e_i t -- all integrated exactly by RK4; q turns about e_i by
    # a t^2 / 2 (RK4 error O(dt^5))
    b, a, dt = np.array([0.3, -0.2, 0.5]), 1.7, 0.05
    x = np.zeros(13); x[3] = 1.0
    u = np.zeros(4)
    acc = b - np.array([0.0, 0.0, QUAD["g"]])
    for axis in range(3):
        ang = np.zeros(3); ang[axis] = a
        layers = [(np.zeros((8, 17)), np.zeros(8)), (np.zeros((6, 8)), np.concatenate([b, ang]))]
        fbar, J = orc.mlp_fwd_jac(layers, np.concatenate([x, u]))
        lin = orc.linearize(QUAD, layers, np.array([1], np.int32), np.array([dt]), np.vstack([x, x]), u[None])
        for phi in (orc.rk4_lin(QUAD, x, u, dt, fbar, J)[0],
                    orc.rk4_true(QUAD, x, u, dt, kind=2, layers=layers), lin[4][0] + x):
            assert np.allclose(phi[0:3], acc * dt * dt / 2, rtol=0, atol=1e-15)
            assert np.allclose(phi[7:10], acc * dt, rtol=0, atol=1e-15)
            assert np.allclose(phi[10:13], ang * dt, rtol=0, atol=1e-15)
            th = a * dt * dt / 2
            qe = np.zeros(4); qe[0] = np.cos(th / 2); qe[1 + axis] = np.sin(th / 2)
            assert np.allclose(phi[3:7], qe, rtol=0, atol=1e-9)


def test_full_residual_stacked_networks(orc):
    # the 6-output network of stacked theta / psi networks has the two
    # networks' values, Jacobians and Hessians as its rows
    theta = W.xavier_mlp([17, 12, 10, 3], 21)
    psi = W.xavier_mlp([17, 9, 14, 3], 22)
    full = stack_residual(theta, psi)
    z = np.random.default_rng(23).normal(0, 0.7, 17)
    f, J, H = orc.mlp_fwd_hess(full, z)
    ft, Jt, Ht = orc.mlp_fwd_hess(theta, z)
    fp, Jp, Hp = orc.mlp_fwd_hess(psi, z)
    assert np.allclose(f, np.concatenate([ft, fp]), rtol=1e-15, atol=1e-16)
    assert np.allclose(J, np.vstack([Jt, Jp]), rtol=1e-15, atol=1e-16)
    assert np.allclose(H, np.concatenate([Ht, Hp]), rtol=1e-14, atol=1e-16)


def test_full_residual_sensitivities_vs_fd(orc):
    layers = W.xavier_mlp([17, 24, 16, 6], 24)
    X, U = W.random_nodes(3, 25)
    for x, u in zip(X, U):
        z = np.concatenate([x, u])
        fbar, J, H = orc.mlp_fwd_hess(layers, z)
        for second in (False, True):
            Hs = H * 20.0 if second else None
            phi, A, B = orc.rk4_lin(QUAD, x, u, 0.05, fbar, J, Hs)
            def ph(zz):
                dz = zz - z
                ff, JJ = fbar + J @ dz, J
                if second:
                    ff = ff + 0.5 * np.einsum('j,rjm,m->r', dz, Hs, dz)
                    JJ = J + Hs @ dz
                return orc.rk4_lin(QUAD, zz[:13], zz[13:], 0.05, ff, JJ, Hs)[0]
            G = np.zeros((13, 17))
            for j in range(17):
                h = 1e-6 * max(1.0, abs(z[j]))
                zp, zm = z.copy(), z.copy()
                zp[j] += h; zm[j] -= h
                G[:, j] = (ph(zp) - ph(zm)) / (2 * h)
            assert _rel(np.hstack([A, B]), G) < 1e-7


def test_full_residual_error_orders(orc):
    # as for the 3-output residual: the local models' step errors against the
    # true dynamics with the same 6-output network fall as dt^3 / dt^4; the
    # angular rows are exercised (the psi block alone changes w)
    layers = W.xavier_mlp([17, 16, 16, 6], 26)
    x = W.random_nodes(1, 27)[0][0].astype(np.float64)
    x[7:10] = [3.0, -2.0, 1.5]
    u = np.array([2.3, 1.5, 2.0, 1.7])
    f, J, H = orc.mlp_fwd_hess(layers, np.concatenate([x, u]))
    e1, e2 = [], []
    for dt in (0.08, 0.04, 0.02):
        true = orc.rk4_true(QUAD, x, u, dt, kind=2, layers=layers)
        e1.append(np.abs(orc.rk4_lin(QUAD, x, u, dt, f, J)[0] - true).max())
        e2.append(np.abs(orc.rk4_lin(QUAD, x, u, dt, f, J, H)[0] - true).max())
    r1 = [e1[0] / e1[1], e1[1] / e1[2]]
    r2 = [e2[0] / e2[1], e2[1] / e2[2]]
    assert all(6 < r < 10 for r in r1), r1
    assert all(12 < r < 20 for r in r2), r2
    # the psi rows move w: dropping them (3-output truncation) is a
    # first-order error, far above the local model's
    f3, J3 = f[:3], J[:3]
    dt = 0.02
    trunc = orc.rk4_lin(QUAD, x, u, dt, f3, J3)[0]
    full = orc.rk4_lin(QUAD, x, u, dt, f, J)[0]
    assert np.abs(trunc[10:13] - full[10:13]).max() > 100 * e1[-1]
