"""FP64 CPU oracle for the Real-time Neural MPC hot path.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the package's smoke check
and by the benchmark's CPU-baseline arm, never by the product path.  The
arithmetic lives in ``rtn_oracle.c`` (plain C, double precision); this module
builds it with gcc on first use and marshals numpy arrays through ctypes.

Parity pins for every routine are in ``tests/test_oracle_pins.py``; none is
unpinned.
"""
import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rtn_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

NX, NU, NZ = 13, 4, 17


def build(force=False):
    """Compile the oracle with gcc (OpenMP over instances in batched calls)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Quad(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("mass", "Jx", "Jy", "Jz", "arm", "c_tau", "u_max", "g")]


def _quad(d):
    return Quad(*[float(d[k]) for k in ("mass", "Jx", "Jy", "Jz", "arm", "c_tau", "u_max", "g")])


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.orc_mse_grad.restype = C.c_double
        _lib.orc_riccati.restype = C.c_int
        _lib.orc_kkt_dense.restype = C.c_int
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(C.POINTER(C.c_int))


def _p(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def pack_mlp(layers):
    """(n_layers, widths int32, flat params) from [(W, b), ...]."""
    if not layers:
        return 0, np.zeros(1, np.int32), np.zeros(1)
    widths = [layers[0][0].shape[1]] + [W.shape[0] for W, _ in layers]
    flat = np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in layers])
    return len(layers), np.array(widths, np.int32), flat.astype(np.float64)


def unpack_mlp(widths, flat):
    out, o = [], 0
    for fi, fo in zip(widths[:-1], widths[1:]):
        W = flat[o:o + fo * fi].reshape(fo, fi); o += fo * fi
        b = flat[o:o + fo]; o += fo
        out.append((W, b))
    return out


def _n_out(layers):
    """Outputs of a quadrotor residual network: 3 (linear acceleration) or 6
    (the full residual of Eq. 7)."""
    if not layers:
        return 3
    no = layers[-1][0].shape[0]
    assert no in (3, 6), no
    return no


class _MLP:
    def __init__(self, layers):
        self.nl, w, p = pack_mlp(layers)
        self.w, self.pw = _i(w)
        self.p, self.pp = _d(p)


def mlp_forward(layers, z):
    m = _MLP(layers)
    z, pz = _d(z)
    out = np.zeros(m.w[-1])
    lib().orc_mlp_forward(m.nl, m.pw, m.pp, pz, _p(out))
    return out


def mlp_fwd_jac(layers, z):
    m = _MLP(layers)
    z, pz = _d(z)
    f = np.zeros(m.w[-1]); J = np.zeros((m.w[-1], m.w[0]))
    lib().orc_mlp_fwd_jac(m.nl, m.pw, m.pp, pz, _p(f), _p(J))
    return f, J


def mlp_fwd_hess(layers, z):
    """Value f [nout], Jacobian J [nout][nin] and Hessian H [nout][nin][nin]
    (forward-over-forward; the H_D of Eq. 4)."""
    m = _MLP(layers)
    z, pz = _d(z)
    nin, nout = m.w[0], m.w[-1]
    f = np.zeros(nout); J = np.zeros((nout, nin)); H = np.zeros((nout, nin, nin))
    lib().orc_mlp_fwd_hess(m.nl, m.pw, m.pp, pz, _p(f), _p(J), _p(H))
    return f, J, H


def mlp_rev_jac(layers, z):
    m = _MLP(layers)
    z, pz = _d(z)
    J = np.zeros((m.w[-1], m.w[0]))
    lib().orc_mlp_rev_jac(m.nl, m.pw, m.pp, pz, _p(J))
    return J


def quad_f(quad, x, u):
    x, px = _d(x); u, pu = _d(u)
    out = np.zeros(NX)
    q = _quad(quad)
    lib().orc_quad_f(C.byref(q), px, pu, _p(out))
    return out


def quad_dfdz(quad, x, u):
    x, px = _d(x); u, pu = _d(u)
    out = np.zeros((NX, NZ))
    q = _quad(quad)
    lib().orc_quad_dfdz(C.byref(q), px, pu, _p(out))
    return out


def qrot(q, v):
    q, pq = _d(q); v, pv = _d(v)
    out = np.zeros(3)
    lib().orc_qrot(pq, pv, _p(out))
    return out


def rk4_lin(quad, x, u, dt, fbar=None, J=None, H=None):
    """RK4 of f_F + f_D* with sensitivities; fbar has 3 entries (linear
    acceleration residual) or 6 (the full residual of Eq. 7, rows 3-5 angular);
    H (no x 17 x 17) selects the second-order local model."""
    x, px = _d(x); u, pu = _d(u)
    phi = np.zeros(NX); A = np.zeros((NX, NX)); B = np.zeros((NX, NU))
    q = _quad(quad)
    ph = None
    no = 3
    if fbar is None:
        pf = pj = None
    else:
        fbar, pf = _d(fbar); J, pj = _d(J)
        no = fbar.size
        assert no in (3, 6) and J.size == no * NZ
        if H is not None:
            H, ph = _d(H)
    lib().orc_rk4_lin_n(C.byref(q), px, pu, no, pf, pj, ph, C.c_double(dt), _p(phi), _p(A), _p(B))
    return phi, A, B


def rk4_true(quad, x, u, dt, kind=0, layers=None):
    m = _MLP(layers or [])
    x, px = _d(x); u, pu = _d(u)
    out = np.zeros(NX)
    q = _quad(quad)
    lib().orc_rk4_true(C.byref(q), kind, m.nl, m.pw, m.pp, px, pu, C.c_double(dt), _p(out))
    return out


def plant_step(quad, x, u, dt, kind=0, layers=None, nsub=4):
    m = _MLP(layers or [])
    x, px = _d(x); u, pu = _d(u)
    out = np.zeros(NX)
    q = _quad(quad)
    lib().orc_plant_step(C.byref(q), kind, m.nl, m.pw, m.pp, px, pu, C.c_double(dt), nsub, _p(out))
    return out


def drag(x):
    x, px = _d(x)
    out = np.zeros(3)
    lib().orc_drag(px, _p(out))
    return out


def drag_targets(X):
    X, px = _d(X)
    Y = np.zeros((X.shape[0], 3))
    lib().orc_drag_targets(X.shape[0], px, _p(Y))
    return Y


def riccati(A, B, c, x, u, xr, ur, Q, R, QN, x0m, nx=NX, nu=NU, return_gains=False):
    N = A.shape[0]
    args = [_d(a) for a in (A, B, c, x, u, xr, ur, Q, R, QN, x0m)]
    dx = np.zeros((N + 1, nx)); du = np.zeros((N, nu))
    K = np.zeros((N, nu, nx)); k = np.zeros((N, nu))
    st = lib().orc_riccati(nx, nu, N, *[a[1] for a in args], _p(dx), _p(du), _p(K), _p(k))
    if return_gains:
        return st, dx, du, K, k
    return st, dx, du


def box_qp(A, B, c, x, u, xr, ur, Q, R, QN, x0m, lb, ub, max_iter=20, nx=NX, nu=NU):
    """The QP with lb <= du <= ub (primal-dual active set on the Riccati
    structure).  Returns (status, dx, du, iterations)."""
    N = A.shape[0]
    args = [_d(a) for a in (A, B, c, x, u, xr, ur, Q, R, QN, x0m, lb, ub)]
    dx = np.zeros((N + 1, nx)); du = np.zeros((N, nu))
    it = C.c_int(0)
    st = lib().orc_box_qp(nx, nu, N, *[a[1] for a in args], int(max_iter), _p(dx), _p(du),
                          C.byref(it))
    return st, dx, du, it.value


def kkt_dense(A, B, c, x, u, xr, ur, Q, R, QN, x0m, nx=NX, nu=NU):
    N = A.shape[0]
    args = [_d(a) for a in (A, B, c, x, u, xr, ur, Q, R, QN, x0m)]
    dx = np.zeros((N + 1, nx)); du = np.zeros((N, nu))
    st = lib().orc_kkt_dense(nx, nu, N, *[a[1] for a in args], _p(dx), _p(du))
    return st, dx, du


def linearize(quad, layers, N, dt, x, u):
    """All nodes: returns fD [n][no], JD [n][no][17], A, B, c (no = the
    network's outputs, 3 or 6)."""
    m = _MLP(layers or [])
    N, pN = _i(N); dt, pdt = _d(dt)
    x, px = _d(x); u, pu = _d(u)
    n = int(N.sum())
    no = _n_out(layers)
    fD = np.zeros((n, no)); JD = np.zeros((n, no, NZ))
    A = np.zeros((n, NX, NX)); B = np.zeros((n, NX, NU)); c = np.zeros((n, NX))
    q = _quad(quad)
    lib().orc_linearize(C.byref(q), m.nl, m.pw, m.pp, len(N), pN, pdt, px, pu, _p(fD), _p(JD),
                        _p(A), _p(B), _p(c))
    return fD, JD, A, B, c


def rti_step(quad, layers, N, dt, Q, R, QN, x, u, xref, uref, x0m, shift=True):
    """Returns (u0 [B][4], x_new, u_new, status [B])."""
    m = _MLP(layers or [])
    N, pN = _i(N); dt, pdt = _d(dt)
    x = np.array(x, dtype=np.float64, copy=True); u = np.array(u, dtype=np.float64, copy=True)
    args = [_d(a) for a in (Q, R, QN)]
    xref, pxr = _d(xref); uref, pur = _d(uref); x0m, px0 = _d(x0m)
    Bn = len(N)
    u0 = np.zeros((Bn, NU)); st = np.zeros(Bn, np.int32)
    q = _quad(quad)
    lib().orc_rti_step(C.byref(q), m.nl, m.pw, m.pp, Bn, pN, pdt, args[0][1], args[1][1], args[2][1],
                       _p(x), _p(u), pxr, pur, px0, int(shift), _p(u0),
                       st.ctypes.data_as(C.POINTER(C.c_int)))
    return u0, x, u, st


def linearize2(quad, layers, N, dt, x, u):
    """Second-order local model: fD [n][no], JD [n][no][17], HD [n][no][17][17], A, B, c."""
    m = _MLP(layers or [])
    N, pN = _i(N); dt, pdt = _d(dt)
    x, px = _d(x); u, pu = _d(u)
    n = int(N.sum())
    no = _n_out(layers)
    fD = np.zeros((n, no)); JD = np.zeros((n, no, NZ)); HD = np.zeros((n, no, NZ, NZ))
    A = np.zeros((n, NX, NX)); B = np.zeros((n, NX, NU)); c = np.zeros((n, NX))
    q = _quad(quad)
    lib().orc_linearize2(C.byref(q), m.nl, m.pw, m.pp, len(N), pN, pdt, px, pu, _p(fD), _p(JD), _p(HD),
                         _p(A), _p(B), _p(c))
    return fD, JD, HD, A, B, c


def rti_step2(quad, layers, N, dt, Q, R, QN, x, u, xref, uref, x0m, shift=True):
    """RTI step with the second-order local model.  Returns (u0, x_new, u_new, status)."""
    m = _MLP(layers or [])
    N, pN = _i(N); dt, pdt = _d(dt)
    x = np.array(x, dtype=np.float64, copy=True); u = np.array(u, dtype=np.float64, copy=True)
    args = [_d(a) for a in (Q, R, QN)]
    xref, pxr = _d(xref); uref, pur = _d(uref); x0m, px0 = _d(x0m)
    Bn = len(N)
    u0 = np.zeros((Bn, NU)); st = np.zeros(Bn, np.int32)
    q = _quad(quad)
    lib().orc_rti_step2(C.byref(q), m.nl, m.pw, m.pp, Bn, pN, pdt, args[0][1], args[1][1], args[2][1],
                        _p(x), _p(u), pxr, pur, px0, int(shift), _p(u0), st.ctypes.data_as(C.POINTER(C.c_int)))
    return u0, x, u, st


def rti_step_box(quad, layers, N, dt, Q, R, QN, x, u, xref, uref, x0m, shift=True, max_iter=20):
    """RTI step with the thrust bounds in the QP.  Returns (u0, x_new, u_new,
    status [B], iterations [B])."""
    m = _MLP(layers or [])
    N, pN = _i(N); dt, pdt = _d(dt)
    x = np.array(x, dtype=np.float64, copy=True); u = np.array(u, dtype=np.float64, copy=True)
    args = [_d(a) for a in (Q, R, QN)]
    xref, pxr = _d(xref); uref, pur = _d(uref); x0m, px0 = _d(x0m)
    Bn = len(N)
    u0 = np.zeros((Bn, NU)); st = np.zeros(Bn, np.int32); its = np.zeros(Bn, np.int32)
    q = _quad(quad)
    ip = C.POINTER(C.c_int)
    lib().orc_rti_step_box(C.byref(q), m.nl, m.pw, m.pp, Bn, pN, pdt, args[0][1], args[1][1],
                           args[2][1], _p(x), _p(u), pxr, pur, px0, int(shift), int(max_iter),
                           _p(u0), st.ctypes.data_as(ip), its.ctypes.data_as(ip))
    return u0, x, u, st, its


def di_rk4_lin(x, u, dt, fbar=None, J=None):
    """Double integrator (Sec. IV): RK4 of f_F + f_D* with sensitivities.
    Returns (phi [2], A [2][2], B [2])."""
    x, px = _d(x)
    phi = np.zeros(2); A = np.zeros((2, 2)); B = np.zeros(2)
    if fbar is None:
        pf = pJ = None
    else:
        fb, pf = _d(np.atleast_1d(fbar)); Jd, pJ = _d(J)
    lib().orc_di_rk4_lin(px, C.c_double(float(u)), pf, pJ, C.c_double(float(dt)), _p(phi), _p(A), _p(B))
    return phi, A, B


def di_linearize(layers, N, dt, x, u):
    """Double integrator, every node: fD [n], JD [n][3], A [n][2][2], B [n][2], c [n][2]."""
    m = _MLP(layers or [])
    N, pN = _i(N); dt, pdt = _d(dt)
    x, px = _d(x); u, pu = _d(u)
    n = int(N.sum())
    fD = np.zeros(n); JD = np.zeros((n, 3))
    A = np.zeros((n, 2, 2)); B = np.zeros((n, 2)); c = np.zeros((n, 2))
    lib().orc_di_linearize(m.nl, m.pw, m.pp, len(N), pN, pdt, px, pu, _p(fD), _p(JD), _p(A), _p(B),
                           _p(c))
    return fD, JD, A, B, c


def di_rti_step(layers, N, dt, Q, R, QN, x, u, xref, uref, x0m, shift=True):
    """Double integrator RTI step.  x [n_states][2], u [n_nodes], xref, uref
    likewise, x0m [B][2].  Returns (u0 [B], x_new, u_new, status [B])."""
    m = _MLP(layers or [])
    N, pN = _i(N); dt, pdt = _d(dt)
    x = np.array(x, dtype=np.float64, copy=True); u = np.array(u, dtype=np.float64, copy=True)
    args = [_d(a) for a in (Q, R, QN)]
    xref, pxr = _d(xref); uref, pur = _d(uref); x0m, px0 = _d(x0m)
    Bn = len(N)
    u0 = np.zeros(Bn); st = np.zeros(Bn, np.int32)
    lib().orc_di_rti_step(m.nl, m.pw, m.pp, Bn, pN, pdt, args[0][1], args[1][1], args[2][1], _p(x),
                          _p(u), pxr, pur, px0, int(shift), _p(u0), st.ctypes.data_as(C.POINTER(C.c_int)))
    return u0, x, u, st


def closed_loop(quad, layers, plant_kind, plant_layers, N, dt, Q, R, QN, x0, xrt, urt, steps,
                box=False, max_iter=20, second=False):
    """Returns traj [steps][B][13] and u0 history [steps][B][4]; second: the
    second-order local model of Eq. 4 in every RTI step (no bounds)."""
    m = _MLP(layers or [])
    pm = _MLP(plant_layers or [])
    N, pN = _i(N); dt, pdt = _d(dt)
    args = [_d(a) for a in (Q, R, QN, x0, xrt, urt)]
    Bn, T = xrt.shape[0], xrt.shape[1]
    traj = np.zeros((steps, Bn, NX)); uh = np.zeros((steps, Bn, NU))
    q = _quad(quad)
    if box:
        lib().orc_closed_loop_box(C.byref(q), m.nl, m.pw, m.pp, plant_kind, pm.nl, pm.pw, pm.pp, Bn,
                                  pN, pdt, *[a[1] for a in args], T, steps, int(max_iter),
                                  _p(traj), _p(uh))
    elif second:
        lib().orc_closed_loop2(C.byref(q), m.nl, m.pw, m.pp, plant_kind, pm.nl, pm.pw, pm.pp, Bn, pN,
                               pdt, *[a[1] for a in args], T, steps, _p(traj), _p(uh))
    else:
        lib().orc_closed_loop(C.byref(q), m.nl, m.pw, m.pp, plant_kind, pm.nl, pm.pw, pm.pp, Bn, pN,
                              pdt, *[a[1] for a in args], T, steps, _p(traj), _p(uh))
    return traj, uh


def mse_grad(layers, Z, Y):
    nl, w, p = pack_mlp(layers)
    w, pw = _i(w); p, pp = _d(p)
    Z, pz = _d(Z); Y, py = _d(Y)
    G = np.zeros_like(p)
    loss = lib().orc_mse_grad(nl, pw, pp, Z.shape[0], pz, py, _p(G))
    return loss, unpack_mlp(w, G)


def adam(flat_p, flat_g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """In place on float64 arrays."""
    for a in (flat_p, flat_g, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib().orc_adam(C.c_size_t(flat_p.size), _p(flat_p), _p(flat_g), _p(m), _p(v), int(t),
                   C.c_double(lr), C.c_double(b1), C.c_double(b2), C.c_double(eps))
