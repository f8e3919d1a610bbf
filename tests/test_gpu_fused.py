"""The fused persistent launch of the RTI step (rtn_options.fused_qp): the RK4
linearisation and the QP of every instance from one work queue.  It runs the
same RK4 and QP device code as the separate launches, compiled into another
kernel (the compiler's choice of fused multiply-adds may differ), so its
results agree with theirs to FP32 rounding: one RTI step (u_0 and the new
iterate within 1e-5 of the largest entry, statuses equal) and a
graph-captured closed loop (plant trajectories within 1e-4 m) on the ragged
workload (N_b in {10..50}, per-instance dt), with the FP32, split-BF16 and
FP8 networks and the nominal model; the step also against the FP64 oracle.  Its bounded waits are made to run out on the host
side of the fault (rtn_inject_wait_stall): every instance reports
RTN_E_TIMEOUT and sends its reference input, and the context recovers."""
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


def f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def ragged(B, seed=0):
    prob = W.make_problem("cfg4_ragged_batch", seed=seed, B=B, bf16=True)
    return prob


def step_inputs(prob):
    N = prob["N"]
    X, U = W.random_nodes(int(N.sum()) + len(N), 5)
    X, U = f32(X), f32(U[:int(N.sum())])
    xref, uref = W.node_refs(prob)
    x0 = f32(X[np.concatenate([[0], np.cumsum(N + 1)])[:-1]] + 0.03)
    return X, U, f32(xref), f32(uref), x0


@pytest.mark.parametrize("precision,net", [("fp32", True), ("bf16x2", True), ("fp8", True), ("fp32", False)])
def test_fused_rti_step_equals_separate_launches(rtn, precision, net):
    prob = ragged(96)
    layers = prob["layers"] if net else None
    if precision == "fp8":
        layers = W.quantize_e4m3(layers)
    N, dt = prob["N"], f32(prob["dt"])
    X, U, xref, uref, x0 = step_inputs(prob)
    out = []
    for fused in (False, True):
        c = rtn.Controller(N, dt, prob["Q"], prob["R"], quad=QUAD, layers=layers, precision=precision, fused_qp=fused)
        c.set_iterate(dev(X), dev(U))
        u0, st = c.rti_step(dev(x0), dev(xref), dev(uref))
        xn, un = c.get_iterate()
        assert c.device_error() == 0
        out.append([u0.cpu(), st.cpu(), xn.cpu(), un.cpu()])
        c.close()
    (u0a, sta, xa, ua), (u0b, stb, xb, ub) = out
    assert torch.equal(sta, stb)
    for a, b in ((u0a, u0b), (xa, xb), (ua, ub)):
        assert (a.double() - b.double()).abs().max() <= 1e-5 * b.double().abs().max()


def test_fused_rti_step_matches_oracle(rtn, orc):
    prob = ragged(24, seed=3)
    layers = [(f32(Wl), f32(bl)) for Wl, bl in prob["layers"]]
    N, dt = prob["N"], f32(prob["dt"])
    X, U, xref, uref, x0 = step_inputs(prob)
    c = rtn.Controller(N, dt, prob["Q"], prob["R"], quad=QUAD, layers=layers, fused_qp=True)
    c.set_iterate(dev(X), dev(U))
    u0, st = c.rti_step(dev(x0), dev(xref), dev(uref))
    assert c.device_error() == 0 and (st.cpu().numpy() == 0).all()
    u0r, _, _, str_ = orc.rti_step(QUAD, layers, N, dt, prob["Q"], prob["R"], prob["QN"], X, U, xref, uref, x0)
    assert (str_ == 0).all()
    assert np.abs(u0.double().cpu().numpy() - u0r).max() / np.abs(u0r).max() < 1e-5


def test_fused_closed_loop_equals_separate_launches(rtn):
    prob = ragged(64, seed=1)
    steps = 6
    N, dt = prob["N"], f32(prob["dt"])
    xrt, urt = W.trajectory_refs(prob, steps)
    xrt, urt = f32(xrt), f32(urt)
    res = []
    for fused in (False, True):
        c = rtn.Controller(N, dt, prob["Q"], prob["R"], quad=QUAD, layers=prob["layers"], precision="bf16x2",
                           fused_qp=fused)
        c.reset(dev(xrt[:, 0] + 0.02))
        xp = dev(xrt[:, 0] + 0.02, torch.float64)
        traj, uo = c.closed_loop(steps, dev(xrt), dev(urt), xp, plant="drag")
        torch.cuda.synchronize()
        assert c.device_error() == 0
        res.append((traj.cpu(), uo.cpu(), xp.cpu()))
        c.close()
    (ta, ua, pa), (tb, ub, pb) = res
    assert (ta[:, :, :3].double() - tb[:, :, :3].double()).abs().max() < 1e-4
    assert (pa[:, :3] - pb[:, :3]).abs().max() < 1e-4


def test_fused_wait_runs_out_and_context_recovers(rtn):
    prob = ragged(40, seed=2)
    N, dt = prob["N"], f32(prob["dt"])
    X, U, xref, uref, x0 = step_inputs(prob)
    c = rtn.Controller(N, dt, prob["Q"], prob["R"], quad=QUAD, layers=prob["layers"], fused_qp=True)
    c.set_wait_budget(200_000)
    c.inject_wait_stall(True)
    c.set_iterate(dev(X), dev(U))
    u0, st = c.rti_step(dev(x0), dev(xref), dev(uref))
    assert c.device_error() == 5
    assert (st.cpu().numpy() == 5).all()  # RTN_E_TIMEOUT per instance
    first = np.concatenate([[0], np.cumsum(N)])[:-1]
    assert np.array_equal(u0.cpu().numpy(), np.float32(uref[first]))
    xn, un = c.get_iterate()
    assert np.array_equal(un.cpu().numpy(), np.float32(U))  # iterate untouched
    c.inject_wait_stall(False)
    c.set_wait_budget(0)
    ref = rtn.Controller(N, dt, prob["Q"], prob["R"], quad=QUAD, layers=prob["layers"])
    c.set_iterate(dev(X), dev(U))
    ref.set_iterate(dev(X), dev(U))
    a, sa = c.rti_step(dev(x0), dev(xref), dev(uref))
    b, sb = ref.rti_step(dev(x0), dev(xref), dev(uref))
    assert c.device_error() == 0 and torch.equal(sa.cpu(), sb.cpu())
    assert (a.double() - b.double()).abs().max() <= 1e-5 * b.double().abs().max()
