"""GPU parity of the runtime-analysis model (Sec. IV): the double integrator
with a residual network, through the C ABI (rtn_create with nx = 2, nu = 1),
against the FP64 oracle."""
import numpy as np
import pytest

import workload as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rtn():
    import paper_2203_07747_b300 as rtn
    rtn.load()
    return rtn


def _net(widths, seed, zero_out=False):
    layers = W.xavier_mlp(widths, seed)
    if zero_out:  # Sec. IV: the network is forced to output zero
        Wl, bl = layers[-1]
        layers[-1] = (np.zeros_like(Wl), np.zeros_like(bl))
    return [(Wl.astype(np.float32).astype(np.float64), bl.astype(np.float32).astype(np.float64))
            for Wl, bl in layers]


def _problem(N, seed):
    rng = np.random.default_rng(seed)
    N = np.asarray(N, np.int32)
    ns, nn = int(N.sum()) + len(N), int(N.sum())
    dt = rng.uniform(0.02, 0.1, len(N))
    x = rng.normal(0, 1, (ns, 2)).astype(np.float32).astype(np.float64)
    u = rng.normal(0, 1, nn).astype(np.float32).astype(np.float64)
    xref = rng.normal(0, 1, (ns, 2)).astype(np.float32).astype(np.float64)
    uref = rng.normal(0, 0.3, nn).astype(np.float32).astype(np.float64)
    x0 = rng.normal(0, 1, (len(N), 2)).astype(np.float32).astype(np.float64)
    return N, dt, x, u, xref, uref, x0


Q, R, QN = np.array([10.0, 1.0]), np.array([0.1]), np.array([20.0, 2.0])


def _t(a, torch):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


@pytest.mark.parametrize("widths", [[3, 16, 16, 1], [3, 128, 128, 128, 128, 1], [3, 512, 512, 1],
                                    [3, 37, 200, 1], [3, 4096, 1]])
def test_di_network_and_linearisation_match_oracle(rtn, orc, widths):
    import torch
    layers = _net(widths, 3)
    N, dt, x, u, *_ = _problem([10, 7, 10, 3], 4)
    ctl = rtn.DIController(N, dt, Q, R, QN, layers=layers)
    fD, JD, A, B, c = ctl.linearize(_t(x, torch), _t(u, torch))
    f_ref, J_ref, A_ref, B_ref, c_ref = orc.di_linearize(layers, N, dt, x, u)
    fD, JD = fD.double().cpu().numpy(), JD.double().cpu().numpy()
    scale = max(np.abs(f_ref).max(), 1e-3)
    assert np.abs(fD - f_ref).max() / scale < 1e-5
    assert np.abs(JD - J_ref).max() / max(np.abs(J_ref).max(), 1e-3) < 1e-5
    for got, ref in ((A, A_ref), (B, B_ref), (c, c_ref)):
        assert np.abs(got.double().cpu().numpy() - ref).max() < 1e-5 * max(1.0, np.abs(ref).max())
    f2, J2 = ctl.mlp_eval(_t(x, torch), _t(u, torch))
    assert np.array_equal(f2.cpu().numpy(), fD.astype(np.float32))
    ctl.close()


@pytest.mark.parametrize("widths,zero", [([3, 32, 32, 1], False), ([3, 128, 128, 128, 128, 128, 1], False),
                                         ([3, 64, 64, 1], True), (None, False)])
def test_di_rti_step_matches_oracle(rtn, orc, widths, zero):
    import torch
    layers = _net(widths, 5, zero_out=zero) if widths else None
    N, dt, x, u, xref, uref, x0 = _problem([10, 10, 4, 17, 1], 6)
    ctl = rtn.DIController(N, dt, Q, R, QN, layers=layers, shift=True)
    ctl.set_iterate(_t(x, torch), _t(u, torch))
    u0, st = ctl.rti_step(_t(x0, torch), _t(xref, torch), _t(uref, torch))
    xg, ug = ctl.get_iterate()
    u0_ref, x_ref, u_ref, st_ref = orc.di_rti_step(layers, N, dt, Q, R, QN, x, u, xref, uref, x0, shift=True)
    assert np.all(st.cpu().numpy() == 0) and np.all(st_ref == 0)
    assert np.abs(u0.double().cpu().numpy() - u0_ref).max() < 1e-5 * max(1.0, np.abs(u0_ref).max())
    assert np.abs(xg.double().cpu().numpy() - x_ref).max() < 1e-5 * max(1.0, np.abs(x_ref).max())
    assert np.abs(ug.double().cpu().numpy() - u_ref).max() < 1e-5 * max(1.0, np.abs(u_ref).max())
    ctl.close()


def test_di_zero_output_network_equals_nominal(rtn):
    # the paper's runtime network outputs zero: the controller's result is
    # the nominal one, to the bit
    import torch
    N, dt, x, u, xref, uref, x0 = _problem([10] * 6, 7)
    outs = []
    for layers in (_net([3, 64, 64, 64, 1], 8, zero_out=True), None):
        ctl = rtn.DIController(N, dt, Q, R, QN, layers=layers)
        ctl.set_iterate(_t(x, torch), _t(u, torch))
        u0, _ = ctl.rti_step(_t(x0, torch), _t(xref, torch), _t(uref, torch))
        xg, ug = ctl.get_iterate()
        outs.append((u0.cpu().numpy(), xg.cpu().numpy(), ug.cpu().numpy()))
        ctl.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_di_closed_loop_converges_to_reference(rtn):
    # repeated RTI steps with the exact double integrator as the plant drive
    # the state to a constant reference
    import torch
    B, Nh, dt = 4, 10, 0.05
    ctl = rtn.DIController(np.full(B, Nh), np.full(B, dt), Q, R, QN, layers=_net([3, 16, 16, 1], 9, zero_out=True))
    target = np.array([1.0, 0.0])
    xref = _t(np.tile(target, (B * (Nh + 1), 1)), torch)
    uref = torch.zeros(B * Nh, device="cuda")
    xs = np.zeros((B, 2))
    ctl.reset(_t(xs, torch))
    for _ in range(200):
        u0, st = ctl.rti_step(_t(xs, torch), xref, uref)
        a = u0.double().cpu().numpy()
        xs = np.stack([xs[:, 0] + xs[:, 1] * dt + a * dt * dt / 2, xs[:, 1] + a * dt], 1)
    assert np.abs(xs - target).max() < 1e-3


def test_di_unsupported_entry_points(rtn):
    ctl = rtn.DIController([10], [0.05], Q, R, layers=_net([3, 16, 1], 1))
    with pytest.raises(rtn.RtnError, match="UNSUPPORTED"):
        rtn.Controller.autotune(ctl)
    with pytest.raises(rtn.RtnError, match="UNSUPPORTED"):
        rtn.Controller.tc_variants(ctl)
    ctl.close()
