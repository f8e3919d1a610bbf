"""rtn_rti_step_host: the RTI step with host buffers, its inputs copied on a
second stream while the linearisation runs, gives bit-for-bit the commands,
statuses and iterates of rtn_rti_step on device buffers, step after step
(the copies of one step must not overtake the QP of the step before)."""
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


@pytest.mark.parametrize("config", ["cfg3_bf16_precision", "cfg4_ragged_batch"])
def test_rti_step_host_matches_device_buffers(rtn, config):
    # uniform horizons, and ragged ones (N_b in {10..50}, per-instance dt_b)
    prob = W.make_problem(config, seed=1, B=96, bf16=True)
    N, B = prob["N"], len(prob["N"])
    dt = np.asarray(prob["dt"], np.float32).astype(np.float64)

    def make():
        return rtn.Controller(N, dt, prob["Q"], prob["R"], QN=prob["QN"], quad=QUAD, layers=prob["layers"],
                              precision="bf16x2")

    dev, host = make(), make()
    X, U = W.random_nodes(dev.n_states, 5)
    xs = torch.as_tensor(X, dtype=torch.float32)
    us = torch.as_tensor(U[:dev.n_nodes], dtype=torch.float32)
    for c in (dev, host):
        c.set_iterate(xs.cuda(), us.cuda())
    xref, uref = W.node_refs(prob)
    h_xr = torch.as_tensor(xref, dtype=torch.float32).pin_memory()
    h_ur = torch.as_tensor(uref, dtype=torch.float32).pin_memory()
    d_xr, d_ur = h_xr.cuda(), h_ur.cuda()
    xo = np.concatenate([[0], np.cumsum(N + 1)])[:-1]
    h_u0 = torch.empty((B, 4), dtype=torch.float32).pin_memory()
    h_st = torch.empty(B, dtype=torch.int32).pin_memory()
    for step in range(4):
        # a different measured state every step: the host copy of step k must
        # not be read by the QP of step k - 1 or be overwritten before it
        h_x0 = (xs[torch.as_tensor(xo)] + 0.01 * (step + 1)).contiguous().pin_memory()
        u0, st = dev.rti_step(h_x0.cuda(), d_xr, d_ur)
        host.rti_step_host(h_x0, h_xr, h_ur, h_u0, h_st)
        torch.cuda.synchronize()
        assert torch.equal(u0.cpu(), h_u0), step
        assert torch.equal(st.cpu(), h_st), step
    xa, ua = dev.get_iterate()
    xb, ub = host.get_iterate()
    assert torch.equal(xa, xb) and torch.equal(ua, ub)
    assert dev.device_error() == 0 and host.device_error() == 0
    dev.close()
    host.close()


def test_rti_step_host_pageable_buffers(rtn):
    # pageable host memory: the driver stages the copies, results unchanged
    prob = W.make_problem("cfg3_bf16_precision", seed=2, B=32, bf16=True)
    N, B = prob["N"], len(prob["N"])
    dt = np.asarray(prob["dt"], np.float32).astype(np.float64)

    def make():
        return rtn.Controller(N, dt, prob["Q"], prob["R"], QN=prob["QN"], quad=QUAD, layers=prob["layers"],
                              precision="bf16x2")

    dev, host = make(), make()
    xref, uref = W.node_refs(prob)
    h_xr = torch.as_tensor(xref, dtype=torch.float32)
    h_ur = torch.as_tensor(uref, dtype=torch.float32)
    xo = np.concatenate([[0], np.cumsum(N + 1)])[:-1]
    h_x0 = (h_xr[torch.as_tensor(xo)] + 0.05).contiguous()
    assert not h_x0.is_pinned()
    h_u0 = torch.empty((B, 4), dtype=torch.float32)
    for step in range(2):
        u0, _ = dev.rti_step(h_x0.cuda(), h_xr.cuda(), h_ur.cuda())
        host.rti_step_host(h_x0, h_xr, h_ur, h_u0)
        torch.cuda.synchronize()
        assert torch.equal(u0.cpu(), h_u0), step
    dev.close()
    host.close()
