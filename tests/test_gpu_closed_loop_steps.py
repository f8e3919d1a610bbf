"""The graph-replayed closed loop (rtn_closed_loop) against the same steps
made one call at a time (rtn_rti_step, then rtn_plant_step): bit-for-bit
equal plant trajectories, commands and iterates for 1, 2 and 3 steps.  The
loop runs each step's plant step on a second graph branch beside the next
step's linearisation, and its first RTI step and last plant step outside
the graph, so these short runs cover every part of that schedule."""
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


@pytest.mark.parametrize("steps", [1, 2, 3])
def test_closed_loop_matches_manual_steps(rtn, steps):
    prob = W.make_problem("cfg3_bf16_precision", seed=3, B=24, bf16=True)
    N, B = prob["N"], len(prob["N"])
    dt = np.asarray(prob["dt"], np.float32).astype(np.float64)

    def make():
        return rtn.Controller(N, dt, prob["Q"], prob["R"], QN=prob["QN"], quad=QUAD, layers=prob["layers"],
                              precision="bf16x2")

    loop, manual = make(), make()
    xrt, urt = W.trajectory_refs(prob, steps)
    x_start = xrt[:, 0] + 0.03
    for c in (loop, manual):
        c.reset(torch.as_tensor(x_start, dtype=torch.float32, device="cuda"))
    xrt_d = torch.as_tensor(xrt, dtype=torch.float32, device="cuda").contiguous()
    urt_d = torch.as_tensor(urt, dtype=torch.float32, device="cuda").contiguous()
    xp_loop = torch.as_tensor(x_start, dtype=torch.float64, device="cuda").contiguous()
    traj, uo = loop.closed_loop(steps, xrt_d, urt_d, xp_loop, plant="drag", record=True)

    # the same steps one call at a time, references sliced at each step
    xo = np.concatenate([[0], np.cumsum(N + 1)])[:-1]
    uo_off = np.concatenate([[0], np.cumsum(N)])[:-1]
    xp = torch.as_tensor(x_start, dtype=torch.float64, device="cuda").contiguous()
    for t in range(steps):
        xr = np.concatenate([xrt[b, t:t + N[b] + 1] for b in range(B)])
        ur = np.concatenate([urt[b, t:t + N[b]] for b in range(B)])
        assert xr.shape[0] == manual.n_states and ur.shape[0] == manual.n_nodes
        u0, st = manual.rti_step(xp.float().contiguous(), torch.as_tensor(xr, dtype=torch.float32, device="cuda"),
                                 torch.as_tensor(ur, dtype=torch.float32, device="cuda"))
        xp = manual.plant_step(xp, u0, kind="drag", nsub=4)
        torch.cuda.synchronize()
        assert torch.equal(uo[t], u0), t
        assert torch.equal(traj[t], xp.float()), t
    assert torch.equal(xp_loop, xp)
    xa, ua = loop.get_iterate()
    xb, ub = manual.get_iterate()
    assert torch.equal(xa, xb) and torch.equal(ua, ub)
    assert loop.device_error() == 0 and manual.device_error() == 0
    assert int(xo[-1]) + N[-1] + 1 == manual.n_states and int(uo_off[-1]) + N[-1] == manual.n_nodes
    loop.close()
    manual.close()
