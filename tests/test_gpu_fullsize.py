"""GPU parity at the headline workload's full size, in the launch
configuration bench.py times: 8192 instances x N = 20 (163,840 nodes), the
17-512x5-3 network with BF16-representable weights, split BF16, the tile
shape the autotuner picks.  The whole batch runs on the GPU; sampled nodes
(spread over the batch, with the first node and the last node of the ragged
final tile) and sampled instances' RTI steps are recomputed one by one by the
FP64 oracle.  Bar: the split-BF16 gate, 1e-3 relative per node (Frobenius
norm of each block)."""
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


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _rel(a, b, floor=1e-12):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), floor))


def f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def test_cfg3_full_size_sampled_against_oracle(rtn, orc):
    prob = W.make_problem("cfg3_bf16_precision", seed=0, bf16=True)
    N = prob["N"]
    B, nn = len(N), int(N.sum())
    assert B == 8192 and nn == 163840
    dt = f32(prob["dt"])
    X, U = W.random_nodes(nn + B, 3)
    X, U = f32(X), f32(U[:nn])
    ctl = rtn.Controller(N, dt, prob["Q"], prob["R"], QN=prob["QN"], quad=QUAD, layers=prob["layers"],
                         precision="bf16x2")
    ctl.autotune()  # the shape bench.py times
    fD, JD, A, Bm, c = (t.double().cpu().numpy() for t in ctl.linearize(_dev(X), _dev(U)))
    assert ctl.device_error() == 0
    xo = np.concatenate([[0], np.cumsum(N + 1)])[:-1]
    uo = np.concatenate([[0], np.cumsum(N)])[:-1]
    inst = np.repeat(np.arange(B), N)
    rng = np.random.default_rng(7)
    nodes = sorted(set(rng.choice(nn, 40, replace=False).tolist()) | {0, nn - 1})
    for n in nodes:
        b = inst[n]
        row = xo[b] + (n - uo[b])
        rf, rJ, rA, rB, rc = orc.linearize(QUAD, prob["layers"], np.array([1], np.int32), dt[b:b + 1],
                                           X[row:row + 2], U[n:n + 1])
        assert _rel(fD[n], rf[0]) < 1e-3, ("f_D", n)
        assert _rel(JD[n], rJ[0]) < 1e-3, ("J_D", n)
        assert _rel(A[n], rA[0]) < 1e-3, ("A", n)
        assert _rel(Bm[n], rB[0]) < 1e-3, ("B", n)
        assert _rel(c[n] + X[row + 1], rc[0] + X[row + 1]) < 1e-3, ("phi", n)

    # one RTI step of the whole batch; sampled instances against the oracle
    xref, uref = W.node_refs(prob)
    xref, uref = f32(xref), f32(uref)
    x0 = f32(X[xo] + 0.02)
    ctl.set_iterate(_dev(X), _dev(U))
    u0, st = ctl.rti_step(_dev(x0), _dev(xref), _dev(uref))
    xn, un = (t.double().cpu().numpy() for t in ctl.get_iterate())
    u0 = u0.double().cpu().numpy()
    assert (st.cpu().numpy() == 0).all() and ctl.device_error() == 0
    for b in sorted({0, B - 1} | set(rng.choice(B, 4, replace=False).tolist())):
        xs = slice(xo[b], xo[b] + N[b] + 1)
        us = slice(uo[b], uo[b] + N[b])
        ru0, rx, ru, rst = orc.rti_step(QUAD, prob["layers"], N[b:b + 1], dt[b:b + 1], prob["Q"], prob["R"],
                                        prob["QN"], X[xs], U[us], xref[xs], uref[us], x0[b:b + 1])
        assert rst[0] == 0
        assert _rel(u0[b], ru0[0]) < 1e-3, ("u_0", b)
        assert _rel(xn[xs], rx) < 1e-3, ("x", b)
        assert _rel(un[us], ru) < 1e-3, ("u", b)
    ctl.close()


@pytest.mark.parametrize("mode", [6, 7])
def test_cfg3_full_size_layered_shapes(rtn, orc, mode):
    # both layered reverse-mode shapes (backward GEMMs on single CTAs, tile
    # mode 6, or on CTA pairs, mode 7) at 163,840 nodes: f_D and J_D of
    # sampled nodes (the first, the last, and 40 spread over the batch)
    # against the oracle
    prob = W.make_problem("cfg3_bf16_precision", seed=0, bf16=True)
    N = prob["N"]
    B, nn = len(N), int(N.sum())
    X, U = W.random_nodes(nn + B, 5)
    X, U = f32(X), f32(U[:nn])
    ctl = rtn.Controller(N, f32(prob["dt"]), prob["Q"], prob["R"], QN=prob["QN"], quad=QUAD,
                         layers=prob["layers"], precision="bf16x2")
    vi = [v[0] for v in ctl.tc_variants() if v[2] == mode]
    assert vi, mode
    ctl.tc_select(vi[0])
    fD, JD = (t.double().cpu().numpy() for t in ctl.mlp_eval(_dev(X), _dev(U)))
    assert ctl.device_error() == 0
    assert np.isfinite(fD).all() and np.isfinite(JD).all()
    xo = np.concatenate([[0], np.cumsum(N + 1)])[:-1]
    uo = np.concatenate([[0], np.cumsum(N)])[:-1]
    inst = np.repeat(np.arange(B), N)
    rng = np.random.default_rng(11)
    for n in sorted(set(rng.choice(nn, 40, replace=False).tolist()) | {0, nn - 1}):
        b = inst[n]
        z = np.concatenate([X[xo[b] + (n - uo[b])], U[n]])
        rf, rJ = orc.mlp_fwd_jac(prob["layers"], z)
        assert _rel(fD[n], rf) < 1e-3, ("f_D", mode, n)
        assert _rel(JD[n], rJ) < 1e-3, ("J_D", mode, n)
    ctl.close()
