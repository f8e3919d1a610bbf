"""GPU parity of the FP8 network path (RTN_FP8) against the FP64 oracle.

The library quantises every weight matrix to e4m3 with the per-layer scale
amax/448 at create; the oracle evaluates the same dequantised weights
(workload.quantize_e4m3, whose result the library reproduces), so the error
measures the arithmetic: the hidden->hidden GEMMs multiply e4m3 weights with
activations / adjoints held as three e4m3 pieces (~12 significant bits) in
kind::f8f6f4 MMAs with FP32 accumulation; the input layer, the folded first
backward layer and the Jacobian GEMM run as in the split-BF16 path.  Gate:
J_D within 1e-3 relative per node (the bar of the BF16 Jacobians), f_D
within 1e-3 of the largest output."""
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


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def rel_rows(a, b, floor=1e-30):
    a = a.reshape(a.shape[0], -1); b = b.reshape(b.shape[0], -1)
    return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), floor)


def fp8_layers(widths, seed, bias=True):
    layers = W.xavier_mlp(widths, seed)
    if bias:
        layers = [(Wl, f32(np.random.default_rng(30 + i).normal(0, 0.05, bl.shape))) for i, (Wl, bl) in enumerate(layers)]
    return W.quantize_e4m3(layers)


def test_library_quantisation_matches_workload(rtn):
    widths = [17, 256, 256, 256, 3]
    raw = W.xavier_mlp(widths, 5)
    ctl = rtn.Controller(np.array([3, 4], np.int32), np.full(2, 0.05), W.Q_DIAG, W.R_DIAG, quad=QUAD, layers=raw,
                         precision="fp8")
    got = ctl.get_params()
    for (Wg, _), (Wq, _) in zip(got, W.quantize_e4m3(raw)):
        assert np.abs(Wg - Wq).max() <= 2.0 ** -23 * np.abs(Wq).max()
    # and quantising already quantised weights changes nothing
    c2 = rtn.Controller(np.array([3, 4], np.int32), np.full(2, 0.05), W.Q_DIAG, W.R_DIAG, quad=QUAD,
                        layers=W.quantize_e4m3(raw), precision="fp8")
    for (Wg, _), (Wq, _) in zip(c2.get_params(), W.quantize_e4m3(raw)):
        assert np.abs(Wg - Wq).max() <= 2.0 ** -23 * np.abs(Wq).max()


@pytest.mark.parametrize("widths,N", [
    ([17, 512, 512, 512, 512, 512, 3], [20] * 9),      # the precision workload's network, ragged tail
    ([17, 256, 256, 256, 256, 3], [17, 50, 10, 33]),   # the ragged workload's network
    ([17, 300, 200, 3], [7, 9]),                       # widths off the tile sizes, one hidden->hidden layer
    ([17, 384, 384, 384, 3], [20] * 70 + [13]),        # several tiles per CTA
])
def test_fp8_network_matches_oracle(rtn, orc, widths, N):
    layers = fp8_layers(widths, 3)
    N = np.asarray(N, np.int32)
    dt = np.full(len(N), 0.05)
    ctl = rtn.Controller(N, dt, W.Q_DIAG, W.R_DIAG, quad=QUAD, layers=layers, precision="fp8")
    assert [v[2] for v in ctl.tc_variants()] == [6]
    X, U = W.random_nodes(ctl.n_states, 6)
    X, U = f32(X), f32(U[:ctl.n_nodes])
    fD, JD = ctl.mlp_eval(dev(X), dev(U))
    assert ctl.device_error() == 0
    fr, Jr, *_ = orc.linearize(QUAD, layers, N, dt, X, U)
    F, J = fD.double().cpu().numpy(), JD.double().cpu().numpy()
    assert np.isfinite(F).all() and np.isfinite(J).all()
    ej = rel_rows(J, Jr)
    assert ej.max() < 1e-3, (ej.max(), np.median(ej))
    assert np.abs(F - fr).max() / np.abs(fr).max() < 1e-3


def test_fp8_rti_step_matches_oracle(rtn, orc):
    prob = W.make_problem("cfg3_bf16_precision", seed=2, B=6)
    layers = W.quantize_e4m3(prob["layers"])
    N, dt = prob["N"], f32(prob["dt"])
    X, U = W.random_nodes(int(N.sum()) + len(N), 3)
    X, U = f32(X), f32(U[:int(N.sum())])
    xref, uref = W.node_refs(prob)
    xref, uref = f32(xref), f32(uref)
    x0 = f32(X[np.concatenate([[0], np.cumsum(N + 1)])[:-1]] + 0.03)
    ctl = rtn.Controller(N, dt, prob["Q"], prob["R"], quad=QUAD, layers=layers, precision="fp8")
    ctl.set_iterate(dev(X), dev(U))
    u0, st = ctl.rti_step(dev(x0), dev(xref), dev(uref))
    assert ctl.device_error() == 0
    u0r, _, _, str_ = orc.rti_step(QUAD, layers, N, dt, prob["Q"], prob["R"], prob["QN"], X, U, xref, uref, x0)
    assert (st.cpu().numpy() == 0).all() and (str_ == 0).all()
    assert np.abs(u0.double().cpu().numpy() - u0r).max() / np.abs(u0r).max() < 1e-3
