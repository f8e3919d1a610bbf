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
    ([17, 512, 300, 512, 3], [20] * 40 + [7]),         # padded to 512: in tile mode 7 the layers with
                                                       # three 128-neuron tiles run on single CTAs
])
def test_fp8_network_matches_oracle(rtn, orc, widths, N):
    # every layered shape the network admits: single CTAs (tile mode 6, the
    # default) and, where the padded width is a multiple of 256, the hidden
    # GEMMs on CTA pairs (mode 7; layers with an odd number of 128-neuron
    # tiles stay on single CTAs)
    layers = fp8_layers(widths, 3)
    N = np.asarray(N, np.int32)
    dt = np.full(len(N), 0.05)
    ctl = rtn.Controller(N, dt, W.Q_DIAG, W.R_DIAG, quad=QUAD, layers=layers, precision="fp8")
    hp = (max(widths[1:-1]) + 127) // 128 * 128
    modes = sorted(v[2] for v in ctl.tc_variants())
    assert modes == ([6, 7] if hp % 256 == 0 else [6]), modes
    X, U = W.random_nodes(ctl.n_states, 6)
    X, U = f32(X), f32(U[:ctl.n_nodes])
    fr, Jr, *_ = orc.linearize(QUAD, layers, N, dt, X, U)
    got = {}
    for vi, _, mode, *_ in ctl.tc_variants():
        ctl.tc_select(vi)
        fD, JD = ctl.mlp_eval(dev(X), dev(U))
        assert ctl.device_error() == 0
        F, J = fD.double().cpu().numpy(), JD.double().cpu().numpy()
        assert np.isfinite(F).all() and np.isfinite(J).all()
        ej = rel_rows(J, Jr)
        assert ej.max() < 1e-3, (mode, ej.max(), np.median(ej))
        assert np.abs(F - fr).max() / np.abs(fr).max() < 1e-3, mode
        got[mode] = (F, J)
    if 7 in got:
        # the two shapes run the same products: they agree far inside the gate
        assert rel_rows(got[7][1], got[6][1]).max() < 1e-4
        assert np.abs(got[7][0] - got[6][0]).max() / np.abs(got[6][0]).max() < 1e-5
    ctl.close()


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


def test_fp8_full_size_pairs(rtn, orc):
    # the precision workload at full size (163,840 nodes) with the FP8 hidden
    # GEMMs on CTA pairs (tile mode 7): f_D and J_D of sampled nodes
    # (the first, the last, 40 spread over the batch) against the oracle on
    # the same dequantised weights
    prob = W.make_problem("cfg3_bf16_precision", seed=0)
    layers = W.quantize_e4m3(prob["layers"])
    N = prob["N"]
    B, nn = len(N), int(N.sum())
    X, U = W.random_nodes(nn + B, 5)
    X, U = f32(X), f32(U[:nn])
    ctl = rtn.Controller(N, f32(prob["dt"]), prob["Q"], prob["R"], QN=prob["QN"], quad=QUAD, layers=layers,
                         precision="fp8")
    vi = [v[0] for v in ctl.tc_variants() if v[2] == 7]
    assert vi
    ctl.tc_select(vi[0])
    fD, JD = (t.double().cpu().numpy() for t in ctl.mlp_eval(dev(X), dev(U)))
    assert ctl.device_error() == 0
    assert np.isfinite(fD).all() and np.isfinite(JD).all()
    xo = np.concatenate([[0], np.cumsum(N + 1)])[:-1]
    uo = np.concatenate([[0], np.cumsum(N)])[:-1]
    inst = np.repeat(np.arange(B), N)
    rng = np.random.default_rng(12)
    for n in sorted(set(rng.choice(nn, 40, replace=False).tolist()) | {0, nn - 1}):
        b = inst[n]
        z = np.concatenate([X[xo[b] + (n - uo[b])], U[n]])
        rf, rJ = orc.mlp_fwd_jac(layers, z)
        assert np.linalg.norm(JD[n] - rJ) / np.linalg.norm(rJ) < 1e-3, ("J_D", n)
        assert np.abs(fD[n] - rf).max() / max(np.abs(rf).max(), 1e-3) < 1e-3, ("f_D", n)
    ctl.close()
