"""The bench's roofline accounting for the layered reverse mode (host
arithmetic only): algorithmic FLOPs and DRAM bytes per launch kind, checked
against totals derived by hand for the 17-512x5-3 network of the cfg3
workload, and against the reverse-mode FLOP count of the whole network."""
import bench

W = [17, 512, 512, 512, 512, 512, 3]


def test_layered_flops_sum_to_reverse_mode_minus_output_layer():
    # every layer GEMM is counted once; the output layer (2 x 3 x h per
    # node) runs on the SIMT cores and carries no GEMM FLOPs
    nn = 1000
    total = sum(bench.lay_flops(k, W, nn) for k in bench.LAY_KERNELS)
    assert total == (bench.rev_flops_per_node(W) - 2 * 3 * W[-2]) * nn


def test_layered_bytes_per_node_by_hand():
    # 4 B per value (FP32, or a BF16 hi + lo pair), per node:
    #   inputs:          x, u in (17) and z out (17)                 136
    #   input GEMM:      z in, a_1 out                 (17 + 512) * 4 = 2116
    #   forward GEMMs:   a_l in, a_{l+1} out, x4; d_5 out        4 * 4096 + 2048 = 18432
    #   output layer:    a_5 in, f_D out               (512 + 3) * 4 = 2060
    #   first backward:  d_5 in, a_4 in, D_4 out (3 rows)  (512 + 512 + 1536) * 4 = 10240
    #   backward x3:     D_{l+1} in, a_l in, D_l out     3 * 14336 = 43008
    #   Jacobian:        D_1 in, J_D out               (1536 + 51) * 4 = 6348
    per_node = {"inputs": 136, "input GEMM": 2116, "forward GEMM": 18432, "output layer": 2060,
                "first backward GEMM": 10240, "backward GEMM": 43008, "Jacobian GEMM": 6348}
    for kind, b in per_node.items():
        assert bench.lay_bytes(kind, W, 1) == b, kind
    assert sum(bench.lay_bytes(k, W, 163840) for k in bench.LAY_KERNELS) == 82340 * 163840


def test_backward_gemm_flops_and_intensity():
    # reverse-mode algorithmic FLOPs of one backward GEMM launch at the cfg3
    # workload: 3 adjoint rows x 2 x 512 x 512 per node, 163,840 nodes; the
    # bench reports this kernel tensor-bound against the BF16 peak.  Its
    # design moves 14,336 B per node (adjoints and a_l through HBM), an
    # intensity of 109.7 FLOP/B, below the BF16 ridge (~274 FLOP/B on the
    # measured peaks): reported beside it as the HBM view
    nn = 163840
    fl = bench.lay_flops("backward GEMM", W, nn) / 3
    assert fl == 3 * 2 * 512 * 512 * nn
    by = bench.lay_bytes("backward GEMM", W, 1) / 3
    assert abs(bench.lay_flops("backward GEMM", W, 1) / 3 / by - 2 * 3 * 512 * 512 / 14336) < 1e-9
    assert bench.A1_METHOD_BYTES_PER_NODE == 284


def test_clock_summary_keeps_the_timed_window():
    # samples outside the timed region (idle before it, the power-capped
    # tail after it) must not decide the reported clocks
    import bench
    ck = bench.Clocks()
    row = lambda sm, cap: [str(sm), "2032", "500.0", "Not Active", "Not Active", "Not Active", cap]
    ck.rows = [(0.0, row(2032, "Not Active")), (1.0, row(1732, "Active")), (1.1, row(1800, "Active")),
               (5.0, row(2032, "Not Active"))]
    ck.mark(0.95, 1.05)
    s = ck.summary()
    assert s["samples"] == 2 and s["sm_mhz"] == 1766.0 and s["sm_min_mhz"] == 1732.0
    assert s["reasons"] == ["sw_power_cap"]
    ck.mark(3.0, 3.01)  # no sample inside: the two nearest
    s = ck.summary()
    assert s["samples"] == 2 and s["sm_min_mhz"] == 1800.0


def test_profiled_figures_follow_the_committed_summary():
    # the layered summary under profiles/ was captured on the current kernel
    # sources in tile mode 7: its DRAM bytes and tensor-pipe activity are read
    # back per launch kind, and nothing is read for another tile mode or a
    # launch kind the summary does not cover
    import bench
    assert bench.profiled_layer_traffic("backward GEMM", 7) > 0
    pipe = bench.profiled_tensor_pipe("backward GEMM", 7)
    assert pipe is not None and 0.0 < pipe <= 100.0
    assert bench.profiled_tensor_pipe("first backward GEMM", 7) is not None
    assert bench.profiled_tensor_pipe("backward GEMM", 6) is None
    assert bench.profiled_tensor_pipe("Jacobian GEMM", 7) is None
