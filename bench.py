"""Benchmark of the Real-time Neural MPC hot path on one B300.

One step = one closed-loop control step of every controller instance: the
RTI step (network value + Jacobian at every node, RK4 sensitivities, Riccati
sweep, feedback update) followed by the plant step, replayed as a CUDA graph
through rtn_closed_loop.  `value` is instance RTI steps per second
(B x K / device time of K steps).  The roofline of the network pass is
tensor-bound: the dominant kernel's reverse-mode algorithmic FLOPs per launch
over its CUDA-event time, against the measured BF16 peak.  The error table
compares the GPU results with the FP64 oracle on a sample of instances, in
the CPU-baseline leg (the one place, with --impl reference, where the bench
runs the oracle).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import hashlib
import json
import re
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workload as W  # noqa: E402

# the headline metric of the precision workload
METRIC = 'SQP-RTI node-linearizations/s + RTI steps/s, BF16 vs FP32 @ ≤1e-3 Jac err'


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d["hbm_gbs"], d["bf16_tflops"], d.get("bf16_tflops_sustained", d["bf16_tflops"]), "measured"
    return 6400.0, 1800.0, 1400.0, "fallback"


LAYERED_PROFILE = "mlp_lay_pass_2048x20_h512x5_bf16x2.md"


def kernel_md5(files):
    """md5 over kernel sources (each profile records it with its file list)."""
    h = hashlib.md5()
    for f in files:
        with open(os.path.join(ROOT, "paper_2203_07747_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def fwd_flops_per_node(widths):
    """Forward-mode algorithmic FLOPs per node.  Hidden->hidden and output
    layers multiply 18 columns (value + 17 tangents); the input layer costs
    its value dot products plus the tangent scaling (its tangent block is the
    weight matrix itself)."""
    f = 2 * 17 * widths[1] + 17 * widths[1]
    for fi, fo in zip(widths[1:-1], widths[2:]):
        f += 2 * 18 * fi * fo
    return f


def rev_flops_per_node(widths):
    """Reverse-mode algorithmic FLOPs per node: the value pass (input layer,
    hidden->hidden layers, output layer) plus three adjoint rows carried back
    through every hidden->hidden layer and the input layer (J_D = W_0' D_1).
    The elementwise scalings by d_l = 1 - a_l^2 are not counted."""
    h1, hl = widths[1], widths[-2]
    mm = sum(fi * fo for fi, fo in zip(widths[1:-1], widths[2:-1]))
    return 2 * 17 * h1 + 2 * 3 * hl + 4 * 2 * mm + 3 * 2 * 17 * h1


class Clocks:
    """nvidia-smi samples during the timed region: every sample carries its
    host arrival time, and the summary keeps those that arrived inside the
    window set by mark() (the timed region, plus 150 ms for the sampler's
    reporting lag), or the two nearest if none did (nvidia-smi refreshes
    its readings about every 100 ms)."""

    def __init__(self):
        self.rows, self.p, self.window = [], None, None

    def mark(self, t0, t1):
        self.window = (t0, t1 + 0.15)

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            dev = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0]
            self.p = subprocess.Popen(["nvidia-smi", "-i", dev, f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "20"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except Exception:
            self.p = None
        return self

    def _read(self):
        for line in self.p.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 7:
                self.rows.append((time.time(), parts))

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        rows = [r for t, r in self.rows]
        if self.window:
            t0, t1 = self.window
            inside = [r for t, r in self.rows if t0 <= t <= t1]
            if not inside:
                mid = 0.5 * (t0 + t1)
                inside = [r for t, r in sorted(self.rows, key=lambda tr: abs(tr[0] - mid))[:2]]
            rows = inside
        sm = [v for v in (num(r[0]) for r in rows) if v is not None]
        mx = [v for v in (num(r[1]) for r in rows) if v is not None]
        pw = [v for v in (num(r[2]) for r in rows) if v is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[3 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "sm_min_mhz": min(sm) if sm else None, "power_w_max": max(pw) if pw else None,
                "reasons": reasons, "samples": len(rows)}


def make(prob, precision, riccati_f64=False, box_qp=False, train_bf16=False):
    import paper_2203_07747_b300 as rtn
    return rtn.Controller(prob["N"], prob["dt"], prob["Q"], prob["R"], QN=prob["QN"], quad=prob["quad"],
                          layers=prob["layers"], precision=precision, riccati_f64=riccati_f64,
                          box_qp=box_qp, train_bf16=train_bf16)


def launches_per_step(ctl, tile_mode=None):
    L = len(ctl.layers) if ctl.layers else 0
    # network: one fused launch, the layered reverse mode 2 L (inputs, input
    # GEMM, forward GEMMs, output, backward GEMMs, Jacobian), the FP32 path L
    # (input, hidden GEMMs, output)
    mlp = 0 if not L else (L if ctl.precision == "fp32" else 2 * L if tile_mode in (6, 7) else 1)
    return mlp + 1 + 1 + 3  # network, RK4, Riccati, plant + record + advance


def rank_barrier():
    """Barrier over the ranks of a torchrun launch (no-op for one process)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def max_over_ranks(v, device):
    """The maximum of a per-rank number over all ranks (the step time of a
    weak-scaled run is the slowest rank's)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(v)
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(instances_per_rank, world, ms_step_max):
    """Whole-job RTI steps/s of a weak-scaled run: every rank steps its own
    instances; the job's step takes the slowest rank's time."""
    return instances_per_rank * world / (ms_step_max * 1e-3)


def time_closed_loop(ctl, prob, steps, warmup):
    """Closed loop on the drag plant; every instance starts on its reference
    state (the random initial states of the workload recipe are used for the
    single-RTI-step measurements)."""
    import torch
    xrt, urt = W.trajectory_refs(prob, steps + warmup)
    xrt_d = torch.as_tensor(xrt, dtype=torch.float32, device="cuda").contiguous()
    urt_d = torch.as_tensor(urt, dtype=torch.float32, device="cuda").contiguous()
    x0 = xrt[:, 0].copy()
    ctl.reset(torch.as_tensor(x0, dtype=torch.float32, device="cuda"))
    xp = torch.as_tensor(x0, dtype=torch.float64, device="cuda").contiguous()
    ctl.closed_loop(warmup, xrt_d, urt_d, xp, plant="drag", record=False)
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # the timed steps continue on the reference window after the warm-up
    xr2, ur2 = xrt_d[:, warmup:].contiguous(), urt_d[:, warmup:].contiguous()
    with Clocks() as ck:
        torch.cuda.synchronize()
        rank_barrier()
        torch.cuda.synchronize()
        t0 = time.time()
        e0.record(s)
        traj, _ = ctl.closed_loop(steps, xr2, ur2, xp, plant="drag", record=True)
        e1.record(s)
        torch.cuda.synchronize()
        ck.mark(t0, time.time())
        rank_barrier()
    ms = e0.elapsed_time(e1)
    pos = traj[:, :, :3].double().cpu().numpy()
    err = np.linalg.norm(pos - xrt[:, warmup + 1:warmup + steps + 1, :3].transpose(1, 0, 2), axis=2)
    time_closed_loop.per_instance = np.sqrt((err ** 2).mean(0))
    return ms / steps, ck.summary(), float(np.sqrt((err ** 2).mean()))


def rmse_distribution(r):
    """Per-instance tracking RMSE [m] summarised over the batch."""
    return {"median": float(np.median(r)), "p90": float(np.percentile(r, 90)), "max": float(r.max()),
            "n_above_1m": int((r > 1.0).sum()), "worst_instances": [int(i) for i in np.argsort(r)[::-1][:4]]}


def time_calls(fn, reps, warm=3):
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        fn()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def e2e_rti(ctl, prob, steps):
    """Through the public API with host buffers (rtn_rti_step_host): per
    step x0, xref, uref from pinned host memory to the device (on a second
    stream, overlapped with the linearisation, which does not read them),
    the RTI step, u0 and the statuses back to pinned host memory."""
    import torch
    xref, uref = W.node_refs(prob)
    h_x0 = torch.as_tensor(prob["x0"], dtype=torch.float32).pin_memory()
    h_xr = torch.as_tensor(xref, dtype=torch.float32).pin_memory()
    h_ur = torch.as_tensor(uref, dtype=torch.float32).pin_memory()
    h_u0 = torch.empty((ctl.B, 4), dtype=torch.float32).pin_memory()
    h_st = torch.empty(ctl.B, dtype=torch.int32).pin_memory()

    def one():
        ctl.rti_step_host(h_x0, h_xr, h_ur, h_u0, h_st)

    ms = time_calls(one, steps)
    bi = sum(h.numel() * 4 for h in (h_x0, h_xr, h_ur))
    return ms, bi, h_u0.numel() * 4 + h_st.numel() * 4


def _rel(a, b):
    """Per-row relative Frobenius error ||a - b|| / max(||b||, 1e-12)."""
    a = a.reshape(a.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-12)


def _stat(e):
    return {"max": float(e.max()), "p99": float(np.percentile(e, 99))}


def error_sample(prob, precision, nb=64):
    """GPU side of the error table: f_D, J_D, A, B (rtn_linearize) and u_0
    (rtn_rti_step) of this precision's path on the first nb instances of the
    workload at seeded random nodes, and J_D with the FP32 weights the BF16
    ones were rounded from.  The oracle side is error_table()."""
    import torch
    sub = W.subset(prob, nb)
    N = sub["N"]
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")
    X, U = W.random_nodes(int(N.sum()) + len(N), 12)
    X, U = f32(X), f32(U[:int(N.sum())])
    xref, uref = W.node_refs(sub)
    xref, uref = f32(xref), f32(uref)
    x0 = f32(X[np.concatenate([[0], np.cumsum(N + 1)])[:-1]] + 0.02)

    def run(problem):
        c = make(problem, precision)
        out = [t.double().cpu().numpy() for t in c.linearize(dev(X), dev(U))[:4]]
        c.set_iterate(dev(X), dev(U))
        out.append(c.rti_step(dev(x0), dev(xref), dev(uref))[0].double().cpu().numpy())
        c.close()
        return out

    smp = {"sub": sub, "X": X, "U": U, "xref": xref, "uref": uref, "x0": x0, "gpu": run(sub)}
    if prob.get("bf16"):
        master = dict(sub)
        master["layers"] = W.xavier_mlp(prob["widths"], prob["seed"], bf16=False)
        smp["master"] = master
        smp["gpu_master_JD"] = run(master)[1]
    if precision == "fp8":
        # the GPU's J_D (quantised weights) against the oracle on the
        # unquantised ones: the effect of the e4m3 weights
        smp["gpu_master_JD"] = smp["gpu"][1]
    return smp


def error_table(smp):
    """Per-node (per-instance for u_0) relative errors, max and p99, of the
    GPU's f_D, J_D, A, B and u_0 against the FP64 oracle on the same inputs
    (the oracle evaluates the same BF16-representable weights, so the errors
    measure arithmetic); and J_D of the GPU path given the FP32 weights
    against the oracle on those weights (BF16 weight rounding included;
    reported, not gated)."""
    import oracle
    oracle.build()
    sub = smp["sub"]
    N, dt = sub["N"], np.asarray(sub["dt"], np.float32).astype(np.float64)
    X, U = smp["X"], smp["U"]
    fD, JD, A, Bm, _ = oracle.linearize(sub["quad"], sub["layers"], N, dt, X, U)
    u0, _, _, _ = oracle.rti_step(sub["quad"], sub["layers"], N, dt, sub["Q"], sub["R"], sub["QN"], X, U,
                                  smp["xref"], smp["uref"], smp["x0"])
    out = {"reference": "FP64 oracle (oracle/rtn_oracle.c) on the same inputs and weights",
           "sample": f"first {len(N)} instances ({int(N.sum())} nodes), seeded random nodes"}
    for name, g, r in zip(("f_D", "J_D", "A", "B", "u_0"), smp["gpu"], (fD, JD, A, Bm, u0)):
        out[name] = _stat(_rel(g, r))
    if "master" in smp:
        m = smp["master"]
        _, Jm, _, _, _ = oracle.linearize(m["quad"], m["layers"], N, dt, X, U)
        out["J_D_vs_fp32_master_weights"] = _stat(_rel(smp["gpu_master_JD"], Jm))
    return out


def cpu_baseline(prob, budget_s=15.0):
    """The oracle's RTI step on a bounded sample of instances of the same
    workload, timed on the host cores (the sample doubles until the budget
    would be exceeded)."""
    import oracle
    oracle.build()
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    nb, total, rate, done = 1, 0.0, None, 0
    while nb <= prob["B"]:
        sub = W.subset(prob, nb)
        N, dt, x0 = sub["N"], sub["dt"], sub["x0"]
        xref, uref = W.node_refs(sub)
        x = np.concatenate([np.repeat(x0[b:b + 1], N[b] + 1, 0) for b in range(nb)])
        u = np.full((int(N.sum()), 4), W.hover_thrust())
        t0 = time.perf_counter()
        oracle.rti_step(sub["quad"], sub["layers"], N, dt, sub["Q"], sub["R"], sub["QN"], x, u,
                        xref, uref, x0)
        el = time.perf_counter() - t0
        total += el
        rate, done = nb / el, nb
        if total + 2.2 * el > budget_s:
            break
        nb *= 2
    # one core: single-instance calls (the OpenMP loop then runs on one thread)
    sub = W.subset(prob, 1)
    N, dt, x0 = sub["N"], sub["dt"], sub["x0"]
    xref, uref = W.node_refs(sub)
    x = np.repeat(x0[0:1], N[0] + 1, 0)
    u = np.full((int(N.sum()), 4), W.hover_thrust())
    t0, k = time.perf_counter(), 0
    while k < 8 and (k == 0 or time.perf_counter() - t0 < 4.0):
        oracle.rti_step(sub["quad"], sub["layers"], N, dt, sub["Q"], sub["R"], sub["QN"], x.copy(), u.copy(),
                        xref, uref, x0)
        k += 1
    single = k / (time.perf_counter() - t0)
    return {"value": rate, "unit": "RTI steps/s", "cores": cores, "kind": "oracle",
            "sample": f"{done} of {prob['B']} instances, one RTI step (FP64 C, OpenMP over instances)",
            "single_core": {"value": single, "unit": "RTI steps/s",
                            "sample": f"{k} single-instance RTI steps, one thread"}}


def bench_ragged(steps=200):
    """cfg4: 4096 instances with horizons N_b ~ U{10..50}, dt_b ~ U[0.02, 0.1],
    17-256x4-3 network (split BF16), closed loop on the drag plant; tracking
    RMSE per instance, without and with the thrust bounds inside the QP.
    Returns the line object and the GPU side of its error table."""
    import torch
    prob = W.make_problem("cfg4_ragged_batch", seed=0, bf16=True)
    ctl = make(prob, "bf16x2")
    vi, _ = ctl.autotune()
    ms, clocks, rmse = time_closed_loop(ctl, prob, steps, 3)
    r_inst = time_closed_loop.per_instance
    x, u = ctl.get_iterate()
    out = ctl.linearize(x, u)
    nn = int(prob["N"].sum())
    ms_lin = time_calls(lambda: ctl.linearize(x, u, out), 10)
    ctl.close()
    cb = make(prob, "bf16x2", box_qp=True)
    cb.tc_select(vi)
    ms_box, _, rmse_box = time_closed_loop(cb, prob, steps, 3)
    r_box = time_closed_loop.per_instance
    cb.close()
    import paper_2203_07747_b300 as rtn
    cf = rtn.Controller(prob["N"], prob["dt"], prob["Q"], prob["R"], QN=prob["QN"], quad=prob["quad"],
                        layers=prob["layers"], precision="bf16x2", fused_qp=True)
    cf.tc_select(vi)
    ms_fused, _, rmse_fused = time_closed_loop(cf, prob, steps, 3)
    cf.close()
    L = len(prob["layers"])
    smp = error_sample(prob, "bf16x2")
    line = {"workload": "cfg4_ragged_batch: 4096 instances, N_b in {10..50} (sum %d nodes), "
                        "dt_b in [0.02, 0.1] s, MLP 17-256x4-3 split BF16, %d-step closed loop, "
                        "drag plant, one CUDA graph per step" % (nn, steps),
            "rti_steps_per_s": prob["B"] / (ms * 1e-3), "ms_per_step": ms,
            "node_linearizations_per_s": nn / (ms_lin * 1e-3),
            "tracking_rmse_m": rmse, "tracking_rmse_per_instance_m": rmse_distribution(r_inst),
            "tracking_note": ("RMSE over all instances is dominated by the instances counted in n_above_1m: "
                              "figure-8s whose peak reference acceleration (~28-32 m/s^2) the unconstrained QP "
                              "(bounds only on the sent u_0) cannot follow; the FP64 oracle loses the same "
                              "instances (tests/test_gpu_long_horizon.py); with the thrust bounds inside the "
                              "QP every instance tracks (box_qp)"),
            "box_qp": {"rti_steps_per_s": prob["B"] / (ms_box * 1e-3), "tracking_rmse_m": rmse_box,
                       "tracking_rmse_per_instance_m": rmse_distribution(r_box)},
            "launches_per_step": 2 * L + 5,
            "fused_lin_qp": {"what": "RK4 linearisation and QP in one persistent launch with a work queue "
                                     "(rtn_options.fused_qp)",
                             "rti_steps_per_s": prob["B"] / (ms_fused * 1e-3), "ms_per_step": ms_fused,
                             "tracking_rmse_m": rmse_fused,
                             "launches_per_step": 2 * L + 4,
                             "note": "the RK4 and QP launches become one launch (its last warp returns the "
                                     "work-queue counters to zero for the next)"},
            "tile_variant": vi}
    return line, smp


def bench_box(prob, precision, tile, steps=20):
    """The thrust bounds inside the QP (primal-dual active set on the Riccati
    structure): the headline closed loop with the box QP, and the QP alone on
    a displaced start (every instance 2 m from its reference, iterate at
    hover there), where thrusts saturate, against the unconstrained QP."""
    import torch
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")
    ctl = make(prob, precision, box_qp=True)
    if tile is not None:
        ctl.tc_select(tile["variant"])
    ms, _, rmse = time_closed_loop(ctl, prob, steps, 3)
    its_loop = ctl.box_iterations()
    xrt, _ = W.trajectory_refs(prob, 1)
    x0 = xrt[:, 0].copy()
    x0[:, 0] += 2.0
    ctl.reset(dev(x0))
    x, u = ctl.get_iterate()
    A, Bm, c = ctl.linearize(x, u)[2:]
    xref, uref = W.node_refs(prob)
    args = (A, Bm, c, x, u, dev(xref), dev(uref), dev(x0))
    ms_box = time_calls(lambda: ctl.qp_solve(*args), 5)
    _, _, st = ctl.qp_solve(*args)
    its = ctl.box_iterations()
    st = st.cpu().numpy()
    ctl.close()
    cu = make(prob, "fp32")
    ms_free = time_calls(lambda: cu.qp_solve(*args), 5)
    _, du_free, _ = cu.qp_solve(*args)
    uf = (u + du_free).cpu().numpy()
    cu.close()
    return {"rti_steps_per_s": prob["B"] / (ms * 1e-3), "ms_per_step": ms, "tracking_rmse_m": rmse,
            "closed_loop_subproblems_last_step": {"mean": float(its_loop.mean()), "max": int(its_loop.max())},
            "displaced_start": {
                "workload": "every instance 2 m from its reference, iterate at hover there, one QP",
                "ms_box_qp": ms_box, "ms_unconstrained_qp": ms_free,
                "unconstrained_step_nodes_outside_bounds_frac": float(((uf < 0) | (uf > prob["quad"]["u_max"])).any(axis=1).mean()) if uf.ndim == 2 else None,
                "subproblems": {"mean": float(its.mean()), "p99": float(np.percentile(its, 99)),
                                "max": int(its.max()), "frac_more_than_one": float((its > 1).mean())},
                "not_converged": int((st == 8).sum())}}


def bench_fp8(prob, bf16_burst, steps=20):
    """The precision workload with the FP8 network path: weights quantised to
    e4m3 with per-layer scale amax/448 (the oracle of the error table gets the
    same dequantised weights), closed loop RTI steps/s, node linearisations/s,
    the network pass against the FP8 tensor peak; the GPU side of its error
    table (the oracle side runs in the CPU-baseline leg)."""
    q = dict(prob)
    q["layers"] = W.quantize_e4m3(prob["layers"])
    q["bf16"] = False
    ctl = make(q, "fp8")
    ms, _, rmse = time_closed_loop(ctl, q, steps, 3)
    x, u = ctl.get_iterate()
    out = ctl.linearize(x, u)
    nn = int(q["N"].sum())
    ms_lin = time_calls(lambda: ctl.linearize(x, u, out), 10)
    ms_mlp = time_calls(lambda: ctl.mlp_eval(x, u, out[0], out[1]), 10)
    flops = rev_flops_per_node(q["widths"]) * nn
    ctl.close()
    smp = error_sample(q, "fp8")
    # J_D against the unquantised network (weight quantisation included)
    master = dict(smp["sub"])
    master["layers"] = prob["layers"]
    smp["master"] = master
    peak8 = 2.0 * bf16_burst
    return {"workload": "cfg3 workload, weights e4m3 with per-layer scale amax/448, FP8 network path "
                        "(hidden GEMMs kind::f8f6f4, activations/adjoints as three e4m3 pieces)",
            "rti_steps_per_s": q["B"] / (ms * 1e-3), "ms_per_step": ms,
            "node_linearizations_per_s": nn / (ms_lin * 1e-3), "ms_network_pass": ms_mlp,
            "tracking_rmse_m": rmse,
            "roofline": {"bound": "tensor", "peak": peak8, "unit": "TFLOP/s",
                         "peak_kind": "fp8 dense = measured bf16 burst x 2 (nominal ratio 4.5 / 2.25)",
                         "achieved": flops / (ms_mlp * 1e-3) / 1e12,
                         "frac": flops / (ms_mlp * 1e-3) / 1e12 / peak8,
                         "note": "whole pass (reverse-mode FLOPs); three e4m3 MMAs per product in the hidden "
                                 "GEMMs, the input / first backward / Jacobian GEMMs in split BF16"}}, smp


def bench_riccati(prob, precision, tile, steps=20):
    """The headline closed loop with the other Riccati arithmetics: the FP32
    sweep with the factorisation of R + B'PB in FP64
    (riccati_f64 = 2) and the FP64 sweep (riccati_f64 = 1); RTI steps/s, the
    QP kernel's time per call and tracking RMSE of each."""
    out = {}
    for name, ric in (("fp32_sweep_fp64_cholesky", "chol64"), ("fp64_sweep", 1)):
        ctl = make(prob, precision, riccati_f64=ric)
        if tile is not None:
            ctl.tc_select(tile["variant"])
        ms, _, rmse = time_closed_loop(ctl, prob, steps, 3)
        x, u = ctl.get_iterate()
        A, Bm, c = ctl.linearize(x, u)[2:]
        xref, uref = W.node_refs(prob)
        import torch
        dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")
        args = (A, Bm, c, x, u, dev(xref), dev(uref), dev(prob["x0"]))
        ms_qp = time_calls(lambda: ctl.qp_solve(*args), 5)
        ctl.close()
        out[name] = {"rti_steps_per_s": prob["B"] / (ms * 1e-3), "ms_per_step": ms, "ms_qp": ms_qp,
                     "tracking_rmse_m": rmse}
    return out


def bench_learned(bf16_burst, epochs=2, steps=100):
    """cfg5: 2^20 seeded samples -> drag residual targets, train 17-512x6-3
    (Adam, lr 1e-3, batch 4096) with BF16 GEMM operands and FP32
    accumulation (and, timed beside it, with split BF16 hi + lo operands),
    then a 4096-instance closed loop on the drag plant with the learned
    network vs the nominal model."""
    import torch
    prob = W.make_problem("cfg5_learned", seed=0, bf16=True)
    n = prob["cfg"]["n_samples"]
    X, U = W.training_samples(n, 0)
    Xd = torch.as_tensor(X, dtype=torch.float32, device="cuda")
    Ud = torch.as_tensor(U, dtype=torch.float32, device="cuda")
    bs, lr = prob["cfg"]["batch"], prob["cfg"]["lr"]
    w = prob["widths"]
    fwd = 2 * sum(a * b for a, b in zip(w[:-1], w[1:]))
    flops = 3 * fwd * epochs * (n // bs) * bs
    runs = {}
    for mode in (True, False):
        learn = make(prob, "bf16x2", train_bf16=mode)
        Yd = learn.drag_targets(Xd)
        # untimed warm-up on a throwaway controller: the first training GEMMs
        # of a process pay the one-time setup
        warm = make(prob, "bf16x2", train_bf16=mode)
        warm.train(Xd[:2 * bs], Ud[:2 * bs], Yd[:2 * bs], epochs=1, batch=bs, lr=lr)
        warm.close()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        losses = learn.train(Xd, Ud, Yd, epochs=epochs, batch=bs, lr=lr)
        t_train = time.perf_counter() - t0
        runs[mode] = (learn, losses, t_train)
    learn, losses, t_train = runs[True]
    split, losses_s, t_split = runs[False]
    split.close()
    learn.autotune()
    _, _, rmse_l = time_closed_loop(learn, prob, steps, 3)
    nominal = make(dict(prob, layers=None), "fp32")
    _, _, rmse_n = time_closed_loop(nominal, prob, steps, 3)
    learn.close(); nominal.close()
    samples = epochs * (n // bs) * bs
    return {"workload": "cfg5_learned: %d samples, MLP %s, Adam lr 1e-3 batch 4096, %d epochs, "
                        "then %d-step closed loop of 4096 instances on the drag plant" % (
                            n, "-".join(map(str, w)), epochs, steps),
            "train_samples_per_s": samples / t_train,
            "train_tflops": flops / t_train / 1e12,
            "ms_per_train_step": 1e3 * t_train / (epochs * (n // bs)),
            "train_precision": "own tcgen05 GEMMs (forward + bias/tanh, backward + tanh', weight gradient split "
                               "over the batch) with BF16 operands (one MMA per product), FP32 accumulation, FP32 "
                               "master weights; fused Adam",
            "train_roofline": {"bound": "tensor", "peak": bf16_burst, "frac": flops / t_train / 1e12 / bf16_burst,
                               "note": "peak = measured BF16 burst; the timing includes the loss, Adam and gather "
                                       "launches and the final repack of the network"},
            "split_operands": {"train_tflops": flops / t_split / 1e12,
                               "ms_per_train_step": 1e3 * t_split / (epochs * (n // bs)),
                               "frac": flops / t_split / 1e12 / bf16_burst,
                               "note": "BF16 hi + lo operands, 3 MMAs per product (frac <= 1/3), the precision of "
                                       "the gradient tests against the oracle (~1e-5)",
                               "loss_last": float(losses_s[-10:].mean())},
            "loss_first": float(losses[:10].mean()), "loss_last": float(losses[-10:].mean()),
            "tracking_rmse_m": {"learned": rmse_l, "nominal": rmse_n}}


# Table II (Sec. IV): hidden layers x width of the zero-output network, and
# the paper's RTN control frequency on the RTX 3000 laptop GPU (context only)
TABLE2 = [(0, 0, 4262), (2, 16, 781), (2, 128, 770), (5, 16, 586), (5, 128, 598), (12, 32, 363),
          (12, 512, 363), (20, 512, 232), (50, 512, 117)]
SWEEP2 = [(16, None), (128, None), (1024, None), (4096, 500.9), (8192, 169.7)]


def di_layers(n_hidden, width, seed=0):
    """Zero-output residual network of the runtime analysis: (p, v, u) ->
    n_hidden tanh layers of `width` -> 1, last layer zero (Sec. IV)."""
    if n_hidden == 0:
        return None
    layers = W.xavier_mlp([3] + [width] * n_hidden + [1], seed)
    Wl, bl = layers[-1]
    layers[-1] = (np.zeros_like(Wl), np.zeros_like(bl))
    return layers


def bench_runtime_analysis(steps=200):
    """f3: control frequency of one double-integrator controller (N = 10)
    with the zero-output networks of Table II and the 2-layer width sweep:
    device-side (one RTI step captured in a CUDA graph, replayed) and through
    the Python API; plus instance RTI steps/s of large batches."""
    import torch
    import paper_2203_07747_b300 as rtn
    Qd, Rd = np.array([10.0, 1.0]), np.array([0.1])

    def one(n_hidden, width, B=1, graph=True):
        s = torch.cuda.Stream()
        ctl = rtn.DIController(np.full(B, 10), np.full(B, 0.05), Qd, Rd, layers=di_layers(n_hidden, width),
                               stream=s)
        x0 = torch.zeros(B, 2, device="cuda")
        xref = torch.zeros(ctl.n_states, 2, device="cuda")
        xref[:, 0] = 1.0
        uref = torch.zeros(ctl.n_nodes, device="cuda")
        u0 = torch.empty(B, device="cuda")
        st = torch.empty(B, dtype=torch.int32, device="cuda")
        res = {}
        with torch.cuda.stream(s):
            for _ in range(10):
                ctl.rti_step(x0, xref, uref, u0, st)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
            n_api = steps if B == 1 else max(5, steps // 20)
            e0.record(s)
            for _ in range(n_api):
                ctl.rti_step(x0, xref, uref, u0, st)
            e1.record(s)
            torch.cuda.synchronize()
            res["ms_api"] = e0.elapsed_time(e1) / n_api
            if graph:
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=s):
                    ctl.rti_step(x0, xref, uref, u0, st)
                for _ in range(10):
                    g.replay()
                torch.cuda.synchronize()
                e0.record(s)
                for _ in range(steps):
                    g.replay()
                e1.record(s)
                torch.cuda.synchronize()
                res["ms_graph"] = e0.elapsed_time(e1) / steps
        assert int((st != 0).sum()) == 0
        ctl.close()
        return res

    def params(n_hidden, width):
        if n_hidden == 0:
            return 0
        w = [3] + [width] * n_hidden + [1]
        return int(sum(a * b + b for a, b in zip(w[:-1], w[1:])))

    out = {"metric": "control frequency of one controller [Hz]: RTI step of the double integrator "
                     "with a zero-output network, N = 10 (Sec. IV, Table II)",
           "note": "hz = device-side (one RTI step in a CUDA graph, replayed); hz_api = through the "
                   "Python binding; paper_rtx3000_hz = the paper's RTN on an RTX 3000 (context)",
           "table2": [], "width_sweep_2_layers": [], "batch": []}
    for n_hidden, width, paper in TABLE2:
        r = one(n_hidden, width)
        out["table2"].append({"hidden_layers": n_hidden, "width": width, "params": params(n_hidden, width),
                              "hz": 1e3 / r["ms_graph"], "hz_api": 1e3 / r["ms_api"],
                              "paper_rtx3000_hz": paper})
    for width, paper in SWEEP2:
        r = one(2, width)
        out["width_sweep_2_layers"].append({"width": width, "params": params(2, width),
                                            "hz": 1e3 / r["ms_graph"], "hz_api": 1e3 / r["ms_api"],
                                            "paper_rtx3000_hz": paper})
    for n_hidden, width in [(2, 128), (5, 128), (12, 512)]:
        B = 8192
        r = one(n_hidden, width, B=B, graph=False)
        out["batch"].append({"instances": B, "hidden_layers": n_hidden, "width": width,
                             "rti_steps_per_s": B / (r["ms_api"] * 1e-3), "ms_per_step": r["ms_api"]})
    out["quadrotor_one_controller"] = bench_one_quadrotor(steps)
    return out


# Table III (Sec. VI): networks N-L-W (hidden layers x width) and the paper's
# average optimisation time of RTN-MPC on one CPU core [ms] (context only)
TABLE3 = [(3, 32, 2.2), (4, 64, 2.3), (5, 128, 3.2)]


def bench_one_quadrotor(steps=200):
    """One quadrotor controller (N = 10, dt = 0.05 s, the residual networks of
    Table III): one RTI step (network + Jacobian, RK4 + sensitivities, QP,
    feedback) captured in a CUDA graph and replayed, split BF16 (tile shape
    autotuned) and FP32-accurate; control frequency against the paper's
    optimisation time on one CPU core (context)."""
    import torch
    import paper_2203_07747_b300 as rtn
    rows = []
    for n_hidden, width, paper_ms in TABLE3:
        prob = W.make_problem("cfg1_single_fp64", seed=0, bf16=True)
        prob["layers"] = W.xavier_mlp([17] + [width] * n_hidden + [3], 0, bf16=True)
        row = {"hidden_layers": n_hidden, "width": width, "paper_cpu_ms": paper_ms}
        for prec in ("bf16x2", "fp32"):
            s = torch.cuda.Stream()
            ctl = rtn.Controller(prob["N"], prob["dt"], prob["Q"], prob["R"], QN=prob["QN"], quad=prob["quad"],
                                 layers=prob["layers"], precision=prec, stream=s)
            if prec != "fp32":
                ctl.autotune()
            xref, uref = W.node_refs(prob)
            xr = torch.as_tensor(xref, dtype=torch.float32, device="cuda")
            ur = torch.as_tensor(uref, dtype=torch.float32, device="cuda")
            x0 = xr[:1].clone() + 0.02
            u0 = torch.empty((1, 4), device="cuda")
            st = torch.empty(1, dtype=torch.int32, device="cuda")
            with torch.cuda.stream(s):
                for _ in range(10):
                    ctl.rti_step(x0, xr, ur, u0, st)
                torch.cuda.synchronize()
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=s):
                    ctl.rti_step(x0, xr, ur, u0, st)
                for _ in range(10):
                    g.replay()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
                e0.record(s)
                for _ in range(steps):
                    g.replay()
                e1.record(s)
                torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            assert int(st.item()) == 0
            row[prec] = {"ms_per_rti_step": ms, "hz": 1e3 / ms}
            ctl.close()
        rows.append(row)
    return {"what": "one quadrotor controller, N = 10, one RTI step per control step, CUDA graph replayed; "
                    "paper_cpu_ms = the paper's RTN-MPC optimisation time on one CPU core (Table III, context)",
            "rows": rows}


LAY_KERNELS = {"input GEMM": "lay_kernel<4>", "forward GEMM": "lay_kernel<0>", "first backward GEMM": "lay_kernel<3>",
               "backward GEMM": "lay_kernel<1>", "Jacobian GEMM": "lay_kernel<2>", "output layer": "lay_fd_kernel",
               "inputs": "lay_z_kernel"}


def lay_kernel_name(kind, mode):
    """Kernel of one kind of layered launch (tile mode 7: the hidden forward
    and backward GEMMs on CTA pairs)."""
    pairs = {"backward GEMM": "lay2_kernel<1> (CTA pairs)", "forward GEMM": "lay2_kernel<0> (CTA pairs)"}
    return pairs[kind] if mode == 7 and kind in pairs else LAY_KERNELS[kind]


def lay_flops(kind, widths, nn):
    """Algorithmic FLOPs of all launches of one kind in a layered pass."""
    w, L = widths, len(widths) - 1
    if kind == "input GEMM":
        return 2 * 17 * w[1] * nn
    if kind == "forward GEMM":
        return sum(2 * w[l] * w[l + 1] for l in range(1, L - 1)) * nn
    if kind == "first backward GEMM":
        return 2 * 3 * w[L - 2] * w[L - 1] * nn
    if kind == "backward GEMM":
        return sum(2 * 3 * w[l] * w[l + 1] for l in range(1, L - 2)) * nn
    if kind == "Jacobian GEMM":
        return 2 * 3 * 17 * w[1] * nn
    return 0


def lay_bytes(kind, widths, nn):
    """Algorithmic DRAM bytes of all launches of one kind in a layered pass:
    every operand a layer GEMM reads and every result it writes, once, 4 B
    per value (FP32, or a BF16 hi + lo pair); weights (L2-resident) and the
    zero padding of z are not counted."""
    w, L = widths, len(widths) - 1
    if kind == "inputs":
        return (17 * 4 + 17 * 4) * nn
    if kind == "input GEMM":
        return (17 + w[1]) * 4 * nn
    if kind == "forward GEMM":
        # a_l in, a_{l+1} out; the last also writes d_{L-1} (the folded
        # first backward GEMM's operand)
        return (sum((w[l] + w[l + 1]) * 4 for l in range(1, L - 1)) + w[L - 1] * 4) * nn
    if kind == "output layer":
        return (w[L - 1] + 3) * 4 * nn
    if kind == "first backward GEMM":
        # d_{L-1} in, a_{L-2} in (d_{L-2} = 1 - a^2), D_{L-2} out
        return (w[L - 1] + w[L - 2] + 3 * w[L - 2]) * 4 * nn
    if kind == "backward GEMM":
        # D_{l+1} in, a_l in (d_l = 1 - a_l^2), D_l out
        return sum((3 * w[l + 1] + w[l] + 3 * w[l]) * 4 for l in range(1, L - 2)) * nn
    if kind == "Jacobian GEMM":
        return (3 * w[1] + 3 * 17) * 4 * nn
    return 0


# bytes per node the method itself needs for a1 (network input z, 17 floats
# in; f_D and J_D, 3 + 51 floats out; weights L2-resident)
A1_METHOD_BYTES_PER_NODE = (17 + 3 + 51) * 4


def layered_roofline(ctl, x, u, out, widths, nn, pass_roof, hbm, bf16_burst, peak_src, mode=6):
    """Roofline of the dominant kernel of the layered pass, tensor-bound: every
    launch of one pass timed with CUDA events on the context's stream, the
    kind with the largest total time; its reverse-mode algorithmic FLOPs per
    launch (3 adjoint rows x 2 h_l h_(l+1) per node for a backward GEMM) over
    its mean launch time, against the measured BF16 burst peak (the kernel is
    timed alone, one pass).  The split-BF16 operands make every product two
    MMAs, so the algorithmic fraction can reach at most 1/2.  `traffic` is
    its DRAM bytes per launch (ncu); the HBM view beside it compares them with
    the activations and adjoints the layered design moves and with the ~284 B
    per node that the method itself needs."""
    import torch
    ctl.mlp_eval(x, u, out[0], out[1])
    # five recorded passes, each launch's median: the GPU's power management
    # moves the SM clock between passes (sw_power_cap), and the clocks seen
    # are reported beside the times
    runs = []
    with Clocks() as ck:
        torch.cuda.synchronize()
        t0 = time.time()
        for _ in range(5):
            ctl.tc_launch_times(True)
            ctl.mlp_eval(x, u, out[0], out[1])
            runs.append(ctl.tc_launch_times(False))
        torch.cuda.synchronize()
        ck.mark(t0, time.time())
    times = [(runs[0][i][0], float(np.median([r[i][1] for r in runs]))) for i in range(len(runs[0]))]
    tot = {}
    for k, ms in times:
        c, t = tot.get(k, (0, 0.0))
        tot[k] = (c + 1, t + ms)
    dom = max((k for k in tot if lay_flops(k, widths, nn) > 0), key=lambda k: tot[k][1])
    c, t = tot[dom]
    fl = lay_flops(dom, widths, nn) / c
    by = lay_bytes(dom, widths, nn) / c
    ms = t / c
    pass_view = {k: pass_roof[k] for k in ("achieved", "unit", "frac", "ms_per_launch",
                                           "algorithmic_flops_per_launch", "peak", "peak_kind")}
    pass_view["kernel"] = pass_roof["kernel"]
    pass_view["dram_bytes"] = profiled_pass_traffic(mode)
    pass_view["design_bytes"] = sum(lay_bytes(k, widths, nn) for k in tot)
    pass_view["method_bytes"] = A1_METHOD_BYTES_PER_NODE * nn
    tflops = fl / (ms * 1e-3) / 1e12
    traffic = profiled_layer_traffic(dom, mode)
    return {"bound": "tensor", "peak": bf16_burst, "peak_kind": f"bf16 burst ({peak_src})", "unit": "TFLOP/s",
            "achieved": tflops, "frac": tflops / bf16_burst, "traffic": traffic,
            "algorithmic_flops_per_launch": fl, "flop_count": "reverse mode (3 adjoint rows per node)",
            "ms_per_launch": ms, "launches_per_pass": c,
            "kernel": f"{lay_kernel_name(dom, mode)}: {dom} of the layered reverse mode ({c} per pass, "
                      f"{100 * t / sum(v[1] for v in tot.values()):.0f}% of the pass)",
            "split_operands": "BF16 hi + lo activations/adjoints: 2 MMAs per product, frac <= 0.5",
            "tensor_pipe_active_pct": profiled_tensor_pipe(dom, mode),
            "tensor_pipe_note": "sm__pipe_tensor_cycles_active of this kernel (ncu --set full, 2,048 "
                                "instances): the pipe counts both MMAs of every split product, frac only "
                                "the method's reverse-mode FLOPs",
            "hbm_view": {"design_bytes_per_launch": by, "achieved_gbs": by / (ms * 1e-3) / 1e9,
                         "frac_of_hbm": by / (ms * 1e-3) / 1e9 / hbm, "hbm_peak": hbm,
                         "method_bytes_per_launch": A1_METHOD_BYTES_PER_NODE * nn,
                         "traffic_over_method_bytes": (traffic / (A1_METHOD_BYTES_PER_NODE * nn)) if traffic else None,
                         "arithmetic_intensity_flop_per_byte": fl / by,
                         "ridge_flop_per_byte": bf16_burst * 1e12 / (hbm * 1e9)},
            "pass": pass_view,
            "launch_ms": [[k, round(v, 4)] for k, v in times],
            "launch_ms_note": "median of 5 recorded passes per launch",
            "clocks": ck.summary()}


def _profile_current(text, mode):
    """The committed layered summary was captured on the current kernel
    sources and the same tile mode."""
    m = re.search(r"kernel sources md5 at capture: (\w+)\s+\(([^)]*)\)", text)
    files = tuple(f.strip() for f in m.group(2).split("+"))
    t = re.search(r"tile shape: npc=\d+ mode=(\d+)", text)
    return m.group(1) == kernel_md5(files) and t is not None and int(t.group(1)) == mode


def profiled_layer_traffic(kind, mode=6):
    """DRAM bytes per launch of one kind of layered launch from the committed
    summary (measured on a smaller case and scaled by nodes), or None when the
    kernel sources or the tile mode differ from the capture's."""
    try:
        text = open(os.path.join(ROOT, "profiles", LAYERED_PROFILE)).read()
        if not _profile_current(text, mode):
            return None
        key = {"backward GEMM": "bwd", "first backward GEMM": "bw0", "forward GEMM": "fwd"}.get(kind)
        r = re.search(r"dram_bytes_per_launch_%s: (\d+)" % key, text) if key else None
        return int(r.group(1)) if r else None
    except (OSError, AttributeError):
        return None


def profiled_tensor_pipe(kind, mode=6):
    """sm__pipe_tensor_cycles_active (% of peak) of one kind of layered
    launch from the committed summary's full-set capture, or None when the
    kernel sources or the tile mode differ from the capture's."""
    try:
        text = open(os.path.join(ROOT, "profiles", LAYERED_PROFILE)).read()
        if not _profile_current(text, mode):
            return None
        key = {"backward GEMM": "bwd", "first backward GEMM": "bw0", "forward GEMM": "fwd"}.get(kind)
        r = re.search(r"tensor_pipe_active_pct_%s: ([0-9.]+)" % key, text) if key else None
        return float(r.group(1)) if r else None
    except (OSError, AttributeError):
        return None


def profiled_pass_traffic(mode=6):
    """DRAM bytes of a whole layered pass from its committed summary."""
    try:
        text = open(os.path.join(ROOT, "profiles", LAYERED_PROFILE)).read()
        if not _profile_current(text, mode):
            return None
        return int(re.search(r"dram_bytes_per_pass: (\d+)", text).group(1))
    except (OSError, AttributeError):
        return None


def hess_flops_per_node(widths):
    """Second-order (forward-over-forward) algorithmic FLOPs per node: 171
    columns per node (value, 17 tangents, 153 second derivatives) through
    every hidden->hidden and the output layer; the input layer costs its value
    dot products, the tangent scaling and the rank-one second-derivative
    products d2 w_j w_m.  Elementwise activation work is not counted."""
    f = 2 * 17 * widths[1] + 17 * widths[1] + 2 * 153 * widths[1]
    for fi, fo in zip(widths[1:-1], widths[2:]):
        f += 2 * 171 * fi * fo
    return f


def bench_network_pass(config, B, reps=3, precision="bf16x2", tile=-1):
    """The network pass (a1) of the workload's network on B instances with
    the layered reverse-mode shape, or tile shape `tile` if >= 0 (split
    BF16, or FP8 on the e4m3-quantised weights): ms per pass after one
    warm-up pass."""
    import torch
    prob = W.make_problem(config, seed=0, B=B, bf16=True)
    if precision == "fp8":
        prob["layers"] = W.quantize_e4m3(prob["layers"])
    ctl = make(prob, precision)
    vi = tile if tile >= 0 else [v[0] for v in ctl.tc_variants() if v[2] == 6][0]
    ctl.tc_select(vi)
    x, u = ctl.get_iterate()
    fD, JD = ctl.mlp_eval(x, u)
    ms = time_calls(lambda: ctl.mlp_eval(x, u, fD, JD), reps, warm=1)
    out = {"instances": B, "nodes": ctl.n_nodes, "variant": vi, "ms_per_pass": ms, "device_error": ctl.device_error()}
    ctl.close()
    return out


def bench_rti_step(config, B, reps=3):
    """One RTI step (a1 network pass, a2 RK4 + sensitivities, a3 + a4
    Riccati QP and feedback) of the workload on B instances with the layered
    reverse-mode shape: ms per step after one warm-up step (the profiling
    command of the RK4 and QP kernels' summaries)."""
    import torch
    prob = W.make_problem(config, seed=0, B=B, bf16=True)
    ctl = make(prob, "bf16x2")
    vi = [v[0] for v in ctl.tc_variants() if v[2] == 6][0]
    ctl.tc_select(vi)
    xref, uref = W.node_refs(prob)
    xref_d = torch.as_tensor(xref, dtype=torch.float32, device="cuda")
    uref_d = torch.as_tensor(uref, dtype=torch.float32, device="cuda")
    xo = np.concatenate([[0], np.cumsum(prob["N"] + 1)])[:-1]
    x0_d = xref_d[torch.as_tensor(xo, device="cuda")] + 0.02
    u0 = torch.empty((B, 4), dtype=torch.float32, device="cuda")
    st = torch.empty(B, dtype=torch.int32, device="cuda")
    ms = time_calls(lambda: ctl.rti_step(x0_d, xref_d, uref_d, u0, st), reps, warm=1)
    out = {"instances": B, "nodes": ctl.n_nodes, "variant": vi, "ms_per_step": ms, "device_error": ctl.device_error()}
    ctl.close()
    return out


def bench_second_order(config, bf16_burst, B=1024, reps=3):
    """f4: the second-order local model (network Hessian H_D, Eq. 4) and the
    6-output full residual (Eq. 7) on the FP32 path, B instances of the
    workload's horizon and network (the 171 second-order columns per node
    need h x 171 x 4 B per node and layer buffer, so B is below the
    headline's).  Node linearisations/s and RTI steps/s, against the
    first-order model on the same workload."""
    import torch
    import paper_2203_07747_b300 as rtn
    prob = W.make_problem(config, seed=0, B=B)
    widths = prob["widths"]
    nn = int(prob["N"].sum())
    xref, uref = W.node_refs(prob)
    xref_d = torch.as_tensor(xref, dtype=torch.float32, device="cuda")
    uref_d = torch.as_tensor(uref, dtype=torch.float32, device="cuda")
    X, U = W.random_nodes(nn + B, 1)
    x_d = torch.as_tensor(X, dtype=torch.float32, device="cuda")
    u_d = torch.as_tensor(U[:nn], dtype=torch.float32, device="cuda")
    xo = np.concatenate([[0], np.cumsum(prob["N"] + 1)])[:-1]
    x0_d = torch.as_tensor(X[xo], dtype=torch.float32, device="cuda")

    def run(layers, second):
        ctl = rtn.Controller(prob["N"], prob["dt"], prob["Q"], prob["R"], QN=prob["QN"], quad=prob["quad"],
                             layers=layers, precision="fp32", second_order=second)
        out = ctl.linearize(x_d, u_d)
        r = {"ms_linearize": time_calls(lambda: ctl.linearize(x_d, u_d, out), reps, warm=1)}
        if second:
            r["ms_network"] = time_calls(lambda: ctl.mlp_hess(x_d, u_d), reps, warm=1)
        else:
            r["ms_network"] = time_calls(lambda: ctl.mlp_eval(x_d, u_d, out[0], out[1]), reps, warm=1)
        u0 = torch.empty(B, 4, device="cuda")
        st = torch.empty(B, dtype=torch.int32, device="cuda")

        def step():
            ctl.set_iterate(x_d, u_d)
            ctl.rti_step(x0_d, xref_d, uref_d, u0, st)
        r["ms_rti"] = time_calls(step, reps, warm=1)
        r["failed_instances"] = int((st != 0).sum())
        ctl.close()
        return r

    full = W.xavier_mlp(widths[:-1] + [6], 5)
    # first and second order: hidden layers on the tensor cores as kind::tf32
    # GEMMs with hi + lo split operands (three MMAs per product, so at most
    # 1/3 of the TF32 peak in algorithmic FLOPs)
    tf32_peak = bf16_burst * 1.1 / 2.25
    out = {"workload": f"{config} network and horizon, {B} instances ({nn} nodes), FP32-accurate paths",
           "peak_kind": "TF32 dense = measured bf16 burst x 1.1/2.25 (nominal ratio); the hi+lo split issues "
                        "3 MMAs per algorithmic product",
           "runs": []}
    for name, layers, second in (("first order, 3 outputs", prob["layers"], False),
                                 ("second order, 3 outputs", prob["layers"], True),
                                 ("first order, full residual (6 outputs)", full, False),
                                 ("second order, full residual (6 outputs)", full, True)):
        r = run(layers, second)
        w = [wl.shape[1] for wl, _ in layers] + [layers[-1][0].shape[0]]
        fl = (hess_flops_per_node(w) if second else fwd_flops_per_node(w)) * nn
        tf = fl / (r["ms_network"] * 1e-3) / 1e12
        out["runs"].append({"model": name, "widths": "-".join(map(str, w)),
                            "node_linearizations_per_s": nn / (r["ms_linearize"] * 1e-3),
                            "rti_steps_per_s": B / (r["ms_rti"] * 1e-3),
                            "network_ms": r["ms_network"], "network_tflops": tf,
                            "roofline": {"bound": "tensor", "peak": tf32_peak, "frac": tf / tf32_peak},
                            "failed_instances": r["failed_instances"]})
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="cfg3_bf16_precision")
    ap.add_argument("--precision", default="auto")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the ragged and learned workloads")
    ap.add_argument("--second-order-only", type=int, default=0, metavar="B",
                    help="run only the second-order / full-residual measurement with B instances")
    ap.add_argument("--tile", type=int, default=-1, metavar="V",
                    help="use tile shape V instead of autotuning (to profile the shape a plain run chose: "
                         "ncu's per-launch overhead changes the autotuner's ranking)")
    ap.add_argument("--network-pass", type=int, default=0, metavar="B",
                    help="time only the network pass (a1) of the workload's network on B instances with "
                         "the layered reverse-mode tile shape, or --tile V (the profiling command of its summary)")
    ap.add_argument("--rti-step", type=int, default=0, metavar="B",
                    help="time only one RTI step of the workload on B instances with the layered reverse-mode "
                         "tile shape (the profiling command of the RK4 and QP kernels' summaries)")
    ap.add_argument("--learned-only", action="store_true",
                    help="run only the training measurement (one epoch) and a short learned closed loop "
                         "(the profiling command of the training kernels' summary)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))

    hbm, bf16_burst, bf16_sus, peak_src = peaks()
    if args.second_order_only:
        print(json.dumps(bench_second_order(args.config, bf16_burst, B=args.second_order_only)))
        return
    if args.network_pass:
        print(json.dumps(bench_network_pass(args.config, args.network_pass,
                                            precision="fp8" if args.precision == "fp8" else "bf16x2",
                                            tile=args.tile)))
        return
    if args.learned_only:
        import torch  # noqa: F401
        print(json.dumps(bench_learned(bf16_burst, epochs=1, steps=10)))
        return
    if args.rti_step:
        print(json.dumps(bench_rti_step(args.config, args.rti_step)))
        return
    # weak scaling: every rank steps its own instances (seeded by rank)
    prob = W.make_problem(args.config, seed=rank, bf16=True)
    widths = prob["widths"]
    B, nn = prob["B"], int(prob["N"].sum())
    cfg = {"workload": f"{args.config}: {B} instances, N={int(prob['N'].max())}, "
                       f"MLP {'-'.join(map(str, widths))} tanh (BF16-representable weights), "
                       "figure-8 references, step = RTI step + drag plant step",
           "instances": B, "nodes": nn,
           "l2": "inputs larger than L2 (A, B, c of all nodes exceed 126 MB)"}

    if args.impl == "reference":
        if rank != 0:
            return
        cb = cpu_baseline(prob)
        line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "RTI steps/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic (seeded workload generator)", "config": cfg, "cpu_baseline": cb,
                "e2e": {"value": cb["value"], "unit": "RTI steps/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    import paper_2203_07747_b300 as rtn
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    rtn.load(build_if_missing=True)

    precs = ["bf16x2", "fp32"] if args.precision == "auto" else [args.precision]
    ctl, prec = None, None
    for p in precs:
        try:
            ctl, prec = make(prob, p), p
            break
        except rtn.RtnError as e:
            if "UNSUPPORTED" not in str(e):
                raise
    cfg["precision"] = prec
    if prec != "fp32":
        # pick the tensor-core tile shape for this network and batch
        if args.tile >= 0:
            ctl.tc_select(args.tile)
            vi, vms = args.tile, None
        else:
            vi, vms = ctl.autotune()
        shape = dict((v[0], v[1:]) for v in ctl.tc_variants())[vi]
        cfg["tile"] = {"variant": vi, "nodes_per_cta": shape[0], "operand_mode": shape[1],
                       "stages": shape[2], "autotune_ms": vms}
    ms_step, clocks, rmse = time_closed_loop(ctl, prob, args.steps, args.warmup)
    ms_step = max_over_ranks(ms_step, "cuda")
    value = weak_value(B, world, ms_step)

    # node linearisations (a1 + a2) and the network kernel alone (a1)
    x, u = ctl.get_iterate()
    out = ctl.linearize(x, u)
    ms_lin = time_calls(lambda: ctl.linearize(x, u, out), max(5, args.steps))
    ms_mlp = time_calls(lambda: ctl.mlp_eval(x, u, out[0], out[1]), max(5, args.steps))
    mode = cfg.get("tile", {}).get("operand_mode")
    rev = mode in (4, 5, 6, 7)  # reverse mode (one CTA / CTA pairs / layered)
    flops = (rev_flops_per_node(widths) if rev else fwd_flops_per_node(widths)) * nn
    if prec == "fp32":
        # FP32-accurate path: TF32 tensor cores with hi + lo split operands
        # (3 MMAs per product: at most 1/3 of the peak in algorithmic FLOPs)
        roof = {"bound": "tensor", "peak": bf16_burst * 1.1 / 2.25,
                "peak_kind": f"TF32 dense = bf16 burst ({peak_src}) x 1.1/2.25 (nominal ratio); hi+lo split"}
    else:
        roof = {"bound": "tensor", "peak": bf16_burst, "peak_kind": f"bf16 burst ({peak_src})"}
    roof.update({"achieved": flops / (ms_mlp * 1e-3) / 1e12, "unit": "TFLOP/s",
                 "algorithmic_flops_per_launch": flops, "ms_per_launch": ms_mlp,
                 "kernel": ("network pass of the layered reverse mode (a1): inputs split, one tensor-core GEMM per "
                            "layer forward (input layer included), output layer, one GEMM per backward layer "
                            "(the first with the last-layer adjoints folded in), the W_0' Jacobian GEMM "
                            "(12 launches at 5 hidden layers)" + ("; the hidden forward and backward GEMMs on "
                                                                   "CTA pairs" if mode == 7 else "")
                            if mode in (6, 7) else
                            "network value + reverse-mode Jacobian (a1, three adjoint rows)" if rev
                            else "network value + forward-mode Jacobian (a1)"),
                 "forward_mode_equivalent_tflops": fwd_flops_per_node(widths) * nn / (ms_mlp * 1e-3) / 1e12,
                 "traffic": None})
    roof["frac"] = roof["achieved"] / roof["peak"]
    if mode in (6, 7):
        roof = layered_roofline(ctl, x, u, out, widths, nn, roof, hbm, bf16_burst, peak_src, mode)

    ms_e2e, bi, bo = e2e_rti(ctl, prob, max(5, args.steps))
    smp = error_sample(prob, prec) if rank == 0 and world == 1 and not args.no_cpu else None
    line = {"metric": METRIC, "value": value, "unit": "RTI steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "fp32", "bf16": "bf16", "bf16x2": "bf16 (hi+lo split operands), fp32 accum"}[prec],
            "data": "synthetic (seeded workload generator)", "config": cfg,
            "node_linearizations_per_s": nn / (ms_lin * 1e-3),
            "jac_rel_err_max": None, "tracking_rmse_m": rmse,
            "tracking_rmse_per_instance_m": rmse_distribution(time_closed_loop.per_instance),
            "roofline": roof, "error_table": None,
            "e2e": {"value": B / (ms_e2e * 1e-3), "unit": "RTI steps/s", "h2d_bytes_per_step": bi,
                    "d2h_bytes_per_step": bo, "path": "rtn_rti_step_host with pinned host buffers (inputs copied on a second stream during the "
                            "linearisation)"},
            "gpu_launches": launches_per_step(ctl, mode) * args.steps, "clocks": clocks}
    ctl.close()
    if prec != "fp32" and not args.no_fp32:
        c32 = make(prob, "fp32")

        ms32, _, _ = time_closed_loop(c32, prob, max(3, args.steps // 4), 2)
        x32, u32 = c32.get_iterate()
        o32 = c32.linearize(x32, u32)
        ml32 = time_calls(lambda: c32.linearize(x32, u32, o32), 5)
        line["fp32_same_workload"] = {"value": B / (ms32 * 1e-3), "unit": "RTI steps/s",
                                      "node_linearizations_per_s": nn / (ml32 * 1e-3)}
        c32.close()
    if rank == 0 and world == 1 and not args.no_extra:
        line["box_qp"] = bench_box(prob, prec, cfg.get("tile"))
        line["riccati_arithmetic"] = bench_riccati(prob, prec, cfg.get("tile"))
        if args.config == "cfg3_bf16_precision":
            line["fp8"], fp8_smp = bench_fp8(prob, bf16_burst)
        line["ragged_batch"], ragged_smp = bench_ragged()
        line["learned_part"] = bench_learned(bf16_burst)
        line["runtime_analysis"] = bench_runtime_analysis()
        line["second_order_and_full_residual"] = bench_second_order(args.config, bf16_burst)
    if rank == 0 and world == 1 and not args.no_cpu:
        # the CPU-baseline leg: the oracle timed on the host cores, and the
        # error tables of the GPU results against it
        line["cpu_baseline"] = cpu_baseline(prob)
        line["error_table"] = error_table(smp)
        line["jac_rel_err_max"] = line["error_table"]["J_D"]["max"]
        if "fp8" in line:
            line["fp8"]["error_table"] = error_table(fp8_smp)
            line["fp8"]["jac_rel_err_max"] = line["fp8"]["error_table"]["J_D"]["max"]
        if "ragged_batch" in line:
            line["ragged_batch"]["error_table"] = error_table(ragged_smp)
            line["ragged_batch"]["jac_rel_err_max"] = line["ragged_batch"]["error_table"]["J_D"]["max"]
    if rank == 0:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
