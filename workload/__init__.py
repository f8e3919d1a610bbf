"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

This module only draws random numbers and lays them out; it holds none of the
method's arithmetic (no dynamics, no network evaluation, no solver).  Both the
product binding and the oracle consume its arrays as plain data, so neither
side depends on the other.

Input recipe (the paper's own workloads -- Circle/Lemniscate tracks on its
simulators and the NeuroBEM data set, Sec. VI -- are not available; these
seeded arrays stand in for them):

* quadrotor: mass 0.75 kg, inertia diag(2.5e-3, 2.1e-3, 4.3e-3) kg m^2,
  arm 0.14 m, thrust per motor in [0, 8.5] N, yaw-torque coefficient 0.05.
* residual network: input 17 = [x; u], tanh hidden layers, linear 3-output
  layer; Xavier-uniform weights U(+-sqrt(6/(fan_in+fan_out))), zero biases.
* initial states: p ~ U[-1,1]^3, v ~ N(0,1)^3, yaw-only attitude with yaw
  ~ U[-pi,pi], omega = 0.
* references: figure-8 Lissajous p(t) = c + [A sin(wt+phi), A/2 sin(2(wt+phi)), 0]
  with A ~ U[1,4] m and period ~ U[3,8] s; circle of radius 2 m at 3 m/s.
  Reference attitude is identity, reference rates zero, reference thrust
  is hover (m g / 4 per motor).
* ragged horizons N_b ~ U{10..50}, dt_b ~ U[0.02, 0.1] s.
* training samples: yaw ~ U[-pi,pi], roll/pitch ~ U[-pi/4, pi/4],
  v ~ U[-12,12]^3, omega ~ U[-3,3]^3, T ~ U[0,8.5]^4, p ~ U[-1,1]^3.
"""
import numpy as np

NX, NU, NIN, NOUT = 13, 4, 17, 3

QUAD = dict(mass=0.75, Jx=2.5e-3, Jy=2.1e-3, Jz=4.3e-3, arm=0.14,
            c_tau=0.05, u_max=8.5, g=9.81)

# Tracking weights: Q = diag(10 I3, 1 I4, 1 I3, 0.1 I3), R = 0.1 I4.
Q_DIAG = np.array([10.0] * 3 + [1.0] * 4 + [1.0] * 3 + [0.1] * 3)
R_DIAG = np.array([0.1] * 4)


def rng(seed, stream=0):
    """Counter-based generator (Philox) keyed by (seed, stream)."""
    return np.random.Generator(np.random.Philox(key=[seed, stream]))


def round_bf16(a):
    """Round float64 values to the nearest bfloat16-representable value
    (round-to-nearest-even through float32).  Used to make network weights
    exactly representable in the tensor-core input format, so that the oracle
    and the GPU evaluate the same network."""
    f = np.asarray(a, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    r = (((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def round_e4m3(x):
    """Round to the nearest e4m3 value (OCP FP8: 3 mantissa bits, exponent
    bias 7, subnormal spacing 2^-9, largest 448), ties to even, saturating."""
    x = np.asarray(x, dtype=np.float64)
    a = np.minimum(np.abs(x), 448.0)
    e = np.floor(np.log2(np.maximum(a, 2.0 ** -6)))
    step = 2.0 ** (e - 3)
    r = np.round(a / step) * step  # numpy rounds halves to even
    return np.sign(x) * np.minimum(r, 448.0)


def quantize_e4m3(layers):
    """Every weight matrix as float32(s * e4m3(W / s)) with the per-layer scale
    s = amax / 448 (in float32), biases unchanged: the weights of the FP8
    workloads, which the library derives the same way and the oracle then
    evaluates as given."""
    out = []
    for W, b in layers:
        W32 = np.asarray(W, np.float32)
        s = np.float32(np.abs(W32).max()) / np.float32(448.0)
        q = round_e4m3(W32.astype(np.float64) / np.float64(np.float32(s))).astype(np.float32)
        out.append(((q * s).astype(np.float32).astype(np.float64), np.asarray(b, np.float64)))
    return out


def xavier_mlp(widths, seed, bf16=False):
    """List of (W[out][in], b[out]) float64 arrays, Xavier-uniform, b = 0."""
    g = rng(seed, 1)
    layers = []
    for fi, fo in zip(widths[:-1], widths[1:]):
        lim = np.sqrt(6.0 / (fi + fo))
        W = g.uniform(-lim, lim, size=(fo, fi))
        if bf16:
            W = round_bf16(W)
        layers.append((W, np.zeros(fo)))
    return layers


def yaw_quat(yaw):
    return np.stack([np.cos(yaw / 2), np.zeros_like(yaw), np.zeros_like(yaw),
                     np.sin(yaw / 2)], -1)


def euler_zyx_quat(yaw, pitch, roll):
    cy, sy = np.cos(yaw / 2), np.sin(yaw / 2)
    cp, sp = np.cos(pitch / 2), np.sin(pitch / 2)
    cr, sr = np.cos(roll / 2), np.sin(roll / 2)
    return np.stack([cr * cp * cy + sr * sp * sy,
                     sr * cp * cy - cr * sp * sy,
                     cr * sp * cy + sr * cp * sy,
                     cr * cp * sy - sr * sp * cy], -1)


def initial_states(B, seed):
    g = rng(seed, 2)
    p = g.uniform(-1, 1, (B, 3))
    q = yaw_quat(g.uniform(-np.pi, np.pi, B))
    v = g.normal(0, 1, (B, 3))
    w = np.zeros((B, 3))
    return np.concatenate([p, q, v, w], 1)


def horizons(B, seed, ragged=False, N=20, dt=0.05):
    if not ragged:
        return np.full(B, N, np.int32), np.full(B, dt)
    g = rng(seed, 3)
    return (g.integers(10, 51, B).astype(np.int32), g.uniform(0.02, 0.1, B))


def figure8_params(B, seed):
    """Per instance: centre (3), amplitude, angular rate, phase."""
    g = rng(seed, 4)
    c = np.concatenate([g.uniform(-1, 1, (B, 2)), np.zeros((B, 1))], 1)
    A = g.uniform(1, 4, B)
    w = 2 * np.pi / g.uniform(3, 8, B)
    ph = g.uniform(0, 2 * np.pi, B)
    return dict(kind="figure8", c=c, A=A, w=w, phase=ph)


def circle_params(B, seed, radius=2.0, speed=3.0):
    g = rng(seed, 5)
    c = np.concatenate([g.uniform(-1, 1, (B, 2)), np.zeros((B, 1))], 1)
    return dict(kind="circle", c=c, A=np.full(B, radius),
                w=np.full(B, speed / radius), phase=g.uniform(0, 2 * np.pi, B))


def reference_states(params, t):
    """Reference states x_r(t) for every instance: t has shape [B, T].
    Returns [B, T, 13] (p, q = identity, v = dp/dt, omega = 0)."""
    c, A, w, ph = params["c"], params["A"][:, None], params["w"][:, None], params["phase"][:, None]
    s = w * t + ph
    if params["kind"] == "figure8":
        px, py = A * np.sin(s), 0.5 * A * np.sin(2 * s)
        vx, vy = A * w * np.cos(s), A * w * np.cos(2 * s)
    else:
        px, py = A * np.cos(s), A * np.sin(s)
        vx, vy = -A * w * np.sin(s), A * w * np.cos(s)
    Bn, T = t.shape
    x = np.zeros((Bn, T, NX))
    x[:, :, 0] = c[:, None, 0] + px
    x[:, :, 1] = c[:, None, 1] + py
    x[:, :, 2] = c[:, None, 2]
    x[:, :, 3] = 1.0
    x[:, :, 7], x[:, :, 8] = vx, vy
    return x


def hover_thrust():
    return QUAD["mass"] * QUAD["g"] / 4.0


def training_samples(n, seed):
    """Seeded (x, u) samples for fitting the residual network."""
    g = rng(seed, 6)
    p = g.uniform(-1, 1, (n, 3))
    q = euler_zyx_quat(g.uniform(-np.pi, np.pi, n), g.uniform(-np.pi / 4, np.pi / 4, n),
                       g.uniform(-np.pi / 4, np.pi / 4, n))
    v = g.uniform(-12, 12, (n, 3))
    w = g.uniform(-3, 3, (n, 3))
    u = g.uniform(0, 8.5, (n, 4))
    return np.concatenate([p, q, v, w], 1), u


def random_nodes(n, seed):
    """Generic linearisation points: states near hover with unit-ish
    quaternions and thrusts inside the box (used by parity tests)."""
    g = rng(seed, 7)
    p = g.uniform(-1, 1, (n, 3))
    q = euler_zyx_quat(g.uniform(-np.pi, np.pi, n), g.uniform(-0.5, 0.5, n), g.uniform(-0.5, 0.5, n))
    q *= g.uniform(0.98, 1.02, (n, 1))
    v = g.normal(0, 1.5, (n, 3))
    w = g.normal(0, 0.8, (n, 3))
    u = g.uniform(0.5, 8.0, (n, 4))
    return np.concatenate([p, q, v, w], 1), u


CONFIGS = {
    # name: (B, widths, ragged, N, dt, precision)
    "cfg1_single_fp64": dict(B=1, widths=[17, 32, 32, 3], N=10, dt=0.05, ragged=False,
                             ref="circle", steps=100),
    "cfg2_fp32_batch": dict(B=1024, widths=[17] + [256] * 5 + [3], N=20, dt=0.05,
                            ragged=False, ref="figure8"),
    "cfg3_bf16_precision": dict(B=8192, widths=[17] + [512] * 5 + [3], N=20, dt=0.05,
                                ragged=False, ref="figure8"),
    "cfg4_ragged_batch": dict(B=4096, widths=[17] + [256] * 4 + [3], ragged=True,
                              ref="figure8", steps=200),
    "cfg5_learned": dict(B=4096, widths=[17] + [512] * 6 + [3], N=20, dt=0.05,
                         ragged=False, ref="figure8", n_samples=1 << 20, batch=4096, lr=1e-3),
}


def make_problem(name, seed=0, B=None, bf16=False):
    """Everything one controller batch needs, as plain arrays."""
    cfg = dict(CONFIGS[name])
    if B is not None:
        cfg["B"] = B
    Bn = cfg["B"]
    N, dt = horizons(Bn, seed, cfg["ragged"], cfg.get("N", 20), cfg.get("dt", 0.05))
    layers = xavier_mlp(cfg["widths"], seed, bf16=bf16)
    x0 = initial_states(Bn, seed)
    refp = circle_params(Bn, seed) if cfg["ref"] == "circle" else figure8_params(Bn, seed)
    return dict(name=name, B=Bn, N=N, dt=dt, layers=layers, widths=cfg["widths"], x0=x0,
                ref=refp, Q=Q_DIAG.copy(), R=R_DIAG.copy(), QN=Q_DIAG.copy(), quad=dict(QUAD),
                cfg=cfg, seed=seed, bf16=bf16)


def node_refs(prob, t0=0.0):
    """Packed reference arrays for one RTI step starting at time t0:
    xref [sum(N_b+1)][13], uref [sum(N_b)][4]."""
    N, dt = prob["N"], prob["dt"]
    Tm = int(N.max()) + 1
    t = t0 + dt[:, None] * np.arange(Tm)[None, :]
    xr = reference_states(prob["ref"], t)
    xref = np.concatenate([xr[b, :N[b] + 1] for b in range(len(N))], 0)
    uref = np.full((int(N.sum()), NU), hover_thrust())
    return xref, uref


def trajectory_refs(prob, steps):
    """Reference samples for a closed loop of `steps` control steps:
    xref [B][steps + Nmax + 1][13] on each instance's own dt grid,
    uref [B][steps + Nmax][4]."""
    N, dt = prob["N"], prob["dt"]
    T = steps + int(N.max()) + 1
    t = dt[:, None] * np.arange(T)[None, :]
    xr = reference_states(prob["ref"], t)
    ur = np.full((len(N), T - 1, NU), hover_thrust())
    return xr, ur


def subset(prob, nb):
    """The first nb instances of a problem (same seeds, same arrays)."""
    out = dict(prob)
    out["B"] = nb
    out["N"], out["dt"], out["x0"] = prob["N"][:nb], prob["dt"][:nb], prob["x0"][:nb]
    out["ref"] = {k: (v if isinstance(v, str) else v[:nb]) for k, v in prob["ref"].items()}
    return out
