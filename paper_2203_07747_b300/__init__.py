"""Python binding of librtn (include/rtn.h): argument marshalling only.

Every step of the hot path runs in the CUDA kernels of ``librtn.so``; this
module checks shapes and dtypes of torch CUDA tensors, passes their device
pointers and the current stream through ctypes, and turns status codes into
exceptions.  There is no CPU fallback: without the built library every call
raises.
"""
import ctypes as C
import os

import numpy as np

from . import _build

NX, NU, NZ, NO = 13, 4, 17, 3
PRECISION = {"fp32": 0, "bf16": 1, "bf16x2": 2, "fp8": 3}
PLANT = {"nominal": 0, "drag": 1, "mlp": 2}
STATUS = {0: "RTN_OK", 1: "RTN_E_INVAL", 2: "RTN_E_CUDA", 3: "RTN_E_NONFINITE",
          4: "RTN_E_NOT_PD", 5: "RTN_E_TIMEOUT", 6: "RTN_E_NOMEM", 7: "RTN_E_UNSUPPORTED",
          8: "RTN_E_NOT_CONVERGED"}

# every symbol include/rtn.h declares
EXPORTS = ["rtn_create", "rtn_destroy", "rtn_last_error", "rtn_sizes", "rtn_reset",
           "rtn_set_iterate", "rtn_get_iterate", "rtn_mlp_eval", "rtn_linearize",
           "rtn_qp_solve", "rtn_rti_step", "rtn_rti_step_host", "rtn_plant_step", "rtn_closed_loop",
           "rtn_mlp_eval_f32_noalloc", "rtn_device_error", "rtn_tc_variants",
           "rtn_tc_variant_info", "rtn_tc_select", "rtn_autotune", "rtn_tc_trace",
           "rtn_tc_trace_read", "rtn_drag_targets", "rtn_mse_grad", "rtn_train",
           "rtn_get_params", "rtn_box_iterations", "rtn_mlp_hess", "rtn_tc_launch_times",
           "rtn_set_wait_budget", "rtn_inject_wait_stall"]

_lib = None


class RtnError(RuntimeError):
    pass


class _Quad(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("mass", "Jx", "Jy", "Jz", "arm", "c_tau", "u_max", "g")]


class _MLP(C.Structure):
    _fields_ = [("n_layers", C.c_int), ("widths", C.POINTER(C.c_int)),
                ("W", C.POINTER(C.POINTER(C.c_float))), ("b", C.POINTER(C.POINTER(C.c_float)))]


class _Opt(C.Structure):
    _fields_ = [("precision", C.c_int), ("riccati_f64", C.c_int), ("shift", C.c_int),
                ("box_qp", C.c_int), ("box_max_iter", C.c_int), ("second_order", C.c_int),
                ("fused_qp", C.c_int), ("train_bf16", C.c_int), ("qp_group", C.c_int)]


def lib_path():
    return _build.LIB


def load(build_if_missing=False):
    """Load librtn.so from the package directory (built in-tree)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if build_if_missing:
            _build.build()
        else:
            raise RtnError("librtn.so is not built (run __graft_entry__.build() or "
                           "python -m paper_2203_07747_b300._build)")
    L = C.CDLL(_build.LIB)
    vp = C.c_void_p
    L.rtn_create.argtypes = [C.POINTER(vp), C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int),
                             C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double),
                             C.POINTER(C.c_double), C.POINTER(_Quad), C.POINTER(_MLP),
                             C.POINTER(_Opt), vp]
    L.rtn_destroy.argtypes = [vp]
    L.rtn_destroy.restype = None
    L.rtn_last_error.argtypes = [vp]
    L.rtn_last_error.restype = C.c_char_p
    L.rtn_sizes.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.rtn_reset.argtypes = [vp, vp]
    L.rtn_set_iterate.argtypes = [vp, vp, vp]
    L.rtn_get_iterate.argtypes = [vp, vp, vp]
    L.rtn_mlp_eval.argtypes = [vp] * 5
    L.rtn_mlp_hess.argtypes = [vp] * 6
    L.rtn_tc_launch_times.argtypes = [vp, C.c_int, C.POINTER(C.c_float), C.POINTER(C.c_int), C.c_int,
                                      C.POINTER(C.c_int)]
    L.rtn_linearize.argtypes = [vp] * 8
    L.rtn_qp_solve.argtypes = [vp] * 12
    L.rtn_rti_step.argtypes = [vp] * 6
    L.rtn_rti_step_host.argtypes = [vp] * 6
    L.rtn_plant_step.argtypes = [vp, C.c_int, vp, vp, vp, C.c_int]
    L.rtn_closed_loop.argtypes = [vp, C.c_int, C.c_int, vp, vp, C.c_int, vp, vp, vp]
    L.rtn_device_error.argtypes = [vp, C.POINTER(C.c_int)]
    L.rtn_set_wait_budget.argtypes = [vp, C.c_longlong]
    L.rtn_inject_wait_stall.argtypes = [vp, C.c_int]
    ip = C.POINTER(C.c_int)
    L.rtn_tc_variants.argtypes = [vp, ip]
    L.rtn_tc_variant_info.argtypes = [vp, C.c_int, ip, ip, ip, ip]
    L.rtn_tc_select.argtypes = [vp, C.c_int]
    L.rtn_autotune.argtypes = [vp, ip, C.POINTER(C.c_float)]
    L.rtn_tc_trace.argtypes = [vp, C.c_int]
    L.rtn_drag_targets.argtypes = [vp, vp, C.c_int, vp]
    L.rtn_mse_grad.argtypes = [vp, vp, vp, vp, C.c_int, vp, vp]
    L.rtn_train.argtypes = [vp, vp, vp, vp, C.c_int, C.c_int, C.c_int, C.c_float, C.POINTER(C.c_float)]
    L.rtn_get_params.argtypes = [vp, C.POINTER(C.c_float), C.POINTER(C.c_float)]
    L.rtn_tc_trace_read.argtypes = [vp, C.POINTER(C.c_ulonglong), C.c_int]
    L.rtn_box_iterations.argtypes = [vp, ip]
    L.rtn_mlp_eval_f32_noalloc.argtypes = [C.c_int, C.POINTER(C.c_int)] + [vp] * 2 + [C.c_int] + \
        [vp] * 5 + [C.c_char_p, C.c_size_t]
    for name in EXPORTS:
        if name not in ("rtn_destroy", "rtn_last_error"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _ptr(t, dtype, shape, name):
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise RtnError(f"{name}: expected a CUDA tensor")
    if t.dtype != dtype:
        raise RtnError(f"{name}: expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise RtnError(f"{name}: must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise RtnError(f"{name}: expected shape {tuple(shape)}, got {tuple(t.shape)}")
    return C.c_void_p(t.data_ptr())


def _hptr(t, dtype, shape, name):
    """A contiguous host tensor's address (page-locked lets the copies overlap)."""
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise RtnError(f"{name}: expected a host tensor")
    if t.dtype != dtype:
        raise RtnError(f"{name}: expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise RtnError(f"{name}: must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise RtnError(f"{name}: expected shape {tuple(shape)}, got {tuple(t.shape)}")
    return C.c_void_p(t.data_ptr())


def _stream_handle(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class Controller:
    """A batch of B controller instances (one RTI-SQP problem each)."""

    def __init__(self, N, dt, Q, R, QN=None, quad=None, layers=None, precision="fp32",
                 riccati_f64=False, shift=True, stream=None, box_qp=False, box_max_iter=20,
                 second_order=False, fused_qp=False, train_bf16=False, qp_group=0):
        import torch
        L = load()
        self.N = np.ascontiguousarray(N, dtype=np.int32)
        self.dt = np.ascontiguousarray(dt, dtype=np.float64)
        self.B = int(self.N.size)
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        R = np.ascontiguousarray(R, dtype=np.float64)
        QN = None if QN is None else np.ascontiguousarray(QN, dtype=np.float64)
        if quad is None:
            import workload
            quad = workload.QUAD
        self.quad = dict(quad)
        q = _Quad(*[float(quad[k]) for k in ("mass", "Jx", "Jy", "Jz", "arm", "c_tau", "u_max", "g")])
        self._keep = []
        mlp_p = None
        self.layers = layers
        if layers:
            widths = [layers[0][0].shape[1]] + [W.shape[0] for W, _ in layers]
            w = (C.c_int * len(widths))(*widths)
            Ws = [np.ascontiguousarray(W, dtype=np.float32) for W, _ in layers]
            bs = [np.ascontiguousarray(b, dtype=np.float32) for _, b in layers]
            self._keep += [w, Ws, bs]
            Wp = (C.POINTER(C.c_float) * len(Ws))(*[a.ctypes.data_as(C.POINTER(C.c_float)) for a in Ws])
            bp = (C.POINTER(C.c_float) * len(bs))(*[a.ctypes.data_as(C.POINTER(C.c_float)) for a in bs])
            self._keep += [Wp, bp]
            mlp = _MLP(len(layers), w, Wp, bp)
            mlp_p = C.byref(mlp)
        # riccati_f64: False/0 FP32 sweep, True/1 FP64 sweep, "chol64"/2 FP32 sweep
        # with the factorisation of R + B'PB in FP64
        ric = 2 if riccati_f64 == "chol64" else int(riccati_f64)
        opt = _Opt(PRECISION[precision], ric, int(bool(shift)), int(bool(box_qp)),
                   int(box_max_iter), int(bool(second_order)), int(bool(fused_qp)), int(bool(train_bf16)),
                   int(qp_group))
        self.box_qp = bool(box_qp)
        self.second_order = bool(second_order)
        # network outputs: 3 (linear acceleration) or 6 (the full residual of
        # Eq. 7: linear, then angular acceleration)
        self.n_out = int(layers[-1][0].shape[0]) if layers else NO
        self.precision = precision
        self.stream = stream
        h = C.c_void_p()
        dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
        st = L.rtn_create(C.byref(h), NX, NU, self.B, self.N.ctypes.data_as(C.POINTER(C.c_int)),
                          dp(self.dt), dp(Q), dp(R), None if QN is None else dp(QN), C.byref(q),
                          mlp_p, C.byref(opt), _stream_handle(stream))
        if st != 0:
            raise RtnError(f"rtn_create: {STATUS.get(st, st)}: {L.rtn_last_error(None).decode()}")
        self._h = h
        nn, ns = C.c_int(), C.c_int()
        L.rtn_sizes(h, C.byref(nn), C.byref(ns))
        self.n_nodes, self.n_states = nn.value, ns.value
        self.device = torch.device("cuda", torch.cuda.current_device())

    def close(self):
        if getattr(self, "_h", None):
            load().rtn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, name):
        if st != 0:
            msg = load().rtn_last_error(self._h).decode()
            raise RtnError(f"{name}: {STATUS.get(st, st)}: {msg}")

    def _empty(self, *shape, dtype=None):
        import torch
        return torch.empty(shape, dtype=dtype or torch.float32, device=self.device)

    def box_iterations(self):
        """Subproblems each instance's last box-constrained QP needed (host array)."""
        out = np.zeros(self.B, np.int32)
        self._check(load().rtn_box_iterations(self._h, out.ctypes.data_as(C.POINTER(C.c_int))),
                    "rtn_box_iterations")
        return out

    def set_wait_budget(self, cycles):
        """Budget [SM cycles] of the layered tensor-core kernels' bounded waits
        (0: the default); a fault-injection aid (rtn_set_wait_budget)."""
        self._check(load().rtn_set_wait_budget(self._h, int(cycles)), "rtn_set_wait_budget")

    def inject_wait_stall(self, enable=True):
        """Fault injection: the layered network kernels first wait on a barrier
        that nothing completes (rtn_inject_wait_stall)."""
        self._check(load().rtn_inject_wait_stall(self._h, int(bool(enable))), "rtn_inject_wait_stall")

    def device_error(self):
        """Synchronise and return (and clear) the device-side status code."""
        code = C.c_int(0)
        self._check(load().rtn_device_error(self._h, C.byref(code)), "rtn_device_error")
        return code.value

    def tc_variants(self):
        """[(index, nodes per CTA (per CTA pair in mode 5), operand mode 0|1|2|4|5|6|7, stages)]
        of the tile shapes that fit."""
        L = load()
        n = C.c_int()
        self._check(L.rtn_tc_variants(self._h, C.byref(n)), "rtn_tc_variants")
        out = []
        for i in range(n.value):
            npc, sp, stg, fits = C.c_int(), C.c_int(), C.c_int(), C.c_int()
            self._check(L.rtn_tc_variant_info(self._h, i, C.byref(npc), C.byref(sp), C.byref(stg),
                                              C.byref(fits)), "rtn_tc_variant_info")
            if fits.value:
                out.append((i, npc.value, sp.value, stg.value))
        return out

    def tc_select(self, idx):
        self._check(load().rtn_tc_select(self._h, int(idx)), "rtn_tc_select")

    def autotune(self):
        """Time every fitting tile shape, keep the fastest: (index, ms)."""
        i, ms = C.c_int(), C.c_float()
        self._check(load().rtn_autotune(self._h, C.byref(i), C.byref(ms)), "rtn_autotune")
        return i.value, ms.value

    def tc_trace(self, enable=True):
        self._check(load().rtn_tc_trace(self._h, int(bool(enable))), "rtn_tc_trace")

    def tc_trace_read(self, n=65536):
        buf = (C.c_ulonglong * n)()
        self._check(load().rtn_tc_trace_read(self._h, buf, n), "rtn_tc_trace_read")
        return np.frombuffer(buf, dtype=np.uint64).copy()

    LAUNCH_KINDS = ("inputs", "input GEMM", "forward GEMM", "output layer", "first backward GEMM",
                    "backward GEMM", "Jacobian GEMM")

    def tc_launch_times(self, enable):
        """Layered reverse mode: enable=True records every launch of the
        following network passes; enable=False returns [(kind, ms)] of the
        last recorded pass and stops recording."""
        if enable:
            self._check(load().rtn_tc_launch_times(self._h, 1, None, None, 0, None), "rtn_tc_launch_times")
            return None
        cap = 64
        ms, kind, cnt = (C.c_float * cap)(), (C.c_int * cap)(), C.c_int()
        self._check(load().rtn_tc_launch_times(self._h, 0, ms, kind, cap, C.byref(cnt)), "rtn_tc_launch_times")
        return [(self.LAUNCH_KINDS[kind[i]], float(ms[i])) for i in range(min(cnt.value, cap))]

    # -- learned part (a6) --------------------------------------------------
    def n_params(self):
        nw = sum(W.shape[0] * W.shape[1] for W, _ in self.layers)
        nb = sum(b.shape[0] for _, b in self.layers)
        return nw, nb

    def drag_targets(self, X):
        import torch
        Y = self._empty(X.shape[0], NO)
        self._check(load().rtn_drag_targets(self._h, _ptr(X, torch.float32, (X.shape[0], NX), "X"),
                                            int(X.shape[0]), _ptr(Y, torch.float32, None, "Y")),
                    "rtn_drag_targets")
        return Y

    def mse_grad(self, X, U, Y):
        import torch
        n = int(X.shape[0])
        nw, nb = self.n_params()
        g = self._empty(nw + nb)
        loss = self._empty(1)
        self._check(load().rtn_mse_grad(self._h, _ptr(X, torch.float32, (n, NX), "X"),
                                        _ptr(U, torch.float32, (n, NU), "U"),
                                        _ptr(Y, torch.float32, (n, self.n_out), "Y"), n,
                                        _ptr(g, torch.float32, None, "grad"),
                                        _ptr(loss, torch.float32, None, "loss")), "rtn_mse_grad")
        return float(loss.item()), g

    def train(self, X, U, Y, epochs, batch, lr):
        import torch
        n = int(X.shape[0])
        steps = epochs * (n // batch)
        losses = (C.c_float * max(steps, 1))()
        self._check(load().rtn_train(self._h, _ptr(X, torch.float32, (n, NX), "X"),
                                     _ptr(U, torch.float32, (n, NU), "U"),
                                     _ptr(Y, torch.float32, (n, self.n_out), "Y"), n, int(epochs), int(batch),
                                     float(lr), losses), "rtn_train")
        return np.frombuffer(losses, dtype=np.float32)[:steps].copy()

    def get_params(self):
        """[(W, b), ...] float64 arrays of the current network."""
        nw, nb = self.n_params()
        W = (C.c_float * nw)()
        b = (C.c_float * nb)()
        self._check(load().rtn_get_params(self._h, W, b), "rtn_get_params")
        W = np.frombuffer(W, dtype=np.float32).astype(np.float64)
        b = np.frombuffer(b, dtype=np.float32).astype(np.float64)
        out, ow, ob = [], 0, 0
        for Wl, bl in self.layers:
            fo, fi = Wl.shape
            out.append((W[ow:ow + fo * fi].reshape(fo, fi), b[ob:ob + fo]))
            ow += fo * fi
            ob += fo
        return out

    # -- iterate ----------------------------------------------------------
    def reset(self, x0):
        import torch
        self._check(load().rtn_reset(self._h, _ptr(x0, torch.float32, (self.B, NX), "x0")), "rtn_reset")

    def set_iterate(self, x, u):
        import torch
        self._check(load().rtn_set_iterate(self._h, _ptr(x, torch.float32, (self.n_states, NX), "x"),
                                           _ptr(u, torch.float32, (self.n_nodes, NU), "u")),
                    "rtn_set_iterate")

    def get_iterate(self):
        import torch
        x, u = self._empty(self.n_states, NX), self._empty(self.n_nodes, NU)
        self._check(load().rtn_get_iterate(self._h, _ptr(x, torch.float32, None, "x"),
                                           _ptr(u, torch.float32, None, "u")), "rtn_get_iterate")
        return x, u

    # -- hot path ---------------------------------------------------------
    def mlp_eval(self, x, u, fD=None, JD=None):
        import torch
        fD = self._empty(self.n_nodes, self.n_out) if fD is None else fD
        JD = self._empty(self.n_nodes, self.n_out, NZ) if JD is None else JD
        self._check(load().rtn_mlp_eval(self._h, _ptr(x, torch.float32, (self.n_states, NX), "x"),
                                        _ptr(u, torch.float32, (self.n_nodes, NU), "u"),
                                        _ptr(fD, torch.float32, (self.n_nodes, self.n_out), "fD"),
                                        _ptr(JD, torch.float32, (self.n_nodes, self.n_out, NZ), "JD")),
                    "rtn_mlp_eval")
        return fD, JD

    def mlp_hess(self, x, u):
        """f_D, J_D and the network Hessian H_D [n][3][17][17] (second_order
        contexts only)."""
        import torch
        n = self.n_nodes
        fD, JD, HD = self._empty(n, self.n_out), self._empty(n, self.n_out, NZ), self._empty(n, self.n_out, NZ, NZ)
        self._check(load().rtn_mlp_hess(self._h, _ptr(x, torch.float32, (self.n_states, NX), "x"),
                                        _ptr(u, torch.float32, (n, NU), "u"),
                                        _ptr(fD, torch.float32, (n, self.n_out), "fD"),
                                        _ptr(JD, torch.float32, (n, self.n_out, NZ), "JD"),
                                        _ptr(HD, torch.float32, (n, self.n_out, NZ, NZ), "HD")), "rtn_mlp_hess")
        return fD, JD, HD

    def linearize(self, x, u, out=None):
        import torch
        n = self.n_nodes
        if out is None:
            out = (self._empty(n, self.n_out), self._empty(n, self.n_out, NZ), self._empty(n, NX, NX),
                   self._empty(n, NX, NU), self._empty(n, NX))
        fD, JD, A, Bm, c = out
        self._check(load().rtn_linearize(
            self._h, _ptr(x, torch.float32, (self.n_states, NX), "x"),
            _ptr(u, torch.float32, (n, NU), "u"), _ptr(fD, torch.float32, (n, self.n_out), "fD"),
            _ptr(JD, torch.float32, (n, self.n_out, NZ), "JD"), _ptr(A, torch.float32, (n, NX, NX), "A"),
            _ptr(Bm, torch.float32, (n, NX, NU), "B"), _ptr(c, torch.float32, (n, NX), "c")),
            "rtn_linearize")
        return fD, JD, A, Bm, c

    def qp_solve(self, A, Bm, c, x, u, xref, uref, x0):
        import torch
        n, ns = self.n_nodes, self.n_states
        dx, du = self._empty(ns, NX), self._empty(n, NU)
        st = self._empty(self.B, dtype=torch.int32)
        f = torch.float32
        self._check(load().rtn_qp_solve(
            self._h, _ptr(A, f, (n, NX, NX), "A"), _ptr(Bm, f, (n, NX, NU), "B"),
            _ptr(c, f, (n, NX), "c"), _ptr(x, f, (ns, NX), "x"), _ptr(u, f, (n, NU), "u"),
            _ptr(xref, f, (ns, NX), "xref"), _ptr(uref, f, (n, NU), "uref"),
            _ptr(x0, f, (self.B, NX), "x0"), _ptr(dx, f, None, "dx"), _ptr(du, f, None, "du"),
            _ptr(st, torch.int32, None, "status")), "rtn_qp_solve")
        return dx, du, st

    def rti_step(self, x0, xref, uref, u0=None, status=None):
        import torch
        f = torch.float32
        u0 = self._empty(self.B, NU) if u0 is None else u0
        status = self._empty(self.B, dtype=torch.int32) if status is None else status
        self._check(load().rtn_rti_step(
            self._h, _ptr(x0, f, (self.B, NX), "x0"), _ptr(xref, f, (self.n_states, NX), "xref"),
            _ptr(uref, f, (self.n_nodes, NU), "uref"), _ptr(u0, f, (self.B, NU), "u0"),
            _ptr(status, torch.int32, (self.B,), "status")), "rtn_rti_step")
        return u0, status

    def rti_step_host(self, x0, xref, uref, u0, status=None):
        """rti_step with host tensors (rtn_rti_step_host): the inputs are
        copied on a second stream while the linearisation runs; u0 (and
        status) are valid once the context's stream is synchronised."""
        import torch
        f = torch.float32
        self._check(load().rtn_rti_step_host(
            self._h, _hptr(x0, f, (self.B, NX), "x0"), _hptr(xref, f, (self.n_states, NX), "xref"),
            _hptr(uref, f, (self.n_nodes, NU), "uref"), _hptr(u0, f, (self.B, NU), "u0"),
            _hptr(status, torch.int32, (self.B,), "status")), "rtn_rti_step_host")
        return u0, status

    def plant_step(self, x, u, kind="nominal", nsub=4, out=None):
        import torch
        out = self._empty(self.B, NX, dtype=torch.float64) if out is None else out
        self._check(load().rtn_plant_step(
            self._h, PLANT[kind], _ptr(x, torch.float64, (self.B, NX), "x"),
            _ptr(u, torch.float32, (self.B, NU), "u"), _ptr(out, torch.float64, (self.B, NX), "x_next"),
            int(nsub)), "rtn_plant_step")
        return out

    def closed_loop(self, steps, xref_traj, uref_traj, x_plant, plant="nominal", record=True):
        """xref_traj [B][T][13], uref_traj [B][T-1][4] float32, x_plant [B][13]
        float64 (updated in place).  Returns (traj [steps][B][13], u [steps][B][4])."""
        import torch
        f = torch.float32
        T = int(xref_traj.shape[1])
        traj = self._empty(steps, self.B, NX) if record else None
        uo = self._empty(steps, self.B, NU) if record else None
        self._check(load().rtn_closed_loop(
            self._h, int(steps), PLANT[plant], _ptr(xref_traj, f, (self.B, T, NX), "xref_traj"),
            _ptr(uref_traj, f, (self.B, T - 1, NU), "uref_traj"), T,
            _ptr(x_plant, torch.float64, (self.B, NX), "x_plant"), _ptr(traj, f, None, "traj"),
            _ptr(uo, f, None, "u_out")), "rtn_closed_loop")
        return traj, uo


class DIController:
    """A batch of B controllers of the runtime-analysis model (Sec. IV): the
    double integrator x = (p, v), u = acceleration, with an optional residual
    network (p, v, u) -> 1 output added to dv/dt.  Same C ABI as Controller
    (rtn_create with nx = 2, nu = 1); FP32 network and QP, no input bounds."""

    def __init__(self, N, dt, Q, R, QN=None, layers=None, shift=True, stream=None):
        import torch
        L = load()
        self.N = np.ascontiguousarray(N, dtype=np.int32)
        self.dt = np.ascontiguousarray(dt, dtype=np.float64)
        self.B = int(self.N.size)
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        R = np.ascontiguousarray(R, dtype=np.float64)
        QN = None if QN is None else np.ascontiguousarray(QN, dtype=np.float64)
        self._keep = []
        mlp_p = None
        self.layers = layers
        if layers:
            widths = [layers[0][0].shape[1]] + [W.shape[0] for W, _ in layers]
            w = (C.c_int * len(widths))(*widths)
            Ws = [np.ascontiguousarray(W, dtype=np.float32) for W, _ in layers]
            bs = [np.ascontiguousarray(b, dtype=np.float32) for _, b in layers]
            Wp = (C.POINTER(C.c_float) * len(Ws))(*[a.ctypes.data_as(C.POINTER(C.c_float)) for a in Ws])
            bp = (C.POINTER(C.c_float) * len(bs))(*[a.ctypes.data_as(C.POINTER(C.c_float)) for a in bs])
            self._keep += [w, Ws, bs, Wp, bp]
            mlp = _MLP(len(layers), w, Wp, bp)
            self._keep.append(mlp)
            mlp_p = C.byref(mlp)
        opt = _Opt(PRECISION["fp32"], 0, int(bool(shift)), 0, 0, 0)
        self.stream = stream
        h = C.c_void_p()
        dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
        st = L.rtn_create(C.byref(h), 2, 1, self.B, self.N.ctypes.data_as(C.POINTER(C.c_int)), dp(self.dt),
                          dp(Q), dp(R), None if QN is None else dp(QN), None, mlp_p, C.byref(opt),
                          _stream_handle(stream))
        if st != 0:
            raise RtnError(f"rtn_create: {STATUS.get(st, st)}: {L.rtn_last_error(None).decode()}")
        self._h = h
        nn, ns = C.c_int(), C.c_int()
        L.rtn_sizes(h, C.byref(nn), C.byref(ns))
        self.n_nodes, self.n_states = nn.value, ns.value
        self.device = torch.device("cuda", torch.cuda.current_device())

    close = Controller.close
    __del__ = Controller.__del__
    _check = Controller._check
    _empty = Controller._empty

    def reset(self, x0):
        import torch
        self._check(load().rtn_reset(self._h, _ptr(x0, torch.float32, (self.B, 2), "x0")), "rtn_reset")

    def set_iterate(self, x, u):
        import torch
        self._check(load().rtn_set_iterate(self._h, _ptr(x, torch.float32, (self.n_states, 2), "x"),
                                           _ptr(u, torch.float32, (self.n_nodes,), "u")), "rtn_set_iterate")

    def get_iterate(self):
        x, u = self._empty(self.n_states, 2), self._empty(self.n_nodes)
        import torch
        self._check(load().rtn_get_iterate(self._h, _ptr(x, torch.float32, None, "x"),
                                           _ptr(u, torch.float32, None, "u")), "rtn_get_iterate")
        return x, u

    def mlp_eval(self, x, u, fD=None, JD=None):
        """Network value [n_nodes] and Jacobian [n_nodes][3] at every node."""
        import torch
        n = self.n_nodes
        fD = self._empty(n) if fD is None else fD
        JD = self._empty(n, 3) if JD is None else JD
        self._check(load().rtn_mlp_eval(self._h, _ptr(x, torch.float32, (self.n_states, 2), "x"),
                                        _ptr(u, torch.float32, (n,), "u"), _ptr(fD, torch.float32, (n,), "fD"),
                                        _ptr(JD, torch.float32, (n, 3), "JD")), "rtn_mlp_eval")
        return fD, JD

    def linearize(self, x, u):
        """(fD [n], JD [n][3], A [n][2][2], B [n][2], c [n][2]) at every node."""
        import torch
        n = self.n_nodes
        fD, JD = self._empty(n), self._empty(n, 3)
        A, Bm, c = self._empty(n, 2, 2), self._empty(n, 2), self._empty(n, 2)
        f = torch.float32
        self._check(load().rtn_linearize(
            self._h, _ptr(x, f, (self.n_states, 2), "x"), _ptr(u, f, (n,), "u"), _ptr(fD, f, (n,), "fD"),
            _ptr(JD, f, (n, 3), "JD"), _ptr(A, f, (n, 2, 2), "A"), _ptr(Bm, f, (n, 2), "B"),
            _ptr(c, f, (n, 2), "c")), "rtn_linearize")
        return fD, JD, A, Bm, c

    def rti_step(self, x0, xref, uref, u0=None, status=None):
        """One RTI step of every instance: returns (u0 [B], status [B])."""
        import torch
        f = torch.float32
        u0 = self._empty(self.B) if u0 is None else u0
        status = self._empty(self.B, dtype=torch.int32) if status is None else status
        self._check(load().rtn_rti_step(
            self._h, _ptr(x0, f, (self.B, 2), "x0"), _ptr(xref, f, (self.n_states, 2), "xref"),
            _ptr(uref, f, (self.n_nodes,), "uref"), _ptr(u0, f, (self.B,), "u0"),
            _ptr(status, torch.int32, (self.B,), "status")), "rtn_rti_step")
        return u0, status
