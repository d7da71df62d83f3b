"""GB300 HOTRG: forward coarse-graining and reverse-mode backward of
differentiable TRG, as a thin Python binding over the C ABI in
``include/hotrg.h`` (argument marshalling only; every step runs in the CUDA
library ``_lib/libhotrg.so``).

The library must be built first (``__graft_entry__.build()`` or
``python paper_1912_02780_gb300/_build.py``).  There is no CPU fallback: if
the library is missing, loading fails with an error.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libhotrg.so")

FP64, BF16X3, BF16X6 = 0, 1, 2
PRECISIONS = {"fp64": FP64, "bf16x3": BF16X3, "bf16x6": BF16X6}

STATUS = {0: "HOTRG_OK", 1: "HOTRG_EINVAL", 2: "HOTRG_ENOMEM", 3: "HOTRG_ECUDA",
          4: "HOTRG_ENOTCONV", 5: "HOTRG_ENONFINITE", 6: "HOTRG_ETIMEOUT",
          7: "HOTRG_ESTATE", 8: "HOTRG_EUNSUPPORTED", 9: "HOTRG_EPENDING"}

# Every symbol declared in include/hotrg.h.
EXPORTS = (
    "hotrg_config_default", "hotrg_config_sizeof", "hotrg_plan_workspace_bytes",
    "hotrg_isometries", "hotrg_set_isometries", "hotrg_isometry_adjoints", "hotrg_mera_update", "hotrg_plan_create",
    "hotrg_plan_destroy", "hotrg_forward_tensor", "hotrg_forward_ising",
    "hotrg_forward_device", "hotrg_backward", "hotrg_backward_device", "hotrg_sync",
    "hotrg_plan_set_steps", "hotrg_plan_set_stream", "hotrg_plan_set_given_steps",
    "hotrg_forward_xy", "hotrg_chain_lnz_steps", "hotrg_isometry_sides",
    "hotrg_group_create", "hotrg_forward_group_tensor", "hotrg_forward_group_ising",
    "hotrg_group_launches", "hotrg_group_destroy", "hotrg_group_workspace_bytes",
    "hotrg_lbfgs_create", "hotrg_lbfgs_layer", "hotrg_lbfgs_destroy",
    "hotrg_diagnostics", "hotrg_eigh_diagnostics", "hotrg_step_dims", "hotrg_status_string", "hotrg_last_error",
    "hotrg_device_supports_split", "hotrg_gemm_split_check", "hotrg_gemm_f64_check",
    "hotrg_profile_enable", "hotrg_profile_read", "hotrg_kernel_launches",
    "hotrg_gemm_split_noalloc",
    "hotrg_server_create", "hotrg_server_submit", "hotrg_server_poll", "hotrg_server_wait",
    "hotrg_server_drain", "hotrg_server_get_stats", "hotrg_server_destroy",
    "hotrg_debug_inject", "hotrg_check_bounded_wait",
)
PROFILE_SLOTS = 32
STAGE_NAMES = {0: "gram", 1: "eigh", 2: "s1", 3: "s2", 4: "s3", 5: "norm", 6: "prep",
               7: "bwd_contract", 8: "bwd_eigh_adj", 9: "bwd_gram_adj", 10: "s2_4plane",
               11: "eigh_prod", 12: "eigh_qr", 13: "eigh_rr", 14: "eigh_res"}


class hotrg_config(ctypes.Structure):
    _fields_ = [("d0", ctypes.c_int), ("d_cut", ctypes.c_int), ("n_steps", ctypes.c_int),
                ("precision", ctypes.c_int), ("split_from_step", ctypes.c_int),
                ("want_grad", ctypes.c_int), ("fixed_w_grad", ctypes.c_int),
                ("eigh_broadening", ctypes.c_double), ("gram_split_from_step", ctypes.c_int),
                ("hi_precision_steps", ctypes.c_int), ("eigh_mode", ctypes.c_int),
                ("eigh_power_iters", ctypes.c_int), ("eigh_block", ctypes.c_int),
                ("epilogue_split", ctypes.c_int), ("split_chunk_elems", ctypes.c_longlong),
                ("w_given", ctypes.c_int), ("eigh_residual_tol", ctypes.c_double),
                ("stage2_n_group", ctypes.c_int), ("stage2_pair", ctypes.c_int),
                ("gemm_sm_reserve", ctypes.c_int), ("eigh_warm_start", ctypes.c_int),
                ("scheme", ctypes.c_int), ("chain_steps", ctypes.c_int),
                ("w_rule", ctypes.c_int)]


class hotrg_request(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("J", ctypes.c_double), ("h", ctypes.c_double),
                ("d_cut", ctypes.c_int), ("n_steps", ctypes.c_int), ("want_grad", ctypes.c_int),
                ("precision", ctypes.c_int), ("split_from_step", ctypes.c_int)]


class hotrg_result(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("status", ctypes.c_int), ("slot", ctypes.c_int),
                ("lnz_per_site", ctypes.c_double), ("dlnz_dbeta", ctypes.c_double),
                ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double),
                ("t_finish", ctypes.c_double)]


class hotrg_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("failed", ctypes.c_uint64), ("plans_created", ctypes.c_uint64),
                ("plans_evicted", ctypes.c_uint64), ("bytes_in_use", ctypes.c_size_t),
                ("peak_bytes", ctypes.c_size_t), ("queue_depth", ctypes.c_int),
                ("busy_slots", ctypes.c_int), ("admission_waits", ctypes.c_uint64),
                ("grouped", ctypes.c_uint64), ("groups", ctypes.c_uint64)]


class HotrgError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        self.status = status
        super().__init__(f"{STATUS.get(status, status)}: {msg}")


_LIB = None
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def lib() -> ctypes.CDLL:
    """Load the CUDA library (raises if it was not built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"HOTRG CUDA library not built: {LIB_PATH} is missing "
                           "(run __graft_entry__.build())")
    L = ctypes.CDLL(LIB_PATH)
    vp = ctypes.c_void_p
    L.hotrg_config_default.argtypes = [ctypes.POINTER(hotrg_config), ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.hotrg_config_default.restype = None
    L.hotrg_plan_workspace_bytes.argtypes = [ctypes.POINTER(hotrg_config), ctypes.POINTER(ctypes.c_size_t)]
    L.hotrg_plan_create.argtypes = [ctypes.POINTER(hotrg_config), vp, ctypes.POINTER(vp)]
    L.hotrg_plan_destroy.argtypes = [vp]
    L.hotrg_plan_destroy.restype = None
    L.hotrg_forward_tensor.argtypes = [vp, _dp, _dp, _dp, _ip]
    L.hotrg_forward_ising.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp, _dp, _ip]
    L.hotrg_forward_device.argtypes = [vp, vp, vp]
    L.hotrg_backward.argtypes = [vp, _dp, _dp]
    L.hotrg_backward_device.argtypes = [vp, vp]
    L.hotrg_sync.argtypes = [vp]
    L.hotrg_plan_set_steps.argtypes = [vp, ctypes.c_int]
    L.hotrg_plan_set_stream.argtypes = [vp, vp]
    L.hotrg_diagnostics.argtypes = [vp, _dp, _dp, _ip]
    L.hotrg_step_dims.argtypes = [vp, ctypes.c_int, _ip, _ip, _ip]
    L.hotrg_eigh_diagnostics.argtypes = [vp, _dp, _ip, _ip, ctypes.POINTER(ctypes.c_longlong)]
    L.hotrg_status_string.argtypes = [ctypes.c_int]
    L.hotrg_status_string.restype = ctypes.c_char_p
    L.hotrg_last_error.argtypes = [vp]
    L.hotrg_last_error.restype = ctypes.c_char_p
    L.hotrg_device_supports_split.argtypes = []
    L.hotrg_gemm_split_check.argtypes = [ctypes.c_int] * 6 + [_dp, _dp, _dp]
    L.hotrg_gemm_f64_check.argtypes = [ctypes.c_int] * 3 + [_dp, _dp, _dp]
    L.hotrg_profile_enable.argtypes = [vp, ctypes.c_int]
    L.hotrg_profile_read.argtypes = [vp, _dp, _ip]
    L.hotrg_kernel_launches.argtypes = []
    L.hotrg_kernel_launches.restype = ctypes.c_ulonglong
    L.hotrg_gemm_split_noalloc.argtypes = [ctypes.c_int] * 5 + [vp, vp, vp, vp]
    L.hotrg_server_create.argtypes = [ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(vp)]
    L.hotrg_server_submit.argtypes = [vp, ctypes.POINTER(hotrg_request), ctypes.POINTER(ctypes.c_uint64)]
    L.hotrg_server_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(hotrg_result)]
    L.hotrg_server_wait.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(hotrg_result)]
    L.hotrg_server_drain.argtypes = [vp]
    L.hotrg_server_get_stats.argtypes = [vp, ctypes.POINTER(hotrg_server_stats)]
    L.hotrg_server_destroy.argtypes = [vp]
    L.hotrg_debug_inject.argtypes = [ctypes.c_int, ctypes.c_int]
    L.hotrg_check_bounded_wait.argtypes = [ctypes.c_double]
    L.hotrg_server_destroy.restype = None
    for name in EXPORTS:
        if name not in ("hotrg_plan_destroy", "hotrg_config_default", "hotrg_status_string",
                        "hotrg_last_error", "hotrg_kernel_launches", "hotrg_server_destroy",
                        "hotrg_config_sizeof", "hotrg_lbfgs_destroy", "hotrg_group_launches",
                        "hotrg_group_destroy"):
            getattr(L, name).restype = ctypes.c_int
    L.hotrg_isometries.argtypes = [vp, _dp]
    L.hotrg_set_isometries.argtypes = [vp, _dp]
    L.hotrg_isometry_adjoints.argtypes = [vp, _dp]
    L.hotrg_mera_update.argtypes = [vp, ctypes.c_int]
    L.hotrg_plan_set_given_steps.argtypes = [vp, ctypes.c_int]
    L.hotrg_forward_xy.argtypes = [vp, ctypes.c_double, ctypes.c_double, _dp, _dp]
    L.hotrg_chain_lnz_steps.argtypes = [vp, _dp]
    L.hotrg_isometry_sides.argtypes = [vp, _ip]
    L.hotrg_group_create.argtypes = [ctypes.POINTER(hotrg_config), ctypes.c_int, vp,
                                     ctypes.POINTER(vp)]
    L.hotrg_forward_group_tensor.argtypes = [vp, ctypes.POINTER(vp), ctypes.c_int, _dp, _dp]
    L.hotrg_forward_group_ising.argtypes = [vp, ctypes.POINTER(vp), ctypes.c_int, _dp, _dp, _dp,
                                            _dp]
    L.hotrg_group_launches.argtypes = [vp]
    L.hotrg_group_launches.restype = ctypes.c_ulonglong
    L.hotrg_group_workspace_bytes.argtypes = [ctypes.POINTER(hotrg_config), ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_size_t)]
    L.hotrg_group_destroy.argtypes = [vp]
    L.hotrg_group_destroy.restype = None
    L.hotrg_lbfgs_create.argtypes = [vp, ctypes.c_int, ctypes.POINTER(vp)]
    L.hotrg_lbfgs_layer.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_int, _dp, _ip, _ip]
    L.hotrg_lbfgs_destroy.argtypes = [vp]
    L.hotrg_lbfgs_destroy.restype = None
    L.hotrg_config_sizeof.argtypes = []
    L.hotrg_config_sizeof.restype = ctypes.c_size_t
    if L.hotrg_config_sizeof() != ctypes.sizeof(hotrg_config):
        raise RuntimeError(f"hotrg_config layout mismatch: library {L.hotrg_config_sizeof()} bytes, "
                           f"binding {ctypes.sizeof(hotrg_config)} bytes (rebuild the library)")
    _LIB = L
    return L


def _p(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def make_config(d0: int, d_cut: int, n_steps: int, precision="fp64", split_from_step: int = 1,
                want_grad: bool = True, fixed_w_grad: bool = False,
                eigh_broadening: float = 1e-12, gram_split_from_step: int = 0,
                hi_precision_steps: int = 2, eigh_mode: int = 0,
                eigh_power_iters: int = 4, eigh_block: int = 0,
                epilogue_split: bool = True, split_chunk_elems: int = 0,
                w_given: bool = False, eigh_residual_tol: float = 0.0,
                stage2_n_group: int = 0, stage2_pair: int = 0,
                gemm_sm_reserve: int = 0, eigh_warm_start: int = 0, scheme: int = 0,
                chain_steps: bool = False, w_rule: int = 0) -> hotrg_config:
    c = hotrg_config()
    lib().hotrg_config_default(ctypes.byref(c), d0, d_cut, n_steps)
    c.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    c.split_from_step = split_from_step
    c.want_grad = int(bool(want_grad))
    c.fixed_w_grad = int(bool(fixed_w_grad))
    c.eigh_broadening = eigh_broadening
    c.gram_split_from_step = gram_split_from_step
    c.hi_precision_steps = hi_precision_steps
    c.eigh_mode = eigh_mode
    c.eigh_power_iters = eigh_power_iters
    c.eigh_block = eigh_block
    c.epilogue_split = int(bool(epilogue_split))
    c.split_chunk_elems = int(split_chunk_elems)
    c.w_given = int(bool(w_given))
    c.eigh_residual_tol = float(eigh_residual_tol)
    c.stage2_n_group = int(stage2_n_group)
    c.stage2_pair = int(stage2_pair)
    c.gemm_sm_reserve = int(gemm_sm_reserve)
    c.eigh_warm_start = int(eigh_warm_start)
    c.scheme = int(scheme)
    c.chain_steps = int(bool(chain_steps))
    c.w_rule = int(w_rule)
    return c


def workspace_bytes(d0, d_cut, n_steps, **kw) -> int:
    c = make_config(d0, d_cut, n_steps, **kw)
    out = ctypes.c_size_t(0)
    s = lib().hotrg_plan_workspace_bytes(ctypes.byref(c), ctypes.byref(out))
    if s:
        raise HotrgError(s, "workspace size")
    return out.value


def device_supports_split() -> bool:
    return lib().hotrg_device_supports_split() == 0


class Plan:
    """One HOTRG problem shape (d0, d_cut, n_steps, precision) bound to a
    CUDA stream; owns all device memory it needs."""

    def __init__(self, d0: int, d_cut: int, n_steps: int, precision="fp64",
                 split_from_step: int = 1, want_grad: bool = True, fixed_w_grad: bool = False,
                 eigh_broadening: float = 1e-12, stream: Optional[int] = None,
                 gram_split_from_step: int = 0, hi_precision_steps: int = 2,
                 eigh_mode: int = 0, eigh_power_iters: int = 4, eigh_block: int = 0,
                 epilogue_split: bool = True, split_chunk_elems: int = 0,
                 w_given: bool = False, eigh_residual_tol: float = 0.0,
                 stage2_n_group: int = 0, stage2_pair: int = 0, gemm_sm_reserve: int = 0,
                 eigh_warm_start: int = 0, scheme: int = 0, chain_steps: bool = False,
                 w_rule: int = 0):
        self.cfg = make_config(d0, d_cut, n_steps, precision, split_from_step, want_grad,
                               fixed_w_grad, eigh_broadening, gram_split_from_step,
                               hi_precision_steps, eigh_mode, eigh_power_iters, eigh_block,
                               epilogue_split, split_chunk_elems, w_given, eigh_residual_tol,
                               stage2_n_group, stage2_pair, gemm_sm_reserve, eigh_warm_start,
                               scheme, chain_steps, w_rule)
        self.d0, self.d_cut, self.n_steps = d0, d_cut, n_steps
        self.n_run = n_steps
        h = ctypes.c_void_p(0)
        s = lib().hotrg_plan_create(ctypes.byref(self.cfg), ctypes.c_void_p(stream or 0), ctypes.byref(h))
        if s:
            raise HotrgError(s, "hotrg_plan_create")
        self._h = h

    def _check(self, s, what):
        if s:
            msg = lib().hotrg_last_error(self._h)
            raise HotrgError(s, f"{what}: {msg.decode() if msg else ''}")

    def set_steps(self, n_steps: int):
        """Run only the first n_steps of this plan from now on (the result of
        a plan created with n_steps)."""
        self._check(lib().hotrg_plan_set_steps(self._h, int(n_steps)), "set_steps")
        self.n_run = int(n_steps)

    def forward_tensor(self, T0: np.ndarray):
        T0 = np.ascontiguousarray(T0, dtype=np.float64)
        if T0.shape != (self.d0,) * 4:
            raise ValueError("T0 must have shape (d0, d0, d0, d0)")
        lnz = ctypes.c_double(0)
        ln = np.zeros(self.n_run)
        sign = ctypes.c_int(0)
        self._check(lib().hotrg_forward_tensor(self._h, _p(T0), ctypes.byref(lnz), _p(ln),
                                               ctypes.byref(sign)), "forward_tensor")
        return lnz.value, ln, sign.value

    def forward_ising(self, beta: float, J: float = 1.0, h: float = 0.0):
        lnz = ctypes.c_double(0)
        ln = np.zeros(self.n_run)
        sign = ctypes.c_int(0)
        self._check(lib().hotrg_forward_ising(self._h, beta, J, h, ctypes.byref(lnz), _p(ln),
                                              ctypes.byref(sign)), "forward_ising")
        return lnz.value, ln, sign.value

    def forward_xy(self, tau: float, J: float = 1.0):
        """Scheme-1 forward of the quantum XY chain's Trotter MPO rho(tau):
        (lnz per copy of T0 at beta = 2^(n+1) tau, log-norms)."""
        lnz = ctypes.c_double(0)
        ln = np.zeros(self.n_run)
        self._check(lib().hotrg_forward_xy(self._h, tau, J, ctypes.byref(lnz), _p(ln)),
                    "forward_xy")
        return lnz.value, ln

    def chain_lnz_steps(self):
        """Scheme 1: lnz of every depth of the last forward (NaN before the
        last unless the plan has chain_steps)."""
        out = np.zeros(self.n_run)
        self._check(lib().hotrg_chain_lnz_steps(self._h, _p(out)), "chain_lnz_steps")
        return out

    def isometry_sides(self):
        """Side (0 left, 1 right) of each step's isometry in the last forward."""
        out = np.zeros(self.n_run, dtype=np.int32)
        self._check(lib().hotrg_isometry_sides(self._h, out.ctypes.data_as(_ip)),
                    "isometry_sides")
        return out

    def set_given_steps(self, k0: int):
        """w_given plans: steps 1..k0 use the stored isometries, later ones
        form theirs from the Gram matrix."""
        self._check(lib().hotrg_plan_set_given_steps(self._h, int(k0)), "set_given_steps")

    def forward_device(self, T0_ptr: int, out_ptr: int):
        self._check(lib().hotrg_forward_device(self._h, ctypes.c_void_p(T0_ptr),
                                               ctypes.c_void_p(out_ptr)), "forward_device")

    def backward(self, want_dbeta: bool = False):
        g = np.zeros((self.d0,) * 4)
        db = ctypes.c_double(0)
        self._check(lib().hotrg_backward(self._h, _p(g), ctypes.byref(db) if want_dbeta else None),
                    "backward")
        return (g, db.value) if want_dbeta else g

    def backward_device(self, grad_ptr: int):
        self._check(lib().hotrg_backward_device(self._h, ctypes.c_void_p(grad_ptr)), "backward_device")

    def sync(self):
        self._check(lib().hotrg_sync(self._h), "sync")

    def diagnostics(self):
        t = np.zeros(self.n_steps)
        g = np.zeros(self.n_steps)
        s = np.zeros(self.n_steps, dtype=np.int32)
        self._check(lib().hotrg_diagnostics(self._h, _p(t), _p(g), s.ctypes.data_as(_ip)), "diagnostics")
        return t, g, s

    def eigh_diagnostics(self):
        """(residual per step, extra power iterations per step, exact-solver flag
        per step, guard firings so far): the subspace eigensolver's accuracy
        guard (NaN residual where it did not run)."""
        r = np.zeros(self.n_steps)
        x = np.zeros(self.n_steps, dtype=np.int32)
        e = np.zeros(self.n_steps, dtype=np.int32)
        f = ctypes.c_longlong(0)
        self._check(lib().hotrg_eigh_diagnostics(self._h, _p(r), x.ctypes.data_as(_ip),
                                                 e.ctypes.data_as(_ip), ctypes.byref(f)),
                    "eigh_diagnostics")
        return r, x, e, int(f.value)

    # ---- differentiable TRG: isometries as parameters ----------------------
    def _w_layout(self):
        shapes, off = [], 0
        for k in range(1, self.n_steps + 1):
            X, _, Xp = self.step_dims(k)
            shapes.append((off, Xp, X * X, X))
            off += Xp * X * X
        return shapes, off

    def _split_w(self, flat):
        """Per-step arrays w[x1, x2, a] (the oracle's layout) from the ABI's rows."""
        shapes, _ = self._w_layout()
        return [flat[o:o + xp * n].reshape(xp, x, x).transpose(1, 2, 0).copy()
                for o, xp, n, x in shapes]

    def isometries(self):
        _, tot = self._w_layout()
        flat = np.zeros(tot)
        self._check(lib().hotrg_isometries(self._h, _p(flat)), "isometries")
        return self._split_w(flat)

    def set_isometries(self, ws):
        shapes, tot = self._w_layout()
        flat = np.zeros(tot)
        for (o, xp, n, x), w in zip(shapes, ws):
            flat[o:o + xp * n] = np.asarray(w, dtype=np.float64).transpose(2, 0, 1).reshape(-1)
        self._check(lib().hotrg_set_isometries(self._h, _p(flat)), "set_isometries")

    def isometry_adjoints(self):
        _, tot = self._w_layout()
        flat = np.zeros(tot)
        self._check(lib().hotrg_isometry_adjoints(self._h, _p(flat)), "isometry_adjoints")
        return self._split_w(flat)

    def mera_update(self, k: int):
        self._check(lib().hotrg_mera_update(self._h, int(k)), "mera_update")

    def step_dims(self, k: int):
        X, Y, Xp = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(lib().hotrg_step_dims(self._h, k, ctypes.byref(X), ctypes.byref(Y), ctypes.byref(Xp)),
                    "step_dims")
        return X.value, Y.value, Xp.value

    def profile(self, enable: bool = True):
        self._check(lib().hotrg_profile_enable(self._h, int(bool(enable))), "profile_enable")

    def profile_read(self):
        """{slot name: (ms, launches)}; FP64-GEMM variants get the suffix _f64."""
        ms = np.zeros(PROFILE_SLOTS)
        cnt = np.zeros(PROFILE_SLOTS, dtype=np.int32)
        self._check(lib().hotrg_profile_read(self._h, _p(ms), cnt.ctypes.data_as(_ip)), "profile_read")
        out = {}
        for i in range(PROFILE_SLOTS):
            if cnt[i]:
                name = STAGE_NAMES.get(i % 16, str(i % 16)) + ("_f64" if i >= 16 else "")
                out[name] = (float(ms[i]), int(cnt[i]))
        return out

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().hotrg_plan_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Group:
    """Grouped forward of several plans of one shape (see include/hotrg.h:
    hotrg_group_*): the same keyword arguments as ``Plan`` describe the
    shape, and every plan passed to it must be created with them.  Each plan
    runs on its own stream (plans on different streams overlap their
    eigensolves); the grouped contractions run on the group's ``stream``."""

    def __init__(self, d0: int, d_cut: int, n_steps: int, precision="fp64", max_count: int = 8,
                 stream: Optional[int] = None, **kw):
        self.cfg = make_config(d0, d_cut, n_steps, precision, **kw)
        self.d0 = d0
        h = ctypes.c_void_p(0)
        s = lib().hotrg_group_create(ctypes.byref(self.cfg), int(max_count),
                                     ctypes.c_void_p(stream or 0), ctypes.byref(h))
        if s:
            raise HotrgError(s, "hotrg_group_create")
        self._h = h

    @staticmethod
    def _handles(plans):
        arr = (ctypes.c_void_p * len(plans))()
        for i, p in enumerate(plans):
            arr[i] = p._h.value
        return arr

    def _check(self, s, plans, what):
        if s:
            msg = lib().hotrg_last_error(plans[0]._h) if plans else b""
            raise HotrgError(s, f"{what}: {msg.decode() if msg else ''}")

    def forward_tensor(self, plans, T0s):
        T0 = np.ascontiguousarray(np.asarray(T0s, dtype=np.float64).reshape(len(plans), -1))
        lnz = np.zeros(len(plans))
        self._check(lib().hotrg_forward_group_tensor(self._h, self._handles(plans), len(plans),
                                                     _p(T0), _p(lnz)), plans, "forward_group")
        return lnz

    def forward_ising(self, plans, betas, J=1.0, h=0.0):
        n = len(plans)
        b = np.ascontiguousarray(np.broadcast_to(np.asarray(betas, dtype=np.float64), (n,)))
        jj = np.ascontiguousarray(np.broadcast_to(np.asarray(J, dtype=np.float64), (n,)))
        hh = np.ascontiguousarray(np.broadcast_to(np.asarray(h, dtype=np.float64), (n,)))
        lnz = np.zeros(n)
        self._check(lib().hotrg_forward_group_ising(self._h, self._handles(plans), n, _p(b),
                                                    _p(jj), _p(hh), _p(lnz)),
                    plans, "forward_group_ising")
        return lnz

    def launches(self) -> int:
        return int(lib().hotrg_group_launches(self._h))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().hotrg_group_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class LBFGS:
    """Quasi-Newton optimiser of one layer's isometry at a time in the
    exponential parametrisation (see include/hotrg.h: hotrg_lbfgs_*), bound to
    a w_given plan that has run a forward."""

    def __init__(self, plan: "Plan", history: int = 10):
        self.plan = plan
        h = ctypes.c_void_p(0)
        plan._check(lib().hotrg_lbfgs_create(plan._h, int(history), ctypes.byref(h)),
                    "lbfgs_create")
        self._h = h

    def layer(self, step: int, n_iter: int, step0: float = 0.1, c1: float = 1e-4,
              max_backtracks: int = 30):
        """n_iter iterations on layer `step`: (ln Z/N at the start and after each
        accepted iteration, forward evaluations)."""
        f = np.zeros(n_iter + 1)
        acc, ev = ctypes.c_int(0), ctypes.c_int(0)
        self.plan._check(lib().hotrg_lbfgs_layer(self._h, int(step), int(n_iter), float(step0),
                                                 float(c1), int(max_backtracks), _p(f),
                                                 ctypes.byref(acc), ctypes.byref(ev)),
                         "lbfgs_layer")
        return f[:acc.value + 1], ev.value

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().hotrg_lbfgs_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Server:
    """Continuous-batching solve server (see include/hotrg.h)."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 4):
        h = ctypes.c_void_p(0)
        s = lib().hotrg_server_create(int(hbm_budget_bytes), int(max_slots), ctypes.byref(h))
        if s:
            raise HotrgError(s, "hotrg_server_create")
        self._h = h

    def submit(self, beta, J=1.0, h=0.0, d_cut=16, n_steps=20, want_grad=False, precision="fp64",
               split_from_step=1) -> int:
        r = hotrg_request(beta, J, h, d_cut, n_steps, int(bool(want_grad)),
                          PRECISIONS[precision] if isinstance(precision, str) else int(precision),
                          split_from_step)
        t = ctypes.c_uint64(0)
        s = lib().hotrg_server_submit(self._h, ctypes.byref(r), ctypes.byref(t))
        if s:
            raise HotrgError(s, "submit")
        return t.value

    def poll(self, ticket: int):
        r = hotrg_result()
        s = lib().hotrg_server_poll(self._h, ticket, ctypes.byref(r))
        if s == 9:
            return None
        if s:
            raise HotrgError(s, "poll")
        return r

    def wait(self, ticket: int) -> hotrg_result:
        r = hotrg_result()
        s = lib().hotrg_server_wait(self._h, ticket, ctypes.byref(r))
        if s:
            raise HotrgError(s, "wait")
        return r

    def drain(self):
        s = lib().hotrg_server_drain(self._h)
        if s:
            raise HotrgError(s, "drain")

    def stats(self) -> dict:
        st = hotrg_server_stats()
        lib().hotrg_server_get_stats(self._h, ctypes.byref(st))
        return {f: getattr(st, f) for f, _ in st._fields_}

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().hotrg_server_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def kernel_launches() -> int:
    return int(lib().hotrg_kernel_launches())


def gemm_split_check(A: np.ndarray, B: np.ndarray, planes: int = 2, kchunk: int = 0,
                     cta_pair: bool = False) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    M, K = A.shape
    N = B.shape[0]
    C = np.zeros((M, N))
    s = lib().hotrg_gemm_split_check(M, N, K, planes, kchunk, int(bool(cta_pair)), _p(A), _p(B),
                                     _p(C))
    if s:
        raise HotrgError(s, "gemm_split_check")
    return C


def gemm_f64_check(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    M, K = A.shape
    N = B.shape[0]
    C = np.zeros((M, N))
    s = lib().hotrg_gemm_f64_check(M, N, K, _p(A), _p(B), _p(C))
    if s:
        raise HotrgError(s, "gemm_f64_check")
    return C
