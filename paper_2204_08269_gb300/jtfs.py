"""Python binding of libjtfs (argument marshalling only; every step of the transform runs in
the library's CUDA kernels).  PyTorch provides device memory and the current stream.

The C ABI is declared in ``include/jtfs.h``; each Python function here calls the function
of the same name.  There is no CPU path: if ``libjtfs.so`` is missing or fails to load,
every call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libjtfs.so")

PRECISIONS = {"fp32": 0, "tf32": 1, "bf16": 2, "fp32_simt": 3}


class _Config(ctypes.Structure):
    _fields_ = [("J", ctypes.c_int32), ("Q", ctypes.c_int32), ("Q2", ctypes.c_int32),
                ("J_fr", ctypes.c_int32), ("Q_fr", ctypes.c_int32), ("T", ctypes.c_int64),
                ("F", ctypes.c_int64), ("average_fr", ctypes.c_int32),
                ("oversampling", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("out_3d", ctypes.c_int32), ("branches", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 3)]


class _Shapes(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "N", "n1", "n2", "n_fr", "C", "n_t", "n_lam_out", "N_fr", "s_F",
        "s0_len", "s1_len", "s2_len", "u1_len", "n_phi", "s2_paths", "out_rows")]


# second-order joint wavelets (jtfs_branch): psi_t x psi_f and psi_t x phi_f are always on
BRANCHES = {"psi_psi": 1, "psi_phi": 2, "phi_psi": 4, "phi_phi": 8}


def _branch_mask(branches):
    """jtfs_config.branches from None (the psi_t paths), a bit mask, or names; the psi_t paths
    (psi_psi, psi_phi) are always included."""
    if branches is None:
        return 0
    if isinstance(branches, int):
        return branches
    m = BRANCHES["psi_psi"] | BRANCHES["psi_phi"]
    for b in branches:
        m |= BRANCHES[b]
    return m


_lib = None
_P = ctypes.c_void_p
_SZ = ctypes.c_size_t
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32


def lib():
    """The loaded libjtfs (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libjtfs.so not found at {LIB_PATH}; run "
                           "`python -m paper_2204_08269_gb300.build` (needs nvcc)")
    L = ctypes.CDLL(LIB_PATH)
    sig = {
        "jtfs_plan_create": ([ctypes.POINTER(_Config), _I64, ctypes.POINTER(_P)], _I32),
        "jtfs_plan_destroy": ([_P], None),
        "jtfs_plan_shapes": ([_P, ctypes.POINTER(_Shapes)], _I32),
        "jtfs_plan_schedule": ([_P, _P, _P, _P], _I32),
        "jtfs_workspace_bytes": ([_P, _I64, _I32, ctypes.POINTER(_SZ)], _I32),
        "jtfs_forward": ([_P, _P, _I64, _P, _P, _P, _P, _P, _SZ, _P], _I32),
        "jtfs_backward": ([_P, _P, _P, _I64, _P, _P, _P, _P, _P, _SZ, _P], _I32),
        "jtfs_forward_backward": ([_P, _P, _I64, _P, _P, _P, _P, _P, _P, _P, _P, _P, _SZ, _P],
                                  _I32),
        "jtfs_host_step_bytes": ([_P, _I64, ctypes.POINTER(_SZ)], _I32),
        "jtfs_scattering1d_forward": ([_P, _P, _I64, _P, _P, _P, _P, _P, _SZ, _P], _I32),
        "jtfs_scattering1d_backward": ([_P, _P, _P, _I64, _P, _P, _P, _P, _P, _SZ, _P], _I32),
        "jtfs_forward_backward_host": ([_P, _P, _I64, _P, _P, _P, _P, _P, _P, _P, _P, _SZ, _P,
                                        _SZ, _P], _I32),
        "jtfs_sync_status": ([_P, _P], _I32),
        "jtfs_plan_set_wait_budget": ([_P, ctypes.c_uint64], _I32),
        "jtfs_plan_set_check_finite": ([_P, _I32], _I32),
        "jtfs_diagnose_wait_timeout": ([_P, ctypes.c_uint64, _P], _I32),
        "jtfs_profile_enable": ([_P, _I32], _I32),
        "jtfs_profile_read": ([_P, _P, _I32, ctypes.POINTER(_I64)], _I32),
        "jtfs_profile_stage_name": ([_I32], ctypes.c_char_p),
        "jtfs_first_order_static": ([_P, _P, _I64, _P, _P, _P], _I32),
        "jtfs_plan_autotune": ([_P, _I64, _P, _SZ, _P, _P], _I32),
        "jtfs_varlen_padded_length": ([ctypes.POINTER(_Config), _I64], _I64),
        "jtfs_varlen_create": ([ctypes.POINTER(_Config), _P, _I64, _I32, ctypes.POINTER(_P)], _I32),
        "jtfs_varlen_destroy": ([_P], None),
        "jtfs_varlen_layout": ([_P, _P, _P, _P, _P], _I32),
        "jtfs_varlen_workspace_bytes": ([_P, ctypes.POINTER(_SZ)], _I32),
        "jtfs_varlen_forward_backward": ([_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _SZ, _P], _I32),
        "jtfs_varlen_capture": ([_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _SZ, _P], _I32),
        "jtfs_varlen_replay": ([_P, _P], _I32),
        "jtfs_varlen_autotune": ([_P, _P, _SZ, _P], _I32),
        "jtfs_varlen_tune_schedule": ([_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _SZ, _P, _P],
                                      _I32),
        "jtfs_mulog_mean": ([_P, _I64, _I64, _I64, _P, _P], _I32),
        "jtfs_mulog": ([_P, _I64, _I64, _I64, _P, ctypes.c_float, _P, _P], _I32),
        "jtfs_mulog_backward": ([_P, _I64, _I64, _I64, _P, ctypes.c_float, _P, _P, _P], _I32),
        "jtfs_status_string": ([_I32], ctypes.c_char_p),
        "jtfs_last_error": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def exported_symbols():
    """Names the binding expects the library to export (one per declaration in jtfs.h)."""
    return ["jtfs_plan_create", "jtfs_plan_destroy", "jtfs_plan_shapes", "jtfs_plan_schedule",
            "jtfs_workspace_bytes", "jtfs_forward", "jtfs_backward", "jtfs_forward_backward",
            "jtfs_host_step_bytes", "jtfs_scattering1d_forward", "jtfs_scattering1d_backward",
            "jtfs_forward_backward_host", "jtfs_sync_status", "jtfs_plan_set_wait_budget",
            "jtfs_plan_set_check_finite", "jtfs_diagnose_wait_timeout", "jtfs_status_string",
            "jtfs_last_error", "jtfs_profile_enable", "jtfs_profile_read",
            "jtfs_profile_stage_name", "jtfs_first_order_static", "jtfs_plan_autotune",
            "jtfs_varlen_padded_length",
            "jtfs_varlen_create", "jtfs_varlen_destroy", "jtfs_varlen_layout",
            "jtfs_varlen_workspace_bytes", "jtfs_varlen_forward_backward", "jtfs_varlen_capture",
            "jtfs_varlen_replay", "jtfs_varlen_autotune", "jtfs_varlen_tune_schedule",
            "jtfs_mulog_mean", "jtfs_mulog",
            "jtfs_mulog_backward"]


class JTFSError(RuntimeError):
    def __init__(self, call, status):
        L = lib()
        msg = L.jtfs_status_string(status).decode()
        detail = L.jtfs_last_error().decode()
        super().__init__(f"{call}: {msg}: {detail}")
        self.status = status


def _check(call, status):
    if status != 0:
        raise JTFSError(call, status)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


@dataclass(frozen=True)
class Shapes:
    N: int
    n1: int
    n2: int
    n_fr: int
    C: int
    n_t: int
    n_lam_out: int
    N_fr: int
    s_F: int
    u1_len: int
    n_phi: int = 0
    s2_paths: int = 0
    out_rows: int = 0

    def s0(self, B):
        return (B, self.n_t)

    def s1(self, B):
        return (B, self.n1, self.n_t)

    def s2(self, B):
        """[B, n2, C, n_lam_out, n_t], or [B, s2_paths, n_lam_out, n_t] with the phi_t paths
        (the n2 C psi_t paths first, then the n_phi phi_t paths)."""
        if self.n_phi:
            return (B, self.s2_paths, self.n_lam_out, self.n_t)
        return (B, self.n2, self.C, self.n_lam_out, self.n_t)

    def out_2d(self, B):
        """The single output of the 2-D layout: [B, 1 + n1 + s2_paths n_lam_out, n_t]."""
        return (B, self.out_rows, self.n_t)


class JTFSPlan:
    """Filterbanks and schedule for signals of length N (Sec. 4.2 parameters), on the
    current CUDA device.  ``precision`` selects the arithmetic of the log-frequency
    contraction: 'fp32' (tensor cores, bf16 hi/lo split), 'tf32', 'bf16' or 'fp32_simt'."""

    def __init__(self, N, J, Q, J_fr, Q_fr, T, F, Q2=1, average_fr=True, oversampling=0,
                 precision="fp32", out_3d=True, branches=None):
        L = lib()
        cfg = _Config(J=J, Q=Q, Q2=Q2, J_fr=J_fr, Q_fr=Q_fr, T=T, F=F,
                      average_fr=1 if average_fr else 0, oversampling=oversampling,
                      precision=PRECISIONS[precision], out_3d=1 if out_3d else 0,
                      branches=_branch_mask(branches))
        self.out_3d = bool(out_3d)
        h = ctypes.c_void_p()
        _check("jtfs_plan_create", L.jtfs_plan_create(ctypes.byref(cfg), N, ctypes.byref(h)))
        self._h = h
        self.device = torch.device("cuda", torch.cuda.current_device())
        sh = _Shapes()
        _check("jtfs_plan_shapes", L.jtfs_plan_shapes(h, ctypes.byref(sh)))
        self.shapes = Shapes(sh.N, sh.n1, sh.n2, sh.n_fr, sh.C, sh.n_t, sh.n_lam_out, sh.N_fr,
                             sh.s_F, sh.u1_len, sh.n_phi, sh.s2_paths, sh.out_rows)
        self.config = dict(N=N, J=J, Q=Q, Q2=Q2, J_fr=J_fr, Q_fr=Q_fr, T=T, F=F,
                           average_fr=average_fr, oversampling=oversampling, precision=precision,
                           out_3d=out_3d, branches=branches)
        self._ws = {}

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.jtfs_plan_destroy(h)
            self._h = None

    def schedule(self):
        import numpy as np
        s1 = np.zeros(self.shapes.n1, dtype=np.int32)
        s2 = np.zeros(self.shapes.n2, dtype=np.int32)
        lm = np.zeros(self.shapes.n2, dtype=np.int32)
        _check("jtfs_plan_schedule", lib().jtfs_plan_schedule(
            self._h, s1.ctypes.data_as(_P), s2.ctypes.data_as(_P), lm.ctypes.data_as(_P)))
        return s1, s2, lm

    def workspace_bytes(self, B, with_grad):
        n = ctypes.c_size_t()
        _check("jtfs_workspace_bytes",
               lib().jtfs_workspace_bytes(self._h, B, 1 if with_grad else 0, ctypes.byref(n)))
        return n.value

    def workspace(self, B, with_grad):
        """The plan's cached device workspace for the current stream.  One buffer is kept per
        stream, so calls issued on different streams (an autograd backward on a side stream,
        for example) never share scratch; calls on one stream run in order."""
        need = self.workspace_bytes(B, with_grad)
        key = ("ws", torch.cuda.current_stream(self.device).cuda_stream)
        buf = self._ws.get(key)
        if buf is None or buf.numel() < need:
            buf = torch.empty(max(need, 256), dtype=torch.uint8, device=self.device)
            self._ws[key] = buf
        return buf

    def _check_x(self, x):
        if not (x.is_cuda and x.dtype == torch.float32 and x.dim() == 2
                and x.shape[1] == self.shapes.N and x.is_contiguous()):
            raise ValueError(f"x must be a contiguous float32 CUDA tensor [B, {self.shapes.N}]")

    def _outputs(self, B, dev):
        sh = self.shapes
        if not self.out_3d:
            return torch.empty(sh.out_2d(B), dtype=torch.float32, device=dev), None, None
        return tuple(torch.empty(f(B), dtype=torch.float32, device=dev)
                     for f in (sh.s0, sh.s1, sh.s2))

    def forward(self, x, keep_checkpoint=True):
        """S0 [B, n_t], S1 [B, n1, n_t], S2 (see Shapes.s2) and the U1 checkpoint; in the 2-D
        layout (out_3d=False) the single [B, out_rows, n_t] output and None, None."""
        self._check_x(x)
        B = x.shape[0]
        sh = self.shapes
        dev = x.device
        s0, s1, s2 = self._outputs(B, dev)
        u1 = torch.empty((B, sh.u1_len), dtype=torch.float32, device=dev) if keep_checkpoint else None
        ws = self.workspace(B, True)
        _check("jtfs_forward", lib().jtfs_forward(
            self._h, _ptr(x), B, _ptr(s0), _ptr(s1), _ptr(s2), _ptr(u1), _ptr(ws), ws.numel(),
            _stream()))
        return s0, s1, s2, u1

    def backward(self, x, u1, g_s0=None, g_s1=None, g_s2=None):
        """g_x = d<g, S(x)>/dx (Sec. 5).  Cotangents may be None (zero)."""
        self._check_x(x)
        B = x.shape[0]
        gx = torch.empty_like(x)
        ws = self.workspace(B, True)
        gs = [None if g is None else g.contiguous() for g in (g_s0, g_s1, g_s2)]
        _check("jtfs_backward", lib().jtfs_backward(
            self._h, _ptr(x), _ptr(u1), B, _ptr(gs[0]), _ptr(gs[1]), _ptr(gs[2]), _ptr(gx),
            _ptr(ws), ws.numel(), _stream()))
        return gx

    def forward_backward(self, x, g_s0=None, g_s1=None, g_s2=None, keep_checkpoint=False):
        """(S0, S1, S2, g_x[, U1 checkpoint]) in one call on device tensors; the backward half
        reuses the forward's intermediate spectra instead of recomputing them."""
        self._check_x(x)
        B = x.shape[0]
        sh = self.shapes
        dev = x.device
        s0, s1, s2 = self._outputs(B, dev)
        gx = torch.empty_like(x)
        u1 = torch.empty((B, sh.u1_len), dtype=torch.float32, device=dev) if keep_checkpoint else None
        ws = self.workspace(B, True)
        gs = [None if g is None else g.contiguous() for g in (g_s0, g_s1, g_s2)]
        _check("jtfs_forward_backward", lib().jtfs_forward_backward(
            self._h, _ptr(x), B, _ptr(gs[0]), _ptr(gs[1]), _ptr(gs[2]), _ptr(s0), _ptr(s1),
            _ptr(s2), _ptr(u1), _ptr(gx), _ptr(ws), ws.numel(), _stream()))
        return (s0, s1, s2, gx, u1) if keep_checkpoint else (s0, s1, s2, gx)

    def scattering1d(self, x, keep_checkpoint=True):
        """Time scattering (Sec. 4.4 baseline) on this plan's filterbanks: S0 [B, n_t], S1
        [B, n1, n_t], S2t [B, n2, n1, n_t] (0 outside the (alpha, lambda') paths) and the U1
        checkpoint."""
        self._check_x(x)
        B = x.shape[0]
        sh = self.shapes
        dev = x.device
        s0 = torch.empty(sh.s0(B), dtype=torch.float32, device=dev)
        s1 = torch.empty(sh.s1(B), dtype=torch.float32, device=dev)
        s2t = torch.empty((B, sh.n2, sh.n1, sh.n_t), dtype=torch.float32, device=dev)
        u1 = torch.empty((B, sh.u1_len), dtype=torch.float32, device=dev) if keep_checkpoint else None
        ws = self.workspace(B, True)
        _check("jtfs_scattering1d_forward", lib().jtfs_scattering1d_forward(
            self._h, _ptr(x), B, _ptr(s0), _ptr(s1), _ptr(s2t), _ptr(u1), _ptr(ws), ws.numel(),
            _stream()))
        return s0, s1, s2t, u1

    def scattering1d_backward(self, x, u1, g_s0=None, g_s1=None, g_s2t=None):
        """g_x of <g, S(x)> for the time scattering outputs (cotangents may be None)."""
        self._check_x(x)
        B = x.shape[0]
        gx = torch.empty_like(x)
        ws = self.workspace(B, True)
        gs = [None if g is None else g.contiguous() for g in (g_s0, g_s1, g_s2t)]
        _check("jtfs_scattering1d_backward", lib().jtfs_scattering1d_backward(
            self._h, _ptr(x), _ptr(u1), B, _ptr(gs[0]), _ptr(gs[1]), _ptr(gs[2]), _ptr(gx),
            _ptr(ws), ws.numel(), _stream()))
        return gx

    def forward_backward_host(self, x_host, g_s0=None, g_s1=None, g_s2=None, outputs=True):
        """End-to-end step from pinned (or pageable) host tensors: H2D, forward, backward,
        D2H, all inside one library call.  Returns (s0, s1, s2, g_x) host tensors."""
        B = x_host.shape[0]
        sh = self.shapes
        n = ctypes.c_size_t()
        _check("jtfs_host_step_bytes", lib().jtfs_host_step_bytes(self._h, B, ctypes.byref(n)))
        key = ("host_dev", torch.cuda.current_stream(self.device).cuda_stream)
        dev_buf = self._ws.get(key)
        if dev_buf is None or dev_buf.numel() < n.value:
            dev_buf = torch.empty(n.value, dtype=torch.uint8, device=self.device)
            self._ws[key] = dev_buf
        ws = self.workspace(B, True)
        pin = x_host.is_pinned()
        gx = torch.empty(x_host.shape, dtype=torch.float32, pin_memory=pin)
        shapes = (sh.s0(B), sh.s1(B), sh.s2(B)) if self.out_3d else (sh.out_2d(B), None, None)
        outs = [torch.empty(s, dtype=torch.float32, pin_memory=pin) if (outputs and s) else None
                for s in shapes]
        _check("jtfs_forward_backward_host", lib().jtfs_forward_backward_host(
            self._h, _ptr(x_host), B, _ptr(g_s0), _ptr(g_s1), _ptr(g_s2), _ptr(outs[0]),
            _ptr(outs[1]), _ptr(outs[2]), _ptr(gx), _ptr(dev_buf), dev_buf.numel(), _ptr(ws),
            ws.numel(), _stream()))
        return outs[0], outs[1], outs[2], gx

    def autotune(self, B):
        """Tunes the launch shape of the second-order FFT stage for batches of B signals;
        returns {threads, samples_per_cta, us_per_launch}."""
        import numpy as np
        ws = self.workspace(B, True)
        c = np.zeros(3, dtype=np.int32)
        _check("jtfs_plan_autotune", lib().jtfs_plan_autotune(
            self._h, B, _ptr(ws), ws.numel(), _stream(), c.ctypes.data_as(_P)))
        return dict(threads=int(c[0]), samples_per_cta=int(c[1]), us_per_launch=int(c[2]))

    def profile(self, on=True):
        _check("jtfs_profile_enable", lib().jtfs_profile_enable(self._h, 1 if on else 0))

    def profile_read(self):
        """({stage: milliseconds}, kernel launches) since the previous read."""
        import numpy as np
        L = lib()
        names = []
        while True:
            n = L.jtfs_profile_stage_name(len(names))
            if n is None:
                break
            names.append(n.decode())
        ms = np.zeros(len(names), dtype=np.float64)
        launches = ctypes.c_int64()
        _check("jtfs_profile_read", L.jtfs_profile_read(self._h, ms.ctypes.data_as(_P), len(names),
                                                        ctypes.byref(launches)))
        return dict(zip(names, ms.tolist())), launches.value

    def sync(self):
        """Waits for the current stream; raises JTFSError on a pending device fault, a bounded
        wait that gave up (status 5) or a non-finite output of an earlier call (status 6)."""
        _check("jtfs_sync_status", lib().jtfs_sync_status(self._h, _stream()))

    def set_wait_budget(self, seconds):
        """Budget of every bounded device wait of later calls (default 2 s)."""
        _check("jtfs_plan_set_wait_budget",
               lib().jtfs_plan_set_wait_budget(self._h, int(seconds * 1e9)))

    def check_finite(self, on=True):
        """Scan every output for NaN / Inf after each call (reported by sync())."""
        _check("jtfs_plan_set_check_finite", lib().jtfs_plan_set_check_finite(self._h, int(on)))


def mulog_mean(s):
    """Eq. 6: mu [P] of a device array S [B, P, ...] (mean over examples of each path's sum)."""
    s = s.contiguous()
    B, P = s.shape[0], s.shape[1]
    M = s[0, 0].numel()
    mu = torch.empty(P, dtype=torch.float32, device=s.device)
    _check("jtfs_mulog_mean", lib().jtfs_mulog_mean(_ptr(s), B, P, M, _ptr(mu), _stream()))
    return mu


def mulog(s, mu, eps=0.1):
    """Eq. 7: log(1 + S / (eps mu[path])) for S [B, P, ...] on the device."""
    s = s.contiguous()
    out = torch.empty_like(s)
    B, P = s.shape[0], s.shape[1]
    _check("jtfs_mulog", lib().jtfs_mulog(_ptr(s), B, P, s[0, 0].numel(), _ptr(mu.contiguous()),
                                          float(eps), _ptr(out), _stream()))
    return out


def mulog_backward(s, mu, g_out, eps=0.1):
    s = s.contiguous()
    gs = torch.empty_like(s)
    B, P = s.shape[0], s.shape[1]
    _check("jtfs_mulog_backward", lib().jtfs_mulog_backward(
        _ptr(s), B, P, s[0, 0].numel(), _ptr(mu.contiguous()), float(eps),
        _ptr(g_out.contiguous()), _ptr(gs), _stream()))
    return gs


class JTFSFunction(torch.autograd.Function):
    """(S0, S1, S2) = JTFS(x) with the hand-written adjoint chain as backward; only the
    first-order scalogram is kept between the passes."""

    @staticmethod
    def forward(ctx, x, plan):
        x = x.contiguous()
        s0, s1, s2, u1 = plan.forward(x)
        ctx.plan = plan
        ctx.save_for_backward(x, u1)
        if not plan.out_3d:
            return s0
        return s0, s1, s2

    @staticmethod
    def backward(ctx, *g):
        x, u1 = ctx.saved_tensors
        g = list(g) + [None] * (3 - len(g))
        gx = ctx.plan.backward(x, u1, *g)
        return gx, None


class JTFS(torch.nn.Module):
    """Joint time-frequency scattering as a module: x [B, N] -> (S0, S1, S2), or the single
    [B, out_rows, n_t] tensor with out_3d=False."""

    def __init__(self, N, J, Q, J_fr, Q_fr, T, F, **kw):
        super().__init__()
        self.plan = JTFSPlan(N, J, Q, J_fr, Q_fr, T, F, **kw)

    def forward(self, x):
        return JTFSFunction.apply(x, self.plan)


def _config(J, Q, J_fr, Q_fr, T, F, Q2=1, average_fr=True, oversampling=0, precision="fp32",
            branches=None):
    return _Config(J=J, Q=Q, Q2=Q2, J_fr=J_fr, Q_fr=Q_fr, T=T, F=F,
                   average_fr=1 if average_fr else 0, oversampling=oversampling,
                   precision=PRECISIONS[precision], out_3d=1, branches=_branch_mask(branches))


def varlen_padded_length(length, J, **kw):
    """Padded length of one signal of an uneven-length batch (host only)."""
    cfg = _config(J=J, Q=kw.pop("Q", 1), J_fr=kw.pop("J_fr", 1), Q_fr=kw.pop("Q_fr", 1),
                  T=kw.pop("T", 1), F=kw.pop("F", 1), **kw)
    return int(lib().jtfs_varlen_padded_length(ctypes.byref(cfg), int(length)))


class JTFSVarlen:
    """Uneven-length batch: signals of lengths ``lengths`` packed back to back, each
    zero-padded to its power-of-two length and keeping ceil(len / T) frames (see jtfs.h)."""

    def __init__(self, lengths, J, Q, J_fr, Q_fr, T, F, chunk=0, **kw):
        import numpy as np
        L = lib()
        self._cfg = _config(J, Q, J_fr, Q_fr, T, F, **kw)
        self.lengths = np.ascontiguousarray(np.asarray(lengths, dtype=np.int64))
        B = len(self.lengths)
        h = ctypes.c_void_p()
        _check("jtfs_varlen_create", L.jtfs_varlen_create(
            ctypes.byref(self._cfg), self.lengths.ctypes.data_as(_P), B, int(chunk),
            ctypes.byref(h)))
        self._h = h
        self.B = B
        offs = [np.zeros(B + 1, dtype=np.int64) for _ in range(4)]
        _check("jtfs_varlen_layout", L.jtfs_varlen_layout(h, *[o.ctypes.data_as(_P) for o in offs]))
        self.x_off, self.s0_off, self.s1_off, self.s2_off = offs
        n = ctypes.c_size_t()
        _check("jtfs_varlen_workspace_bytes", L.jtfs_varlen_workspace_bytes(h, ctypes.byref(n)))
        self.device = torch.device("cuda", torch.cuda.current_device())
        self._ws = torch.empty(max(n.value, 256), dtype=torch.uint8, device=self.device)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.jtfs_varlen_destroy(h)
            self._h = None

    def outputs(self):
        dev = self.device
        return [torch.empty(int(o[-1]), dtype=torch.float32, device=dev)
                for o in (self.s0_off, self.s1_off, self.s2_off, self.x_off)]

    def _args(self, x, g, outs):
        g = list(g) + [None] * (3 - len(g))
        return [_ptr(x), _ptr(g[0]), _ptr(g[1]), _ptr(g[2]), _ptr(outs[0]), _ptr(outs[1]),
                _ptr(outs[2]), _ptr(outs[3]), _ptr(self._ws), self._ws.numel()]

    def forward_backward(self, x_packed, g=(), outs=None):
        """(S0, S1, S2, g_x) packed; g = (g_s0, g_s1, g_s2) packed cotangents (None = 0)."""
        outs = outs or self.outputs()
        _check("jtfs_varlen_forward_backward",
               lib().jtfs_varlen_forward_backward(self._h, *self._args(x_packed, g, outs), _stream()))
        return outs

    def capture(self, x_packed, g=(), outs=None):
        """Captures the step on the current (non-default) stream into a CUDA graph bound to
        these buffers; returns the output buffers the graph writes."""
        outs = outs or self.outputs()
        self._bound = (x_packed, tuple(g), outs)   # keep the buffers alive
        _check("jtfs_varlen_capture",
               lib().jtfs_varlen_capture(self._h, *self._args(x_packed, g, outs), _stream()))
        return outs

    def replay(self):
        _check("jtfs_varlen_replay", lib().jtfs_varlen_replay(self._h, _stream()))

    def autotune(self):
        _check("jtfs_varlen_autotune", lib().jtfs_varlen_autotune(
            self._h, _ptr(self._ws), self._ws.numel(), _stream()))

    def tune_schedule(self, x_packed, g=(), outs=None):
        """Times the step with every sub-batch size up to the creation's ``chunk`` and keeps
        the fastest; returns that size.  Capture the graph afterwards."""
        import numpy as np
        outs = outs or self.outputs()
        c = np.zeros(1, dtype=np.int32)
        _check("jtfs_varlen_tune_schedule", lib().jtfs_varlen_tune_schedule(
            self._h, *self._args(x_packed, g, outs), _stream(), c.ctypes.data_as(_P)))
        return int(c[0])
