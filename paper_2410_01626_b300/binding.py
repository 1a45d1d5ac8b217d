"""Thin ctypes binding of the fmmcph C ABI (argument marshalling only).

Every step of the evaluation runs in the library's CUDA kernels; this module
only passes device pointers, sizes and the current CUDA stream.  There is no
CPU fallback: if the shared library cannot be loaded, importing the package
raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import build as _build

P = ctypes.c_void_p
I = ctypes.c_int

FMM_FP32, FMM_MIXED_TF32, FMM_MIXED_3XTF32, FMM_MIXED_3XBF16, FMM_MIXED_FP16 = 0, 1, 2, 3, 4
PRECISIONS = {"fp32": FMM_FP32, "tf32": FMM_MIXED_TF32, "3xtf32": FMM_MIXED_3XTF32, "3xbf16": FMM_MIXED_3XBF16,
              "fp16": FMM_MIXED_FP16}
# lambda dependence within a site (Sec. 2.1, Eq. 1): interpolated charges, or interpolated Hamiltonian
INTERPOLATIONS = {"charge": 0, "hamiltonian": 1}
DEV_DOMAIN, DEV_SITE, DEV_TIMEOUT, DEV_BOUNDS = 1, 2, 4, 8
KE_DEFAULT = 138.935458
# stage intervals of one evaluation (fmm_stage_times): the chain binning .. final, the near field
# ("p2p", concurrent with p2m .. m2m), and the coarse levels' M2L and L2L, which run on a side
# branch beside the finest levels' M2L (0 where an evaluation has no such branch)
STAGES = ("binning", "p2m", "m2m", "root", "m2l", "l2l", "outputs", "final", "p2p", "m2l_coarse", "l2l_coarse")


class FmmBox(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_double * 3), ("edge", ctypes.c_double)]


class FmmOptions(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("coulomb_k", ctypes.c_double), ("interpolation", ctypes.c_int),
                ("m2l_tile_rows", ctypes.c_int), ("p2p_leaves_per_block", ctypes.c_int), ("reserved", ctypes.c_int * 5)]


EXPORTS = {
    "fmm_create": (I, [ctypes.POINTER(FmmBox), I, I, I, ctypes.POINTER(FmmOptions), ctypes.POINTER(P)]),
    "fmm_set_charges": (I, [P, I, I, P, P, P, P, P]),
    "fmm_set_charges4": (I, [P, I, I, P, P, P, P, P, P, P]),
    "fmm_set_lambda": (I, [P, P, P]),
    "fmm_bind_lambda": (I, [P, P]),
    "fmm_eval": (I, [P, P, P, P, P, P, P]),
    "fmm_eval_host": (I, [P, P, P, P, P, P]),
    "fmm_eval_host_async": (I, [P, P, P, P, P, P]),
    "fmm_adjoint": (I, [P, P, P, P, P, P, P, P, P, P]),
    "fmm_adjoint4": (I, [P, P, P, P, P, P, P, P, P, P, P, P]),
    "fmm_get_binning": (I, [P, P, P, P, P, P]),
    "fmm_status_word": (I, [P, ctypes.POINTER(I), P]),
    "fmm_stage_times": (I, [P, P, I]),
    "fmm_set_profiling": (I, [P, I]),
    "fmm_launches_per_eval": (I, [P]),
    "fmm_host_operator": (I, [I, I, P, P]),
    "fmm_host_regular": (I, [I, P, P]),
    "fmm_set_wait_limit": (I, [P, ctypes.c_longlong]),
    "fmm_inject_alloc_failure": (I, [I]),
    "fmm_binning_noalloc": (I, [ctypes.POINTER(FmmBox), I, I, I, P, P, P, P, P, P, P]),
    "fmm_lambda_step": (I, [I, P, P, P, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                            ctypes.c_ulonglong, ctypes.c_ulonglong, I, ctypes.c_double, ctypes.c_double, P]),
    "fmm_lambda_step_bias": (I, [I, P, P, P, P, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_ulonglong, ctypes.c_ulonglong, I, ctypes.c_double, ctypes.c_double, P]),
    "fmm_lambda_pfc": (I, [ctypes.c_double] * 9 + [ctypes.POINTER(ctypes.c_double)]),
    "fmm_batch_create": (I, [I, P, ctypes.POINTER(P)]),
    "fmm_batch_eval": (I, [P, P, P, P, P, P]),
    "fmm_batch_destroy": (None, [P]),
    "fmm_host_alloc": (I, [ctypes.c_size_t, ctypes.POINTER(P)]),
    "fmm_host_free": (None, [P]),
    "fmm_destroy": (None, [P]),
    "fmm_error_string": (ctypes.c_char_p, [I]),
    "fmm_last_error": (ctypes.c_char_p, []),
    "fmm_build_flags": (I, []),
    "fmm_inject_copy_loss": (I, [P, I]),
    "fmm_stream_wait_eval": (I, [P, P]),
}

_lib = None


def _checked() -> bool:
    return os.environ.get("FMMCPH_BOUNDS_CHECK", "") not in ("", "0")


def library_path() -> str:
    """The library this process loads: the bounds-checked build when the environment variable
    FMMCPH_BOUNDS_CHECK is set (to anything but 0) before the first load, else the normal one."""
    return _build.LIB_CHECKED if _checked() else _build.LIB


def load(build_if_missing: bool = True):
    """Load (building first if needed) the shared library."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if build_if_missing and not os.path.exists(path):
        _build.build(checked=_checked())
    lib = ctypes.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class FmmError(RuntimeError):
    def __init__(self, code, what=""):
        msg = load().fmm_error_string(code).decode()
        detail = load().fmm_last_error().decode() if code == 3 else ""
        super().__init__(f"{what}: {msg} (status {code})" + (f" [{detail}]" if detail else ""))
        self.code = code


def _check(code, what):
    if code != 0:
        raise FmmError(code, what)


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev(t, dtype, name):
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


class FMM:
    """One solver handle: a cubic box, boundary, multipole order p and tree depth."""

    def __init__(self, edge, periodic, p, depth, origin=(0.0, 0.0, 0.0), precision="fp32", ke=None,
                 interpolation="charge", m2l_rows=0, p2p_warps=0):
        lib = load()
        box = FmmBox((ctypes.c_double * 3)(*[float(o) for o in origin]), float(edge))
        opt = FmmOptions(PRECISIONS[precision] if isinstance(precision, str) else int(precision),
                         float(ke) if ke else 0.0, INTERPOLATIONS[interpolation], int(m2l_rows), int(p2p_warps),
                         (ctypes.c_int * 5)())
        h = ctypes.c_void_p()
        _check(lib.fmm_create(ctypes.byref(box), int(bool(periodic)), int(p), int(depth), ctypes.byref(opt),
                              ctypes.byref(h)), "fmm_create")
        self._h = h
        self._lib = lib
        self.edge, self.periodic, self.p, self.depth = float(edge), bool(periodic), int(p), int(depth)
        self.origin = tuple(float(o) for o in origin)
        self.precision = precision
        self.interpolation = interpolation
        self.ke = float(ke) if ke else KE_DEFAULT
        self.n = 0
        self.K = 0
        self.nlam = 0  # lambda coordinates: K (two-form sites) or 2K (four-form sites)
        self.forms = 2

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.fmm_destroy(self._h)
        self._h = None

    __del__ = close

    def set_charges(self, qA, qB, site, lam):
        n = qA.numel()
        K = lam.numel()
        _dev(qA, torch.float32, "qA"), _dev(qB, torch.float32, "qB"), _dev(site, torch.int32, "site")
        if K:
            _dev(lam, torch.float32, "lambda")
        _check(self._lib.fmm_set_charges(self._h, n, K, _ptr(qA), _ptr(qB), _ptr(site), _ptr(lam) if K else None,
                                         _stream()), "fmm_set_charges")
        self.n, self.K, self.nlam, self.forms = n, K, K, 2
        self._site = site

    def set_charges4(self, qA, qB, qC, qD, site, lam):
        """Sites with two lambda coordinates over four charge forms (Sec. 2.1, Eq. 2):
        q = (1 - lp)[(1 - lt) qA + lt qB] + lp[(1 - lt) qC + lt qD]; lam = [2K] = (lp, lt) per
        site.  dV/dlambda then has 2K entries in the same order."""
        n = qA.numel()
        if lam.numel() % 2:
            raise ValueError("lambda must hold (lambda_p, lambda_t) for every site")
        K = lam.numel() // 2
        for t, nm in ((qA, "qA"), (qB, "qB"), (qC, "qC"), (qD, "qD")):
            _dev(t, torch.float32, nm)
        _dev(site, torch.int32, "site")
        if K:
            _dev(lam, torch.float32, "lambda")
        _check(self._lib.fmm_set_charges4(self._h, n, K, _ptr(qA), _ptr(qB), _ptr(qC), _ptr(qD), _ptr(site),
                                          _ptr(lam) if K else None, _stream()), "fmm_set_charges4")
        self.n, self.K, self.nlam, self.forms = n, K, 2 * K, 4
        self._site = site

    def set_lambda(self, lam):
        _dev(lam, torch.float32, "lambda")
        _check(self._lib.fmm_set_lambda(self._h, _ptr(lam), _stream()), "fmm_set_lambda")

    def bind_lambda(self, lam):
        if lam is not None:
            _dev(lam, torch.float32, "lambda")
        self._bound = lam
        _check(self._lib.fmm_bind_lambda(self._h, _ptr(lam)), "fmm_bind_lambda")

    def outputs(self, device=None, phi=False):
        dev = device or torch.device("cuda")
        E = torch.empty(1, dtype=torch.float64, device=dev)
        F = torch.empty(self.n, 3, dtype=torch.float32, device=dev)
        dV = torch.empty(self.nlam, dtype=torch.float32, device=dev)
        ph = torch.empty(self.n, dtype=torch.float32, device=dev) if phi else None
        return E, F, dV, ph

    def eval_into(self, x, E, F=None, dVdl=None, phi=None):
        _dev(x, torch.float32, "x")
        if x.numel() != 3 * self.n:
            raise ValueError("x must have shape [n_atoms, 3]")
        _check(self._lib.fmm_eval(self._h, _ptr(x), _ptr(E), _ptr(F), _ptr(dVdl) if self.K else None, _ptr(phi),
                                  _stream()), "fmm_eval")

    def eval(self, x, phi=False):
        E, F, dV, ph = self.outputs(x.device, phi)
        self.eval_into(x, E, F, dV, ph)
        return E, F, dV, ph

    def eval_host(self, x_host, E_host, F_host, dV_host):
        """Host buffers (numpy or pinned CPU tensors); copies inside the call."""
        def hp(a):
            if a is None:
                return None
            if isinstance(a, torch.Tensor):
                return ctypes.c_void_p(a.data_ptr())
            return a.ctypes.data_as(ctypes.c_void_p)
        _check(self._lib.fmm_eval_host(self._h, hp(x_host), hp(E_host), hp(F_host), hp(dV_host), _stream()),
               "fmm_eval_host")

    def stream_wait_eval(self):
        """Make the current stream wait for the end of the last evaluation's kernels (not for
        the result copies of eval_host(_async) that follow them)."""
        _check(self._lib.fmm_stream_wait_eval(self._h, _stream()), "fmm_stream_wait_eval")

    def eval_host_async(self, x_host, E_host, F_host, dV_host):
        """As eval_host without waiting: the results are in the host buffers once the current
        stream has reached the end of the call (page-locked buffers; keep them and x_host
        unchanged until then).  Consecutive calls overlap one call's position copy with the
        previous call's evaluation."""
        def hp(a):
            if a is None:
                return None
            if isinstance(a, torch.Tensor):
                return ctypes.c_void_p(a.data_ptr())
            return a.ctypes.data_as(ctypes.c_void_p)
        _check(self._lib.fmm_eval_host_async(self._h, hp(x_host), hp(E_host), hp(F_host), hp(dV_host), _stream()),
               "fmm_eval_host_async")

    def adjoint(self, gbar, F, phi, dVdl, grad_x=True, grad_qA=True, grad_qB=True, grad_lam=True):
        dev = F.device
        gx = torch.empty(self.n, 3, dtype=torch.float32, device=dev) if grad_x else None
        ga = torch.empty(self.n, dtype=torch.float32, device=dev) if grad_qA else None
        gb = torch.empty(self.n, dtype=torch.float32, device=dev) if grad_qB else None
        gl = torch.empty(self.nlam, dtype=torch.float32, device=dev) if grad_lam else None
        _check(self._lib.fmm_adjoint(self._h, _ptr(gbar), _ptr(F), _ptr(phi), _ptr(dVdl) if self.K else None,
                                     _ptr(gx), _ptr(ga), _ptr(gb), _ptr(gl) if self.K else None, _stream()),
               "fmm_adjoint")
        return gx, ga, gb, gl

    def adjoint4(self, gbar, F, phi, dVdl, grad_x=True, grad_q=(True, True, True, True), grad_lam=True):
        """Reverse mode for four-form sites: (dL/dx, (dL/dq^A .. dL/dq^D), dL/dlambda)."""
        dev = F.device
        gx = torch.empty(self.n, 3, dtype=torch.float32, device=dev) if grad_x else None
        gq = [torch.empty(self.n, dtype=torch.float32, device=dev) if w else None for w in grad_q]
        gl = torch.empty(self.nlam, dtype=torch.float32, device=dev) if grad_lam else None
        _check(self._lib.fmm_adjoint4(self._h, _ptr(gbar), _ptr(F), _ptr(phi), _ptr(dVdl) if self.K else None,
                                      _ptr(gx), *[_ptr(t) for t in gq], _ptr(gl) if self.K else None, _stream()),
               "fmm_adjoint4")
        return gx, gq, gl

    def binning(self):
        dev = torch.device("cuda")
        nleaf = 1 << (3 * self.depth)
        key = torch.empty(self.n, dtype=torch.int32, device=dev)
        perm = torch.empty(self.n, dtype=torch.int32, device=dev)
        start = torch.empty(nleaf, dtype=torch.int32, device=dev)
        count = torch.empty(nleaf, dtype=torch.int32, device=dev)
        _check(self._lib.fmm_get_binning(self._h, _ptr(key), _ptr(perm), _ptr(start), _ptr(count), _stream()),
               "fmm_get_binning")
        return key, perm, start, count

    def status_word(self):
        s = ctypes.c_int(0)
        _check(self._lib.fmm_status_word(self._h, ctypes.byref(s), _stream()), "fmm_status_word")
        return s.value

    def set_wait_limit(self, cycles=0):
        """Limit (GPU clock cycles) of the kernels' bounded waits (tensor-core M2L, M2M and L2L,
        near-field staging); 0 = the default (about 2 s)."""
        _check(self._lib.fmm_set_wait_limit(self._h, int(cycles)), "fmm_set_wait_limit")

    def inject_copy_loss(self, mask=0):
        """Test hook: the bulk copies of the kernels in `mask` (1 = M2M/L2L operator copies,
        2 = near-field staging) are announced but never issued, so their waits run out."""
        _check(self._lib.fmm_inject_copy_loss(self._h, int(mask)), "fmm_inject_copy_loss")

    def set_profiling(self, on=True, serial=False):
        """Per-stage event timing (stage_times); with ``serial`` every stage runs alone."""
        _check(self._lib.fmm_set_profiling(self._h, (2 if serial else 1) if on else 0), "fmm_set_profiling")

    def stage_times(self):
        ms = (ctypes.c_float * len(STAGES))()
        k = self._lib.fmm_stage_times(self._h, ctypes.cast(ms, ctypes.c_void_p), len(STAGES))
        return dict(zip(STAGES[:k], list(ms)[:k]))

    def launches_per_eval(self):
        return int(self._lib.fmm_launches_per_eval(self._h))


def pinned_empty(shape, dtype=torch.float32):
    """Page-locked host tensor from the library's allocator (fmm_host_alloc), for the buffers of
    FMM.eval_host; the memory is released (fmm_host_free) when the last tensor using it is gone."""
    import weakref
    import numpy as np
    shape = tuple(int(d) for d in (shape if isinstance(shape, (tuple, list)) else (shape,)))
    count = int(np.prod(shape)) if shape else 1
    itemsize = torch.empty((), dtype=dtype).element_size()
    nbytes = max(1, count * itemsize)
    ptr = P()
    _check(load().fmm_host_alloc(nbytes, ctypes.byref(ptr)), "fmm_host_alloc")
    raw = (ctypes.c_uint8 * nbytes).from_address(ptr.value)
    arr = np.frombuffer(raw, dtype=np.uint8)
    weakref.finalize(arr, load().fmm_host_free, ptr.value)
    return torch.from_numpy(arr)[: count * itemsize].view(dtype).view(shape)


def host_operator(kind, p, o=(0, 0, 0)):
    """FP64 real-form operator from the library's host code (no GPU needed)."""
    lib = load()
    nc = (p + 1) ** 2
    out = np.empty((nc, nc))
    oo = np.ascontiguousarray(o, np.int32)
    _check(lib.fmm_host_operator(int(kind), int(p), oo.ctypes.data_as(ctypes.c_void_p),
                                 out.ctypes.data_as(ctypes.c_void_p)), "fmm_host_operator")
    return out


def host_regular(p, u):
    lib = load()
    out = np.empty((p + 1) ** 2)
    uu = np.ascontiguousarray(u, np.float64)
    _check(lib.fmm_host_regular(int(p), uu.ctypes.data_as(ctypes.c_void_p), out.ctypes.data_as(ctypes.c_void_p)),
           "fmm_host_regular")
    return out


def lambda_step(lam, vel, dVdl, step, seed, dt=0.002, mass=60.0, gamma=1.0, kT=2.494339, first=False,
                lo=-0.1, hi=1.1, bias=None):
    """One device-side BAOAB step of the lambda particles (in place); ``bias`` ([n, 5] float:
    a0, a1, barrier, delta, kwall per coordinate, see ``lambda_bias``) adds the double-well force."""
    _dev(lam, torch.float32, "lambda"), _dev(vel, torch.float32, "velocity"), _dev(dVdl, torch.float32, "dVdl")
    if bias is None:
        _check(load().fmm_lambda_step(lam.numel(), _ptr(lam), _ptr(vel), _ptr(dVdl), dt, mass, gamma, kT, int(seed),
                                      int(step), int(bool(first)), lo, hi, _stream()), "fmm_lambda_step")
        return
    _dev(bias, torch.float32, "bias")
    if bias.numel() != 5 * lam.numel():
        raise ValueError("bias must hold 5 values per lambda coordinate")
    _check(load().fmm_lambda_step_bias(lam.numel(), _ptr(lam), _ptr(vel), _ptr(dVdl), _ptr(bias), dt, mass, gamma,
                                       kT, int(seed), int(step), int(bool(first)), lo, hi, _stream()),
           "fmm_lambda_step_bias")


def lambda_pfc(pH, pKa_ref, barrier, kT=2.494339, a0=0.0, a1=1.0, kwall=1000.0, lo=0.0, hi=1.0):
    """Well offset delta of the double well (partition function correction, host FP64); the
    partition functions run over [lo, b] and [b, hi], by default Sec. 2.3's [0, 0.5] and
    [0.5, 1]."""
    d = ctypes.c_double()
    _check(load().fmm_lambda_pfc(float(pH), float(pKa_ref), float(barrier), float(kT), float(a0), float(a1),
                                 float(kwall), float(lo), float(hi), ctypes.byref(d)), "fmm_lambda_pfc")
    return d.value


def lambda_bias(pH, pKa_ref, barrier, kT=2.494339, a0=0.0, a1=1.0, kwall=1000.0, pfc_lo=0.0, pfc_hi=1.0,
                device="cuda"):
    """Bias parameters [n, 5] for ``lambda_step`` from per-coordinate pKa_ref and barrier
    (sequences of equal length, or scalars): the double well with the pH offset from
    ``lambda_pfc`` over [pfc_lo, pfc_hi] (Sec. 2.3: [0, 1])."""
    import numpy as np
    pk = np.atleast_1d(np.asarray(pKa_ref, np.float64))
    bh = np.broadcast_to(np.atleast_1d(np.asarray(barrier, np.float64)), pk.shape)
    rows = [[a0, a1, b, lambda_pfc(pH, p, b, kT, a0, a1, kwall, pfc_lo, pfc_hi), kwall] for p, b in zip(pk, bh)]
    return torch.tensor(rows, dtype=torch.float32, device=device)


class Batch:
    """Independent replicas evaluated as parallel branches of one CUDA graph."""

    def __init__(self, solvers):
        self.solvers = list(solvers)
        arr = (ctypes.c_void_p * len(self.solvers))(*[s._h.value for s in self.solvers])
        b = ctypes.c_void_p()
        _check(load().fmm_batch_create(len(self.solvers), ctypes.cast(arr, ctypes.c_void_p), ctypes.byref(b)),
               "fmm_batch_create")
        self._b = b

    def eval_into(self, xs, Es, Fs=None, dVs=None):
        n = len(self.solvers)
        def arr(ts):
            if ts is None:
                return None
            a = (ctypes.c_void_p * n)(*[(t.data_ptr() if t is not None and t.numel() else None) for t in ts])
            return ctypes.cast(a, ctypes.c_void_p)
        self._keep = (arr(xs), arr(Es), arr(Fs), arr(dVs))
        _check(load().fmm_batch_eval(self._b, *self._keep, _stream()), "fmm_batch_eval")

    def close(self):
        if getattr(self, "_b", None) is not None and self._b.value:
            load().fmm_batch_destroy(self._b)
        self._b = None

    __del__ = close
