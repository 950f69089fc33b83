"""Python face of the linewidth library: same operations as the C ABI.

Arrays may be numpy arrays (host) or torch tensors (host or CUDA).  With CUDA
tensors the call runs asynchronously on the current torch stream and returns
CUDA tensors; with host arrays it stages through device memory and returns
numpy arrays.  Every step of the path runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib

FP64, FP32, BF16X3, TF32X3 = 0, 1, 2, 3
PRECISIONS = {"fp64": FP64, "fp32": FP32, "bf16x3": BF16X3, "tf32x3": TF32X3}


class EPWError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_lib.STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(status: int):
    if status != _lib.EPW_OK:
        msg = _lib.load().epw_last_error().decode(errors="replace")
        raise EPWError(status, msg)


def _is_torch(x):
    return type(x).__module__.startswith("torch")


class _Arg:
    """Pointer to a contiguous array (kept alive while the call runs)."""

    def __init__(self, x, dtype):
        self.keep = None
        self.device = False
        if x is None:
            self.ptr = None
            return
        if _is_torch(x):
            import torch
            tdt = {np.float64: torch.float64, np.int32: torch.int32, np.complex128: torch.complex128}[dtype]
            t = x.detach()
            if t.dtype != tdt:
                t = t.to(tdt)
            t = t.contiguous()
            self.keep = t
            self.device = t.is_cuda
            self.ptr = t.data_ptr()
        else:
            a = np.ascontiguousarray(x, dtype=dtype)
            self.keep = a
            self.ptr = a.ctypes.data


def _stream_of(*args):
    if any(a.device for a in args):
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(0)


class Model:
    """A Wannier model resident on the current CUDA device (epw_load_wannier).

    ``wm`` is any object with the attributes nw, nat, mass, Re, wRe, H, Rph,
    wRph, Phi, Rp, wRp, g (see the layouts in include/epw.h).
    """

    def __init__(self, wm, g_is_c64: bool = False):
        lib = _lib.load()
        self.nw, self.nat = int(wm.nw), int(wm.nat)
        self.nm = 3 * self.nat
        c = np.ascontiguousarray
        gdt = np.complex64 if g_is_c64 else np.complex128
        self._keep = [
            c(wm.mass, np.float64), c(wm.Re, np.int32), c(wm.wRe, np.float64), c(wm.H, np.complex128),
            c(wm.Rph, np.int32), c(wm.wRph, np.float64), c(wm.Phi, np.complex128),
            c(wm.Rp, np.int32), c(wm.wRp, np.float64), c(wm.g, gdt),
        ]
        k = self._keep
        self.nRe, self.nRph, self.nRp = len(k[1]), len(k[4]), len(k[7])
        self.g_shape = (self.nRe, self.nRp, self.nm, self.nw, self.nw)
        d = _lib.WannierDesc(self.nw, self.nat, k[0].ctypes.data,
                             self.nRe, k[1].ctypes.data, k[2].ctypes.data, k[3].ctypes.data,
                             self.nRph, k[4].ctypes.data, k[5].ctypes.data, k[6].ctypes.data,
                             self.nRp, k[7].ctypes.data, k[8].ctypes.data, k[9].ctypes.data, int(g_is_c64))
        h = ctypes.c_void_p()
        _check(lib.epw_load_wannier(ctypes.byref(d), ctypes.byref(h)))
        self._h = h
        self._keep = None
        if getattr(wm, "polar", None) is not None:
            self.set_polar(wm.polar)

    def set_polar(self, polar):
        """Long-range vertex of polar materials (epw_set_polar); polar has A, eps_inf, Zstar [nat,3,3],
        alpha, prefactor, gmax (None removes it)."""
        lib = _lib.load()
        if polar is None:
            _check(lib.epw_set_polar(self._h, None))
            return
        Z = np.ascontiguousarray(polar.Zstar, dtype=np.float64)
        if Z.shape != (self.nat, 3, 3):
            raise ValueError(f"Zstar shape {Z.shape} != {(self.nat, 3, 3)}")
        d = _lib.PolarDesc((ctypes.c_double * 9)(*np.asarray(polar.A, dtype=np.float64).ravel()),
                           (ctypes.c_double * 9)(*np.asarray(polar.eps_inf, dtype=np.float64).ravel()),
                           Z.ctypes.data, float(polar.alpha), float(polar.prefactor), int(polar.gmax))
        _check(lib.epw_set_polar(self._h, ctypes.byref(d)))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.load().epw_free_model(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def set_vertex(self, g):
        """Replace g(Re,Rp) (layout of the model's g; host array or CUDA tensor)."""
        ga = _Arg(g, np.complex128)
        if tuple(ga.keep.shape) != self.g_shape:
            raise ValueError(f"vertex shape {tuple(ga.keep.shape)} != {self.g_shape}")
        self._autograd_vertex = None  # the vertex the autograd interface last loaded is gone
        _check(_lib.load().epw_set_vertex(self._h, ga.ptr, 0, _stream_of(ga)))

    def reserve(self, nk: int, nq: int, precision: int = FP64):
        _check(_lib.load().epw_reserve(self._h, int(nk), int(nq), int(precision)))

    def sync(self, stream=None):
        _check(_lib.load().epw_sync(self._h, ctypes.c_void_p(stream or 0)))

    def timing(self, enable: bool):
        """Bracket each dominant-kernel launch with CUDA events (measurement hook)."""
        _check(_lib.load().epw_timing_enable(self._h, int(enable)))

    def timing_read(self):
        """(summed device ms, launches) of the dominant kernel since the last read."""
        ms = ctypes.c_double(0.0)
        n = ctypes.c_int(0)
        _check(_lib.load().epw_timing_read(self._h, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def timing_read_tags(self):
        """((ms, launches) of the dominant kernel, (ms, launches) of the secondary one) since
        the last read; the secondary one is the per-pair eigensolve kernel of the wide-shape
        tensor-core form."""
        ms = (ctypes.c_double * 2)()
        n = (ctypes.c_int * 2)()
        _check(_lib.load().epw_timing_read_tags(self._h, ms, n))
        return (ms[0], n[0]), (ms[1], n[1])

    # ------------------------------------------------------------- linewidth
    def linewidth(self, k, q, wq=None, *, T: float, EF: float, sigma: float, omega_min: float = 1e-5,
                  precision: int = FP64, out=None):
        """Im Sigma_nk [nk, nw] (eV), Eq. (linewidthel) on shell."""
        lib = _lib.load()
        ka, qa, wa = _Arg(k, np.float64), _Arg(q, np.float64), _Arg(wq, np.float64)
        nk = int(np.prod(ka.keep.shape)) // 3
        nq = int(np.prod(qa.keep.shape)) // 3
        if out is None:
            if ka.device:
                import torch
                out = torch.empty((nk, self.nw), dtype=torch.float64, device=ka.keep.device)
            else:
                out = np.zeros((nk, self.nw))
        oa = _Arg(out, np.float64)
        if oa.keep is not out and not _is_torch(out):
            raise ValueError("out must be a contiguous float64 array")
        pr = _lib.Params(float(T), float(EF), float(sigma), float(omega_min), int(precision), 0)
        _check(lib.epw_linewidth(self._h, nk, ka.ptr, nq, qa.ptr, wa.ptr, ctypes.byref(pr), oa.ptr,
                                 _stream_of(ka, qa, wa, oa)))
        return out

    def phonon_selfenergy(self, k, q, wk=None, *, T: float, EF: float, sigma: float, omega_min: float = 1e-5,
                          precision: int = FP64):
        """(Pi''_qnu [nq, 3nat], lambda_qnu [nq, 3nat], nesting [nq], N(E_F)): per-q sums over the k list
        (Eqs. linewidthph on shell, lambdaEQ, nestingfct)."""
        lib = _lib.load()
        ka, qa, wa = _Arg(k, np.float64), _Arg(q, np.float64), _Arg(wk, np.float64)
        nk = int(np.prod(ka.keep.shape)) // 3
        nq = int(np.prod(qa.keep.shape)) // 3
        if qa.device:
            import torch
            mk = lambda *shape: torch.zeros(shape, dtype=torch.float64, device=qa.keep.device)
        else:
            mk = lambda *shape: np.zeros(shape)
        pi, lam, zeta, dos = mk(nq, self.nm), mk(nq, self.nm), mk(nq), mk(1)
        outs = [_Arg(x, np.float64) for x in (pi, lam, zeta, dos)]
        pr = _lib.Params(float(T), float(EF), float(sigma), float(omega_min), int(precision), 0)
        _check(lib.epw_phonon_selfenergy(self._h, nk, ka.ptr, wa.ptr, nq, qa.ptr, ctypes.byref(pr),
                                         *[o.ptr for o in outs], _stream_of(ka, qa, wa, *outs)))
        return pi, lam, zeta, (float(dos[0]) if not _is_torch(dos) else dos)

    def selfenergy(self, k, q, omega, wq=None, *, T: float, EF: float, delta: float, omega_min: float = 1e-5,
                   precision: int = FP64, spectral: bool = True):
        """(Sigma_nk(omega) [nk, nw, nomega] complex, A_nk(omega) [nk, nw, nomega] or None):
        Eqs. elselfenergy and spectral_funct on the frequency grid `omega` (eV from E_F)."""
        lib = _lib.load()
        ka, qa, wa, oa = _Arg(k, np.float64), _Arg(q, np.float64), _Arg(wq, np.float64), _Arg(omega, np.float64)
        nk = int(np.prod(ka.keep.shape)) // 3
        nq = int(np.prod(qa.keep.shape)) // 3
        nom = int(np.prod(oa.keep.shape))
        if ka.device:
            import torch
            sig = torch.zeros((nk, self.nw, nom), dtype=torch.complex128, device=ka.keep.device)
            spec = torch.zeros((nk, self.nw, nom), dtype=torch.float64, device=ka.keep.device) if spectral else None
        else:
            sig = np.zeros((nk, self.nw, nom), dtype=np.complex128)
            spec = np.zeros((nk, self.nw, nom)) if spectral else None
        sa, pa = _Arg(sig, np.complex128), _Arg(spec, np.float64)
        pr = _lib.Params(float(T), float(EF), 1.0, float(omega_min), int(precision), 0)
        _check(lib.epw_selfenergy(self._h, nk, ka.ptr, nq, qa.ptr, wa.ptr, ctypes.byref(pr), float(delta), nom,
                                  oa.ptr, sa.ptr, pa.ptr, _stream_of(ka, qa, wa, oa, sa, pa)))
        return sig, spec

    def linewidth_noalloc(self, k, q, wq=None, *, T: float, EF: float, sigma: float, omega_min: float = 1e-5,
                          precision: int = FP64, out=None):
        """epw_linewidth_noalloc: like linewidth, but the library allocates no device memory.

        For callers that must not allocate (see include/epw.h).  k, q, wq and
        out must be CUDA tensors; out is allocated here by torch only when the
        caller does not pass one.
        """
        lib = _lib.load()
        ka, qa, wa = _Arg(k, np.float64), _Arg(q, np.float64), _Arg(wq, np.float64)
        nk = int(np.prod(ka.keep.shape)) // 3
        nq = int(np.prod(qa.keep.shape)) // 3
        if out is None:
            import torch
            out = torch.empty((nk, self.nw), dtype=torch.float64, device=ka.keep.device)
        oa = _Arg(out, np.float64)
        pr = _lib.Params(float(T), float(EF), float(sigma), float(omega_min), int(precision), 0)
        _check(lib.epw_linewidth_noalloc(self._h, nk, ka.ptr, nq, qa.ptr, wa.ptr, ctypes.byref(pr), oa.ptr,
                                         _stream_of(ka, qa, wa, oa)))
        return out

    # ---------------------------------------------------------------- interp
    def interp(self, k, q, precision: int = FP64, omega_min: float = 1e-5, want_g: bool = True):
        """(eps_k [nk,nw], eps_kq [nk,nq,nw], omega [nq,3nat], g [nk,nq,3nat,nw,nw]) as numpy arrays."""
        lib = _lib.load()
        ka, qa = _Arg(k, np.float64), _Arg(q, np.float64)
        nk = int(np.prod(ka.keep.shape)) // 3
        nq = int(np.prod(qa.keep.shape)) // 3
        eps_k = np.zeros((nk, self.nw))
        eps_kq = np.zeros((nk, nq, self.nw))
        omega = np.zeros((nq, self.nm))
        g = np.zeros((nk, nq, self.nm, self.nw, self.nw), dtype=np.complex128) if want_g else None
        _check(lib.epw_interp_g(self._h, nk, ka.ptr, nq, qa.ptr, int(precision), float(omega_min),
                                eps_k.ctypes.data, eps_kq.ctypes.data, omega.ctypes.data,
                                None if g is None else g.ctypes.data, _stream_of(ka, qa)))
        return eps_k, eps_kq, omega, g

    # -------------------------------------------------------------- backward
    def linewidth_backward(self, k, q, grad, wq=None, *, T: float, EF: float, sigma: float,
                           omega_min: float = 1e-5, precision: int = FP64, want_dg: bool = True):
        """Adjoint of sum(grad * Im Sigma): (dg like g, dL/dT, dL/dE_F)."""
        lib = _lib.load()
        ka, qa, wa, ca = _Arg(k, np.float64), _Arg(q, np.float64), _Arg(wq, np.float64), _Arg(grad, np.float64)
        nk = int(np.prod(ka.keep.shape)) // 3
        nq = int(np.prod(qa.keep.shape)) // 3
        dT = ctypes.c_double(0.0)
        dE = ctypes.c_double(0.0)
        if ka.device:
            import torch
            dg = torch.zeros(self.g_shape, dtype=torch.complex128, device=ka.keep.device) if want_dg else None
            dptr = dg.data_ptr() if want_dg else None
        else:
            dg = np.zeros(self.g_shape, dtype=np.complex128) if want_dg else None
            dptr = dg.ctypes.data if want_dg else None
        pr = _lib.Params(float(T), float(EF), float(sigma), float(omega_min), int(precision), 0)
        st = _stream_of(ka, qa, wa, ca)
        _check(lib.epw_linewidth_backward(self._h, nk, ka.ptr, nq, qa.ptr, wa.ptr, ctypes.byref(pr), ca.ptr,
                                          dptr, ctypes.byref(dT), ctypes.byref(dE), st))
        return dg, dT.value, dE.value


def launch_count() -> int:
    return int(_lib.load().epw_launch_count())


def plan_linewidth(nw: int, nat: int, nRe: int, nRp: int, nRph: int, nk: int, nq: int, precision: int = BF16X3,
                   same_ep: bool = False, same_eph: bool = False, polar: bool = False):
    """(workspace bytes, k per pass) that Model.linewidth takes for a model of this shape on nk x nq
    points with host inputs (epw_plan_linewidth): no model, no device work."""
    lib = _lib.load()
    ws = ctypes.c_size_t(0)
    kp = ctypes.c_int(0)
    _check(lib.epw_plan_linewidth(int(nw), int(nat), int(nRe), int(nRp), int(nRph), int(bool(same_ep)),
                                  int(bool(same_eph)), int(bool(polar)), int(nk), int(nq), int(precision),
                                  ctypes.byref(ws), ctypes.byref(kp)))
    return int(ws.value), int(kp.value)


def eliashberg(omega, lam, grid, sigma_ph: float, wq=None):
    """alpha^2 F on `grid` (Eq. isotropiceliash) from w_qnu and lambda_qnu [nq, 3nat] (epw_eliashberg)."""
    lib = _lib.load()
    oa, la, ga, wa = _Arg(omega, np.float64), _Arg(lam, np.float64), _Arg(grid, np.float64), _Arg(wq, np.float64)
    nq, nm = (oa.keep.shape[0], oa.keep.shape[1]) if oa.keep.ndim == 2 else (0, 0)
    if tuple(la.keep.shape) != tuple(oa.keep.shape):
        raise ValueError("omega and lambda must have the same shape [nq, nmodes]")
    ng = int(np.prod(ga.keep.shape))
    if ga.device:
        import torch
        out = torch.zeros(ng, dtype=torch.float64, device=ga.keep.device)
    else:
        out = np.zeros(ng)
    o = _Arg(out, np.float64)
    _check(lib.epw_eliashberg(nq, nm, oa.ptr, la.ptr, wa.ptr, ng, ga.ptr, float(sigma_ph), o.ptr,
                              _stream_of(oa, la, ga, wa, o)))
    return out


class Batch:
    """Many linewidth problems (possibly different models and sizes) as one CUDA graph.

    ``jobs`` is a list of dicts with keys model (Model), k, q (CUDA float64
    tensors [n, 3]), wq (CUDA tensor or None), T, EF, sigma, optional
    omega_min and precision, and optional out (CUDA float64 [nk, nw]; made
    here when absent).  Creating the batch autotunes, captures the graph and
    runs every job once; ``run()`` replays it on the current torch stream.
    Shapes and buffers are fixed; the contents of k, q, wq may change.
    """

    def __init__(self, jobs):
        import torch
        lib = _lib.load()
        self._keep = []
        self.outputs = []
        arr = (_lib.LinewidthJob * max(len(jobs), 1))()
        for i, j in enumerate(jobs):
            m = j["model"]
            ka, qa, wa = _Arg(j["k"], np.float64), _Arg(j["q"], np.float64), _Arg(j.get("wq"), np.float64)
            for a in (ka, qa) + ((wa,) if wa.keep is not None else ()):
                if not a.device:
                    raise ValueError("batch jobs take CUDA tensors")
            nk = int(np.prod(ka.keep.shape)) // 3
            nq = int(np.prod(qa.keep.shape)) // 3
            out = j.get("out")
            if out is None:
                out = torch.empty((nk, m.nw), dtype=torch.float64, device=ka.keep.device)
            oa = _Arg(out, np.float64)
            self._keep += [ka, qa, wa, oa, m]
            self.outputs.append(oa.keep)
            pr = _lib.Params(float(j["T"]), float(j["EF"]), float(j["sigma"]), float(j.get("omega_min", 1e-5)),
                             int(j.get("precision", FP64)), 0)
            arr[i] = _lib.LinewidthJob(m.handle, nk, nq, ka.ptr, qa.ptr, wa.ptr, pr, oa.ptr)
        self._jobs = arr
        h = ctypes.c_void_p()
        torch.cuda.synchronize()
        _check(lib.epw_batch_create(len(jobs), arr, ctypes.byref(h)))
        self._h = h

    def run(self):
        import torch
        _check(_lib.load().epw_batch_run(self._h, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
        return self.outputs

    def info(self):
        """(graph branches, workspace bytes, kernel nodes of the graph: the kernels one replay launches)."""
        b, w, n = ctypes.c_int(), ctypes.c_size_t(), ctypes.c_size_t()
        _check(_lib.load().epw_batch_info(self._h, ctypes.byref(b), ctypes.byref(w), ctypes.byref(n)))
        return b.value, w.value, n.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.load().epw_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
