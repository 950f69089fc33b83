"""FP64 CPU oracle for the Wannier-interpolated electron linewidth (EPW, Eq. linewidthel).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark may use it; the product path never does.  It shares no code
with the CUDA path (plain C in ``epw_oracle.c``, built here with gcc/OpenMP).

Parity status of each function (what pins it against something other than
itself is listed in the tests named):

* ``eigh``            -- pinned to LAPACK (numpy.linalg.eigh) and residuals
                         (tests/test_oracle_pins.py).
* ``bands``/``phonons`` -- closed-form tight-binding bands and spring-model
                         phonons; a two-atom chain with unequal masses (both
                         branches); time reversal; acoustic sum rule.
* ``g_wannier``       -- two-step (Rp then Re) order against the direct double
                         sum; round trip through a coarse grid; closed form.
* ``linewidth``       -- closed-form one-band model (no Fourier sum, no
                         eigensolve on the check side); the two-atom chain with
                         the vertex on either atom (per-atom masses in the mode
                         factors); constant-vertex (Einstein) reduction; gauge
                         invariance; non-negativity.
* ``selfenergy``      -- closed-form one-band Sigma(omega); the spectral function
                         point by point with its Re Sigma(0) shift; unit norm.
* polar vertex        -- one-band closed form at G = 0; the G sum (|n_i| <= 2,
                         anisotropic eps, full Born charges) against an integral
                         representation of the lattice sum; 1/|q| divergence.
* ``interp``          -- gauge-invariant degenerate-subspace sums against the
                         closed form and the symmetries above.
* ``linewidth_grad``  -- central finite differences of ``linewidth``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "epw_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libepw_oracle.so")
_lock = threading.Lock()
_lib = None

KB_EV = 8.617333262e-5


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP).  Returns the library path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-fopenmp",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Model(ctypes.Structure):
    _fields_ = [
        ("nw", ctypes.c_int), ("nat", ctypes.c_int), ("mass", ctypes.c_void_p),
        ("nRe", ctypes.c_int), ("Re", ctypes.c_void_p), ("wRe", ctypes.c_void_p), ("H", ctypes.c_void_p),
        ("nRph", ctypes.c_int), ("Rph", ctypes.c_void_p), ("wRph", ctypes.c_void_p), ("Phi", ctypes.c_void_p),
        ("nRp", ctypes.c_int), ("Rp", ctypes.c_void_p), ("wRp", ctypes.c_void_p), ("g", ctypes.c_void_p),
        ("polar", ctypes.c_int), ("pA", ctypes.c_void_p), ("peps", ctypes.c_void_p), ("pZ", ctypes.c_void_p),
        ("palpha", ctypes.c_double), ("ppref", ctypes.c_double), ("pgmax", ctypes.c_int),
    ]


class _Params(ctypes.Structure):
    _fields_ = [("T", ctypes.c_double), ("EF", ctypes.c_double),
                ("sigma", ctypes.c_double), ("omega_min", ctypes.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I = ctypes.c_int
            lib.oracle_eigh.argtypes = [I, P, P, P]
            lib.oracle_eigh.restype = I
            for name, args in [
                ("oracle_bands", [P, I, P, P, P]),
                ("oracle_phonons", [P, I, P, P, P]),
                ("oracle_interp", [P, I, P, I, P, ctypes.c_double, P, P, P, P]),
                ("oracle_linewidth", [P, I, P, I, P, P, P, P]),
                ("oracle_linewidth_grad", [P, I, P, I, P, P, P, P, P, P, P]),
                ("oracle_phonon_self", [P, I, P, P, I, P, P, P, P, P, P]),
                ("oracle_selfenergy", [P, I, P, I, P, P, P, ctypes.c_double, I, P, P, P]),
            ]:
                getattr(lib, name).argtypes = args
                getattr(lib, name).restype = I
            lib.oracle_g_wannier_direct.argtypes = [P, P, P, P]
            lib.oracle_g_wannier_direct.restype = None
            lib.oracle_g_Re_q.argtypes = [P, P, P]
            lib.oracle_g_Re_q.restype = None
            for name in ("oracle_bose", "oracle_gauss"):
                getattr(lib, name).argtypes = [ctypes.c_double, ctypes.c_double]
                getattr(lib, name).restype = ctypes.c_double
            lib.oracle_gauss_diff.argtypes = [ctypes.c_double] * 3
            lib.oracle_gauss_diff.restype = ctypes.c_double
            for name in ("oracle_fermi", "oracle_fermi_slope"):
                getattr(lib, name).argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
                getattr(lib, name).restype = ctypes.c_double
            lib.oracle_eliashberg.argtypes = [I, I, P, P, P, I, P, ctypes.c_double, P]
            lib.oracle_eliashberg.restype = None
            lib.oracle_fermi_diff.argtypes = [ctypes.c_double] * 4
            lib.oracle_fermi_diff.restype = ctypes.c_double
            lib.oracle_num_threads.argtypes = []
            lib.oracle_num_threads.restype = I
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class _Bound:
    """Keeps contiguous copies alive while the C struct points at them."""

    def __init__(self, m):
        c = np.ascontiguousarray
        self.keep = [
            c(m.mass, np.float64), c(m.Re, np.int32), c(m.wRe, np.float64), c(m.H, np.complex128),
            c(m.Rph, np.int32), c(m.wRph, np.float64), c(m.Phi, np.complex128),
            c(m.Rp, np.int32), c(m.wRp, np.float64), c(m.g, np.complex128),
        ]
        k = self.keep
        pol = getattr(m, "polar", None)
        if pol is not None:
            self.keep += [c(pol.A, np.float64), c(pol.eps_inf, np.float64), c(pol.Zstar, np.float64)]
            pargs = (1, _p(k[10]).value, _p(k[11]).value, _p(k[12]).value, float(pol.alpha), float(pol.prefactor),
                     int(pol.gmax))
        else:
            pargs = (0, None, None, None, 0.0, 0.0, 0)
        self.s = _Model(m.nw, m.nat, _p(k[0]).value,
                        len(m.Re), _p(k[1]).value, _p(k[2]).value, _p(k[3]).value,
                        len(m.Rph), _p(k[4]).value, _p(k[5]).value, _p(k[6]).value,
                        len(m.Rp), _p(k[7]).value, _p(k[8]).value, _p(k[9]).value, *pargs)

    @property
    def ptr(self):
        return ctypes.cast(ctypes.pointer(self.s), ctypes.c_void_p)


def _pts(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1, 3))


def num_threads() -> int:
    return _load().oracle_num_threads()


def eigh(A: np.ndarray):
    """Cyclic Jacobi on the Hermitian part of A: (ascending eigenvalues, eigenvector columns, sweeps)."""
    lib = _load()
    n = A.shape[0]
    a = np.ascontiguousarray(A, dtype=np.complex128).copy()
    w = np.zeros(n)
    V = np.zeros((n, n), dtype=np.complex128)
    sweeps = lib.oracle_eigh(n, _p(a), _p(w), _p(V))
    if sweeps < 0:
        raise RuntimeError("oracle eigh did not converge")
    return w, V, sweeps


def bands(model, k):
    lib = _load()
    k = _pts(k)
    b = _Bound(model)
    eps = np.zeros((len(k), model.nw))
    U = np.zeros((len(k), model.nw, model.nw), dtype=np.complex128)
    if lib.oracle_bands(b.ptr, len(k), _p(k), _p(eps), _p(U)) != 0:
        raise RuntimeError("oracle bands: eigensolve did not converge")
    return eps, U


def phonons(model, q):
    lib = _load()
    q = _pts(q)
    b = _Bound(model)
    nm = 3 * model.nat
    w = np.zeros((len(q), nm))
    ev = np.zeros((len(q), nm, nm), dtype=np.complex128)
    if lib.oracle_phonons(b.ptr, len(q), _p(q), _p(w), _p(ev)) != 0:
        raise RuntimeError("oracle phonons: eigensolve did not converge")
    return w, ev


def g_wannier_direct(model, k, q):
    """g_{kappa alpha}(k,q) in the Wannier basis by the direct (Re,Rp) double sum: [3nat,nw,nw]."""
    lib = _load()
    b = _Bound(model)
    out = np.zeros((3 * model.nat, model.nw, model.nw), dtype=np.complex128)
    lib.oracle_g_wannier_direct(b.ptr, _p(_pts(k)[0].copy()), _p(_pts(q)[0].copy()), _p(out))
    return out


def g_Re_q(model, q):
    """First interpolation step g(Re,q): [nRe,3nat,nw,nw]."""
    lib = _load()
    b = _Bound(model)
    out = np.zeros((len(model.Re), 3 * model.nat, model.nw, model.nw), dtype=np.complex128)
    lib.oracle_g_Re_q(b.ptr, _p(_pts(q)[0].copy()), _p(out))
    return out


def interp(model, k, q, omega_min=1e-5):
    """(eps_k [nk,nw], eps_kq [nk,nq,nw], omega [nq,3nat], g [nk,nq,3nat,nw,nw])."""
    lib = _load()
    k, q = _pts(k), _pts(q)
    b = _Bound(model)
    nk, nq, nw, nm = len(k), len(q), model.nw, 3 * model.nat
    eps_k = np.zeros((nk, nw))
    eps_kq = np.zeros((nk, nq, nw))
    omega = np.zeros((nq, nm))
    g = np.zeros((nk, nq, nm, nw, nw), dtype=np.complex128)
    if lib.oracle_interp(b.ptr, nk, _p(k), nq, _p(q), omega_min, _p(eps_k), _p(eps_kq), _p(omega), _p(g)) != 0:
        raise RuntimeError("oracle interp: eigensolve did not converge")
    return eps_k, eps_kq, omega, g


def linewidth(model, k, q, wq=None, T=300.0, EF=0.0, sigma=0.05, omega_min=1e-5):
    """Im Sigma_nk [nk, nw] in eV (Eq. linewidthel, on shell)."""
    lib = _load()
    k, q = _pts(k), _pts(q)
    b = _Bound(model)
    wq_a = None if wq is None else np.ascontiguousarray(wq, dtype=np.float64)
    out = np.zeros((len(k), model.nw))
    pr = _Params(T, EF, sigma, omega_min)
    rc = lib.oracle_linewidth(b.ptr, len(k), _p(k), len(q), _p(q),
                              None if wq_a is None else _p(wq_a), ctypes.byref(pr), _p(out))
    if rc != 0:
        raise RuntimeError("oracle linewidth: eigensolve did not converge")
    return out


def phonon_self(model, k, q, wk=None, T=300.0, EF=0.0, sigma=0.05, omega_min=1e-5):
    """(Pi''_qnu [nq, 3nat] (Eq. linewidthph, on shell), lambda_qnu [nq, 3nat] (Eq. lambdaEQ),
    nesting zeta_q [nq] (Eq. nestingfct), N(E_F)) from sums over the k list (weights wk, default 1/nk)."""
    lib = _load()
    k, q = _pts(k), _pts(q)
    b = _Bound(model)
    nm = 3 * model.nat
    wk_a = None if wk is None else np.ascontiguousarray(wk, dtype=np.float64)
    pi = np.zeros((len(q), nm))
    lam = np.zeros((len(q), nm))
    zeta = np.zeros(len(q))
    dos = np.zeros(1)
    pr = _Params(T, EF, sigma, omega_min)
    rc = lib.oracle_phonon_self(b.ptr, len(k), _p(k), None if wk_a is None else _p(wk_a), len(q), _p(q),
                                ctypes.byref(pr), _p(pi), _p(lam), _p(zeta), _p(dos))
    if rc != 0:
        raise RuntimeError("oracle phonon self-energy: eigensolve did not converge")
    return pi, lam, zeta, float(dos[0])


def selfenergy(model, k, q, omega, wq=None, T=300.0, EF=0.0, delta=0.01, omega_min=1e-5):
    """(Sigma_nk(omega) [nk, nw, nomega] complex (Eq. elselfenergy, i delta broadening, omega from E_F),
    A_nk(omega) [nk, nw, nomega] (Eq. spectral_funct))."""
    lib = _load()
    k, q = _pts(k), _pts(q)
    b = _Bound(model)
    om = np.ascontiguousarray(omega, dtype=np.float64)
    wq_a = None if wq is None else np.ascontiguousarray(wq, dtype=np.float64)
    sig = np.zeros((len(k), model.nw, len(om)), dtype=np.complex128)
    spec = np.zeros((len(k), model.nw, len(om)))
    pr = _Params(T, EF, 1.0, omega_min)
    rc = lib.oracle_selfenergy(b.ptr, len(k), _p(k), len(q), _p(q), None if wq_a is None else _p(wq_a),
                               ctypes.byref(pr), float(delta), len(om), _p(om), _p(sig), _p(spec))
    if rc != 0:
        raise RuntimeError("oracle self-energy: eigensolve did not converge")
    return sig, spec


def eliashberg(omega, lam, grid, sigma_ph, wq=None):
    """alpha^2 F(omega) on `grid` (Eq. isotropiceliash) from w_qnu, lambda_qnu [nq, nm]."""
    lib = _load()
    om = np.ascontiguousarray(omega, dtype=np.float64)
    la = np.ascontiguousarray(lam, dtype=np.float64)
    gr = np.ascontiguousarray(grid, dtype=np.float64)
    wq_a = None if wq is None else np.ascontiguousarray(wq, dtype=np.float64)
    out = np.zeros(len(gr))
    lib.oracle_eliashberg(om.shape[0], om.shape[1], _p(om), _p(la), None if wq_a is None else _p(wq_a), len(gr),
                          _p(gr), float(sigma_ph), _p(out))
    return out


def linewidth_grad(model, k, q, wq=None, T=300.0, EF=0.0, sigma=0.05, omega_min=1e-5, cot=None):
    """Adjoint of L = sum_{k,n} cot_nk Im Sigma_nk: (dg like model.g, dL/dT, dL/dE_F)."""
    lib = _load()
    k, q = _pts(k), _pts(q)
    b = _Bound(model)
    wq_a = None if wq is None else np.ascontiguousarray(wq, dtype=np.float64)
    c = np.ones((len(k), model.nw)) if cot is None else np.ascontiguousarray(cot, dtype=np.float64)
    dg = np.zeros_like(np.ascontiguousarray(model.g, dtype=np.complex128))
    dT = ctypes.c_double(0.0)
    dE = ctypes.c_double(0.0)
    pr = _Params(T, EF, sigma, omega_min)
    rc = lib.oracle_linewidth_grad(b.ptr, len(k), _p(k), len(q), _p(q),
                                   None if wq_a is None else _p(wq_a), ctypes.byref(pr), _p(c),
                                   _p(dg), ctypes.byref(dT), ctypes.byref(dE))
    if rc != 0:
        raise RuntimeError("oracle linewidth_grad: eigensolve did not converge")
    return dg, dT.value, dE.value


def bose(w, T):
    return _load().oracle_bose(float(w), float(T))


def fermi(e, EF, T):
    return _load().oracle_fermi(float(e), float(EF), float(T))


def fermi_slope(e, EF, T):
    return _load().oracle_fermi_slope(float(e), float(EF), float(T))


def fermi_diff(ea, eb, EF, T):
    return _load().oracle_fermi_diff(float(ea), float(eb), float(EF), float(T))


def gauss(x, sigma):
    return _load().oracle_gauss(float(x), float(sigma))


def gauss_diff(x, w, sigma):
    """delta(x + w) - delta(x - w) of the Gaussian delta, in the sinh form without cancellation."""
    return _load().oracle_gauss_diff(float(x), float(w), float(sigma))
