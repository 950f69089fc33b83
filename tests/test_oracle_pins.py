"""Pins of the FP64 CPU oracle against things other than itself.

Each check would fail for a plausible slip in the oracle (dropped term, wrong
sign or index, transposed operand):

* eigensolver      vs LAPACK (numpy.linalg.eigh) and HU = U eps residuals;
* bands / phonons  vs the closed forms of a nearest-neighbour model;
* Fourier sums     round trip through a coarse grid (exact for any data), both
                   the direct double sum and the first (Rp) step of the
                   two-step order, with Wigner-Seitz weights for even grids;
* two-step order   vs the direct double sum, rotated with LAPACK eigenvectors
                   (also a gauge-invariance check: different eigensolvers);
* gauge            random unitaries inside exactly degenerate subspaces of U_k,
                   U_k+q and e_q leave the degenerate-block sums of |g|^2 unchanged;
* linewidth        vs the closed-form one-band model (no Fourier sum and no
                   eigensolve on the checking side);
* symmetries       time reversal with real inputs, acoustic sum rule,
                   non-negativity;
* occupations      closed forms, limits, n(-w) = -1 - n(w), unit-norm delta;
* adjoint          central finite differences of the forward oracle;
* masses           a two-atom chain with unequal masses: both phonon branches and
                   the linewidth with the vertex on either atom (1/sqrt(M_k M_k')
                   in D(q), 1/sqrt(2 M_k w) per atom in the mode factors);
* constant vertex  Einstein phonons with g_a(k,q) = c_a: Im Sigma from the band
                   energies alone (degenerate modes summed);
* spectral fn      A_nk(w) point by point from the closed-form Sigma of the
                   one-band model with its Re Sigma(0) shift;
* polar G sum      |n_i| <= 2, diagonal anisotropic eps, full Born charges,
                   against an integral representation of the lattice sum.
"""
import dataclasses
import itertools
import math

import numpy as np
import pytest

import workloads as W
from tests._util import degenerate_sums, ws_vectors

KB = 8.617333262e-5


def test_eigh_matches_lapack(oracle_lib):
    rng = np.random.default_rng(1)
    for n in (1, 2, 3, 4, 5, 6, 8, 9, 12, 18):
        A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        A = A + A.conj().T
        w, V, _ = oracle_lib.eigh(A)
        assert np.allclose(w, np.linalg.eigvalsh(A), atol=1e-12 * n)
        assert np.abs(A @ V - V * w).max() < 1e-12 * n
        assert np.abs(V.conj().T @ V - np.eye(n)).max() < 1e-13 * n
        assert np.all(np.diff(w) >= 0)


def test_eigh_degenerate_and_nonhermitian_input(oracle_lib):
    rng = np.random.default_rng(2)
    n = 6
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    d = np.array([-1.0, -1.0, 0.5, 0.5, 0.5, 2.0])
    A = Q @ np.diag(d) @ Q.conj().T
    w, V, _ = oracle_lib.eigh(A)
    assert np.allclose(w, d, atol=1e-13)
    assert np.abs(A @ V - V * w).max() < 1e-12
    # Only the Hermitian part enters.
    B = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    w2, _, _ = oracle_lib.eigh(B)
    assert np.allclose(w2, np.linalg.eigvalsh(0.5 * (B + B.conj().T)), atol=1e-12)


def _tb():
    return W.tight_binding_model(eps0=0.2, t=0.5, K=0.01, g0=0.05, mass=1.3)


def test_tight_binding_bands_and_phonons(oracle_lib):
    m = _tb()
    rng = np.random.default_rng(3)
    k = rng.random((20, 3))
    eps, _ = oracle_lib.bands(m, k)
    ref = 0.2 - 2 * 0.5 * np.cos(2 * np.pi * k).sum(axis=1)
    assert np.allclose(eps[:, 0], ref, atol=1e-13)
    w, ev = oracle_lib.phonons(m, k)
    wref = np.sort(2 * np.sqrt(0.01 / 1.3) * np.abs(np.sin(np.pi * k)), axis=1)
    assert np.allclose(w, wref, atol=1e-12)


def test_tight_binding_vertex_closed_form(oracle_lib):
    m = _tb()
    rng = np.random.default_rng(4)
    for _ in range(5):
        k, q = rng.random(3), rng.random(3)
        g = oracle_lib.g_wannier_direct(m, k, q)
        assert np.allclose(g[:, 0, 0], 0.05 * np.sin(2 * np.pi * q), atol=1e-14)
        gReq = oracle_lib.g_Re_q(m, q)
        i0 = [i for i, R in enumerate(m.Re) if not R.any()][0]
        assert np.allclose(gReq[i0, :, 0, 0], 0.05 * np.sin(2 * np.pi * q), atol=1e-14)
        assert np.abs(np.delete(gReq, i0, axis=0)).max() == 0.0


def _bose(w, T):
    if T == 0 or w / (KB * T) > 700:
        return 0.0
    return 1.0 / (math.exp(w / (KB * T)) - 1.0)


def _fermi(e, EF, T):
    if T == 0:
        return 1.0 if e < EF else (0.0 if e > EF else 0.5)
    x = (e - EF) / (KB * T)
    return 0.0 if x > 700 else 1.0 / (math.exp(x) + 1.0)


def _gauss(x, s):
    return math.exp(-(x / s) ** 2) / (s * math.sqrt(math.pi))


def _tb_linewidth_closed_form(k, q, T, EF, sigma, eps0=0.2, t=0.5, K=0.01, g0=0.05, M=1.3, wmin=1e-5):
    out = np.zeros(len(k))
    for ik, kk in enumerate(k):
        ek = eps0 - 2 * t * np.cos(2 * np.pi * kk).sum()
        s = 0.0
        for qq in q:
            ekq = eps0 - 2 * t * np.cos(2 * np.pi * (kk + qq)).sum()
            f = _fermi(ekq, EF, T)
            for a in range(3):
                w = 2 * math.sqrt(K / M) * abs(math.sin(math.pi * qq[a]))
                if w < wmin:
                    continue
                g2 = g0**2 * math.sin(2 * math.pi * qq[a]) ** 2 / (2 * M * w)
                n = _bose(w, T)
                s += g2 * ((n + f) * _gauss(ek - ekq + w, sigma) + (n + 1 - f) * _gauss(ek - ekq - w, sigma))
        out[ik] = math.pi * s / len(q)
    return out


@pytest.mark.parametrize("T,EF,sigma", [(300.0, 0.1, 0.05), (10.0, -0.3, 0.02), (0.0, 0.0, 0.08)])
def test_linewidth_closed_form_one_band(oracle_lib, T, EF, sigma):
    m = _tb()
    k = W.uniform_grid(3) + 0.05
    q = W.uniform_grid(6)
    got = oracle_lib.linewidth(m, k, q, None, T, EF, sigma)[:, 0]
    ref = _tb_linewidth_closed_form(k, q, T, EF, sigma)
    assert np.all(ref > 0)
    assert np.allclose(got, ref, rtol=1e-11, atol=1e-14 * ref.max())


def _inverse_dft(vals, pts, R):
    """X(R) = (1/Npts) sum_p e^{-2 pi i p.R} vals[p]   (vals [Npts, ...])."""
    ph = np.exp(-2j * np.pi * (pts @ R.T))  # [Npts, nR]
    return np.tensordot(ph, vals, axes=(0, 0)) / len(pts)


@pytest.mark.parametrize("N", [2, 3])
def test_round_trip_through_coarse_grid(oracle_lib, N):
    """Wannierize random coarse-grid data, interpolate back at the same points: exact."""
    rng = np.random.default_rng(10 + N)
    R, wR = ws_vectors(N)
    nw, nat = 2, 1
    kc = W.uniform_grid(N)
    Hc = rng.standard_normal((len(kc), nw, nw)) + 1j * rng.standard_normal((len(kc), nw, nw))
    Hc = Hc + Hc.conj().transpose(0, 2, 1)
    HR = _inverse_dft(Hc, kc, R)
    gc = rng.standard_normal((len(kc), len(kc), 3, nw, nw)) + 1j * rng.standard_normal((len(kc), len(kc), 3, nw, nw))
    tmp = _inverse_dft(gc, kc, R)  # over k -> [nR, nq, ...]
    gR = _inverse_dft(np.moveaxis(tmp, 1, 0), kc, R)  # over q -> [nRp, nRe, ...]
    gR = np.moveaxis(gR, 0, 1).copy()  # [nRe, nRp, ...]
    m = W.WannierModel("sc", nw, nat, np.ones(1), R, wR, HR, R, wR, np.zeros((len(R), 3, 3), complex), R, wR, gR)
    eps, _ = oracle_lib.bands(m, kc)
    assert np.allclose(eps, np.linalg.eigvalsh(Hc), atol=1e-12)
    for ik, iq in [(0, 0), (1, len(kc) - 1), (len(kc) // 2, 3)]:
        got = oracle_lib.g_wannier_direct(m, kc[ik], kc[iq])
        assert np.allclose(got, gc[ik, iq], atol=1e-12)
        # first step of the two-step order: g(Re,q) = inverse DFT over k of g_c(., q)
        got_req = oracle_lib.g_Re_q(m, kc[iq]) * wR[:, None, None, None]
        assert np.allclose(got_req, _inverse_dft(gc[:, iq], kc, R) * wR[:, None, None, None], atol=1e-12)


def _small_model(seed, nw=3, nat=2, real=False):
    rng = np.random.default_rng(seed)
    return W.make_model("diamond", nw, nat, [1.0, 1.2], 20, 20, rng, real=real)


def test_two_step_order_matches_direct_sum_and_lapack_rotation(oracle_lib):
    m = _small_model(20)
    rng = np.random.default_rng(21)
    k = rng.random((3, 3))
    q = rng.random((4, 3))
    eps_k, eps_kq, omega, g = oracle_lib.interp(m, k, q)
    nw, nm = m.nw, 3 * m.nat
    for ik in range(len(k)):
        for iq in range(len(q)):
            gw = oracle_lib.g_wannier_direct(m, k[ik], q[iq])
            # LAPACK eigenvectors (a different gauge from the oracle's Jacobi)
            Hk = sum(np.exp(2j * np.pi * k[ik] @ R) * H for R, H in zip(m.Re, m.H))
            Hkq = sum(np.exp(2j * np.pi * (k[ik] + q[iq]) @ R) * H for R, H in zip(m.Re, m.H))
            D = sum(np.exp(2j * np.pi * q[iq] @ R) * P for R, P in zip(m.Rph, m.Phi))
            msq = np.repeat(np.sqrt(m.mass), 3)
            D = D / np.outer(msq, msq)
            ek, Uk = np.linalg.eigh(Hk)
            ekq, Ukq = np.linalg.eigh(Hkq)
            w2, e = np.linalg.eigh(D)
            w = np.sqrt(np.abs(w2)) * np.sign(w2)
            assert np.allclose(ek, eps_k[ik], atol=1e-12)
            assert np.allclose(ekq, eps_kq[ik, iq], atol=1e-12)
            assert np.allclose(w, omega[iq], atol=1e-12)
            keep = w >= 1e-5
            mrep = np.repeat(m.mass, 3)
            E = np.where(keep[None, :], e / np.sqrt(2 * np.outer(mrep, np.where(keep, w, 1.0))), 0)
            gB = np.einsum("im,aij,jn->amn", Ukq.conj(), gw, Uk)
            ref = np.einsum("amn,av->vmn", gB, E)
            a = degenerate_sums(np.abs(g[ik, iq]) ** 2, ekq, ek, w, 1e-8)
            b = degenerate_sums(np.abs(ref) ** 2, ekq, ek, w, 1e-8)
            assert np.allclose(a, b, rtol=1e-10, atol=1e-14 * b.max())


def test_time_reversal_with_real_inputs(oracle_lib):
    m = _small_model(30, nw=2, nat=2, real=True)
    rng = np.random.default_rng(31)
    k = rng.random((4, 3))
    q = W.uniform_grid(3)  # closed under q -> -q (mod 1)
    e1, _ = oracle_lib.bands(m, k)
    e2, _ = oracle_lib.bands(m, -k)
    assert np.allclose(e1, e2, atol=1e-12)
    w1, _ = oracle_lib.phonons(m, k)
    w2, _ = oracle_lib.phonons(m, -k)
    assert np.allclose(w1, w2, atol=1e-12)
    s1 = oracle_lib.linewidth(m, k, q, None, 300.0, 0.0, 0.1)
    s2 = oracle_lib.linewidth(m, -k, q, None, 300.0, 0.0, 0.1)
    assert np.allclose(s1, s2, rtol=1e-10, atol=1e-14)
    a = oracle_lib.interp(m, k[:2], q[:5])
    b = oracle_lib.interp(m, -k[:2], -q[:5])
    for ik in range(2):
        for iq in range(5):
            sa = degenerate_sums(np.abs(a[3][ik, iq]) ** 2, a[1][ik, iq], a[0][ik], a[2][iq], 1e-8)
            sb = degenerate_sums(np.abs(b[3][ik, iq]) ** 2, b[1][ik, iq], b[0][ik], b[2][iq], 1e-8)
            assert np.allclose(sa, sb, rtol=1e-9, atol=1e-14)


def test_acoustic_sum_rule_and_stability(oracle_lib):
    m = _small_model(40)
    w, _ = oracle_lib.phonons(m, np.zeros((1, 3)))
    assert np.abs(w[0, :3]).max() < 1e-6
    assert w[0, 3:].min() > 1e-4
    wq, _ = oracle_lib.phonons(m, np.random.default_rng(41).random((50, 3)))
    assert wq.min() > 0 and wq.max() <= 0.1 + 1e-12


def test_linewidth_non_negative_and_weighting(oracle_lib):
    m = _small_model(50, nw=2, nat=1)
    rng = np.random.default_rng(51)
    k = rng.random((3, 3))
    q = rng.random((10, 3))
    s = oracle_lib.linewidth(m, k, q, None, 100.0, 0.0, 0.05)
    assert np.all(s >= 0)
    # explicit weights: the BZ sum is linear in w_q
    wq = rng.random(10)
    s1 = oracle_lib.linewidth(m, k, q, wq, 100.0, 0.0, 0.05)
    parts = [oracle_lib.linewidth(m, k, q[i:i + 1], wq[i:i + 1], 100.0, 0.0, 0.05) for i in range(10)]
    assert np.allclose(s1, sum(parts), rtol=1e-12)


def test_occupations_and_delta(oracle_lib):
    for w, T in [(0.01, 300.0), (0.2, 50.0), (1e-4, 10.0)]:
        assert math.isclose(oracle_lib.bose(w, T), 1 / math.expm1(w / (KB * T)), rel_tol=1e-14)
        assert math.isclose(oracle_lib.bose(-w, T), -1 - oracle_lib.bose(w, T), rel_tol=1e-12)
    assert oracle_lib.bose(0.05, 0.0) == 0.0
    assert oracle_lib.bose(5.0, 1.0) == 0.0  # overflow-safe limit
    for e, EF, T in [(0.1, 0.0, 300.0), (-0.02, 0.01, 77.0), (0.5, 0.0, 300.0)]:
        assert math.isclose(oracle_lib.fermi(e, EF, T), 1 / (math.exp((e - EF) / (KB * T)) + 1), rel_tol=1e-13)
        assert math.isclose(oracle_lib.fermi(e, EF, T) + oracle_lib.fermi(2 * EF - e, EF, T), 1.0, rel_tol=1e-14)
    assert oracle_lib.fermi(-0.1, 0.0, 0.0) == 1.0 and oracle_lib.fermi(0.1, 0.0, 0.0) == 0.0
    assert oracle_lib.fermi(0.0, 0.0, 0.0) == 0.5
    # f (1 - f) against the occupations where 1 - f is exact enough, against the
    # slope -kT df/de by central differences, and against exp(-|x|) deep in the tails.
    for e, EF, T in [(0.03, 0.0, 300.0), (-0.01, 0.02, 77.0)]:
        f = oracle_lib.fermi(e, EF, T)
        assert math.isclose(oracle_lib.fermi_slope(e, EF, T), f * (1 - f), rel_tol=1e-13)
        h = 1e-7
        d = (oracle_lib.fermi(e + h, EF, T) - oracle_lib.fermi(e - h, EF, T)) / (2 * h)
        assert math.isclose(oracle_lib.fermi_slope(e, EF, T), -KB * T * d, rel_tol=1e-6)
    for x in (40.0, -40.0, 300.0):
        T = 300.0
        assert math.isclose(oracle_lib.fermi_slope(x * KB * T, 0.0, T), math.exp(-abs(x)), rel_tol=1e-12)
    assert oracle_lib.fermi_slope(0.1, 0.0, 0.0) == 0.0
    s = 0.02
    x = np.linspace(-12 * s, 12 * s, 20001)
    vals = np.array([oracle_lib.gauss(v, s) for v in x])
    assert abs(np.trapezoid(vals, x) - 1.0) < 1e-10
    assert math.isclose(oracle_lib.gauss(0.0, s), 1 / (s * math.sqrt(math.pi)), rel_tol=1e-15)
    assert math.isclose(oracle_lib.gauss(s, s), math.exp(-1) / (s * math.sqrt(math.pi)), rel_tol=1e-15)


def test_adjoint_matches_finite_differences(oracle_lib):
    rng = np.random.default_rng(60)
    m = W.make_model("sc", 2, 1, [1.0], None, None, rng, box=1, omega_max=0.2)
    k = rng.random((3, 3))
    q = rng.random((6, 3))
    T, EF, sig = 300.0, 0.2, 0.2
    cot = rng.random((3, 2))
    dg, dT, dEF = oracle_lib.linewidth_grad(m, k, q, None, T, EF, sig, cot=cot)

    def L(model, T=T, EF=EF):
        return float((oracle_lib.linewidth(model, k, q, None, T, EF, sig) * cot).sum())

    h = 1e-6
    L0 = L(m)
    assert L0 > 0
    idxs = [tuple(int(rng.integers(s)) for s in m.g.shape) for _ in range(6)]
    for idx in idxs:
        for part, unit in (("re", 1.0), ("im", 1j)):
            gp = m.g.copy()
            gm = m.g.copy()
            gp[idx] += h * unit
            gm[idx] -= h * unit
            mp = W.WannierModel(**{**m.__dict__, "g": gp})
            mm = W.WannierModel(**{**m.__dict__, "g": gm})
            fd = (L(mp) - L(mm)) / (2 * h)
            an = dg[idx].real if part == "re" else dg[idx].imag
            assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3 * np.abs(dg).max()), (idx, part, fd, an)
    fdT = (L(m, T=T + 1e-3) - L(m, T=T - 1e-3)) / 2e-3
    assert abs(fdT - dT) <= 1e-6 * abs(dT)
    fdE = (L(m, EF=EF + 1e-6) - L(m, EF=EF - 1e-6)) / 2e-6
    assert abs(fdE - dEF) <= 1e-6 * abs(dEF)


def test_fermi_difference_without_cancellation(oracle_lib):
    """f(ea) - f(eb) against 600-digit arithmetic (the plain difference of the two occupations),
    where forming two rounded double occupations cancels."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 600
    T, EF = 300.0, 0.1
    kT = KB * T
    for xa, xb in [(1.0, 2.0), (-3.0, 5.0), (40.0, 40.001), (-40.0, -40.0001), (-30.0, 29.0), (25.0, -31.0),
                   (1e-3, -1e-3), (300.0, 301.0), (-500.0, -400.0)]:
        ea, eb = EF + xa * kT, EF + xb * kT
        # the same rounded arguments as the oracle forms (the conditioning of b - a is the input's)
        a = mpmath.mpf((ea - EF) / (KB * T))
        b = mpmath.mpf((eb - EF) / (KB * T))
        ref = float(1 / (1 + mpmath.e ** a) - 1 / (1 + mpmath.e ** b))
        got = oracle_lib.fermi_diff(ea, eb, EF, T)
        assert abs(got - ref) <= 1e-13 * abs(ref) + 1e-300, (xa, xb, got, ref)
    assert oracle_lib.fermi_diff(-0.1, 0.1, 0.0, 0.0) == 1.0
    assert oracle_lib.fermi_diff(0.0, 0.1, 0.0, 0.0) == 0.5


def test_gauss_difference_without_cancellation(oracle_lib):
    """delta(x + w) - delta(x - w) of the Gaussian delta against 100-digit arithmetic (the plain
    difference of the two Gaussians), from w ~ 1e-9 sigma (where two rounded double Gaussians
    cancel to all but a few digits) through w ~ sigma and across the switch to the plain
    difference at |2 x w| = sigma^2.  Also the symmetries: odd in x, odd in w."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 100
    sig = 0.05
    for a in (-3.0, -1.2, -0.3, -1e-4, 0.0, 2e-6, 0.25, 0.9, 1.7, 4.0):
        for b in (1e-9, 3e-6, 1e-3, 0.02, 0.3, 0.55, 1.0, 2.5):
            x, w = a * sig, b * sig
            X, Wm, S = mpmath.mpf(x), mpmath.mpf(w), mpmath.mpf(sig)
            ref = float((mpmath.e ** (-((X + Wm) / S) ** 2) - mpmath.e ** (-((X - Wm) / S) ** 2))
                        / (S * mpmath.sqrt(mpmath.pi)))
            got = oracle_lib.gauss_diff(x, w, sig)
            assert abs(got - ref) <= 1e-13 * abs(ref) + 1e-300, (a, b, got, ref)
            assert oracle_lib.gauss_diff(-x, w, sig) == -got
            assert oracle_lib.gauss_diff(x, -w, sig) == -got
    # the plain difference of two double Gaussians loses most digits at w = 1e-9 sigma
    x, w = 0.5 * sig, 1e-9 * sig
    plain = oracle_lib.gauss(x + w, sig) - oracle_lib.gauss(x - w, sig)
    exact = oracle_lib.gauss_diff(x, w, sig)
    assert abs(plain - exact) > 1e-9 * abs(exact)


def test_adjoint_fermi_level_with_soft_modes(oracle_lib):
    """dL/dE_F weights each term by d+ - d-, which is O(w / sigma) for soft modes: with every
    phonon below sigma / 50 (a soft spring), the oracle's sinh form of the difference still
    matches a central finite difference of the linewidth in E_F."""
    rng = np.random.default_rng(61)
    m = W.make_model("sc", 2, 1, [1.0], None, None, rng, box=1, omega_max=0.002)
    k = rng.random((3, 3))
    q = rng.random((6, 3))
    T, EF, sig = 300.0, 0.2, 0.2
    cot = rng.random((3, 2))
    _, _, dEF = oracle_lib.linewidth_grad(m, k, q, None, T, EF, sig, cot=cot, omega_min=1e-7)

    def L(EF):
        return float((oracle_lib.linewidth(m, k, q, None, T, EF, sig, omega_min=1e-7) * cot).sum())

    fdE = (L(EF + 1e-5) - L(EF - 1e-5)) / 2e-5
    assert abs(dEF) > 0
    assert abs(fdE - dEF) <= 1e-6 * abs(dEF), (fdE, dEF)


# ------------------------------------------------- phonon self-energy (oracle)
def _two_band_tb(eps=(-0.3, 0.4), t=0.5, K=0.01, M=1.3, c=((0.05, 0.03), (0.08, 0.02))):
    """Two bands that never mix (H(k) diagonal, band 0 below band 1 everywhere) with
    g_mn,a(Re=0, Rp=+-e_a) = -+ i c_mn / 2, so that g_mn,a(k,q) = c_mn sin(2 pi q_a)."""
    m = W.tight_binding_model(eps0=0.0, t=t, K=K, g0=1.0, mass=M)
    nR = len(m.Re)
    H = np.zeros((nR, 2, 2), dtype=np.complex128)
    g = np.zeros((nR, nR, 3, 2, 2), dtype=np.complex128)
    for b in range(2):
        H[:, b, b] = m.H[:, 0, 0]
        i0 = [i for i, R in enumerate(m.Re) if not R.any()][0]
        H[i0, b, b] = eps[b]
    for mm in range(2):
        for n in range(2):
            g[:, :, :, mm, n] = m.g[:, :, :, 0, 0] * c[mm][n]
    return dataclasses.replace(m, nw=2, H=H, g=g), eps, t, K, M, np.array(c)


def _phonon_closed_form(k, q, T, EF, sigma, bands, K, M, c, wmin=1e-5):
    """Pi'', lambda, zeta, N(E_F) for models with k-independent |g_mn,a|^2 = c_mn^2 sin^2(2 pi q_a) / (2 M w_a)
    and band energies bands(k) -> [nw]; modes sorted by frequency like the oracle's."""
    nk = len(k)
    ek = np.array([bands(kk) for kk in k])
    dos = sum(_gauss(e - EF, sigma) for row in ek for e in row) / nk
    pi_out, lam_out, zeta = [], [], []
    for qq in q:
        ekq = np.array([bands(kk + qq) for kk in k])
        w = 2 * math.sqrt(K / M) * np.abs(np.sin(np.pi * qq))
        z = 0.0
        P = np.zeros(3)
        L = np.zeros(3)
        for ik in range(nk):
            for n in range(ek.shape[1]):
                fn = _fermi(ek[ik, n], EF, T)
                for mm in range(ek.shape[1]):
                    fm = _fermi(ekq[ik, mm], EF, T)
                    dd = _gauss(ek[ik, n] - EF, sigma) * _gauss(ekq[ik, mm] - EF, sigma)
                    z += dd / nk
                    for a in range(3):
                        if w[a] < wmin:
                            continue
                        g2 = c[mm, n] ** 2 * math.sin(2 * math.pi * qq[a]) ** 2 / (2 * M * w[a])
                        P[a] += g2 * (fn - fm) * _gauss(ek[ik, n] - ekq[ik, mm] - w[a], sigma) / nk
                        L[a] += g2 * dd / nk
        order = np.argsort(w)
        pi_out.append(2 * math.pi * P[order])
        lam_out.append(np.where(w[order] >= wmin, L[order] / (dos * np.maximum(w[order], wmin)), 0.0))
        zeta.append(z)
    return np.array(pi_out), np.array(lam_out), np.array(zeta), dos


@pytest.mark.parametrize("T,EF,sigma", [(300.0, 0.1, 0.08), (50.0, -0.4, 0.05)])
def test_phonon_self_energy_closed_form_one_band(oracle_lib, T, EF, sigma):
    m = _tb()
    rng = np.random.default_rng(70)
    k = W.uniform_grid(6) + 0.03
    q = rng.random((5, 3))  # generic q: three distinct frequencies
    pi, lam, zeta, dos = oracle_lib.phonon_self(m, k, q, None, T, EF, sigma)
    bands = lambda kk: [0.2 - 2 * 0.5 * np.cos(2 * np.pi * kk).sum()]
    rpi, rlam, rz, rdos = _phonon_closed_form(k, q, T, EF, sigma, bands, 0.01, 1.3, np.array([[0.05]]))
    assert math.isclose(dos, rdos, rel_tol=1e-12)
    assert np.allclose(zeta, rz, rtol=1e-11, atol=1e-14 * np.abs(rz).max())
    assert np.allclose(pi, rpi, rtol=1e-10, atol=1e-13 * np.abs(rpi).max())
    assert np.allclose(lam, rlam, rtol=1e-10, atol=1e-13 * np.abs(rlam).max())
    assert np.abs(rpi).max() > 0 and np.abs(rlam).max() > 0


def test_phonon_self_energy_closed_form_two_bands(oracle_lib):
    """Asymmetric interband couplings pin the band indices: n at k, m at k+q."""
    m, eps, t, K, M, c = _two_band_tb()
    rng = np.random.default_rng(71)
    k = W.uniform_grid(5) + 0.02
    q = rng.random((4, 3))
    T, EF, sigma = 300.0, 0.05, 0.1
    pi, lam, zeta, dos = oracle_lib.phonon_self(m, k, q, None, T, EF, sigma)
    bands = lambda kk: [e - 2 * t * np.cos(2 * np.pi * kk).sum() for e in eps]
    rpi, rlam, rz, rdos = _phonon_closed_form(k, q, T, EF, sigma, bands, K, M, c)
    assert math.isclose(dos, rdos, rel_tol=1e-12)
    assert np.allclose(zeta, rz, rtol=1e-11, atol=1e-14 * np.abs(rz).max())
    assert np.allclose(pi, rpi, rtol=1e-10, atol=1e-13 * np.abs(rpi).max())
    assert np.allclose(lam, rlam, rtol=1e-10, atol=1e-13 * np.abs(rlam).max())
    # the transposed couplings give a different answer (the pin sees the index order)
    tpi, _, _, _ = _phonon_closed_form(k, q, T, EF, sigma, bands, K, M, c.T)
    assert not np.allclose(tpi, rpi, rtol=1e-3)


def test_phonon_self_energy_time_reversal(oracle_lib):
    rng = np.random.default_rng(72)
    m = W.make_model("fcc", 2, 1, [1.0], 20, 20, rng, real=True)
    k = W.uniform_grid(4) + 0.0
    q = rng.random((3, 3))
    a = oracle_lib.phonon_self(m, k, q, None, 300.0, 0.0, 0.1)
    b = oracle_lib.phonon_self(m, k, -q, None, 300.0, 0.0, 0.1)
    for x, y in zip(a[:3], b[:3]):
        assert np.allclose(x, y, rtol=1e-9, atol=1e-12 * (np.abs(x).max() + 1e-300))


def test_eliashberg_function_pins(oracle_lib):
    """Eq. (isotropiceliash): one mode at w0 gives lambda w0 / 2 times a normalised Gaussian at w0;
    for any spectrum, 2 int a2F(w)/w dw = sum_q w_q sum_nu lambda_qnu (widths small against w)."""
    s = 1e-4
    grid = np.linspace(0.0, 0.12, 24001)
    a2f = oracle_lib.eliashberg(np.array([[0.05]]), np.array([[0.8]]), grid, s)
    ref = 0.5 * 0.05 * 0.8 * np.exp(-((grid - 0.05) / s) ** 2) / (s * math.sqrt(math.pi))
    assert np.allclose(a2f, ref, rtol=1e-13, atol=1e-13 * ref.max())
    rng = np.random.default_rng(80)
    om = 0.01 + 0.09 * rng.random((40, 6))
    lam = rng.random((40, 6))
    wq = rng.random(40)
    wq /= wq.sum()
    a2f = oracle_lib.eliashberg(om, lam, grid, s, wq)
    integral = 2 * np.trapezoid(a2f / np.maximum(grid, 1e-12), grid)
    assert abs(integral - (wq[:, None] * lam).sum()) < 1e-5 * (wq[:, None] * lam).sum()


# ------------------------------------------- complex self-energy (oracle)
def test_selfenergy_closed_form_one_band(oracle_lib):
    """Eq. (elselfenergy) on the one-band model: a sum of analytic terms (no Fourier sum, no eigensolve)."""
    m = _tb()
    rng = np.random.default_rng(90)
    k = rng.random((3, 3))
    q = W.uniform_grid(4) + 0.01
    omega = np.linspace(-0.3, 0.3, 13)
    T, EF, delta = 300.0, 0.05, 0.02
    sig, _ = oracle_lib.selfenergy(m, k, q, omega, None, T, EF, delta)
    for ik, kk in enumerate(k):
        ref = np.zeros(len(omega), dtype=complex)
        for qq in q:
            x = 0.2 - 2 * 0.5 * np.cos(2 * np.pi * (kk + qq)).sum() - EF
            f = _fermi(x + EF, EF, T)
            for a in range(3):
                w = 2 * math.sqrt(0.01 / 1.3) * abs(math.sin(math.pi * qq[a]))
                if w < 1e-5:
                    continue
                g2 = 0.05**2 * math.sin(2 * math.pi * qq[a]) ** 2 / (2 * 1.3 * w)
                n = _bose(w, T)
                ref += g2 * ((n + f) / (omega - x + w + 1j * delta) + (n + 1 - f) / (omega - x - w + 1j * delta))
        ref /= len(q)
        assert np.allclose(sig[ik, 0], ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max())


def test_spectral_function_normalisation(oracle_lib):
    """int A_nk(w) dw = 1: with Sigma analytic in the upper half plane (positive weights over
    w - a + i delta) and a real constant shift, -Im G / pi is a normalised density.  Only the
    squared Sigma'' in the denominator of Eq. (spectral_funct) has this property."""
    rng = np.random.default_rng(91)
    # a coupling weak enough that the spectral weight lies well inside the +-40 eV grid
    m = W.make_model("fcc", 2, 1, [1.0], 20, 20, rng, g_amp=0.01)
    k = rng.random((2, 3))
    q = W.uniform_grid(3) + 0.05
    omega = np.linspace(-40.0, 40.0, 160001)
    sig, spec = oracle_lib.selfenergy(m, k, q, omega, None, 300.0, 0.0, 0.05)
    norm = np.trapezoid(spec, omega, axis=-1)
    assert np.all(np.abs(norm - 1.0) < 1e-5), norm
    assert np.all(-sig.imag >= 0)


# ------------------------------------------------------ polar vertex (oracle)
def test_polar_vertex_closed_form_one_band(oracle_lib):
    """One band, one atom, simple cubic (a = 1), Z* = z I, eps_inf = e I and the G = 0 term alone:
    g^L_a = i pref z q_a damp / (2 pi e |q|^2 sqrt(2 M w_a)) with damp = exp(-e (2 pi |q|)^2 / (4 alpha)),
    imaginary against the real short-range g0 sin(2 pi q_a) / sqrt(2 M w_a): |g|^2 is the sum of squares."""
    m = _tb()
    z, e, alpha, pref = 1.7, 5.0, 0.8, 0.03
    m = dataclasses.replace(m, polar=W.models.PolarTerms(A=np.eye(3), eps_inf=e * np.eye(3), Zstar=z * np.eye(3)[None],
                                                         alpha=alpha, prefactor=pref, gmax=0))
    k = W.uniform_grid(3) + 0.05
    q = W.uniform_grid(6) + 0.013  # no q on a reciprocal lattice vector
    T, EF, sigma, M = 300.0, 0.1, 0.05, 1.3
    got = oracle_lib.linewidth(m, k, q, None, T, EF, sigma)[:, 0]
    ref = np.zeros(len(k))
    for ik, kk in enumerate(k):
        ek = 0.2 - 2 * 0.5 * np.cos(2 * np.pi * kk).sum()
        s = 0.0
        for qq in q:
            ekq = 0.2 - 2 * 0.5 * np.cos(2 * np.pi * (kk + qq)).sum()
            f = _fermi(ekq, EF, T)
            q2 = float((qq**2).sum())
            damp = math.exp(-e * (2 * math.pi) ** 2 * q2 / (4 * alpha))
            for a in range(3):
                w = 2 * math.sqrt(0.01 / M) * abs(math.sin(math.pi * qq[a]))
                gs = 0.05 * math.sin(2 * math.pi * qq[a]) / math.sqrt(2 * M * w)
                gl = pref * z * qq[a] * damp / (2 * math.pi * e * q2 * math.sqrt(2 * M * w))
                g2 = gs * gs + gl * gl
                n = _bose(w, T)
                s += g2 * ((n + f) * _gauss(ek - ekq + w, sigma) + (n + 1 - f) * _gauss(ek - ekq - w, sigma))
        ref[ik] = math.pi * s / len(q)
    assert np.allclose(got, ref, rtol=1e-11, atol=1e-14 * np.abs(ref).max())
    # and the long-range part is not negligible here
    base = oracle_lib.linewidth(dataclasses.replace(m, polar=None), k, q, None, T, EF, sigma)[:, 0]
    assert np.abs(got - base).max() > 0.1 * np.abs(base).max()


def test_polar_vertex_diverges_as_one_over_q(oracle_lib):
    """|g^L| |q| tends to a constant as q -> 0 along a direction (the G = 0 term of Eq. long-range),
    for an optical mode of a two-atom model with neutral Born charges."""
    rng = np.random.default_rng(95)
    m = W.make_model("diamond", 1, 2, [1.0, 1.2], 20, 20, rng)
    m = dataclasses.replace(m, polar=W.models.polar_terms("diamond", 2, rng, prefactor=0.05, gmax=2))
    short = dataclasses.replace(m, polar=None)
    qhat = np.array([0.3, -0.2, 0.5])
    k = np.array([[0.1, 0.2, 0.3]])
    vals = []
    for t in (1e-3, 1e-4, 1e-5):
        q = (t * qhat)[None]
        _, _, om, g = oracle_lib.interp(m, k, q)
        _, _, _, gs = oracle_lib.interp(short, k, q)
        gl = np.abs(g[0, 0, -1, 0, 0] - gs[0, 0, -1, 0, 0])  # highest (optical) mode, one band
        vals.append(gl * t)
    assert vals[0] > 0
    assert abs(vals[1] - vals[2]) < 1e-3 * vals[2]
    assert abs(vals[0] - vals[2]) < 1e-1 * vals[2]


def _random_unitary_in_blocks(vals, tol, rng):
    """A unitary that mixes only eigenvectors whose (ascending) values lie within tol."""
    from tests._util import group_labels
    lab = group_labels(vals, tol)
    n = len(vals)
    W = np.zeros((n, n), dtype=complex)
    for b in range(lab.max() + 1):
        idx = np.where(lab == b)[0]
        z = rng.standard_normal((len(idx), len(idx))) + 1j * rng.standard_normal((len(idx), len(idx)))
        Q, R = np.linalg.qr(z)
        W[np.ix_(idx, idx)] = Q * (np.diag(R) / np.abs(np.diag(R)))
    return W


def test_gauge_invariance_in_degenerate_subspaces(oracle_lib):
    """Random unitaries inside degenerate subspaces of U_k, U_k+q and e_q leave |g|^2 summed
    over the degenerate blocks unchanged (the gauge-invariant quantity compared throughout).
    Every band is doubly degenerate (H(R) = h(R) x I_2) and the sc spring model has degenerate
    transverse modes on the q axes, so the gauge freedom is exercised."""
    rng = np.random.default_rng(910)
    m1 = W.make_model("sc", 1, 1, [1.0], None, None, rng, box=1)
    H2 = np.stack([np.kron(h, np.eye(2)) for h in m1.H])
    nR = len(m1.Re)
    g2 = (rng.standard_normal((nR, nR, 3, 2, 2)) + 1j * rng.standard_normal((nR, nR, 3, 2, 2))) * 0.05
    m = dataclasses.replace(m1, nw=2, H=H2, g=g2)
    k = rng.random((2, 3))
    q = np.array([[0.25, 0.0, 0.0], [0.0, 0.375, 0.0], [0.13, 0.41, 0.77]])
    eps_k, eps_kq, omega, g = oracle_lib.interp(m, k, q)
    msq = np.repeat(np.sqrt(m.mass), 3)
    mrep = np.repeat(m.mass, 3)
    changed = 0.0
    for ik in range(len(k)):
        for iq in range(len(q)):
            G = oracle_lib.g_wannier_direct(m, k[ik], q[iq])
            Hk = sum(np.exp(2j * np.pi * k[ik] @ R) * Hr for R, Hr in zip(m.Re, m.H))
            Hkq = sum(np.exp(2j * np.pi * (k[ik] + q[iq]) @ R) * Hr for R, Hr in zip(m.Re, m.H))
            D = sum(np.exp(2j * np.pi * q[iq] @ R) * P for R, P in zip(m.Rph, m.Phi)) / np.outer(msq, msq)
            ek, Uk = np.linalg.eigh(Hk)
            ekq, Ukq = np.linalg.eigh(Hkq)
            w2, e = np.linalg.eigh(D)
            w = np.sqrt(np.abs(w2)) * np.sign(w2)
            Uk = Uk @ _random_unitary_in_blocks(ek, 1e-9, rng)
            Ukq = Ukq @ _random_unitary_in_blocks(ekq, 1e-9, rng)
            e = e @ _random_unitary_in_blocks(w2, 1e-12, rng)
            keep = w >= 1e-5
            E = np.where(keep[None, :], e / np.sqrt(2 * np.outer(mrep, np.where(keep, w, 1.0))), 0)
            gB = np.einsum("im,aij,jn->amn", Ukq.conj(), G, Uk)
            ref = np.einsum("amn,av->vmn", gB, E)
            a = degenerate_sums(np.abs(g[ik, iq]) ** 2, ekq, ek, w, 1e-9)
            b = degenerate_sums(np.abs(ref) ** 2, ekq, ek, w, 1e-9)
            assert np.allclose(a, b, rtol=1e-10, atol=1e-14 * b.max())
            changed = max(changed, np.abs(np.abs(g[ik, iq]) ** 2 - np.abs(ref) ** 2).max() / b.max())
    # the rotated gauge really differs element by element
    assert changed > 1e-3


# ------------------------------------------------ unequal masses (two-atom chain)
def _chain_closed_form(q, M, Kx):
    """Branches of the x-polarised chain: eigenvalues lam_+- of
    [[2K/M0, b], [conj b, 2K/M1]], b = -K (1 + e^{-2 pi i q_x}) / sqrt(M0 M1), and the
    weights |e_0|^2, |e_1|^2 of each eigenvector on the two atoms."""
    M0, M1 = M
    s = Kx * (1.0 / M0 + 1.0 / M1)
    root = np.sqrt(s * s - 4.0 * Kx * Kx * np.sin(np.pi * q[:, 0]) ** 2 / (M0 * M1))
    lam = np.stack([s - root, s + root], axis=1)  # acoustic, optical
    b2 = Kx * Kx * np.abs(1.0 + np.exp(-2j * np.pi * q[:, 0])) ** 2 / (M0 * M1)
    d = lam - 2.0 * Kx / M0
    e0 = b2[:, None] / (b2[:, None] + d * d)
    return np.sqrt(lam), e0, 1.0 - e0


def test_two_atom_chain_phonons_closed_form(oracle_lib):
    M, K = (1.0, 2.5), (0.010, 0.017, 0.029)
    m = W.diatomic_chain_model(M=M, Kdiag=K)
    rng = np.random.default_rng(140)
    q = rng.random((40, 3))
    w, _ = oracle_lib.phonons(m, q)
    ref = np.concatenate([_chain_closed_form(q, M, Kc)[0] for Kc in K], axis=1)
    assert np.allclose(np.sort(w, axis=1), np.sort(ref, axis=1), rtol=1e-10, atol=1e-13)


@pytest.mark.parametrize("couple,comp", [(0, 0), (1, 0), (0, 1), (1, 2)])
def test_two_atom_chain_linewidth_per_atom_mass(oracle_lib, couple, comp):
    """The vertex on one displacement component of one atom: |g_nu|^2 = g0^2 sin^2(2 pi q_x)
    |e_couple|^2 / (2 M_couple w_nu) on the two branches of that polarisation, 0 on the others
    (no Fourier sum, no eigensolve here)."""
    M, K, g0 = (1.0, 2.5), (0.010, 0.017, 0.029), 0.05
    m = W.diatomic_chain_model(M=M, Kdiag=K, couple=couple, comp=comp, g0=g0)
    k = W.uniform_grid(2) + 0.07
    q = W.uniform_grid(6) + 0.031
    T, EF, sigma = 300.0, 0.05, 0.05
    got = oracle_lib.linewidth(m, k, q, None, T, EF, sigma)[:, 0]
    w, e0, e1 = _chain_closed_form(q, M, K[comp])
    wt = e0 if couple == 0 else e1
    ref = np.zeros(len(k))
    for ik, kk in enumerate(k):
        ek = 0.2 - 2 * 0.5 * np.cos(2 * np.pi * kk).sum()
        s = 0.0
        for iq, qq in enumerate(q):
            ekq = 0.2 - 2 * 0.5 * np.cos(2 * np.pi * (kk + qq)).sum()
            f = _fermi(ekq, EF, T)
            for br in range(2):
                wv = w[iq, br]
                g2 = g0 ** 2 * math.sin(2 * math.pi * qq[0]) ** 2 * wt[iq, br] / (2 * M[couple] * wv)
                n = _bose(wv, T)
                s += g2 * ((n + f) * _gauss(ek - ekq + wv, sigma) + (n + 1 - f) * _gauss(ek - ekq - wv, sigma))
        ref[ik] = math.pi * s / len(q)
    assert np.all(ref > 0)
    assert np.allclose(got, ref, rtol=1e-10, atol=1e-14 * ref.max())


# --------------------------------------------- constant vertex (Einstein phonons)
@pytest.mark.parametrize("T,EF", [(300.0, 0.1), (0.0, -0.2)])
def test_constant_vertex_einstein_reduction(oracle_lib, T, EF):
    """g_a(k,q) = c_a and w_qnu = w0 for all three (degenerate) modes: sum_nu |g_nu|^2 =
    |c|^2 / (2 M w0) whatever the eigenvectors, so Im Sigma_k = pi |c|^2/(2 M w0) sum_q w_q
    [(n + f) d(e_k - e_k+q + w0) + (n + 1 - f) d(e_k - e_k+q - w0)] from band energies alone."""
    M, w0, c = 1.4, 0.06, np.array([0.03, -0.02j, 0.05])
    m = W.einstein_model(M=M, w0=w0, c=c)
    k = W.uniform_grid(3) + 0.05
    q = W.uniform_grid(7)
    sigma = 0.04
    got = oracle_lib.linewidth(m, k, q, None, T, EF, sigma)[:, 0]
    c2 = float(np.sum(np.abs(c) ** 2)) / (2 * M * w0)
    n = _bose(w0, T)
    ref = np.zeros(len(k))
    for ik, kk in enumerate(k):
        ek = 0.2 - 2 * 0.5 * np.cos(2 * np.pi * kk).sum()
        s = 0.0
        for qq in q:
            ekq = 0.2 - 2 * 0.5 * np.cos(2 * np.pi * (kk + qq)).sum()
            f = _fermi(ekq, EF, T)
            s += (n + f) * _gauss(ek - ekq + w0, sigma) + (n + 1 - f) * _gauss(ek - ekq - w0, sigma)
        ref[ik] = math.pi * c2 * s / len(q)
    assert np.all(ref > 0)
    assert np.allclose(got, ref, rtol=1e-11, atol=1e-14 * ref.max())


# ------------------------------------- spectral function point by point (one band)
def test_spectral_function_pointwise_with_shift(oracle_lib):
    """Eq. (spectral_funct) with Sigma~' = Sigma'(w) - Sigma'(0) (Eq. realpartselfenergy, w from E_F),
    from the closed-form Sigma(w) of the one-band model on the grid and at w = 0."""
    m = _tb()
    rng = np.random.default_rng(92)
    k = rng.random((3, 3))
    q = W.uniform_grid(4) + 0.01
    omega = np.linspace(-0.4, 0.4, 41)
    T, EF, delta = 300.0, 0.05, 0.02

    def sigma_cf(kk, om):
        out = np.zeros(len(om), dtype=complex)
        for qq in q:
            x = 0.2 - 2 * 0.5 * np.cos(2 * np.pi * (kk + qq)).sum() - EF
            f = _fermi(x + EF, EF, T)
            for a in range(3):
                w = 2 * math.sqrt(0.01 / 1.3) * abs(math.sin(math.pi * qq[a]))
                if w < 1e-5:
                    continue
                g2 = 0.05 ** 2 * math.sin(2 * math.pi * qq[a]) ** 2 / (2 * 1.3 * w)
                nb = _bose(w, T)
                out += g2 * ((nb + f) / (om - x + w + 1j * delta) + (nb + 1 - f) / (om - x - w + 1j * delta))
        return out / len(q)

    _, spec = oracle_lib.selfenergy(m, k, q, omega, None, T, EF, delta)
    for ik, kk in enumerate(k):
        s = sigma_cf(kk, omega)
        s0 = sigma_cf(kk, np.zeros(1))[0]
        xn = 0.2 - 2 * 0.5 * np.cos(2 * np.pi * kk).sum() - EF
        s2 = -s.imag
        ref = np.abs(s2) / (math.pi * ((omega - xn - (s.real - s0.real)) ** 2 + s2 ** 2))
        assert np.allclose(spec[ik, 0], ref, rtol=1e-10, atol=1e-14 * ref.max())
        # the shift matters: without it the spectral function differs
        unshifted = np.abs(s2) / (math.pi * ((omega - xn - s.real) ** 2 + s2 ** 2))
        assert np.abs(unshifted - ref).max() > 1e-3 * ref.max()


# ------------------------------------------ polar G sum beyond G = 0 (one atom)
def _polar_F_integral(q, eps_d, Z, alpha, gmax):
    """F_a = sum_{|n_i| <= gmax} (x Z)_a e^{-x.eps.x/(4 alpha)} / (x.eps.x), x = 2 pi (q + n) (sc, a = 1),
    for diagonal eps, through e^{-s/(4 alpha)}/s = int_{1/(4 alpha)}^inf e^{-s t} dt: the sum over the
    G box becomes a product of one-axis sums under a one-dimensional integral,
      sum_G x_c e^{-s t} = S1_c(t) prod_{d != c} S0_d(t),
      S0_d(t) = sum_n e^{-eps_d x_d^2 t},  S1_c(t) = sum_n x_c e^{-eps_c x_c^2 t}."""
    from scipy.integrate import quad
    ns = np.arange(-gmax, gmax + 1)
    xs = [2 * np.pi * (q[c] + ns) for c in range(3)]

    def S0(d, t):
        return float(np.sum(np.exp(-eps_d[d] * xs[d] ** 2 * t)))

    def S1(c, t):
        return float(np.sum(xs[c] * np.exp(-eps_d[c] * xs[c] ** 2 * t)))

    I = np.zeros(3)
    for c in range(3):
        others = [d for d in range(3) if d != c]
        f = lambda t, c=c, o=others: S1(c, t) * S0(o[0], t) * S0(o[1], t)  # noqa: E731
        I[c] = quad(f, 1.0 / (4 * alpha), np.inf, epsabs=0.0, epsrel=1e-13, limit=400)[0]
    return I @ Z  # F_a = sum_c I_c Z[c][a]


def test_polar_g_sum_anisotropic_beyond_gamma(oracle_lib):
    """One band, one atom (the tight-binding model, Cartesian modes), diagonal anisotropic eps_inf,
    a full Born-charge tensor, G box |n_i| <= 2: the long-range vertex of each mode,
    |g^L_a| = pref |F_a| / sqrt(2 M w_a), against the integral representation of the G sum."""
    m = _tb()
    eps_d = np.array([4.0, 6.5, 9.0])
    Z = np.array([[1.3, 0.4, -0.2], [0.1, 0.8, 0.5], [-0.6, 0.3, 1.7]])
    alpha, pref, gmax, M = 40.0, 0.04, 2, 1.3
    mp = dataclasses.replace(m, polar=W.models.PolarTerms(A=np.eye(3), eps_inf=np.diag(eps_d), Zstar=Z[None],
                                                          alpha=alpha, prefactor=pref, gmax=gmax))
    rng = np.random.default_rng(96)
    k = rng.random((1, 3))
    q = rng.random((6, 3)) - 0.5
    _, _, om, g = oracle_lib.interp(mp, k, q)
    _, _, _, gs = oracle_lib.interp(m, k, q)
    for iq, qq in enumerate(q):
        F = _polar_F_integral(qq, eps_d, Z, alpha, gmax)
        gl = np.abs(g[0, iq, :, 0, 0] - gs[0, iq, :, 0, 0])  # modes in ascending w
        wa = 2 * math.sqrt(0.01 / M) * np.abs(np.sin(np.pi * qq))
        order = np.argsort(wa)
        ref = pref * np.abs(F[order]) / np.sqrt(2 * M * wa[order])
        assert np.allclose(om[iq], wa[order], rtol=1e-12)
        assert np.allclose(gl, ref, rtol=1e-9, atol=1e-15), (gl, ref)
        # terms beyond G = 0 matter at this alpha
        F0 = _polar_F_integral(qq, eps_d, Z, alpha, 0)
        assert np.abs(F - F0).max() > 1e-3 * np.abs(F).max()
