"""Synthetic Wannier models and k/q point sets.

Conventions (shared by every consumer, stated once here):

* k, q and lattice vectors R are in crystal (fractional) coordinates; R are
  integer triples.  Cartesian lengths (used only for decay envelopes and shell
  ordering) use the lattice matrix ``A`` whose rows are the primitive vectors in
  units of the lattice parameter a = 1.
* Energies are in eV, temperatures in K.
* H[iR, i, j]            electronic Hamiltonian H(Re)_{ij}, nw x nw, complex128.
* Phi[iR, ka, kb]        force constants Phi_{kappa alpha, kappa' beta}(R), 3nat x 3nat.
* g[iRe, iRp, ka, m, n]  Wannier-space vertex g_{kappa alpha}(Re, Rp)_{mn}.
* All R sets are closed under R -> -R and every Hermiticity relation
  (H(-R) = H(R)^dagger, Phi(-R) = Phi(R)^T) holds exactly.

Nothing here evaluates the method (no Fourier sums, eigensolves, occupations or
delta functions); a few quantities (the energy window of the k lists) need band
energies and therefore come from stored files written by a script that uses the
CPU oracle.
"""
from __future__ import annotations

import dataclasses
import math
import os
from typing import Optional

import numpy as np

SEED_BASE = 160403525

# Primitive vectors (rows) in units of a, and atomic positions (Cartesian, units of a).
LATTICES = {
    "sc": (np.eye(3), np.zeros((1, 3))),
    "fcc": (np.array([[0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]]), np.zeros((1, 3))),
    "diamond": (
        np.array([[0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]]),
        np.array([[0.0, 0.0, 0.0], [0.25, 0.25, 0.25]]),
    ),
    "hex": (
        np.array([[1.0, 0.0, 0.0], [-0.5, math.sqrt(3.0) / 2.0, 0.0], [0.0, 0.0, 1.6]]),
        np.array([[0.0, 0.0, 0.0], [0.5, math.sqrt(3.0) / 6.0, 0.8], [0.0, math.sqrt(3.0) / 3.0, 0.8]]),
    ),
}


@dataclasses.dataclass
class PolarTerms:
    """Inputs of the long-range vertex: lattice vectors A (rows, units of a), the high-frequency
    dielectric tensor, Born effective charges Z*[kappa][b][alpha], the damping alpha of the G sum
    (1/a^2), the overall prefactor (eV) and the G box |n_i| <= gmax."""

    A: np.ndarray
    eps_inf: np.ndarray
    Zstar: np.ndarray
    alpha: float
    prefactor: float
    gmax: int


def polar_terms(lattice: str, nat: int, rng: np.random.Generator, prefactor: float = 0.05, alpha: float = 1.0,
                gmax: int = 2) -> PolarTerms:
    """Seeded synthetic polar inputs: eps_inf symmetric positive definite (eigenvalues 4..10), Z* random
    3x3 per atom with the charge-neutrality sum rule sum_kappa Z*_kappa = 0 (a single atom gets
    Z* = 0 unless given explicitly)."""
    A, _ = LATTICES[lattice]
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    eps = Q @ np.diag(4.0 + 6.0 * rng.random(3)) @ Q.T
    Z = rng.standard_normal((nat, 3, 3))
    Z -= Z.mean(axis=0, keepdims=True)
    return PolarTerms(A=np.array(A, dtype=np.float64), eps_inf=0.5 * (eps + eps.T), Zstar=Z, alpha=alpha,
                      prefactor=prefactor, gmax=gmax)


def _canonical_order(R: np.ndarray, A: np.ndarray) -> np.ndarray:
    """Sort integer vectors by Cartesian length, then lexicographically."""
    lengths = np.round(np.linalg.norm(R @ A, axis=1), 9)
    order = np.lexsort((R[:, 2], R[:, 1], R[:, 0], lengths))
    return R[order]


def box_vectors(n: int) -> np.ndarray:
    """All integer triples in {-n..n}^3 (the (2n+1)^3 box), canonically ordered."""
    r = np.arange(-n, n + 1)
    R = np.stack(np.meshgrid(r, r, r, indexing="ij"), axis=-1).reshape(-1, 3)
    return _canonical_order(R, np.eye(3)).astype(np.int32)


def lattice_shells(A: np.ndarray, target: int, search: int = 8) -> np.ndarray:
    """Whole shells of lattice vectors (by Cartesian length) until the count >= target.

    The set contains the origin, is closed under R -> -R (shells are), and is
    returned in canonical order (length, then lexicographic).
    """
    r = np.arange(-search, search + 1)
    R = np.stack(np.meshgrid(r, r, r, indexing="ij"), axis=-1).reshape(-1, 3)
    lengths = np.round(np.linalg.norm(R @ A, axis=1), 9)
    shells = np.unique(lengths)
    chosen = []
    count = 0
    for s in shells:
        members = R[lengths == s]
        chosen.append(members)
        count += len(members)
        if count >= target:
            break
    if count < target:
        raise ValueError("search box too small for the requested shell count")
    return _canonical_order(np.concatenate(chosen), A).astype(np.int32)


def uniform_grid(n: int) -> np.ndarray:
    """Gamma-centred uniform n^3 grid in crystal coordinates, points in [0,1)^3."""
    i = np.arange(n) / n
    return np.stack(np.meshgrid(i, i, i, indexing="ij"), axis=-1).reshape(-1, 3).copy()


def random_points(rng: np.random.Generator, n: int) -> np.ndarray:
    """n points uniform in [0,1)^3 (crystal coordinates)."""
    return rng.random((n, 3))


def _cnormal(rng: np.random.Generator, shape) -> np.ndarray:
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2.0)


def _positive(R: np.ndarray) -> bool:
    for c in R:
        if c != 0:
            return c > 0
    return False


def _index_of(Rset: np.ndarray) -> dict:
    return {tuple(int(x) for x in r): i for i, r in enumerate(Rset)}


@dataclasses.dataclass
class WannierModel:
    """Real-space inputs of the interpolation (one material)."""

    lattice: str
    nw: int
    nat: int
    mass: np.ndarray  # [nat]
    Re: np.ndarray  # [nRe,3] int32
    wRe: np.ndarray  # [nRe]
    H: np.ndarray  # [nRe,nw,nw] complex128
    Rph: np.ndarray  # [nRph,3] int32
    wRph: np.ndarray  # [nRph]
    Phi: np.ndarray  # [nRph,3nat,3nat] complex128
    Rp: np.ndarray  # [nRp,3] int32
    wRp: np.ndarray  # [nRp]
    g: np.ndarray  # [nRe,nRp,3nat,nw,nw] complex128
    polar: Optional["PolarTerms"] = None  # long-range part of the vertex (polar materials)

    @property
    def nmodes(self) -> int:
        return 3 * self.nat

    def nbytes_g(self) -> int:
        return self.g.nbytes


def _hamiltonian(rng, Re, A, nw, amp, decay, onsite):
    """H(R) complex, decaying as amp*exp(-|R|/decay); H(-R) = H(R)^dagger; H(0) Hermitian."""
    idx = _index_of(Re)
    H = np.zeros((len(Re), nw, nw), dtype=np.complex128)
    for i, R in enumerate(Re):
        if not (_positive(R) or not R.any()):
            continue
        env = amp * math.exp(-np.linalg.norm(R @ A) / decay)
        X = _cnormal(rng, (nw, nw)) * env
        if not R.any():
            X = 0.5 * (X + X.conj().T)
            X[np.diag_indices(nw)] = rng.uniform(-onsite, onsite, nw)
            H[i] = X
        else:
            H[i] = X
            H[idx[tuple(int(x) for x in -R)]] = X.conj().T
    return H


def _springs(rng, Rph, A, tau, mass, decay, omega_max):
    """Force constants of a random central-plus-transverse spring network.

    Each bond (kappa in cell 0, kappa' in cell R) carries a random symmetric
    positive semi-definite 3x3 stiffness K_b (decaying as exp(-|d|/decay)); the
    force constants are the second derivatives of the spring energy, which makes
    Phi(-R) = Phi(R)^T, the acoustic sum rule exact and every omega^2 >= 0.
    The stiffness is scaled so that a norm bound on the dynamical matrix equals
    omega_max^2 (so every omega <= omega_max).
    """
    nat = len(tau)
    idx = _index_of(Rph)
    Phi = np.zeros((len(Rph), 3 * nat, 3 * nat))
    i0 = idx[(0, 0, 0)]
    for i, R in enumerate(Rph):
        zero = not R.any()
        if not (zero or _positive(R)):
            continue
        for a in range(nat):
            for b in range(nat):
                if zero and b <= a:
                    continue
                d = R @ A + tau[b] - tau[a]
                L = rng.standard_normal((3, 3))
                K = (L @ L.T) / 3.0 * math.exp(-np.linalg.norm(d) / decay)
                sa, sb = slice(3 * a, 3 * a + 3), slice(3 * b, 3 * b + 3)
                j = idx[tuple(int(x) for x in -R)]
                Phi[i, sa, sb] -= K
                Phi[j, sb, sa] -= K.T
                Phi[i0, sa, sa] += K
                Phi[i0, sb, sb] += K
    # ||D(q)||_2 <= sum_R ||Phi(R)||_F / min(M): scale that bound to omega_max^2.
    bound = sum(np.linalg.norm(P) for P in Phi) / float(np.min(mass))
    Phi *= omega_max**2 / bound
    return Phi.astype(np.complex128)


def make_model(
    lattice: str,
    nw: int,
    nat: int,
    masses,
    nRe_target: Optional[int],
    nRp_target: Optional[int],
    rng: np.random.Generator,
    box: Optional[int] = None,
    h_amp: float = 1.0,
    h_decay: float = 0.7,
    onsite: float = 1.0,
    g_amp: float = 0.1,
    ge_decay: float = 1.0,
    gp_decay: float = 1.5,
    ph_decay: float = 0.7,
    omega_max: float = 0.1,
    real: bool = False,
) -> WannierModel:
    """Draw one synthetic Wannier model.

    ``box`` selects the (2*box+1)^3 box for all R sets instead of shells.
    ``real`` makes H, Phi and g real (used for time-reversal checks).
    The phonon R set is the electronic one.
    """
    A, tau = LATTICES[lattice]
    tau = tau[:nat] if len(tau) >= nat else np.concatenate(
        [tau, rng.random((nat - len(tau), 3)) @ A], axis=0)
    mass = np.asarray(masses, dtype=np.float64)
    if box is not None:
        Re = box_vectors(box)
        Rp = Re.copy()
    else:
        Re = lattice_shells(A, nRe_target)
        Rp = lattice_shells(A, nRp_target)
    Rph = Re.copy()
    H = _hamiltonian(rng, Re, A, nw, h_amp, h_decay, onsite)
    Phi = _springs(rng, Rph, A, tau, mass, ph_decay, omega_max)
    le = np.linalg.norm(Re @ A, axis=1)
    lp = np.linalg.norm(Rp @ A, axis=1)
    env = g_amp * np.exp(-le[:, None] / ge_decay - lp[None, :] / gp_decay)
    g = _cnormal(rng, (len(Re), len(Rp), 3 * nat, nw, nw)) * env[:, :, None, None, None]
    if real:
        H = _real_hermitian(H, Re)
        g = g.real.astype(np.complex128)
    return WannierModel(
        lattice=lattice, nw=nw, nat=nat, mass=mass,
        Re=Re, wRe=np.ones(len(Re)), H=H,
        Rph=Rph, wRph=np.ones(len(Rph)), Phi=Phi,
        Rp=Rp, wRp=np.ones(len(Rp)), g=g,
    )


def _real_hermitian(H, Re):
    """Real H(R) with H(-R) = H(R)^T (keeps the R -> -R pairing of the complex draw)."""
    idx = _index_of(Re)
    out = np.zeros_like(H)
    for i, R in enumerate(Re):
        j = idx[tuple(int(x) for x in -R)]
        out[i] = H[i].real
        out[j] = H[i].real.T
    for i, R in enumerate(Re):
        if not R.any():
            out[i] = 0.5 * (H[i].real + H[i].real.T)
    return out.astype(np.complex128)


def tight_binding_model(eps0=0.2, t=0.5, K=0.01, g0=0.05, mass=1.0) -> WannierModel:
    """One band, one atom, simple cubic, nearest neighbours only.

    H(0)=eps0, H(+-e_a)=-t; central springs of stiffness K on the six bonds;
    g_a(Re=0, Rp=+-e_a) = -+ i g0/2 (cartesian component a only).  Every
    interpolated quantity of this model has a closed form (used by the tests).
    """
    Re = box_vectors(1)
    idx = _index_of(Re)
    H = np.zeros((len(Re), 1, 1), dtype=np.complex128)
    H[idx[(0, 0, 0)], 0, 0] = eps0
    Phi = np.zeros((len(Re), 3, 3), dtype=np.complex128)
    Phi[idx[(0, 0, 0)]] = 2.0 * K * np.eye(3)
    g = np.zeros((len(Re), len(Re), 3, 1, 1), dtype=np.complex128)
    i0 = idx[(0, 0, 0)]
    for a in range(3):
        e = np.zeros(3, dtype=int)
        e[a] = 1
        for s in (+1, -1):
            j = idx[tuple(int(x) for x in s * e)]
            H[j, 0, 0] = -t
            Phi[j, a, a] = -K
            g[i0, j, a, 0, 0] = -s * 0.5j * g0
    return WannierModel(
        lattice="sc", nw=1, nat=1, mass=np.array([mass]),
        Re=Re, wRe=np.ones(len(Re)), H=H,
        Rph=Re.copy(), wRph=np.ones(len(Re)), Phi=Phi,
        Rp=Re.copy(), wRp=np.ones(len(Re)), g=g,
    )


def diatomic_chain_model(M=(1.0, 2.5), Kdiag=(0.010, 0.017, 0.029), couple=0, comp=0, g0=0.05, eps0=0.2, t=0.5):
    """One band; a simple cubic cell (a = 1) with two atoms, kappa = 0 at the origin and
    kappa = 1 at (1/2, 0, 0), masses M; chains along x: each atom bonded to its two x
    neighbours of the other kind by the spring tensor diag(Kdiag) (one chain per Cartesian
    polarisation).  Electrons as in tight_binding_model.  The vertex couples only the
    displacement component `comp` of atom `couple`: g_{couple,comp}(Re=0, Rp=+-e_x) = -+ i g0/2.

    Force constants Phi(R)_{kappa alpha, kappa' beta}: atom kappa in cell 0 with atom kappa'
    in cell R.  Every interpolated quantity has a closed form (used by the tests).
    """
    Re = box_vectors(1)
    idx = _index_of(Re)
    H = np.zeros((len(Re), 1, 1), dtype=np.complex128)
    H[idx[(0, 0, 0)], 0, 0] = eps0
    for a in range(3):
        for sgn in (+1, -1):
            e = [0, 0, 0]
            e[a] = sgn
            H[idx[tuple(e)], 0, 0] = -t
    Kt = np.diag(np.asarray(Kdiag, dtype=np.float64))
    Phi = np.zeros((len(Re), 6, 6), dtype=np.complex128)
    i0, ip, im = idx[(0, 0, 0)], idx[(1, 0, 0)], idx[(-1, 0, 0)]
    Phi[i0, 0:3, 0:3] = 2.0 * Kt
    Phi[i0, 3:6, 3:6] = 2.0 * Kt
    Phi[i0, 0:3, 3:6] = -Kt  # atom 0 with atom 1 of the same cell
    Phi[i0, 3:6, 0:3] = -Kt
    Phi[im, 0:3, 3:6] = -Kt  # atom 0 with atom 1 of the cell at -e_x
    Phi[ip, 3:6, 0:3] = -Kt  # atom 1 with atom 0 of the cell at +e_x
    g = np.zeros((len(Re), len(Re), 6, 1, 1), dtype=np.complex128)
    for sgn in (+1, -1):
        g[i0, idx[(sgn, 0, 0)], 3 * couple + comp, 0, 0] = -sgn * 0.5j * g0
    return WannierModel(
        lattice="sc", nw=1, nat=2, mass=np.asarray(M, dtype=np.float64),
        Re=Re, wRe=np.ones(len(Re)), H=H,
        Rph=Re.copy(), wRph=np.ones(len(Re)), Phi=Phi,
        Rp=Re.copy(), wRp=np.ones(len(Re)), g=g,
    )


def einstein_model(M=1.4, w0=0.06, c=(0.03, -0.02j, 0.05), eps0=0.2, t=0.5):
    """One band, one atom, simple cubic: tight-binding electrons, dispersionless (Einstein)
    phonons Phi(0) = M w0^2 I (three modes of frequency w0) and a constant vertex
    g_a(Re=0, Rp=0) = c_a, so that g_a(k,q) = c_a for every k and q."""
    Re = box_vectors(1)
    idx = _index_of(Re)
    H = np.zeros((len(Re), 1, 1), dtype=np.complex128)
    H[idx[(0, 0, 0)], 0, 0] = eps0
    for a in range(3):
        for sgn in (+1, -1):
            e = [0, 0, 0]
            e[a] = sgn
            H[idx[tuple(e)], 0, 0] = -t
    Phi = np.zeros((len(Re), 3, 3), dtype=np.complex128)
    Phi[idx[(0, 0, 0)]] = M * w0 * w0 * np.eye(3)
    g = np.zeros((len(Re), len(Re), 3, 1, 1), dtype=np.complex128)
    g[idx[(0, 0, 0)], idx[(0, 0, 0)], :, 0, 0] = np.asarray(c, dtype=np.complex128)
    return WannierModel(
        lattice="sc", nw=1, nat=1, mass=np.array([M]),
        Re=Re, wRe=np.ones(len(Re)), H=H,
        Rph=Re.copy(), wRph=np.ones(len(Re)), Phi=Phi,
        Rp=Re.copy(), wRp=np.ones(len(Re)), g=g,
    )


@dataclasses.dataclass
class Workload:
    """One run of the linewidth path: a model, k and q lists, and parameters."""

    name: str
    model: WannierModel
    k: np.ndarray  # [nk,3]
    q: np.ndarray  # [nq,3]
    wq: np.ndarray  # [nq]
    T: float  # K
    EF: float  # eV
    sigma: float  # eV
    omega_min: float = 1e-5  # eV

    @property
    def pairs(self) -> int:
        return len(self.k) * len(self.q)


def load_kpoint_file(path: str):
    """Read a stored k list: a '# EF=<value>' header then one 'kx ky kz' per line."""
    EF = None
    rows = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line:
                continue
            if line.startswith("#"):
                for tok in line[1:].split():
                    if tok.startswith("EF="):
                        EF = float(tok[3:])
                continue
            rows.append([float(x) for x in line.split()])
    return np.array(rows), EF


GOLDEN_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden")

# Workload registry: name -> (description, builder).  Builders take an optional
# q subsample size (for CPU-timed samples) and return a Workload.


def _c1(nq_sub=None):
    rng = np.random.default_rng(SEED_BASE + 0)
    m = make_model("sc", 1, 1, [1.0], None, None, rng, box=1,
                   h_decay=0.7, ge_decay=0.7, gp_decay=0.7, ph_decay=0.7)
    k = uniform_grid(8)
    q = uniform_grid(8)
    if nq_sub:
        q = q[:nq_sub]
    return Workload("sc_nw1_nat1_k8^3_q8^3", m, k, q, np.full(len(q), 1.0 / 512), 300.0, 0.0, 0.050)


def _c2(nq_sub=None, kfile="kwindow_fcc_nw4.txt", T=300.0):
    rng = np.random.default_rng(SEED_BASE + 1)
    m = make_model("fcc", 4, 1, [1.0], 120, 120, rng)
    k, EF = load_kpoint_file(os.path.join(GOLDEN_DIR, kfile))
    q = uniform_grid(40)
    nq_full = len(q)
    if nq_sub:
        q = q[np.random.default_rng(SEED_BASE + 101).choice(nq_full, nq_sub, replace=False)]
    return Workload("fcc_nw4_nat1_k1000win_q40^3", m, k, q, np.full(len(q), 1.0 / nq_full), T, EF, 0.020)


def diamond_nw8_model():
    """Diamond two-atom basis, nw=8, masses 1 and 1.2, 249 Re = Rp (whole fcc shells)."""
    rng = np.random.default_rng(SEED_BASE + 2)
    return make_model("diamond", 8, 2, [1.0, 1.2], 249, 249, rng)


def _c3(nq_sub=None, kfile="kwindow_diamond_nw8.txt", T=300.0):
    """2000 k near the band edges; 60^3 grid plus 10^5 random q, equal weights; sigma 10 meV."""
    m = diamond_nw8_model()
    k, EF = load_kpoint_file(os.path.join(GOLDEN_DIR, kfile))
    q = np.concatenate([uniform_grid(60), random_points(np.random.default_rng(SEED_BASE + 302), 100000)])
    nq_full = len(q)
    if nq_sub:
        q = q[np.random.default_rng(SEED_BASE + 102).choice(nq_full, nq_sub, replace=False)]
    return Workload("diamond_nw8_nat2_k2000edge_q60^3+1e5", m, k, q, np.full(len(q), 1.0 / nq_full), T, EF, 0.010)


def _c5(nq_sub=None):
    rng = np.random.default_rng(SEED_BASE + 4)
    m = make_model("hex", 5, 3, [1.0, 1.1, 1.2], 300, 300, rng)
    k = uniform_grid(20)
    q = uniform_grid(40)
    nq_full = len(q)
    if nq_sub:
        q = q[np.random.default_rng(SEED_BASE + 104).choice(nq_full, nq_sub, replace=False)]
    return Workload("hex_nw5_nat3_k20^3_q40^3", m, k, q, np.full(len(q), 1.0 / nq_full), 50.0, 0.0, 0.015)


# ------------------------------------------------------------ uneven batch
BATCH_NW = (1, 2, 4, 5, 8, 12, 18)


@dataclasses.dataclass
class BatchSpec:
    lattice: str
    nw: int
    nat: int
    nRe: int     # shell target of the electronic (and phonon) R set
    nRp: int     # shell target of the vertex's phonon-displacement R set, drawn independently
    nk: int
    nq_grid: int  # q on an N^3 grid
    seed: int


def batch_specs(n: int = 64, seed: int = SEED_BASE + 3, nR_range=(27, 400), nk_range=(50, 5000),
                nq_range=(16, 48), cap_bytes: float = 64e9, max_nw: int = 18, max_modes: int = 18):
    """Seeded draw of uneven systems: nw from BATCH_NW, nat 1..6, shell targets for Re
    and for Rp each uniform in nR_range (independently), nk log-uniform in nk_range, q
    grids N^3 with N uniform in nq_range.  Redrawn (next seed) until the vertices
    g(Re,Rp) of all systems take at most cap_bytes as complex64.  max_nw / max_modes keep
    only systems within given per-pair limits (each drawn system is kept or dropped
    whole, so the others keep their sizes)."""
    lats = ("sc", "fcc", "diamond", "hex")
    s = seed
    while True:
        rng = np.random.default_rng(s)
        out = []
        for i in range(n):
            lat = lats[rng.integers(len(lats))]
            nw = int(BATCH_NW[rng.integers(len(BATCH_NW))])
            nat = int(rng.integers(1, 7))
            nRe = int(rng.integers(nR_range[0], nR_range[1] + 1))
            nRp = int(rng.integers(nR_range[0], nR_range[1] + 1))
            nk = int(round(math.exp(rng.uniform(math.log(nk_range[0]), math.log(nk_range[1])))))
            N = int(rng.integers(nq_range[0], nq_range[1] + 1))
            out.append(BatchSpec(lat, nw, nat, nRe, nRp, nk, N, int(rng.integers(1 << 30))))
        gbytes = sum(8.0 * b.nRe * b.nRp * 3 * b.nat * b.nw * b.nw for b in out)
        if gbytes <= cap_bytes:
            return [b for b in out if b.nw <= max_nw and 3 * b.nat <= max_modes]
        s += 1


def batch_system(spec: BatchSpec):
    """(model, k [nk,3], q [N^3,3]) of one drawn system; masses 1 + 0.1 i; E_F = 0."""
    rng = np.random.default_rng(spec.seed)
    m = make_model(spec.lattice, spec.nw, spec.nat, [1.0 + 0.1 * i for i in range(spec.nat)], spec.nRe, spec.nRp,
                   rng)
    k = random_points(rng, spec.nk)
    q = uniform_grid(spec.nq_grid)
    return m, k, q


WORKLOADS = {
    "sc_nw1": _c1,
    "fcc_nw4": _c2,
    "diamond_nw8": _c3,
    "hex_nw5": _c5,
}


def make_workload(name: str, nq_sub=None, **kw) -> Workload:
    return WORKLOADS[name](nq_sub=nq_sub, **kw)
