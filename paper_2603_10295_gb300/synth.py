"""Seeded synthetic inputs shaped like the paper's silicon, MoS2 and stanene workloads.

This module builds *inputs* only: lattice vectors, Wigner-Seitz-like R sets, a
Hermitian-paired Wannier Hamiltonian H(Re), pair-spring force constants Phi(Rp)
obeying the acoustic sum rule, the Wannier-space coupling g(Re,Rp) (Eq. 3) and
fine k/q lists.  It holds none of the interpolation arithmetic; both the CPU
oracle and the CUDA path consume the arrays it returns.

Recipe (one numpy ``default_rng(seed)``, draws in this order):
  1. H(R): for R = 0 a complex N(0,1) matrix A gives H(0) = (A + A^H)/2; for each
     R whose first nonzero coordinate is positive and whose -R is also in the set,
     A (real part then imaginary part, each N(0,1)) times exp(-|R|/lam_H) gives
     H(R) = A and H(-R) = A^H.  An R whose -R is outside the set keeps H(R) = 0.
  2. Springs: for every unordered pair {(kappa,0), (kappa',R)} with R = 0 or R
     "positive" (and -R in the set), B ~ N(0,1)^{3x3} and
     K = s exp(-|R|/lam_Phi) B B^T / 3, s = 10 eV/A^2.  Off-site blocks get -K,
     on-site blocks get +K (acoustic sum rule holds exactly).
  3. g(Re,Rp) [Np][Nm][Ne][Nb][Nb]: real part, then imaginary part, each N(0,1),
     times 0.1 eV exp(-(|Re|+|Rp|)/lam_g).
  4. k points (if random), 5. q points.
|R| is the Cartesian length of n1 a1 + n2 a2 + n3 a3 (cell to cell).
Units: eV, Angstrom, amu.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SPRING_SCALE_EV_A2 = 10.0


@dataclasses.dataclass
class Workload:
    name: str
    nb: int
    na: int
    masses: np.ndarray          # [na] amu
    lattice: np.ndarray         # [3][3] rows a1, a2, a3 (Angstrom)
    Re: np.ndarray              # [ne][3] int32
    Rp: np.ndarray              # [np][3] int32
    we: np.ndarray              # [ne] f64
    wp: np.ndarray              # [np] f64
    H_Re: np.ndarray            # [ne][nb][nb] complex128, eV
    Phi_Rp: np.ndarray          # [np][nm][nm] f64, eV/A^2
    g_ReRp: np.ndarray          # [np][nm][ne][nb][nb] complex128, eV
    kpts: np.ndarray            # [nk][3] f64, crystal coordinates
    qpts: np.ndarray            # [nq][3] f64
    kgrid: tuple | None = None  # (n1, n2, n3) when kpts is a uniform grid

    @property
    def nm(self) -> int:
        return 3 * self.na

    @property
    def ne(self) -> int:
        return len(self.Re)

    @property
    def np_(self) -> int:
        return len(self.Rp)


def fcc_lattice(a: float) -> np.ndarray:
    return 0.5 * a * np.array([[0.0, 1.0, 1.0], [1.0, 0.0, 1.0], [1.0, 1.0, 0.0]])


def hex_lattice(a: float, c: float = 20.0) -> np.ndarray:
    return np.array([[a, 0.0, 0.0], [-0.5 * a, 0.5 * math.sqrt(3.0) * a, 0.0], [0.0, 0.0, c]])


def chain_lattice_b(a: float) -> np.ndarray:
    """Ribbon periodic along the second lattice vector; the other two never appear (n1 = n3 = 0)."""
    return np.array([[30.0, 0.0, 0.0], [0.0, a, 0.0], [0.0, 0.0, 30.0]])


def box_vectors(r1, r2, r3) -> np.ndarray:
    """All integer vectors of a box, first coordinate slowest; each r is an iterable of ints."""
    out = [(i, j, k) for i in r1 for j in r2 for k in r3]
    return np.asarray(out, dtype=np.int32)


def centred_range(n: int) -> range:
    """{-n/2, ..., n/2-1} for even n, {-(n-1)/2, ..., (n-1)/2} for odd n."""
    return range(-(n // 2), n - n // 2)


def cart_length(R: np.ndarray, lattice: np.ndarray) -> np.ndarray:
    return np.linalg.norm(R.astype(np.float64) @ lattice, axis=-1)


def _index_of(R: np.ndarray) -> dict:
    return {tuple(int(x) for x in r): i for i, r in enumerate(R)}


def _positive(r) -> bool:
    for x in r:
        if x != 0:
            return x > 0
    return False


def draw_hamiltonian(rng, R, lattice, nb, lam, real=False):
    """H(R) with H(-R) = H(R)^H.  real: H(R) real (H(-R) = H(R)^T), i.e. a Hamiltonian with
    time-reversal symmetry, H(-k) = conj H(k) (draws one real matrix per +-R pair)."""
    ne = len(R)
    H = np.zeros((ne, nb, nb), dtype=np.complex128)
    idx = _index_of(R)
    L = cart_length(R, lattice)

    def draw():
        if real:
            return rng.standard_normal((nb, nb)).astype(np.complex128)
        return rng.standard_normal((nb, nb)) + 1j * rng.standard_normal((nb, nb))

    for i, r in enumerate(R):
        r = tuple(int(x) for x in r)
        j = idx.get(tuple(-x for x in r))
        if j is None:
            continue
        if i == j:
            A = draw()
            H[i] = 0.5 * (A + A.conj().T)
        elif _positive(r):
            A = draw() * math.exp(-L[i] / lam)
            H[i] = A
            H[j] = A.conj().T
    return H


def draw_force_constants(rng, R, lattice, na, lam, scale=SPRING_SCALE_EV_A2):
    nR = len(R)
    nm = 3 * na
    Phi = np.zeros((nR, nm, nm), dtype=np.float64)
    idx = _index_of(R)
    L = cart_length(R, lattice)
    i0 = idx.get((0, 0, 0))
    if i0 is None:
        raise ValueError("R set must contain the origin")
    for i, r in enumerate(R):
        r = tuple(int(x) for x in r)
        j = idx.get(tuple(-x for x in r))
        if j is None:
            continue
        if i != i0 and not _positive(r):
            continue
        for ka in range(na):
            for kb in range(na):
                if i == i0 and kb <= ka:
                    continue
                B = rng.standard_normal((3, 3))
                K = scale * math.exp(-L[i] / lam) * (B @ B.T) / 3.0
                sa, sb = slice(3 * ka, 3 * ka + 3), slice(3 * kb, 3 * kb + 3)
                Phi[i, sa, sb] -= K
                Phi[j, sb, sa] -= K.T
                Phi[i0, sa, sa] += K
                Phi[i0, sb, sb] += K
    return Phi


def draw_coupling(rng, Re, Rp, lattice, na, nb, lam, amp=0.1):
    ne, np_ = len(Re), len(Rp)
    nm = 3 * na
    shape = (np_, nm, ne, nb, nb)
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    g = re + 1j * im
    del re, im
    Le = cart_length(Re, lattice)
    Lp = cart_length(Rp, lattice)
    decay = amp * np.exp(-(Lp[:, None] + Le[None, :]) / lam)      # [np][ne]
    g *= decay[:, None, :, None, None]
    return g


def uniform_grid(n1, n2, n3) -> np.ndarray:
    g = np.stack(np.meshgrid(np.arange(n1) / n1, np.arange(n2) / n2, np.arange(n3) / n3, indexing="ij"), -1)
    return g.reshape(-1, 3).astype(np.float64)


def random_points(rng, n, dims) -> np.ndarray:
    """Uniform random points in [0,1) along the periodic directions `dims` (others 0)."""
    out = np.zeros((n, 3))
    r = rng.random((n, len(dims)))
    for c, d in enumerate(dims):
        out[:, d] = r[:, c]
    return out


# name -> parameters.  Each config is a synthetic stand-in for one of the paper's
# workloads (silicon mobility, MoS2 self-energy, zigzag stanene nanoribbon).
CONFIGS = {
    "si_tiny": dict(lattice=("fcc", 5.43), nb=8, masses=[28.0855] * 2,
                    box=(range(-1, 2), range(-1, 2), range(-1, 2)),
                    lam=(2.0, 2.0, 3.0), k=("random", 64), q=("random", 16), dims=(0, 1, 2)),
    "si_full": dict(lattice=("fcc", 5.43), nb=8, masses=[28.0855] * 2,
                    box=(centred_range(6), centred_range(6), centred_range(6)),
                    lam=(2.0, 2.0, 3.0), k=("grid", (40, 40, 40)), q=("random", 1000), dims=(0, 1, 2)),
    "mos2": dict(lattice=("hex", 3.16), nb=11, masses=[95.95, 32.06, 32.06],
                 box=(centred_range(12), centred_range(12), range(0, 1)),
                 lam=(3.0, 3.0, 3.0), k=("grid", (200, 200, 1)), q=("random", 2000), dims=(0, 1)),
    "mos2_diff": dict(lattice=("hex", 3.16), nb=11, masses=[95.95, 32.06, 32.06],
                      box=(centred_range(12), centred_range(12), range(0, 1)),
                      lam=(3.0, 3.0, 3.0), k=("grid", (48, 48, 1)), q=("random", 256), dims=(0, 1)),
    "stanene": dict(lattice=("chain_b", 4.67), nb=120, masses=[118.71] * 60,
                    box=(range(0, 1), range(-7, 8), range(0, 1)),
                    lam=(5.0, 5.0, 5.0), k=("grid", (1, 512, 1)), q=("random", 1400), dims=(1,)),
}

STANENE_Q_BATCHES = (17, 400, 113, 256, 64, 331, 29, 190)


def _lattice(spec):
    kind, a = spec
    if kind == "fcc":
        return fcc_lattice(a)
    if kind == "hex":
        return hex_lattice(a)
    if kind == "chain_b":
        return chain_lattice_b(a)
    raise ValueError(kind)


def make_workload(name: str, seed: int = 0, nq: int | None = None, nk: int | None = None,
                  nb: int | None = None, box=None, with_coupling: bool = True, na: int | None = None,
                  real_h: bool = False) -> Workload:
    """Build a named workload.  nq/nk/nb/na/box override the config (smaller cases for tests);
    real_h draws real H(R) (time-reversal symmetric bands, eps(-k) = eps(k))."""
    cfg = dict(CONFIGS[name])
    rng = np.random.default_rng(seed)
    lat = _lattice(cfg["lattice"])
    nb = cfg["nb"] if nb is None else nb
    masses = np.asarray(cfg["masses"], dtype=np.float64)
    if na is not None:
        masses = np.resize(masses, na)
    na = len(masses)
    R = box_vectors(*(box if box is not None else cfg["box"]))
    lamH, lamP, lamG = cfg["lam"]
    H = draw_hamiltonian(rng, R, lat, nb, lamH, real=real_h)
    Phi = draw_force_constants(rng, R, lat, na, lamP)
    g = draw_coupling(rng, R, R, lat, na, nb, lamG) if with_coupling else None
    kspec, qspec = cfg["k"], cfg["q"]
    kgrid = None
    if kspec[0] == "grid" and nk is None:
        kgrid = tuple(kspec[1])
        kpts = uniform_grid(*kgrid)
    else:
        kpts = random_points(rng, nk if nk is not None else kspec[1], cfg["dims"])
    qpts = random_points(rng, nq if nq is not None else qspec[1], cfg["dims"])
    ones = np.ones(len(R))
    return Workload(name=name, nb=nb, na=na, masses=masses, lattice=lat, Re=R, Rp=R.copy(),
                    we=ones, wp=ones.copy(), H_Re=H, Phi_Rp=Phi, g_ReRp=g, kpts=kpts, qpts=qpts,
                    kgrid=kgrid)
