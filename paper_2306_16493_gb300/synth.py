"""Seeded synthetic Wannier-basis inputs for EPWI transport.

This module only *makes inputs*: lattices, masses, lattice-vector sets with their
weights, H(R_e), Phi(R_p) and g(R_e, R_p).  It contains none of the interpolation,
diagonalisation, scattering-rate or transport arithmetic, so both the CUDA path and
the CPU oracle may consume its output without sharing any of the method's code.

The paper reads these arrays from EPW (Sec. III A, description of the CPU flow);
real DFPT data is not available here, so every system is drawn from a documented
random recipe:

* PRNG: SplitMix64 (Steele, Lea & Flood 2014) on a counter, 53-bit uniform doubles,
  Box-Muller normals.  Draw order is fixed per system.
* R-sets: the cube n in {-r..r}^3.  r = 1 has unit weights; r >= 2 uses
  Wigner-Seitz-style boundary weights w = prod_a (1/2 if |n_a| = r else 1), so
  sum(w) = (2r)^3 and the set is symmetric under R -> -R.
* H(R): complex normal (E|z|^2 = sigma_H^2, sigma_H = 1 eV) times exp(-|R|/2 A) for
  R != 0; at R = 0 the diagonal is uniform in [-2, 2] eV and the off-diagonal is
  complex normal with sigma_H.  Then H(R) <- (H(R) + H(-R)^dagger) / 2.
* Semiconductor variant: decoupled valence and conduction Wannier blocks built as
  E_v - D - t_s S(k) - C(k)^dag C(k) and E_c + D + t_s S(k) + B(k)^dag B(k), so the gap
  E_c - E_v is exact and both band edges sit at Gamma (see ``_semiconductor``).
* Phi(R): central springs between atom pairs within the two nearest neighbour shells,
  K = K0 exp(-r/2 A) LogNormal(0, 0.2), Phi_ab(R) = -K rhat rhat^T, the self term set by
  the acoustic sum rule.  K0 is chosen so that the Loewner bound
  D(q) <= 2 blockdiag(Phi_aa(0)/M_a), evaluated with the row-sum norm, caps the
  phonon energy at the requested maximum.
* g(R_e, R_p): complex normal times 0.05 eV/A times exp(-|R_e|/2 - |R_p|/2), layout
  [nRe][nRp][3 nat][nw][nw] (mu, i, j), i pairing with k+q and j with k.

All arrays are unweighted: the R weights are separate and are applied by the consumer.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# CODATA 2018 constants used only to convert the requested phonon energy cap into a
# force-constant scale.
_HBAR_JS = 1.054571817e-34
_AMU_KG = 1.66053906660e-27
_EV_J = 1.602176634e-19
#: hbar^2 / (amu * A^2) expressed in eV.
HBAR2_OVER_AMU_A2_EV = _HBAR_JS ** 2 / (_AMU_KG * 1e-20) / _EV_J


class SplitMix64:
    """Counter-based SplitMix64 stream (vectorised over numpy uint64)."""

    _GAMMA = np.uint64(0x9E3779B97F4A7C15)
    _M1 = np.uint64(0xBF58476D1CE4E5B9)
    _M2 = np.uint64(0x94D049BB133111EB)

    def __init__(self, seed: int):
        self.state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)

    def next_u64(self, n: int) -> np.ndarray:
        with np.errstate(over="ignore"):
            idx = np.arange(1, n + 1, dtype=np.uint64)
            z = self.state + idx * self._GAMMA
            self.state = self.state + np.uint64(n) * self._GAMMA
            z = (z ^ (z >> np.uint64(30))) * self._M1
            z = (z ^ (z >> np.uint64(27))) * self._M2
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, n: int) -> np.ndarray:
        """n doubles in [0, 1) with 53 random bits."""
        return (self.next_u64(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def normal(self, n: int) -> np.ndarray:
        """n standard normals by Box-Muller (both outputs of each pair are used)."""
        m = (n + 1) // 2
        u1 = 1.0 - self.uniform(m)          # (0, 1]
        u2 = self.uniform(m)
        r = np.sqrt(-2.0 * np.log(u1))
        out = np.empty(2 * m)
        out[0::2] = r * np.cos(2.0 * np.pi * u2)
        out[1::2] = r * np.sin(2.0 * np.pi * u2)
        return out[:n]

    def complex_normal(self, shape, sigma=1.0) -> np.ndarray:
        n = int(np.prod(shape))
        if n < self._CHUNK:
            z = self.normal(2 * n)
            return (sigma / math.sqrt(2.0)) * (z[0::2] + 1j * z[1::2]).reshape(shape)
        return self._complex_normal_chunked(n, sigma).reshape(shape)

    # Large draws: element j of complex_normal depends only on the stream values at counter
    # offsets j + 1 (u1) and n + j + 1 (u2), so chunks are computed independently, in
    # threads, with the same elementwise operations as ``normal`` (identical results).
    _CHUNK = 1 << 21

    def _complex_normal_chunked(self, n: int, sigma: float) -> np.ndarray:
        from concurrent.futures import ThreadPoolExecutor
        import os

        out = np.empty(n, np.complex128)
        s0 = self.state
        scale = sigma / math.sqrt(2.0)

        def draw(start, count):
            with np.errstate(over="ignore"):
                z = s0 + np.arange(start + 1, start + count + 1, dtype=np.uint64) * self._GAMMA
                z = (z ^ (z >> np.uint64(30))) * self._M1
                z = (z ^ (z >> np.uint64(27))) * self._M2
                z = z ^ (z >> np.uint64(31))
            return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

        def work(a):
            b = min(n, a + self._CHUNK)
            u1 = 1.0 - draw(a, b - a)
            u2 = draw(n + a, b - a)
            r = np.sqrt(-2.0 * np.log(u1))
            out[a:b] = scale * (r * np.cos(2.0 * np.pi * u2) + 1j * (r * np.sin(2.0 * np.pi * u2)))

        with ThreadPoolExecutor(max_workers=max(1, os.cpu_count() or 1)) as ex:
            list(ex.map(work, range(0, n, self._CHUNK)))
        with np.errstate(over="ignore"):
            self.state = self.state + np.uint64(2 * n) * self._GAMMA
        return out


@dataclasses.dataclass
class System:
    """One crystal in the Wannier basis (all arrays C row-major, unweighted)."""

    name: str
    lattice: np.ndarray      # (3, 3) rows a1, a2, a3 in A
    tau: np.ndarray          # (nat, 3) Cartesian atom positions in A (input recipe only)
    mass: np.ndarray         # (nat,) amu
    nw: int
    Re: np.ndarray           # (nRe, 3) int32 lattice coordinates
    we: np.ndarray           # (nRe,) weights
    H: np.ndarray            # (nRe, nw, nw) complex128, eV
    Rp: np.ndarray           # (nRp, 3) int32
    wp: np.ndarray           # (nRp,)
    Phi: np.ndarray          # (nRp, 3nat, 3nat) float64, eV/A^2
    g: np.ndarray            # (nRe, nRp, 3nat, nw, nw) complex128, eV/A
    n_valence: int = 0       # number of valence Wannier functions (semiconductor), else 0
    seed: int = 0

    @property
    def nat(self) -> int:
        return int(self.mass.shape[0])

    @property
    def nm(self) -> int:
        return 3 * self.nat

    @property
    def volume(self) -> float:
        return float(abs(np.linalg.det(self.lattice)))


def r_cube(r: int, ws_weights: bool):
    """Lattice coordinates n in {-r..r}^3 (n3 fastest) and their weights."""
    ax = np.arange(-r, r + 1)
    n = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), axis=-1).reshape(-1, 3)
    if ws_weights:
        w = np.prod(np.where(np.abs(n) == r, 0.5, 1.0), axis=1)
    else:
        w = np.ones(len(n))
    return n.astype(np.int32), w


def ws_rset(lat, nsc: int, tol: float = 1e-6):
    """Wigner-Seitz set of the nsc x nsc x nsc supercell of ``lat``: the lattice vectors R (in
    lattice coordinates n, R = n @ lat) that are no farther from the origin than from any
    supercell image nsc T @ lat, with weight 1 / (number of images at that same distance),
    so that sum(w) = nsc^3.  Unlike ``r_cube`` this set is not a cube in lattice coordinates
    (for fcc and nsc = 4: 93 vectors up to |n_a| = 3).  Sorted by n (n3 fastest); closed
    under R -> -R."""
    lat = np.asarray(lat, float)
    ax = np.arange(-2 * nsc, 2 * nsc + 1)
    n = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), axis=-1).reshape(-1, 3)
    tr = np.stack(np.meshgrid(*(np.arange(-2, 3),) * 3, indexing="ij"), axis=-1).reshape(-1, 3)
    R = n @ lat
    d0 = np.linalg.norm(R, axis=1)
    dT = np.linalg.norm(R[:, None, :] + ((nsc * tr) @ lat)[None, :, :], axis=-1)
    eps = tol * nsc * np.abs(lat).max()
    inside = d0 <= dT.min(axis=1) + eps
    deg = (np.abs(dT - d0[:, None]) <= eps).sum(axis=1)
    sel = np.nonzero(inside)[0]
    return n[sel].astype(np.int32), 1.0 / deg[sel]


def _minus_index(R: np.ndarray) -> np.ndarray:
    lut = {tuple(v): i for i, v in enumerate(R.tolist())}
    return np.array([lut[tuple((-v).tolist())] for v in R])


def fcc_cell(a: float):
    lat = 0.5 * a * np.array([[0.0, 1.0, 1.0], [1.0, 0.0, 1.0], [1.0, 1.0, 0.0]])
    return lat, np.zeros((1, 3))


def diamond_cell(a: float):
    lat, _ = fcc_cell(a)
    return lat, np.array([[0.0, 0.0, 0.0], [0.25 * a, 0.25 * a, 0.25 * a]])


def cubic_cell(nat: int, a: float = 4.05):
    """Cells with more atoms for the batched workload (conventional fcc, 3x2x1 sc)."""
    if nat == 4:
        lat = a * np.eye(3)
        tau = a * np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]], float)
        return lat, tau
    if nat == 6:
        s = 2.8
        lat = np.diag([3 * s, 2 * s, s])
        tau = np.array([[i * s, j * s, 0.0] for i in range(3) for j in range(2)])
        return lat, tau
    raise ValueError(nat)


def _hamiltonian(rng: SplitMix64, lat, Re, nw, sigma_h=1.0, onsite=2.0):
    nR = len(Re)
    Rc = Re @ lat
    dist = np.linalg.norm(Rc, axis=1)
    H = rng.complex_normal((nR, nw, nw), sigma_h) * np.exp(-dist / 2.0)[:, None, None]
    i0 = int(np.where((Re == 0).all(1))[0][0])
    diag = rng.uniform(nw) * 2.0 * onsite - onsite
    H[i0][np.diag_indices(nw)] = diag
    mi = _minus_index(Re)
    H = 0.5 * (H + np.conj(np.transpose(H[mi], (0, 2, 1))))
    return H, i0


def _springs(rng: SplitMix64, lat, tau, mass, Rp, wp, omega_max_ev):
    nat = len(tau)
    nm = 3 * nat
    Rc = Rp @ lat
    # distances of every (a, b, R) bond, to find the two nearest shells
    d = np.linalg.norm(tau[None, :, None, :] + Rc[:, None, None, :] - tau[None, None, :, :],
                       axis=-1)  # [R][b][a]: vector from a to b+R
    dpos = np.unique(np.round(d[d > 1e-8], 6))
    cutoff = dpos[1] + 1e-4 if len(dpos) > 1 else dpos[0] + 1e-4
    Phi = np.zeros((len(Rp), nm, nm))
    mi = _minus_index(Rp)
    # enumerate unordered bonds: (a, b, R) ~ (b, a, -R)
    for iR in range(len(Rp)):
        for a in range(nat):
            for b in range(nat):
                key = (iR, a, b)
                partner = (mi[iR], b, a)
                if partner < key:
                    continue
                r = d[iR, b, a]
                if r < 1e-8 or r > cutoff:
                    continue
                if wp[iR] != 1.0:
                    raise ValueError("spring reaches a boundary-weighted image")
                ln = rng.normal(1)[0]
                K = math.exp(-r / 2.0) * math.exp(0.2 * ln)
                rh = (tau[b] + Rc[iR] - tau[a]) / r
                blk = -K * np.outer(rh, rh)
                Phi[iR, 3 * a:3 * a + 3, 3 * b:3 * b + 3] += blk
                if partner != key:
                    Phi[mi[iR], 3 * b:3 * b + 3, 3 * a:3 * a + 3] += blk.T
    i0 = int(np.where((Rp == 0).all(1))[0][0])
    for a in range(nat):
        s = np.zeros((3, 3))
        for iR in range(len(Rp)):
            for b in range(nat):
                if iR == i0 and b == a:
                    continue
                s += wp[iR] * Phi[iR, 3 * a:3 * a + 3, 3 * b:3 * b + 3]
        Phi[i0, 3 * a:3 * a + 3, 3 * a:3 * a + 3] = -s
    # scale K0 with the Loewner row-sum bound of the dynamical matrix
    bound = 0.0
    for a in range(nat):
        blk = Phi[i0, 3 * a:3 * a + 3, 3 * a:3 * a + 3]
        bound = max(bound, 2.0 * np.abs(blk).sum(1).max() / mass[a])
    K0 = (omega_max_ev ** 2 / HBAR2_OVER_AMU_A2_EV) / bound
    return Phi * K0


def _gmat(rng: SplitMix64, lat, Re, Rp, nm, nw, scale=0.05):
    de = np.linalg.norm(Re @ lat, axis=1)
    dp = np.linalg.norm(Rp @ lat, axis=1)
    env = scale * np.exp(-de / 2.0)[:, None] * np.exp(-dp / 2.0)[None, :]
    g = rng.complex_normal((len(Re), len(Rp), nm, nw, nw))
    return g * env[:, :, None, None, None]


def _semiconductor(rng: SplitMix64, lat, R, w, nv, nc, gap_ev, sigma_b=0.5, t_s=0.25,
                   split=0.1):
    """Decoupled valence and conduction Wannier blocks with an exact gap at Gamma.

    Conduction: H_c(k) = E_c + D + t_s S(k) + B(k)^dag B(k); valence:
    H_v(k) = E_v - D - t_s S(k) - C(k)^dag C(k), with D = diag(0, split, 2 split, ...),
    S(k) = sum over the nearest lattice vectors of (1 - cos k.R) >= 0 (zero only at Gamma)
    and B(R), C(R) complex normal (sigma_b) times exp(-|R|/2) on |n_a| <= 1 with
    sum_R B(R) = sum_R C(R) = 0.  Every term beyond E_c (E_v) is positive (negative)
    semidefinite and vanishes at Gamma for the first band, so the conduction minimum is
    E_c = gap and the valence maximum is E_v = 0, both at Gamma, on any Gamma-centred grid.
    In R space B(k)^dag B(k) = sum_R e^{ik.R} sum_R' B(R')^dag B(R'+R).
    """
    nR = len(R)
    lut = {tuple(v): i for i, v in enumerate(R.tolist())}
    i0 = lut[(0, 0, 0)]
    inner = np.where(np.abs(R).max(1) <= 1)[0]
    dist = np.linalg.norm(R @ lat, axis=1)
    nz = dist > 1e-9
    nn = np.where(nz & (np.abs(dist - dist[nz].min()) < 1e-6))[0]
    H = np.zeros((nR, nv + nc, nv + nc), complex)

    def square(nb):
        B = rng.complex_normal((len(inner), nb, nb), sigma_b) \
            * np.exp(-dist[inner] / 2.0)[:, None, None]
        B[np.where(inner == i0)[0][0]] -= B.sum(0)
        out = np.zeros((nR, nb, nb), complex)
        for a, ia in enumerate(inner):
            for b, ib in enumerate(inner):
                d = tuple((R[ib] - R[ia]).tolist())
                if d in lut:
                    out[lut[d]] += B[a].conj().T @ B[b]
                else:
                    raise ValueError("R-set too small for the conduction block")
        if np.any(w[np.abs(out).reshape(nR, -1).max(1) > 0] != 1.0):
            raise ValueError("semiconductor block reaches a boundary-weighted image")
        return out

    def scalar(nb, sign, e0):
        out = np.zeros((nR, nb, nb), complex)
        out[i0] += (e0 + sign * t_s * len(nn)) * np.eye(nb) + sign * np.diag(split * np.arange(nb))
        for i in nn:
            out[i] += -sign * t_s * np.eye(nb)
        return out

    cblk = scalar(nc, +1.0, gap_ev) + square(nc)
    vblk = scalar(nv, -1.0, 0.0) - square(nv)
    H[:, :nv, :nv] = vblk
    H[:, nv:, nv:] = cblk
    return H


def make_system(name: str, lat, tau, mass, nw, r, ws, seed, omega_max_ev,
                n_valence=0, gap_ev=1.1, rset=None) -> System:
    rng = SplitMix64(seed)
    R, w = r_cube(r, ws) if rset is None else rset
    mass = np.asarray(mass, float) * np.ones(len(tau))
    H, i0 = _hamiltonian(rng, lat, R, nw)
    if n_valence:
        H = _semiconductor(rng, lat, R, w, n_valence, nw - n_valence, gap_ev)
    Phi = _springs(rng, lat, np.asarray(tau, float), mass, R, w, omega_max_ev)
    g = _gmat(rng, lat, R, R, 3 * len(tau), nw)
    return System(name=name, lattice=np.asarray(lat, float), tau=np.asarray(tau, float),
                  mass=mass, nw=nw, Re=R.copy(), we=w.copy(), H=H, Rp=R.copy(),
                  wp=w.copy(), Phi=Phi, g=g, n_valence=n_valence, seed=seed)


def tiny_system(seed: int = 1) -> System:
    """fcc 1 atom, a = 4.05 A, M = 27 amu, nw = 4, 3^3 R-sets (unit weights)."""
    lat, tau = fcc_cell(4.05)
    return make_system("tiny", lat, tau, 27.0, 4, 1, False, seed, 0.040)


def al_like_system(seed: int = 2) -> System:
    """fcc Al-like metal: nw = 4, 3 modes, 5^3 Wigner-Seitz-weighted R-sets."""
    lat, tau = fcc_cell(4.05)
    return make_system("al_like", lat, tau, 27.0, 4, 2, True, seed, 0.040)


def al_like_ws_system(seed: int = 2, nsc: int = 4) -> System:
    """fcc Al-like metal on genuine Wigner-Seitz R-sets: nw = 4, 3 modes, Re = Rp = the WS set
    of the nsc^3 supercell (93 vectors for nsc = 4, fractional weights summing to 64)."""
    lat, tau = fcc_cell(4.05)
    return make_system("al_like_ws", lat, tau, 27.0, 4, 0, False, seed, 0.040, rset=ws_rset(lat, nsc))


def point_group(lat) -> list:
    """The lattice's point group as integer matrices M acting on lattice coordinates (n -> M n,
    columns): every M with entries in {-1, 0, 1}, |det M| = 1 and M^T G M = G for the metric
    G = A A^T (A rows = a_1, a_2, a_3).  48 matrices for fcc and simple cubic."""
    lat = np.asarray(lat, float)
    G = lat @ lat.T
    ops = []
    for e in np.ndindex(*(3,) * 9):
        M = np.array(e).reshape(3, 3) - 1
        if round(abs(np.linalg.det(M))) == 1 and np.allclose(M.T @ G @ M, G, atol=1e-9 * np.abs(G).max()):
            ops.append(M.astype(np.int64))
    return ops


def kpoint_ops(ops) -> np.ndarray:
    """The k-space action of lattice operations M: fractional k -> M^{-T} k (integer for a
    unimodular M), so that e^{2 pi i k.n} is invariant when n -> M n.  [nops][3][3] int32."""
    return np.array([np.rint(np.linalg.inv(M).T).astype(np.int32) for M in ops])


def symmetrize(sysm: System, ops) -> System:
    """The crystal made invariant under the lattice operations ``ops`` (a group; one atom at the
    origin, s-like Wannier functions): H(R) is averaged over each orbit, H(M R) = H(R);
    Phi(M R) = S Phi(R) S^T and g_mu(M Re, M Rp) = sum_nu S_mu,nu g_nu(Re, Rp) with the Cartesian
    rotation S = A^T M A^{-T}, made exact by group averaging.  Both R-sets must be closed under
    the group with invariant weights (a Wigner-Seitz set is).  Averaging keeps Hermiticity, the
    acoustic sum rule and Phi(-R) = Phi(R)^T."""
    if sysm.nat != 1:
        raise ValueError("symmetrize: one atom at the origin only")
    A = sysm.lattice
    S = [A.T @ M @ np.linalg.inv(A.T) for M in ops]

    def index(R):
        lut = {tuple(v): i for i, v in enumerate(R.tolist())}
        idx = []
        for M in ops:
            idx.append(np.array([lut[tuple((M @ v).tolist())] for v in R]))
        return idx
    ie, ip = index(sysm.Re), index(sysm.Rp)
    for k in range(len(ops)):
        if not (np.allclose(sysm.we[ie[k]], sysm.we) and np.allclose(sysm.wp[ip[k]], sysm.wp)):
            raise ValueError("symmetrize: weights are not invariant")
    H = sum(sysm.H[ie[k]] for k in range(len(ops))) / len(ops)
    Phi = sum(np.einsum("ba,rbc,cd->rad", S[k], sysm.Phi[ip[k]], S[k]) for k in range(len(ops))) / len(ops)
    g = sum(np.einsum("ba,rpbij->rpaij", S[k], sysm.g[ie[k]][:, ip[k]]) for k in range(len(ops))) / len(ops)
    return dataclasses.replace(sysm, name=sysm.name + "_sym", H=H, Phi=Phi, g=g)


def al_like_sym_system(seed: int = 2) -> System:
    """The Wigner-Seitz Al-like metal (``al_like_ws_system``) made invariant under the 48
    operations of the fcc point group (``symmetrize``): eps(M^{-T} k) = eps(k) and the SERTA
    rates are equal on every star of k-points."""
    s = al_like_ws_system(seed)
    return symmetrize(s, point_group(s.lattice))


def si_like_system(seed: int = 3) -> System:
    """Diamond Si-like semiconductor: nw = 8 (4 valence + 4 conduction), 6 modes, 7^3 R."""
    lat, tau = diamond_cell(5.43)
    return make_system("si_like", lat, tau, 28.0, 8, 3, True, seed, 0.060,
                       n_valence=4, gap_ev=1.1)


def time_reversal_symmetric(sysm: System) -> System:
    """The same crystal with real Wannier-basis H(R) and g(Re, Rp) (their real parts).

    With H(-R) = H(R)^T real, H(-k) = H(k)^* and eps(-k) = eps(k), v(-k) = -v(k); with real g,
    |g(-k,-q)| = |g(k,q)|.  A Gamma-centred grid is closed under k -> -k, so every sum of an
    odd function of k vanishes exactly, as for a crystal with time-reversal symmetry."""
    return dataclasses.replace(sysm, name=sysm.name + "_tr", H=sysm.H.real.astype(complex),
                               g=sysm.g.real.astype(complex))


def einstein_system(t_ev: float = 0.5, a: float = 3.0, spring: float = 5.0,
                    g_ev_a: float = 0.05) -> System:
    """Isotropic-scattering test crystal: simple cubic, one s-like Wannier function with
    nearest-neighbour hopping -t (eps(k) = -2t sum_i cos 2 pi k_i), one atom of 27 amu held by
    an on-site spring only (three degenerate, dispersionless modes), and a coupling that is
    local in both lattice vectors (only Re = Rp = 0, the same real value for each Cartesian
    direction).  3^3 R-sets with unit weights.  No random numbers."""
    R, w = r_cube(1, False)
    nR = len(R)
    H = np.zeros((nR, 1, 1), complex)
    for i, v in enumerate(R.tolist()):
        if sum(abs(x) for x in v) == 1:
            H[i, 0, 0] = -t_ev
    i0 = int(np.nonzero((R == 0).all(axis=1))[0][0])
    Phi = np.zeros((nR, 3, 3))
    Phi[i0] = spring * np.eye(3)
    g = np.zeros((nR, nR, 3, 1, 1), complex)
    g[i0, i0, :, 0, 0] = g_ev_a
    return System(name="einstein", lattice=a * np.eye(3), tau=np.zeros((1, 3)),
                  mass=np.array([27.0]), nw=1, Re=R.copy(), we=w.copy(), H=H, Rp=R.copy(),
                  wp=w.copy(), Phi=Phi, g=g, n_valence=0, seed=0)


def batch_system(s: int) -> tuple[System, int]:
    """System s (0..63) of the uneven batch: s = 16 a + 4 b + c.

    nat = [1, 2, 4, 6][c], nw = [4, 8, 16, 24][b], grid = [24, 36, 48, 60][a] per axis,
    R cube side = [3, 5, 7][(a + b + c) mod 3]; metal generator, seed 100 + s.
    Returns the system and its grid size.
    """
    a, b, c = s // 16, (s // 4) % 4, s % 4
    nat = [1, 2, 4, 6][c]
    nw = [4, 8, 16, 24][b]
    grid = [24, 36, 48, 60][a]
    r = [1, 2, 3][(a + b + c) % 3]
    if nat == 1:
        lat, tau = fcc_cell(4.05)
    elif nat == 2:
        lat, tau = diamond_cell(5.43)
    else:
        lat, tau = cubic_cell(nat)
    sysm = make_system(f"batch{s}", lat, tau, 27.0, nw, r, r >= 2, 100 + s, 0.040)
    return sysm, grid
