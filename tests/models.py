"""Closed-form test systems (inputs only) and their analytic band, phonon and coupling values.

One-band nearest-neighbour tight binding on a simple-cubic lattice (lattice constant a):
H(0) = eps0, H(+-a_hat) = -t, so eps(k) = eps0 - 2 t sum_a cos(2 pi k_a) and
v_a = (2 t a / hbar) sin(2 pi k_a).
Axial springs K along +-a_hat on one atom of mass M: Phi(0) = 2K I, Phi(+-a_hat)_aa = -K, so
D(q) is diagonal, (hbar omega_a)^2 = C 4K/M sin^2(pi q_a) with C = hbar^2/(amu A^2).
Deformation-potential coupling g^a(Re = 0, Rp = +-a_hat) = +-D/(2a): the Wannier sum gives
G^a(k, q) = i (D/a) sin(2 pi q_a) and g_nu=a = G^a (C / (2 M hbar omega_a))^{1/2}, so
|g_a|^2 = (D/a)^2 sin^2(2 pi q_a) C / (2 M hbar omega_a), independent of k.
"""
import numpy as np

from paper_2306_16493_gb300.synth import HBAR2_OVER_AMU_A2_EV, System, r_cube

C_EV = HBAR2_OVER_AMU_A2_EV


def tb_dp_system(a=3.0, t=0.8, eps0=0.3, K=2.0, M=20.0, D=1.5, r=1) -> System:
    R, w = r_cube(r, False)
    lut = {tuple(v): i for i, v in enumerate(R.tolist())}
    i0 = lut[(0, 0, 0)]
    H = np.zeros((len(R), 1, 1), complex)
    H[i0, 0, 0] = eps0
    Phi = np.zeros((len(R), 3, 3))
    Phi[i0] = 2.0 * K * np.eye(3)
    g = np.zeros((len(R), len(R), 3, 1, 1), complex)
    for ax in range(3):
        for s in (1, -1):
            n = [0, 0, 0]
            n[ax] = s
            iR = lut[tuple(n)]
            H[iR, 0, 0] = -t
            Phi[iR, ax, ax] = -K
            g[i0, iR, ax, 0, 0] = s * D / (2.0 * a)
    return System(name="tb_dp", lattice=a * np.eye(3), tau=np.zeros((1, 3)),
                  mass=np.array([M]), nw=1, Re=R, we=w, H=H, Rp=R.copy(), wp=w.copy(),
                  Phi=Phi, g=g)


def tb_eps(kfrac, a=3.0, t=0.8, eps0=0.3):
    return eps0 - 2.0 * t * np.cos(2 * np.pi * kfrac).sum(-1)


def tb_vel(kfrac, a=3.0, t=0.8, hbar_evs=6.582119569e-16):
    return 2.0 * t * a / hbar_evs * np.sin(2 * np.pi * kfrac) * 1e-10


def spring_hw(qfrac, K=2.0, M=20.0):
    return np.sqrt(C_EV * 4.0 * K / M) * np.abs(np.sin(np.pi * qfrac))


def dp_g2(qfrac, a=3.0, K=2.0, M=20.0, D=1.5):
    hw = spring_hw(qfrac, K, M)
    with np.errstate(divide="ignore", invalid="ignore"):
        return (D / a) ** 2 * np.sin(2 * np.pi * qfrac) ** 2 * C_EV / (2.0 * M * hw)
