"""The sieve kernel's decision rule (Sec. III A) against the FP64 definition, on the CPU.

The GPU sieve decides a candidate (k, q) from hm = hbar omega_max(q) and the smallest distance
d = min |e_n(k) - e_m(k+q)| in FP32, with the rounding margin delta of the kernel's arguments:
reject when d > hm + c eta + delta, accept when hm <= c eta - 2 delta and d <= hm + c eta -
delta, and otherwise run the per-mode FP32 test with its FP64 re-check.  This file emulates
that FP32 arithmetic step by step (NumPy float32 rounds to nearest like the kernel) and checks
that every decision equals the FP64 definition: some window band n, band m, kept mode nu and
sign s with |(e_n + s w_nu) - e_m| <= c eta.  The inputs are random and adversarial: final
energies placed exactly on, and within a few ulps or a fraction of delta of, every boundary of
the rule and of the definition."""
import numpy as np
import pytest

F = np.float32


def definition(en, em, w, ceta, omega_min):
    """FP64, in the oracle's rounding order."""
    for n in en:
        for m in em:
            for x in w:
                if not (x >= omega_min):
                    continue
                if abs((n + x) - m) <= ceta or abs((n - x) - m) <= ceta:
                    return True
    return False


def kernel_rule(en, em, w, ceta, omega_min, eabs_max):
    """The distance rule, then the per-mode FP32 test and FP64 re-check, as the kernel runs them."""
    delta = 1e-6 + 4e-7 * (2.0 * eabs_max + 1.0)
    ceta32, delta32 = F(ceta), F(delta)
    lim_extra = F(ceta + float(delta32) + 1e-5)
    kept = [x for x in w if x >= omega_min]
    hm = F(max(kept)) if kept else F(-1.0)
    if hm < 0:
        return False
    e32 = [F(x) for x in en]
    m32 = [F(x) for x in em]
    d = F(3.0e38)
    for a in e32:
        for b in m32:
            d = min(d, abs(F(a - b)))
    rej, acc = F(ceta32 + delta32), F(ceta32 - delta32)
    hm_fast = F(ceta32 - F(2.0) * delta32)
    if not (d <= F(hm + rej)):
        return False
    if hm <= hm_fast and d <= F(hm + acc):
        return True
    # per-mode FP32 test with an ambiguity band, then FP64 for ambiguous candidates
    lim = F(hm + lim_extra)
    inner, outer = F(ceta32 - delta32), F(ceta32 + delta32)
    w32 = [F(x) if x >= omega_min else F(-1.0) for x in w]
    ambiguous = False
    for b in m32:
        for a in e32:
            dd = F(a - b)
            if not (abs(dd) <= lim):
                continue
            for x in w32:
                if x < 0:
                    continue
                xm = min(abs(F(dd + x)), abs(F(dd - x)))
                if xm <= inner:
                    return True
                if xm <= outer:
                    ambiguous = True
    if not ambiguous:
        return False
    return definition(en, em, w, ceta, omega_min)


def _cases(rng, n):
    omega_min = 1e-4
    for _ in range(n):
        eta = rng.choice([0.003, 0.005, 0.01, 0.02])
        ceta = 6.0 * eta
        E = rng.uniform(2.0, 20.0)
        nsel = int(rng.integers(1, 4))
        en = rng.uniform(-E, E, nsel)
        # modes: some below omega_min (dropped), the top one sometimes right at c eta
        w = np.sort(rng.uniform(0.0, 0.08, 3))
        if rng.random() < 0.1:
            w[0] = rng.uniform(0.0, omega_min)
        if rng.random() < 0.2:
            w[-1] = ceta + rng.choice([-2, -1, 0, 1, 2]) * 1e-6 * rng.random()
        delta = 1e-6 + 4e-7 * (2.0 * E + 1.0)
        em = np.sort(rng.uniform(-E, E, 4))
        # one final band on a boundary of the definition or of the rule
        n0 = en[int(rng.integers(nsel))]
        kind = int(rng.integers(5))
        s = rng.choice([-1.0, 1.0])
        x = w[int(rng.integers(3))]
        hm = w[w >= omega_min].max() if (w >= omega_min).any() else 0.0
        if kind == 0:                  # |(e_n + s w) - e_m| = c eta (+ tiny)
            target = n0 + s * x + rng.choice([-1.0, 1.0]) * ceta
        elif kind == 1:                # distance = hm + c eta (+- a fraction of delta)
            target = n0 + s * (hm + ceta)
        elif kind == 2:                # distance = hm + c eta - delta
            target = n0 + s * (hm + ceta - delta)
        elif kind == 3:                # distance = w - c eta (the inner edge of a mode)
            target = n0 + s * (x - ceta)
        else:                          # anywhere near the window energy
            target = n0 + rng.uniform(-0.3, 0.3)
        tiny = rng.choice([0.0, 1.0, -1.0]) * rng.choice([1e-15, 1e-9, 1e-7, 0.5 * delta, 2 * delta])
        em[int(rng.integers(4))] = np.clip(target + tiny, -E, E)
        yield en, em, w, ceta, omega_min, E


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_distance_rule_equals_the_fp64_definition(seed):
    rng = np.random.default_rng(seed)
    hits = 0
    for en, em, w, ceta, omega_min, E in _cases(rng, 4000):
        want = definition(en, em, w, ceta, omega_min)
        got = kernel_rule(en, em, w, ceta, omega_min, E)
        assert got == want, (en, em, w, ceta)
        hits += want
    assert 200 < hits < 3800          # both outcomes are well represented


def test_a_dropped_margin_would_be_caught():
    """The same adversarial cases catch an accept rule without the rounding margin: accepting
    whenever d <= hm + c eta in FP32 disagrees with the definition somewhere."""
    rng = np.random.default_rng(9)
    bad = 0
    for en, em, w, ceta, omega_min, E in _cases(rng, 4000):
        kept = [x for x in w if x >= omega_min]
        if not kept:
            continue
        hm = F(max(kept))
        d = min(abs(F(F(a) - F(b))) for a in en for b in em)
        naive = bool(d <= F(hm + F(ceta)))
        bad += naive != definition(en, em, w, ceta, omega_min)
    assert bad > 0
