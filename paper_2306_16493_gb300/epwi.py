"""Python binding of the C ABI in include/epwi.h (ctypes; argument marshalling only).

Every step of the path runs in libepwi.so's CUDA kernels; this module converts numpy
arrays to pointers and status codes to exceptions.  It raises at import time if the
compiled library is missing: there is no CPU fallback.  The functions keep the C names
(``epwi_create``, ``epwi_setup``, ...); ``Context`` bundles them for convenience.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libepwi.so")

EPWI_FP64, EPWI_TF32X3, EPWI_BF16X3, EPWI_FP16X3, EPWI_FP32 = 0, 1, 2, 3, 4
#: split-precision (tcgen05) modes built into this library
SPLIT_MODES = ("fp16x3", "tf32x3", "bf16x3")
PRECISIONS = {"fp64": EPWI_FP64, "tf32x3": EPWI_TF32X3, "bf16x3": EPWI_BF16X3,
              "fp16x3": EPWI_FP16X3, "fp32": EPWI_FP32}
STATUS = {0: "EPWI_OK", 1: "EPWI_EINVAL", 2: "EPWI_ENOMEM", 3: "EPWI_ECUDA", 4: "EPWI_ESTATE",
          5: "EPWI_ETIMEOUT", 6: "EPWI_ENUMERIC", 7: "EPWI_ETOOSMALL", 8: "EPWI_EUNSUPPORTED"}


class EpwiError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class epwi_c64(C.Structure):
    _fields_ = [("re", C.c_double), ("im", C.c_double)]


class epwi_system(C.Structure):
    _fields_ = [("lattice", C.c_double * 9), ("nat", C.c_int32), ("mass", C.c_void_p),
                ("nw", C.c_int32), ("nRe", C.c_int32), ("Re", C.c_void_p), ("we", C.c_void_p),
                ("H", C.c_void_p), ("nRp", C.c_int32), ("Rp", C.c_void_p), ("wp", C.c_void_p),
                ("Phi", C.c_void_p), ("g", C.c_void_p)]


class epwi_options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("sieve_c", C.c_double), ("omega_min_eV", C.c_double),
                ("device", C.c_int32), ("cuda_stream", C.c_void_p), ("kpoint_chunk", C.c_int32),
                ("tc_a_operand", C.c_int32), ("ordering", C.c_int32)]


class epwi_stats(C.Structure):
    _fields_ = [("n_kpoints", C.c_int64), ("n_states", C.c_int64), ("n_pairs", C.c_int64),
                ("n_tiles", C.c_int64), ("n_chunks", C.c_int64), ("ms_eigs", C.c_double),
                ("ms_sieve", C.c_double), ("ms_restage", C.c_double), ("ms_scatter", C.c_double),
                ("ms_reduce", C.c_double), ("restage_bytes", C.c_int64),
                ("scatter_flops", C.c_double), ("precision", C.c_int32), ("sm_count", C.c_int32),
                ("tc_grid", C.c_int64), ("tc_ctas_per_sm", C.c_int32), ("tc_regs", C.c_int32),
                ("tc_smem", C.c_int64), ("tc_smem_avail2", C.c_int64),
                ("ms_proposal", C.c_double), ("ms_sampling", C.c_double),
                ("proposal_flops", C.c_double), ("sym_kpoints", C.c_int64), ("sym_states", C.c_int64)]


class epwi_ibte_stats(C.Structure):
    _fields_ = [("n_states", C.c_int64), ("n_pairs", C.c_int64), ("n_entries", C.c_int64),
                ("entry_bytes", C.c_int32), ("iters", C.c_int32), ("change", C.c_double),
                ("ms_rates", C.c_double), ("ms_iterate", C.c_double), ("ms_step", C.c_double),
                ("bytes_per_step", C.c_double), ("index_bytes", C.c_int64)]


class epwi_mlp_train_options(C.Structure):
    _fields_ = [("epochs", C.c_int32), ("batch", C.c_int32), ("lr", C.c_double),
                ("background", C.c_double), ("floor_rel", C.c_double), ("seed", C.c_uint64)]


class epwi_batch_stats(C.Structure):
    _fields_ = [("n_systems", C.c_int64), ("n_states", C.c_int64), ("n_pairs", C.c_int64),
                ("n_items", C.c_int64), ("graph_nodes", C.c_int64), ("persistent_ctas", C.c_int64),
                ("smem_bytes", C.c_int64), ("runs", C.c_int64), ("ms_plan", C.c_double),
                ("ms_graph", C.c_double), ("ms_persistent", C.c_double),
                ("scatter_flops", C.c_double), ("restage_flops", C.c_double)]


EPWI_MLP_NPARAM = 34433
EPWI_PROPOSAL_UNIFORM, EPWI_PROPOSAL_LEARNED = 0, 1


def _load() -> C.CDLL:
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_2306_16493_gb300.build` (needs nvcc)")
    lib = C.CDLL(LIB_PATH)
    P, I32, I64, D, V = C.c_void_p, C.c_int32, C.c_int64, C.c_double, None
    sig = {
        "epwi_default_options": (V, [P]),
        "epwi_create": (I32, [P, P]),
        "epwi_destroy": (V, [P]),
        "epwi_last_error": (C.c_char_p, [P]),
        "epwi_set_precision": (I32, [P, I32]),
        "epwi_set_stream": (I32, [P, P]),
        "epwi_setup": (I32, [P, P]),
        "epwi_eigs": (I32, [P, P, P]),
        "epwi_band_range": (I32, [P, P, P]),
        "epwi_band_edges": (I32, [P, I32, P, P]),
        "epwi_find_mu": (I32, [P, D, D, I32, P]),
        "epwi_carrier_density": (I32, [P, D, D, I32, P]),
        "epwi_scatter_rates": (I32, [P, D, D, D, D, D, P, P]),
        "epwi_get_rates": (I32, [P, I64, P, P, P]),
        "epwi_conductivity": (I32, [P, P]),
        "epwi_mobility": (I32, [P, D, P]),
        "epwi_transport": (I32, [P, P, P, P]),
        "epwi_ibte": (I32, [P, D, D, D, D, D, I32, D, P, P]),
        "epwi_get_mfp": (I32, [P, I64, P]),
        "epwi_ibte_transport": (I32, [P, P, P, P]),
        "epwi_get_ibte_stats": (I32, [P, P]),
        "epwi_get_bands": (I32, [P, P, P, P]),
        "epwi_get_phonons": (I32, [P, P, P]),
        "epwi_get_sieve": (I32, [P, I64, P, P]),
        "epwi_g2": (I32, [P, I64, P, P, I32, I32, P]),
        "epwi_get_stats": (I32, [P, P]),
        "epwi_kernel_launches": (I64, []),
        "epwi_fma_peak": (I32, [I32, I32, P, D, P, P]),
        "epwi_set_symmetry": (I32, [P, I32, P]),
        "epwi_conductivity_noalloc": (I32, [I64, P, P, P, D, D, D, I64, P, P]),
        "epwi_mlp_default_train_options": (V, [P]),
        "epwi_mlp_train": (I32, [P, D, D, D, D, D, P, P]),
        "epwi_mlp_set_params": (I32, [P, P]),
        "epwi_mlp_get_params": (I32, [P, P, P, P]),
        "epwi_mlp_forward": (I32, [P, I64, P, P]),
        "epwi_mlp_forward_tc": (I32, [P, I64, P, P]),
        "epwi_mlp_loss_grad": (I32, [P, I64, P, P, P, P]),
        "epwi_mlp_get_training_set": (I32, [P, I64, P, P, P, P, P]),
        "epwi_scatter_rates_is": (I32, [P, D, D, D, D, D, I64, D, I32, I32, C.c_uint64, P, P]),
        "epwi_get_is_pairs": (I32, [P, I64, P, P, P, P]),
        "epwi_batch_create": (I32, [P, P]),
        "epwi_batch_destroy": (V, [P]),
        "epwi_batch_last_error": (C.c_char_p, [P]),
        "epwi_batch_setup": (I32, [P, I32, P, P]),
        "epwi_batch_plan": (I32, [P, D, P, D, P, P, I32, P]),
        "epwi_batch_add": (I32, [P, P, P, P]),
        "epwi_batch_band_range": (I32, [P, I32, P, P]),
        "epwi_batch_run": (I32, [P, P]),
        "epwi_batch_get_rates": (I32, [P, I32, I64, P, P, P, P]),
        "epwi_batch_set_tile": (I32, [P, I32, I32, I32]),
        "epwi_batch_get_tile": (I32, [P, I32, P, P, P]),
        "epwi_batch_get_stats": (I32, [P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _check(ctx, st: int):
    if st != 0:
        msg = _lib.epwi_last_error(ctx).decode() if ctx else ""
        raise EpwiError(st, msg)


# ------------------------------------------------------------------ C-named functions
def epwi_default_options() -> epwi_options:
    o = epwi_options()
    _lib.epwi_default_options(C.byref(o))
    return o


def epwi_create(options: epwi_options | None = None):
    h = C.c_void_p()
    st = _lib.epwi_create(C.byref(h), C.byref(options) if options is not None else None)
    if st != 0:
        raise EpwiError(st, "epwi_create failed")
    return h


def epwi_destroy(ctx):
    _lib.epwi_destroy(ctx)


def epwi_set_precision(ctx, precision: int):
    _check(ctx, _lib.epwi_set_precision(ctx, int(precision)))


def epwi_set_stream(ctx, stream: int | None):
    _check(ctx, _lib.epwi_set_stream(ctx, C.c_void_p(stream or 0)))


def _system_struct(sysm):
    """epwi_system for sysm (an object with the fields of synth.System) and the arrays it
    points into (keep them alive while the struct is in use)."""
    keep = dict(
        mass=np.ascontiguousarray(sysm.mass, np.float64),
        Re=np.ascontiguousarray(sysm.Re, np.int32), we=np.ascontiguousarray(sysm.we, np.float64),
        H=np.ascontiguousarray(sysm.H, np.complex128),
        Rp=np.ascontiguousarray(sysm.Rp, np.int32), wp=np.ascontiguousarray(sysm.wp, np.float64),
        Phi=np.ascontiguousarray(sysm.Phi, np.float64),
        g=np.ascontiguousarray(sysm.g, np.complex128))
    s = epwi_system()
    s.lattice[:] = np.ascontiguousarray(sysm.lattice, np.float64).ravel().tolist()
    s.nat = len(keep["mass"])
    s.nw = int(sysm.nw)
    s.nRe = len(keep["Re"])
    s.nRp = len(keep["Rp"])
    for k in ("mass", "Re", "we", "H", "Rp", "wp", "Phi", "g"):
        setattr(s, k, _ptr(keep[k]))
    return s, keep


def epwi_setup(ctx, sysm):
    """sysm: an object with the fields of synth.System (numpy arrays, unweighted)."""
    s, keep = _system_struct(sysm)
    _check(ctx, _lib.epwi_setup(ctx, C.byref(s)))


def epwi_eigs(ctx, kgrid, qgrid=None):
    k = np.ascontiguousarray(kgrid, np.int32)
    q = np.ascontiguousarray(kgrid if qgrid is None else qgrid, np.int32)
    _check(ctx, _lib.epwi_eigs(ctx, _ptr(k), _ptr(q)))


def epwi_band_range(ctx):
    lo, hi = C.c_double(), C.c_double()
    _check(ctx, _lib.epwi_band_range(ctx, C.byref(lo), C.byref(hi)))
    return lo.value, hi.value


def epwi_band_edges(ctx, n_valence: int):
    v, c = C.c_double(), C.c_double()
    _check(ctx, _lib.epwi_band_edges(ctx, int(n_valence), C.byref(v), C.byref(c)))
    return v.value, c.value


def epwi_find_mu(ctx, T, n_cm3, n_valence):
    m = C.c_double()
    _check(ctx, _lib.epwi_find_mu(ctx, float(T), float(n_cm3), int(n_valence), C.byref(m)))
    return m.value


def epwi_carrier_density(ctx, T, mu, n_valence):
    n = C.c_double()
    _check(ctx, _lib.epwi_carrier_density(ctx, float(T), float(mu), int(n_valence), C.byref(n)))
    return n.value


def epwi_scatter_rates(ctx, T, mu, smear, emin, emax):
    ns, npair = C.c_int64(), C.c_int64()
    _check(ctx, _lib.epwi_scatter_rates(ctx, float(T), float(mu), float(smear), float(emin),
                                        float(emax), C.byref(ns), C.byref(npair)))
    return ns.value, npair.value


def epwi_get_rates(ctx, n_states: int):
    k = np.empty(n_states, np.int32)
    b = np.empty(n_states, np.int32)
    r = np.empty(n_states, np.float64)
    _check(ctx, _lib.epwi_get_rates(ctx, n_states, _ptr(k), _ptr(b), _ptr(r)))
    return k, b, r


def epwi_conductivity(ctx):
    s = np.empty(9, np.float64)
    _check(ctx, _lib.epwi_conductivity(ctx, _ptr(s)))
    return s.reshape(3, 3)


def epwi_mobility(ctx, n_cm3):
    m = np.empty(9, np.float64)
    _check(ctx, _lib.epwi_mobility(ctx, float(n_cm3), _ptr(m)))
    return m.reshape(3, 3)


def epwi_get_bands(ctx, nk: int, nw: int):
    e = np.empty((nk, nw))
    V = np.empty((nk, nw, nw), np.complex128)
    v = np.empty((nk, nw, 3))
    _check(ctx, _lib.epwi_get_bands(ctx, _ptr(e), _ptr(V), _ptr(v)))
    return e, V, v


def epwi_get_phonons(ctx, nq: int, nm: int):
    w = np.empty((nq, nm))
    u = np.empty((nq, nm, nm), np.complex128)
    _check(ctx, _lib.epwi_get_phonons(ctx, _ptr(w), _ptr(u)))
    return w, u


def epwi_get_sieve(ctx, n_kpoints: int):
    k = np.empty(n_kpoints, np.int32)
    c = np.empty(n_kpoints, np.int64)
    _check(ctx, _lib.epwi_get_sieve(ctx, n_kpoints, _ptr(k), _ptr(c)))
    return k, c


def epwi_g2(ctx, ik, iq, band_lo: int, nsel: int, nm: int, nw: int):
    ik = np.ascontiguousarray(ik, np.int32)
    iq = np.ascontiguousarray(iq, np.int32)
    out = np.empty((len(ik), nsel, nm, nw))
    _check(ctx, _lib.epwi_g2(ctx, len(ik), _ptr(ik), _ptr(iq), int(band_lo), int(nsel), _ptr(out)))
    return out


def epwi_conductivity_noalloc(n_states: int, eps_dev: int, vel_dev: int, inv_tau_dev: int,
                              mu_eV: float, T_K: float, volume_A3: float, nk: int, stream: int | None,
                              sigma_dev: int):
    """Device-pointer variant of epwi_conductivity that allocates nothing (pointers as ints)."""
    st = _lib.epwi_conductivity_noalloc(int(n_states), C.c_void_p(eps_dev), C.c_void_p(vel_dev),
                                        C.c_void_p(inv_tau_dev), float(mu_eV), float(T_K),
                                        float(volume_A3), int(nk), C.c_void_p(stream or 0),
                                        C.c_void_p(sigma_dev))
    if st != 0:
        raise EpwiError(st, "epwi_conductivity_noalloc failed")


def epwi_kernel_launches() -> int:
    return int(_lib.epwi_kernel_launches())


def epwi_fma_peak(fp64: bool, device: int = 0, stream: int | None = None, target_ms: float = 50.0):
    """Measured FMA throughput (TFLOP/s, ms of the best launch) of FP32 or FP64 FMAs."""
    tf, ms = C.c_double(), C.c_double()
    st = _lib.epwi_fma_peak(int(bool(fp64)), int(device), C.c_void_p(stream or 0), float(target_ms),
                            C.byref(tf), C.byref(ms))
    if st != 0:
        raise EpwiError(st, "epwi_fma_peak failed")
    return tf.value, ms.value


def epwi_get_stats(ctx) -> dict:
    s = epwi_stats()
    _check(ctx, _lib.epwi_get_stats(ctx, C.byref(s)))
    return {name: getattr(s, name) for name, _ in epwi_stats._fields_}


def epwi_ibte(ctx, T, mu, smear, emin, emax, max_iter=100, tol=1e-8):
    """Iterative BTE; returns (iterations, last relative change)."""
    it, ch = C.c_int32(), C.c_double()
    _check(ctx, _lib.epwi_ibte(ctx, T, mu, smear, emin, emax, int(max_iter), float(tol),
                               C.byref(it), C.byref(ch)))
    return it.value, ch.value


def epwi_get_mfp(ctx, n_states) -> np.ndarray:
    F = np.empty((max(int(n_states), 0), 3))
    _check(ctx, _lib.epwi_get_mfp(ctx, int(n_states), _ptr(F)))
    return F


def epwi_ibte_transport(ctx):
    sig, S, kap = np.empty((3, 3)), np.empty((3, 3)), np.empty((3, 3))
    _check(ctx, _lib.epwi_ibte_transport(ctx, _ptr(sig), _ptr(S), _ptr(kap)))
    return sig, S, kap


def epwi_get_ibte_stats(ctx) -> dict:
    s = epwi_ibte_stats()
    _check(ctx, _lib.epwi_get_ibte_stats(ctx, C.byref(s)))
    return {name: getattr(s, name) for name, _ in epwi_ibte_stats._fields_}


def epwi_mlp_default_train_options() -> epwi_mlp_train_options:
    o = epwi_mlp_train_options()
    _lib.epwi_mlp_default_train_options(C.byref(o))
    return o


def epwi_mlp_train(ctx, T, mu, smear, emin, emax, options: epwi_mlp_train_options | None = None):
    o = options or epwi_mlp_default_train_options()
    loss = C.c_double()
    _check(ctx, _lib.epwi_mlp_train(ctx, T, mu, smear, emin, emax, C.byref(o), C.byref(loss)))
    return loss.value


def epwi_mlp_set_params(ctx, params):
    p = np.ascontiguousarray(params, np.float32)
    assert p.size == EPWI_MLP_NPARAM
    _check(ctx, _lib.epwi_mlp_set_params(ctx, _ptr(p)))


def epwi_mlp_get_params(ctx):
    p = np.empty(EPWI_MLP_NPARAM, np.float32)
    sc, sh = C.c_double(), C.c_double()
    _check(ctx, _lib.epwi_mlp_get_params(ctx, _ptr(p), C.byref(sc), C.byref(sh)))
    return p, sc.value, sh.value


def epwi_mlp_forward(ctx, x):
    x = np.ascontiguousarray(x, np.float32).reshape(-1, 9)
    y = np.empty(len(x), np.float32)
    _check(ctx, _lib.epwi_mlp_forward(ctx, len(x), _ptr(x), _ptr(y)))
    return y


def epwi_mlp_forward_tc(ctx, x):
    x = np.ascontiguousarray(x, np.float32).reshape(-1, 9)
    y = np.empty(len(x), np.float32)
    _check(ctx, _lib.epwi_mlp_forward_tc(ctx, len(x), _ptr(x), _ptr(y)))
    return y


def epwi_mlp_loss_grad(ctx, x, y):
    x = np.ascontiguousarray(x, np.float32).reshape(-1, 9)
    y = np.ascontiguousarray(y, np.float32)
    g = np.empty(EPWI_MLP_NPARAM, np.float32)
    loss = C.c_double()
    _check(ctx, _lib.epwi_mlp_loss_grad(ctx, len(x), _ptr(x), _ptr(y), C.byref(loss), _ptr(g)))
    return loss.value, g


def epwi_mlp_get_training_set(ctx):
    n = C.c_int64()
    _check(ctx, _lib.epwi_mlp_get_training_set(ctx, 0, None, None, None, None, C.byref(n)))
    m = n.value
    ids = np.empty((m, 4), np.int32)
    t = np.empty(m)
    x = np.empty((m, 9), np.float32)
    y = np.empty(m, np.float32)
    _check(ctx, _lib.epwi_mlp_get_training_set(ctx, m, _ptr(ids), _ptr(t), _ptr(x), _ptr(y),
                                               C.byref(n)))
    return ids, t, x, y


def epwi_scatter_rates_is(ctx, T, mu, smear, emin, emax, samples_per_k, alpha=0.1,
                          cell_stride=1, proposal=EPWI_PROPOSAL_LEARNED, seed=1):
    ns, npairs = C.c_int64(), C.c_int64()
    _check(ctx, _lib.epwi_scatter_rates_is(ctx, T, mu, smear, emin, emax, int(samples_per_k),
                                           float(alpha), int(cell_stride), int(proposal),
                                           int(seed), C.byref(ns), C.byref(npairs)))
    return ns.value, npairs.value


def epwi_get_is_pairs(ctx):
    n = C.c_int64()
    _check(ctx, _lib.epwi_get_is_pairs(ctx, 0, None, None, None, C.byref(n)))
    m = n.value
    ik = np.empty(m, np.int32)
    iq = np.empty(m, np.int32)
    w = np.empty(m)
    _check(ctx, _lib.epwi_get_is_pairs(ctx, m, _ptr(ik), _ptr(iq), _ptr(w), C.byref(n)))
    return ik, iq, w


def _bcheck(b, st: int):
    if st != 0:
        msg = _lib.epwi_batch_last_error(b).decode() if b else ""
        raise EpwiError(st, msg)


class Batch:
    """Uneven systems in one planned step (epwi_batch_* calls)."""

    def __init__(self, device=0, stream=None):
        o = epwi_default_options()
        o.device = device
        o.cuda_stream = stream or 0
        h = C.c_void_p()
        st = _lib.epwi_batch_create(C.byref(h), C.byref(o))
        if st != 0:
            raise EpwiError(st, "epwi_batch_create failed")
        self.h = h
        self.nsys = 0
        self._keep = []

    def close(self):
        if self.h:
            _lib.epwi_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def setup(self, systems, grids):
        arr = (epwi_system * len(systems))()
        keep = []
        for i, sysm in enumerate(systems):
            arr[i], k = _system_struct(sysm)
            keep.append(k)
        g = np.ascontiguousarray(np.asarray(grids, np.int32).reshape(-1, 3))
        _bcheck(self.h, _lib.epwi_batch_setup(self.h, len(systems), arr, _ptr(g)))
        self.nsys = len(systems)
        self._keep = keep

    def add(self, sysm, grid):
        """Appends one system (its arrays may be dropped afterwards); returns its index."""
        s, keep = _system_struct(sysm)
        g = np.ascontiguousarray(np.asarray(grid, np.int32).reshape(3))
        idx = C.c_int32()
        _bcheck(self.h, _lib.epwi_batch_add(self.h, C.byref(s), _ptr(g), C.byref(idx)))
        self.nsys = idx.value + 1
        return idx.value

    def band_range(self, s):
        lo, hi = C.c_double(), C.c_double()
        _bcheck(self.h, _lib.epwi_batch_band_range(self.h, s, C.byref(lo), C.byref(hi)))
        return lo.value, hi.value

    def plan(self, T, mu, smear, emin, emax, autotune=True):
        mu = np.ascontiguousarray(mu, float)
        lo = np.ascontiguousarray(emin, float)
        hi = np.ascontiguousarray(emax, float)
        n = C.c_int64()
        _bcheck(self.h, _lib.epwi_batch_plan(self.h, T, _ptr(mu), smear, _ptr(lo), _ptr(hi),
                                             int(bool(autotune)), C.byref(n)))
        return n.value

    def run(self):
        sig = np.empty((self.nsys, 3, 3))
        _bcheck(self.h, _lib.epwi_batch_run(self.h, _ptr(sig)))
        return sig

    def rates(self, s):
        n = C.c_int64()
        _bcheck(self.h, _lib.epwi_batch_get_rates(self.h, s, 0, None, None, None, C.byref(n)))
        k = np.empty(n.value, np.int32)
        b = np.empty(n.value, np.int32)
        r = np.empty(n.value)
        _bcheck(self.h, _lib.epwi_batch_get_rates(self.h, s, n.value, _ptr(k), _ptr(b), _ptr(r),
                                                  C.byref(n)))
        return k, b, r

    def set_tile(self, s, mt, kc):
        _bcheck(self.h, _lib.epwi_batch_set_tile(self.h, s, mt, kc))

    def tile(self, s):
        mt, kc, src = C.c_int32(), C.c_int32(), C.c_int32()
        _bcheck(self.h, _lib.epwi_batch_get_tile(self.h, s, C.byref(mt), C.byref(kc), C.byref(src)))
        return mt.value, kc.value, src.value

    def stats(self):
        st = epwi_batch_stats()
        _bcheck(self.h, _lib.epwi_batch_get_stats(self.h, C.byref(st)))
        return {name: getattr(st, name) for name, _ in epwi_batch_stats._fields_}


# ------------------------------------------------------------------ convenience wrapper
class Context:
    """One library context (device memory, stream, last results)."""

    def __init__(self, precision="fp64", device=0, stream=None, sieve_c=6.0, omega_min=1e-4,
                 kpoint_chunk=0, tc_a_operand=0, ordering="q-batch"):
        o = epwi_default_options()
        o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        o.device = device
        o.cuda_stream = stream or 0
        o.sieve_c = sieve_c
        o.omega_min_eV = omega_min
        o.kpoint_chunk = kpoint_chunk
        o.tc_a_operand = tc_a_operand
        o.ordering = {"q-batch": 0, "k-batch": 1}[ordering] if isinstance(ordering, str) else int(ordering)
        self.h = epwi_create(o)
        self.nk = self.nw = self.nm = 0
        self.n_states = 0

    def close(self):
        if self.h:
            epwi_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_precision(self, p):
        epwi_set_precision(self.h, PRECISIONS[p] if isinstance(p, str) else p)

    def setup(self, sysm):
        epwi_setup(self.h, sysm)
        self.nw, self.nm = int(sysm.nw), 3 * len(sysm.mass)

    def eigs(self, grid):
        grid = [grid] * 3 if np.isscalar(grid) else list(grid)
        epwi_eigs(self.h, grid, grid)
        self.nk = int(np.prod(grid))

    def band_range(self):
        return epwi_band_range(self.h)

    def band_edges(self, nv):
        return epwi_band_edges(self.h, nv)

    def find_mu(self, T, n_cm3, nv):
        return epwi_find_mu(self.h, T, n_cm3, nv)

    def carrier_density(self, T, mu, nv):
        return epwi_carrier_density(self.h, T, mu, nv)

    def scatter_rates(self, T, mu, smear, emin, emax):
        self.n_states, n_pairs = epwi_scatter_rates(self.h, T, mu, smear, emin, emax)
        return self.n_states, n_pairs

    def rates(self):
        return epwi_get_rates(self.h, self.n_states)

    def conductivity(self):
        return epwi_conductivity(self.h)

    def transport(self):
        """(sigma [S/m], Seebeck [V/K], kappa_e [W/(m K)]) as 3x3 arrays."""
        sig, S, kap = np.empty((3, 3)), np.empty((3, 3)), np.empty((3, 3))
        _check(self.h, _lib.epwi_transport(self.h, _ptr(sig), _ptr(S), _ptr(kap)))
        return sig, S, kap

    def mobility(self, n_cm3):
        return epwi_mobility(self.h, n_cm3)

    def ibte(self, T, mu, smear, emin, emax, max_iter=100, tol=1e-8):
        """Iterative BTE (also leaves the SERTA rates); returns (iterations, change)."""
        it, ch = epwi_ibte(self.h, T, mu, smear, emin, emax, max_iter, tol)
        self.n_states = epwi_get_ibte_stats(self.h)["n_states"]
        return it, ch

    def mfp(self):
        """Mean free paths F [n_states, 3] (m) of the last ibte call, in rates order."""
        return epwi_get_mfp(self.h, self.n_states)

    def ibte_transport(self):
        """(sigma, Seebeck, kappa_e) from the mean free paths, as 3x3 arrays."""
        return epwi_ibte_transport(self.h)

    def ibte_stats(self):
        return epwi_get_ibte_stats(self.h)

    def bands(self):
        return epwi_get_bands(self.h, self.nk, self.nw)

    def phonons(self):
        return epwi_get_phonons(self.h, self.nk, self.nm)

    def set_symmetry(self, kops):
        """Point-group operations on grid index vectors ([nops][3][3] int), or None to clear."""
        ops = np.ascontiguousarray(np.zeros((0, 3, 3)) if kops is None else kops, dtype=np.int32)
        _check(self.h, _lib.epwi_set_symmetry(self.h, int(len(ops)), _ptr(ops) if len(ops) else None))

    def sieve(self):
        st = self.stats()
        return epwi_get_sieve(self.h, st["n_kpoints"])

    def g2(self, ik, iq, band_lo, nsel):
        return epwi_g2(self.h, ik, iq, band_lo, nsel, self.nm, self.nw)

    def stats(self):
        return epwi_get_stats(self.h)

    def mlp_train(self, T, mu, smear, emin, emax, **opts):
        o = epwi_mlp_default_train_options()
        for k, v in opts.items():
            setattr(o, k, v)
        return epwi_mlp_train(self.h, T, mu, smear, emin, emax, o)

    def scatter_rates_is(self, T, mu, smear, emin, emax, samples_per_k, alpha=0.1,
                         cell_stride=1, proposal="learned", seed=1):
        pr = {"uniform": EPWI_PROPOSAL_UNIFORM, "learned": EPWI_PROPOSAL_LEARNED}[proposal]
        self.n_states, n_pairs = epwi_scatter_rates_is(self.h, T, mu, smear, emin, emax,
                                                       samples_per_k, alpha, cell_stride, pr,
                                                       seed)
        return self.n_states, n_pairs
