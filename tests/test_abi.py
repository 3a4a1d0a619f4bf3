"""The C ABI library loads and exports every function that include/epwi.h declares (CPU only:
no call here touches a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "epwi.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(epwi_[a-z0-9_]+)\s*\(",
                       text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("epwi_create", "epwi_setup", "epwi_eigs", "epwi_scatter_rates",
                 "epwi_conductivity", "epwi_mobility", "epwi_find_mu", "epwi_mlp_train",
                 "epwi_scatter_rates_is", "epwi_conductivity_noalloc"):
        assert must in names, must


def test_library_exports_every_declared_symbol():
    from paper_2306_16493_gb300 import epwi
    lib = ctypes.CDLL(epwi.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_knows_every_symbol():
    from paper_2306_16493_gb300 import epwi
    src = open(os.path.join(ROOT, "paper_2306_16493_gb300", "epwi.py")).read()
    missing = [n for n in declared_functions() if f'"{n}"' not in src]
    assert not missing, missing


def test_host_only_defaults():
    """Pure host calls (no device work): the option defaults documented in the header."""
    from paper_2306_16493_gb300 import epwi
    o = epwi.epwi_default_options()
    assert o.precision == epwi.EPWI_FP64 and o.sieve_c == 6.0 and o.omega_min_eV == 1e-4
    t = epwi.epwi_mlp_default_train_options()
    assert (t.epochs, t.batch, t.lr, t.background, t.floor_rel, t.seed) == (100, 512, 2e-3, 1.0,
                                                                            1e-8, 1)


def test_parameter_count_matches_oracle():
    from oracle import mlp_oracle
    from paper_2306_16493_gb300 import epwi
    assert epwi.EPWI_MLP_NPARAM == mlp_oracle.N_PARAM
    m = re.search(r"#define EPWI_MLP_NPARAM (\d+)", open(HEADER).read())
    assert int(m.group(1)) == mlp_oracle.N_PARAM


def test_default_options_match_the_header():
    """epwi_default_options is host code: the ctypes mirror of epwi_options reads back the
    documented defaults, including the fields appended last (tc_a_operand, ordering)."""
    from paper_2306_16493_gb300 import epwi
    o = epwi.epwi_default_options()
    assert o.precision == epwi.EPWI_FP64
    assert o.sieve_c == 6.0 and o.omega_min_eV == 1e-4
    assert o.device == 0 and not o.cuda_stream and o.kpoint_chunk == 0
    assert o.tc_a_operand == 0 and o.ordering == 0
    # the Python mirror's size equals the struct the library fills (no trailing field lost)
    import ctypes as C
    buf = (C.c_uint8 * (C.sizeof(epwi.epwi_options) + 64))(*([0xAB] * (C.sizeof(epwi.epwi_options) + 64)))
    epwi._lib.epwi_default_options(C.cast(buf, C.c_void_p))
    assert all(b == 0xAB for b in bytes(buf)[C.sizeof(epwi.epwi_options):])
