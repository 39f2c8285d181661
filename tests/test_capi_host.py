"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point include/afqmc.h declares, and rejects invalid input before
touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from synth import small_system

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "afqmc.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1804_03310_gb300 import build
    build.build()
    from paper_1804_03310_gb300.afqmc import load_library
    return load_library()


def declared_symbols():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(afqmc_[a-z_]+)\s*\(", txt)))


def test_header_declares_the_calls():
    names = declared_symbols()
    for must in ("afqmc_create", "afqmc_propagate", "afqmc_orthonormalize",
                 "afqmc_local_energy", "afqmc_weights", "afqmc_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_params_default(lib):
    from paper_1804_03310_gb300.afqmc import default_params
    p = default_params()
    assert p.taylor_order == 6 and p.fb_cap == 1.0 and np.isnan(p.e_shift)
    assert p.ortho_every == 2 and p.measure_every == 20 and p.pc_every == 20


def _create(system, **kw):
    from paper_1804_03310_gb300 import Afqmc
    return Afqmc.from_system(system, **kw)


@pytest.mark.parametrize("mutate,needle", [
    (lambda s: s.replace(L=s.L + np.triu(np.ones_like(s.L[0]), 1)[None] * 0.1), "symmetric"),
    (lambda s: s.replace(h1=s.h1 + np.triu(np.ones_like(s.h1), 1)), "symmetric"),
    (lambda s: s.replace(C_up=s.C_up * 2.0), "orthonormal"),
    (lambda s: s.replace(occ_up=np.array([[0, 0]], dtype=np.int32)), "repeated"),
    (lambda s: s.replace(occ_dn=np.array([[0, 99]], dtype=np.int32)), "range"),
])
def test_invalid_inputs_rejected_before_device(lib, mutate, needle):
    from paper_1804_03310_gb300 import AfqmcError
    s = mutate(small_system(M=6, n_up=2, n_dn=2, n_chol=3))
    with pytest.raises(AfqmcError) as e:
        _create(s)
    assert e.value.status == 1 and needle in str(e.value)


@pytest.mark.parametrize("kw,needle", [
    (dict(taylor_order=0), "taylor_order"),
    (dict(dtau=-1.0), "dtau"),
    (dict(n_walkers=0), "n_walkers"),
    (dict(precision=9), "precision"),
])
def test_invalid_params_rejected(lib, kw, needle):
    from paper_1804_03310_gb300 import AfqmcError
    s = small_system(M=6, n_up=2, n_dn=2, n_chol=3)
    with pytest.raises(AfqmcError) as e:
        _create(s, **kw)
    assert e.value.status == 1 and needle in str(e.value)


def test_oversized_problem_rejected(lib):
    from paper_1804_03310_gb300 import AfqmcError
    s = small_system(M=6, n_up=2, n_dn=2, n_chol=3)
    big = s.replace(h1=np.eye(300), L=np.zeros((1, 300, 300)),
                    C_up=np.eye(300), C_dn=np.eye(300))
    with pytest.raises(AfqmcError) as e:
        _create(big)
    assert "M must be" in str(e.value)


def test_state_codec_round_trip():
    from paper_1804_03310_gb300.afqmc import HEADER, decode_state, encode_state
    rng = np.random.default_rng(0)
    W, M, nu, nd = 3, 5, 2, 1
    h = np.zeros(1, dtype=HEADER)
    h["magic"] = b"AFQMCST1"
    h["M"], h["n_up"], h["n_dn"], h["n_walkers"], h["step"] = M, nu, nd, W, 7
    Pu = rng.normal(size=(W, M, nu)) + 1j * rng.normal(size=(W, M, nu))
    Pd = rng.normal(size=(W, M, nd)) + 1j * rng.normal(size=(W, M, nd))
    w = rng.uniform(size=W)
    lo = rng.normal(size=W) + 1j * rng.normal(size=W)
    tmpl = h.tobytes() + bytes(W * (nu + nd) * M * 16 + W * 8 + W * 16)
    buf = encode_state(tmpl, Pu, Pd, w, lo)
    d = decode_state(buf)
    assert np.array_equal(d["Phi_up"], Pu) and np.array_equal(d["Phi_dn"], Pd)
    assert np.array_equal(d["weight"], w) and np.array_equal(d["logO"], lo)
    assert d["step"] == 7
