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
    (dict(weight_mode=2), "weight_mode"),
    (dict(mf_subtract=-1), "mf_subtract"),
    (dict(weight_mode=1, n_det=2), "one-determinant"),
    (dict(block_sparse=3), "block_sparse"),
    (dict(block_sparse=1), "not block-diagonal"),
    (dict(fp64_islands=3), "fp64_islands"),
])
def test_invalid_params_rejected(lib, kw, needle):
    from paper_1804_03310_gb300 import AfqmcError
    kw = dict(kw)
    s = small_system(M=6, n_up=2, n_dn=2, n_chol=3, n_det=kw.pop("n_det", 1))
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


def _inputs(system, **kw):
    from paper_1804_03310_gb300 import Inputs
    return Inputs.from_system(system, **kw)


def test_footprint_is_host_only_and_grows_with_walkers(lib):
    from paper_1804_03310_gb300 import afqmc_footprint
    s = small_system(M=12, n_up=3, n_dn=2, n_chol=7)
    r1, s1 = afqmc_footprint(_inputs(s.replace(n_walkers=16)))
    r2, s2 = afqmc_footprint(_inputs(s.replace(n_walkers=32)))
    r3, _ = afqmc_footprint(_inputs(s.replace(n_walkers=48)))
    # setup staging does not depend on the walker count; resident memory is
    # affine in it
    assert s1 == s2 and s1 > 0
    assert r2 > r1 and (r3 - r2) == (r2 - r1)
    # the walker-proportional part holds at least three copies of the
    # orbitals (propagation buffers) and the one-body operator per walker
    M, N, G = 12, 5, 7
    per_walker = (r2 - r1) / 16
    assert per_walker >= 16 * (3 * N * M + M * M)
    # the tensor-core modes keep extra operand copies
    rt, _ = afqmc_footprint(_inputs(s, precision="tf32x3"))
    rf, _ = afqmc_footprint(_inputs(s, precision="fp32"))
    assert rt > rf


def test_footprint_rejects_what_create_rejects(lib):
    from paper_1804_03310_gb300 import AfqmcError, afqmc_footprint
    s = small_system(M=6, n_up=2, n_dn=2, n_chol=3)
    with pytest.raises(AfqmcError) as e:
        afqmc_footprint(_inputs(s, taylor_order=0))
    assert e.value.status == 1
    inp = _inputs(s)
    inp.params.graphs = 2
    with pytest.raises(AfqmcError) as e:
        afqmc_footprint(inp)
    assert "graphs" in str(e.value)


def test_multidet_footprint_counts_active_orbitals(lib):
    from paper_1804_03310_gb300 import afqmc_footprint
    s = small_system(M=12, n_up=3, n_dn=3, n_chol=5, n_det=6, seed=1)
    r_md, _ = afqmc_footprint(_inputs(s))
    r_sd, _ = afqmc_footprint(_inputs(s.replace(occ_up=s.occ_up[:1], occ_dn=s.occ_dn[:1],
                                                ci=s.ci[:1])))
    assert r_md > r_sd


def test_batch_and_server_validate_before_device(lib):
    from paper_1804_03310_gb300.afqmc import afqmc_server_config
    out = C.c_void_p()
    assert lib.afqmc_batch_create(None, 0, 10, C.byref(out)) == 1
    assert lib.afqmc_batch_propagate(None, 1) == 1
    cfg = afqmc_server_config()
    cfg.max_active = 1000
    assert lib.afqmc_server_create(C.byref(cfg), C.byref(out)) == 1
    assert b"max_active" in lib.afqmc_last_error(None)
    cfg.max_active = 4
    cfg.reserved[0] = 1
    assert lib.afqmc_server_create(C.byref(cfg), C.byref(out)) == 1
