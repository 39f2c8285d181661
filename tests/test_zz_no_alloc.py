"""The allocation-free comb, afqmc_comb_static, against the context's comb.

afqmc_comb_static serves callers that cannot allocate device memory (their
device memory belongs to another allocator, or their host forbids device
allocation after start-up): they hand it their own device buffers and it
keeps its scratch in a fixed device array inside the library. Here it must
pick exactly the parents and the new weight that afqmc_population_control
picks for the same weights, on two calls in a row, so that nothing left in
the shared array by the first call leaks into the second. This file is
collected last on purpose.
"""
import math

import numpy as np
import pytest

from synth import small_system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1804_03310_gb300 import build
    build.build()


def context_comb(weights, seed):
    """Parents and new weight chosen by the existing entry point: walkers are
    tagged by an orbital phase, combed by the context, and identified again."""
    from paper_1804_03310_gb300 import Afqmc
    from paper_1804_03310_gb300.afqmc import decode_state, encode_state
    W = len(weights)
    s = small_system(M=5, n_up=1, n_dn=1, n_chol=2, n_walkers=W, seed=seed,
                     ortho_every=0, measure_every=0, pc_every=0)
    gpu = Afqmc.from_system(s)
    st = gpu.afqmc_get_state()
    d = decode_state(st)
    tag = np.exp(1j * np.arange(W) / W)
    Pu = d["Phi_up"] * tag[:, None, None]
    gpu.afqmc_set_state(encode_state(st, Pu, d["Phi_dn"], weights, d["logO"]))
    gpu.afqmc_population_control()
    out = gpu.walkers()
    # the context divides the common weight S/n out and keeps its log
    assert np.all(out["weight"] == 1.0)
    wnew = math.exp(gpu.afqmc_log_weight_scale())
    gpu.close()
    parent = np.argmin(np.abs(out["Phi_up"][:, 0, 0][:, None] - Pu[:, 0, 0][None, :]), axis=1)
    return parent, wnew, s.seed, s.run_id


def static_comb(weights, seed, run_id, step=0):
    import torch
    from paper_1804_03310_gb300.afqmc import afqmc_comb_static
    n = len(weights)
    w = torch.tensor(weights, dtype=torch.float64, device="cuda")
    parent = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    wnew = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    afqmc_comb_static(w.data_ptr(), n, seed, run_id, step, parent.data_ptr(),
                      wnew.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    return parent.cpu().numpy().astype(np.int64), float(wnew.item())


def test_static_comb_matches_context_comb_on_two_calls():
    rng = np.random.default_rng(2024)
    # the second call is smaller, so prefix sums left by the first call past
    # its end would change its answer if they were read
    for W, seed in ((1000, 7), (100, 3)):
        w = rng.uniform(0.0, 2.0, size=W)
        w[rng.uniform(size=W) < 0.2] = 0.0
        w[0] = max(w[0], 0.1)
        p_ctx, w_ctx, s_seed, s_run = context_comb(w, seed)
        p_st, wn = static_comb(w, s_seed, s_run)
        assert np.array_equal(p_st, p_ctx)
        assert abs(w_ctx - wn) <= 1e-15 * wn


def test_static_comb_reports_an_impossible_comb_by_a_negative_weight():
    """All-zero or non-finite weights leave nothing to comb: the call returns
    d_wnew = -1 with the identity in d_parent (its only signal; the kernel's
    status word stays in the library's array). A normal call right after
    must not be disturbed by the status left behind."""
    rng = np.random.default_rng(5)
    n = 77
    zero = np.zeros(n)
    nan = rng.uniform(0.5, 1.5, size=n)
    nan[13] = np.nan
    inf = rng.uniform(0.5, 1.5, size=n)
    inf[40] = np.inf
    for w in (zero, nan, inf):
        p, wn = static_comb(w, 3, 0)
        assert wn == -1.0
        assert np.array_equal(p, np.arange(n))
    w = rng.uniform(0.0, 2.0, size=n)
    p_ctx, w_ctx, s_seed, s_run = context_comb(w, 9)
    p_st, wn = static_comb(w, s_seed, s_run)
    assert np.array_equal(p_st, p_ctx)
    assert np.all(w_ctx == wn)


def test_static_comb_rejects_oversized_population():
    from paper_1804_03310_gb300 import AfqmcError
    from paper_1804_03310_gb300.afqmc import COMB_STATIC_MAX_WALKERS, afqmc_comb_static
    with pytest.raises(AfqmcError) as e:
        afqmc_comb_static(16, COMB_STATIC_MAX_WALKERS + 1, 0, 0, 0, 16, 16)
    assert e.value.status == 1 and "n_walkers" in str(e.value)
