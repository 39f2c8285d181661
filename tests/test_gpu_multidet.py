"""Multi-determinant trials (Sherman-Morrison-Woodbury path) against the oracle,
which sums the determinants one by one with full inverses."""
import numpy as np
import pytest

from fock import FockSpace
from gpu_helpers import side_by_side
from oracle import afqmc as O
from synth import config_c4, small_system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="session", autouse=True)
def built():
    from paper_1804_03310_gb300 import build
    build.build()


def gpu_ctx(system, **kw):
    from paper_1804_03310_gb300 import Afqmc
    return Afqmc.from_system(system, **kw)


def run_pair(system, precision, n_steps, rtol, walkers=None, energy_at=()):
    # at tau = 0 every walker is the reference determinant, whose overlap
    # with the excited determinants vanishes (a 0/0 local energy); the first
    # comparisons come after one step
    gpu = gpu_ctx(system, precision=precision)
    orc = O.OracleRun(system, walker_ids=walkers)
    worst = side_by_side(gpu, orc, n_steps, rtol, walkers=walkers, energy_at=energy_at,
                         label=precision)
    gpu.close()
    return worst


def scrambled(system, rng):
    """Same trial with every determinant's columns permuted and complex CI
    coefficients: the library must fold the column-order signs in."""
    ou = system.occ_up.copy()
    od = system.occ_dn.copy()
    for i in range(1, system.n_det):
        ou[i] = ou[i][rng.permutation(ou.shape[1])]
        od[i] = od[i][rng.permutation(od.shape[1])]
    ci = system.ci * np.exp(1j * rng.uniform(0, 2 * np.pi, system.n_det))
    return system.replace(occ_up=ou, occ_dn=od, ci=ci)


@pytest.mark.parametrize("n_det", [2, 20])
def test_small_multidet_fp64(n_det):
    s = small_system(M=12, n_up=3, n_dn=3, n_chol=15, seed=3, n_det=n_det,
                     n_walkers=16, dtau=0.01, l_sigma=0.08, ortho_every=2,
                     measure_every=4, pc_every=4)
    s = scrambled(s, np.random.default_rng(n_det))
    w = run_pair(s, "fp64", 8, 1e-10, energy_at=(1, 4, 8))
    print(f"multidet n_det={n_det} fp64 worst", w)


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
@pytest.mark.parametrize("M", [12, 14])
def test_small_multidet_tensor_cores(prec, M):
    """Multi-determinant trials in the tensor-core modes: M % 4 == 0 puts the
    half steps on the tensor cores as well, M = 14 keeps them on the CUDA
    cores."""
    s = small_system(M=M, n_up=3, n_dn=2, n_chol=15, seed=4, n_det=20, n_walkers=16,
                     dtau=0.01, l_sigma=0.05, ortho_every=2, measure_every=4, pc_every=0)
    s = scrambled(s, np.random.default_rng(7))
    w = run_pair(s, prec, 8, 1e-4, energy_at=(1, 4, 8))
    print(f"multidet M={M} {prec} worst", w)


def test_unequal_spins_multidet_fp64():
    s = small_system(M=9, n_up=4, n_dn=2, n_chol=11, seed=9, n_det=12, n_walkers=8,
                     dtau=0.01, l_sigma=0.08, ortho_every=2, measure_every=3,
                     pc_every=0)
    s = scrambled(s, np.random.default_rng(2))
    run_pair(s, "fp64", 6, 1e-10, energy_at=(3, 6))


def test_exact_trial_zero_variance_gpu():
    """The exact 2e/4o ground state as a 16-determinant trial: every walker's
    local energy is the exact energy at every step."""
    from test_oracle_pins import fci_trial_2e4o
    fs = FockSpace(4)
    s = small_system(M=4, n_up=1, n_dn=1, n_chol=4, seed=8, l_sigma=0.3, n_walkers=32,
                     dtau=0.02, ortho_every=2, measure_every=0, pc_every=0)
    e0, ou, od, ci = fci_trial_2e4o(fs, s)
    s = s.replace(occ_up=ou, occ_dn=od, ci=ci)
    gpu = gpu_ctx(s, precision="fp64")
    for _ in range(6):
        gpu.afqmc_propagate(1)
        e, _ = gpu.afqmc_local_energy()
        w, _ = gpu.afqmc_weights()
        live = w > 0
        assert np.max(np.abs(e[live] - e0)) < 1e-10
    gpu.close()


def test_c4_full_size_sampled_fp64():
    """200-determinant workload at full size, two sampled walkers followed for
    the first 20 steps (comb off)."""
    s = config_c4(pc_every=0)
    w = run_pair(s, "fp64", 20, 1e-10, walkers=[0, 1023], energy_at=(20,))
    print("c4 fp64 worst", w)


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3", "fp32"])
def test_c4_full_size_sampled_reduced(prec):
    s = config_c4(pc_every=0)
    w = run_pair(s, prec, 20, 1e-4, walkers=[0, 511, 1023], energy_at=(20,))
    print(f"c4 {prec} worst", w)
