"""Parity of the local-energy weight form and of the mean-field subtraction
(Sec. II) with the FP64 oracle, through the C ABI.

Each variant is followed walker by walker for 20 shared-draw steps at the
bars of the plain step (1e-10 relative on the FP64 path, 1e-4 in the
reduced modes): weights, overlaps, orbitals, Green's functions and local
energies, as in tests/gpu_helpers.py. The full-size shapes are followed on
sampled walkers with the comb moved past step 20.
"""
import numpy as np
import pytest

from gpu_helpers import side_by_side as run_side_by_side
from oracle import afqmc as O
from synth import config_c1, config_c2, config_c3, config_c4, small_system

pytestmark = pytest.mark.gpu

# (weight_mode, mf_subtract): the plain hybrid form is covered elsewhere
VARIANTS = [(0, 1), (1, 0), (1, 1)]


@pytest.fixture(scope="session", autouse=True)
def built():
    from paper_1804_03310_gb300 import build
    build.build()


def side_by_side(system, precision, n_steps, rtol, walkers=None, energy_at=()):
    from paper_1804_03310_gb300 import Afqmc
    gpu = Afqmc.from_system(system, precision=precision)
    orc = O.OracleRun(system, walker_ids=walkers)
    assert abs(gpu.afqmc_energy_shift() - orc.e_shift) <= 1e-10 * max(1.0, abs(orc.e_shift))
    worst = run_side_by_side(gpu, orc, n_steps, rtol, walkers=walkers, energy_at=energy_at,
                             label=f"{precision} mode={system.weight_mode} "
                                   f"mf={system.mf_subtract}")
    gpu.close()
    return worst


@pytest.mark.parametrize("mode,mf", VARIANTS)
def test_c1_twenty_steps_fp64(mode, mf):
    s = config_c1().replace(weight_mode=mode, mf_subtract=mf)
    w = side_by_side(s, "fp64", 20, 1e-10, energy_at=(5, 10, 20))
    print(f"c1 fp64 mode={mode} mf={mf} worst", w)


@pytest.mark.parametrize("mode,mf", VARIANTS)
@pytest.mark.parametrize("M,nu,nd,G,W", [
    (7, 3, 2, 5, 5),
    (33, 17, 16, 67, 67),
    (12, 4, 0, 9, 3),
    (70, 5, 9, 130, 40),
])
def test_ragged_sizes_fp64(M, nu, nd, G, W, mode, mf):
    """The gentler of the two ragged-size recipes (eigenvector trial,
    dt = 0.01): in the local-energy form a weight takes dt E_L each step,
    and with a random trial at dt = 0.02 the M = 70 walkers reach the trial's
    nodes within a few steps, where |E_L| grows to 1e3-1e4 Ha and its
    conditioning, not the kernels, decides the last digits (the oracle's
    own E_L moves by 1e-12 relative under a 1e-14 change of the walker)."""
    s = small_system(M=M, n_up=nu, n_dn=nd, n_chol=G, seed=M + G,
                     l_sigma=0.05 * (10.0 / M) ** 0.5, n_walkers=W, dtau=0.01,
                     ortho_every=3, measure_every=4, pc_every=4,
                     trial="eig").replace(weight_mode=mode, mf_subtract=mf)
    side_by_side(s, "fp64", 8, 1e-10, energy_at=(4, 8))


@pytest.mark.parametrize("mode,mf", VARIANTS)
@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3", "fp32"])
def test_c2_full_size_sampled_reduced(prec, mode, mf):
    s = config_c2(pc_every=0).replace(weight_mode=mode, mf_subtract=mf)
    w = side_by_side(s, prec, 20, 1e-4, walkers=[0, 700, 1023], energy_at=(10, 20))
    print(f"c2 {prec} mode={mode} mf={mf} worst", w)


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_c3_full_size_sampled_local_energy_mean_field(prec):
    s = config_c3(pc_every=0).replace(weight_mode=1, mf_subtract=1)
    w = side_by_side(s, prec, 20, 1e-10 if prec == "fp64" else 1e-4, walkers=[0, 2047],
                     energy_at=(10, 20))
    print(f"c3 {prec} local energy, mean field worst", w)


@pytest.mark.parametrize("prec,rtol", [("fp64", 1e-10), ("tf32x3", 1e-4), ("bf16x3", 1e-4)])
def test_multidet_mean_field(prec, rtol):
    s = small_system(M=12, n_up=3, n_dn=3, n_chol=16, seed=21, n_walkers=24, dtau=0.01,
                     l_sigma=0.1, ortho_every=2, measure_every=5, pc_every=0,
                     trial="eig", n_det=20).replace(mf_subtract=1)
    w = side_by_side(s, prec, 20, rtol, energy_at=(5, 10, 20))
    print(f"multidet mean field {prec} worst", w)


def test_c4_full_size_sampled_mean_field():
    s = config_c4(pc_every=0).replace(mf_subtract=1)
    w = side_by_side(s, "tf32x3", 20, 1e-4, walkers=[0, 1023], energy_at=(20,))
    print("c4 tf32x3 mean field worst", w)


def test_force_bias_vanishes_at_the_reference_with_the_mean_field():
    """The walkers start at the reference determinant, whose mean field is
    subtracted: the first step's force bias is zero, the second's matches
    the oracle."""
    from paper_1804_03310_gb300 import Afqmc
    s = config_c1().replace(mf_subtract=1)
    gpu = Afqmc.from_system(s, precision="fp64")
    orc = O.OracleRun(s)
    gpu.afqmc_propagate(1)
    orc.step()
    assert np.abs(gpu.afqmc_force_bias()).max() < 1e-12
    gpu.afqmc_propagate(1)
    orc.step()
    xb = gpu.afqmc_force_bias()
    err = np.max(np.abs(xb - orc.last["xbar"])) / np.max(np.abs(orc.last["xbar"]))
    assert err < 1e-12
    gpu.close()


def test_mean_field_subtraction_keeps_more_walkers_alive():
    """What the subtraction is for: with the reference's mean field taken
    out of the force bias the overlap phases shrink, so the phaseless cut
    removes fewer walkers (H-chain shape, 60 steps, comb off)."""
    from paper_1804_03310_gb300 import Afqmc
    alive = {}
    for mf in (0, 1):
        s = config_c2(pc_every=0, measure_every=0).replace(mf_subtract=mf, dtau=0.02)
        gpu = Afqmc.from_system(s, precision="tf32x3")
        gpu.afqmc_propagate(60)
        w, _ = gpu.afqmc_weights()
        alive[mf] = int(np.count_nonzero(w > 0))
        gpu.close()
    print("walkers alive after 60 steps (no subtraction, subtraction):", alive)
    assert alive[1] > 4 * alive[0]
