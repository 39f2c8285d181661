"""Block-diagonal Cholesky vectors (shell-structured inputs): the one-body
operator is built on the blocks' entries only and its Taylor series is
applied block by block between the dense half steps. Same arithmetic as
the dense path, so the same bars against the FP64 oracle: 1e-10 relative
per walker on the FP64 path, 1e-4 in the reduced modes, every step for 20
shared-draw steps (full-size shapes on sampled walkers, comb moved past
step 20)."""
import numpy as np
import pytest

from gpu_helpers import side_by_side as run_side_by_side
from oracle import afqmc as O
from synth import config_c3, make_system, small_system

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-4, "tf32x3": 1e-4, "bf16x3": 1e-4}


@pytest.fixture(scope="session", autouse=True)
def built():
    from paper_1804_03310_gb300 import build
    build.build()


def shells(M, nu, nd, G, W, n_det=1, **kw):
    return make_system(f"shells_m{M}", M=M, n_up=nu, n_dn=nd, n_chol=G, ham_seed=M + G,
                       l_kind="shells", l_sigma=0.1, trial="eig", n_det=n_det, dtau=0.01,
                       n_walkers=W, n_steps=100, seed=M + G, ortho_every=2,
                       measure_every=4, pc_every=4, **kw)


def side_by_side(system, precision, n_steps, walkers=None, energy_at=(), expect_sparse=True,
                 **kw):
    from paper_1804_03310_gb300 import Afqmc
    gpu = Afqmc.from_system(system, precision=precision, **kw)
    if precision not in ("fp64", "fp32"):
        assert (gpu.afqmc_get_tuning()["taylor_fused"] == 4) == expect_sparse
    orc = O.OracleRun(system, walker_ids=walkers)
    w = run_side_by_side(gpu, orc, n_steps, TOL[precision], walkers=walkers,
                         energy_at=energy_at, label=f"{precision} block-sparse")
    gpu.close()
    return w


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("M,nu,nd,G,W", [
    (20, 4, 3, 30, 16),     # blocks 1,3,5,7,1,3: M % 4 == 0, half steps on the tensor cores
    (37, 6, 6, 50, 9),      # ragged: the last block cut short, half steps on the CUDA cores
    (70, 9, 8, 120, 5),     # M > 64
])
def test_shell_systems_match_oracle(M, nu, nd, G, W, prec):
    w = side_by_side(shells(M, nu, nd, G, W), prec, 8, energy_at=(4, 8))
    print(f"shells {M} {prec} worst", w)


@pytest.mark.parametrize("prec", ["fp64", "tf32x3", "bf16x3"])
def test_c3_full_size_block_sparse(prec):
    """The TM-atom shape (shells 1/3/5/7, M = 150) on the block-diagonal path."""
    s = config_c3(pc_every=0)
    w = side_by_side(s, prec, 20, walkers=[0, 2047], energy_at=(10, 20))
    print(f"c3 block-sparse {prec} worst", w)


def test_dense_path_when_asked():
    w = side_by_side(shells(20, 4, 3, 30, 16), "tf32x3", 4, expect_sparse=False,
                     block_sparse=2)
    print("shells 20 forced dense worst", w)


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_multidet_and_weight_forms_on_shells(prec):
    md = shells(20, 4, 3, 30, 12, n_det=10).replace(mf_subtract=1, pc_every=0)
    w = side_by_side(md, prec, 12, energy_at=(4, 12))
    print(f"shells multidet mean field {prec} worst", w)
    le = shells(20, 4, 3, 30, 12).replace(weight_mode=1, mf_subtract=1)
    w = side_by_side(le, prec, 12, energy_at=(4, 12))
    print(f"shells local energy mean field {prec} worst", w)


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_large_blocks_and_scattered_members(prec):
    """Blocks above 8 orbitals (the shared-memory form of the series) whose
    members are not contiguous: the same random permutation applied to the
    basis of a block-diagonal Hamiltonian."""
    s = small_system(M=40, n_up=5, n_dn=4, n_chol=24, seed=17, l_sigma=0.1, n_walkers=10,
                     dtau=0.01, ortho_every=2, measure_every=4, pc_every=4)
    mask = np.zeros((40, 40))
    for a in range(0, 40, 10):      # four blocks of 10: 400 entries = M^2 / 4
        mask[a:a + 10, a:a + 10] = 1.0
    perm = np.random.default_rng(3).permutation(40)
    mask = mask[np.ix_(perm, perm)]
    s = s.replace(L=s.L * mask[None])
    w = side_by_side(s, prec, 8, energy_at=(4, 8))
    print(f"large scattered blocks {prec} worst", w)
