"""Long-run mixed-estimator energies: reduced precision against FP64.

The reduced-precision paths must reproduce the FP64 GPU path's mixed
estimate (Sec. II, sum_w W Re E_L / sum_w W, measured every 0.1 Ha^-1 as in
Sec. IV.A): the error the precision adds must stay within 0.5 mHa, and
independent long runs must agree within their combined error bar. The FP64
path itself agrees with the FP64 oracle walker by walker over the first 20
shared-draw steps (test_gpu_step.py), so it stands in for the oracle at
lengths the oracle cannot follow.

Checks:

* paired, at every workload shape (the plain 10-orbital system, the
  H-chain, TM-atom and multi-determinant shapes at full size): both runs
  draw the same fields and the comb is off, so walker i of one run is
  walker i of the other for the whole run; the difference of the two mixed
  estimates, measurement by measurement, is the precision error alone, free
  of statistical noise, whether or not the energy is still drifting: it
  must stay within 0.5 mHa;
* independent, on the plain 10-orbital system, whose mixed estimate is
  stationary after about 1 Ha^-1 (the larger synthetic shapes start tens of
  Ha above their ground state and keep drifting for longer than a test can
  follow): with the comb on, the runs part ways after a few hundred
  steps (a tooth of the comb lands on the other side of a walker boundary),
  so their long-run means differ by statistical noise of about 1 mHa at this
  length (50 million walker-steps each); they must agree within twice the
  combined reblocked error bar. These runs use the weight cap option
  (below).
"""
import numpy as np
import pytest

from synth import config_c1, config_c2, config_c3, config_c4

pytestmark = pytest.mark.gpu

MHA = 1e-3


def reblocked_error(x):
    """Standard error of the mean of a serially correlated series: the largest
    naive error over pairwise-averaging levels that keep at least 4 blocks
    (Flyvbjerg and Petersen's blocking analysis)."""
    x = np.asarray(x, dtype=np.float64)
    best = 0.0
    while len(x) >= 4:
        best = max(best, float(np.std(x, ddof=1) / np.sqrt(len(x))))
        n = len(x) // 2 * 2
        x = 0.5 * (x[0:n:2] + x[1:n:2])
    return best


def run_energies(system, precision, n_steps):
    from paper_1804_03310_gb300 import Afqmc, build
    build.build()
    with Afqmc.from_system(system, precision=precision) as ctx:
        ctx.afqmc_propagate(n_steps)
        h = ctx.afqmc_energy_history()
    assert len(h) == n_steps // system.measure_every
    assert np.all(np.isfinite(h[:, 1]))
    return h[:, 1]


PAIRED = config_c1().replace(n_walkers=512, pc_every=0)
PAIRED_STEPS = 600
# With the paper's uncapped hybrid weights, a walker passing next to a node of
# the trial now and then takes a runaway weight that the comb copies to the
# whole population (seen on the FP64 path too, for some seeds); the long runs
# cap weights at 20x the last comb's common weight, the same on both paths.
INDEP = config_c1().replace(n_walkers=16384, weight_cap=20)
INDEP_STEPS = 3000
EQUIL = 20          # measurements dropped as equilibration (2 Ha^-1)


@pytest.fixture(scope="module")
def fp64_paired():
    return run_energies(PAIRED, "fp64", PAIRED_STEPS)


@pytest.fixture(scope="module")
def fp64_indep():
    return run_energies(INDEP, "fp64", INDEP_STEPS)


@pytest.mark.parametrize("prec", ["tf32x3", "fp32"])
def test_paired_energy_matches_fp64(fp64_paired, prec):
    red = run_energies(PAIRED, prec, PAIRED_STEPS)
    d = red - fp64_paired
    print(f"paired c1 {prec}: max |dE| = {np.max(np.abs(d)) / MHA:.5f} mHa, "
          f"mean dE = {np.mean(d) / MHA:.5f} mHa over {len(d)} measurements")
    assert np.max(np.abs(d)) <= 0.5 * MHA


# full-size shapes, comb off, one measurement every 20 steps
SHAPES = {
    "c2": (config_c2(pc_every=0), 200),
    "c3": (config_c3(pc_every=0), 100),
    # comb off: the multi-determinant shape loses walkers to the phaseless
    # cut from about step 50 (a third gone by step 70, all by step 170), so
    # its paired window is 60 steps
    "c4": (config_c4(pc_every=0), 60),
}
_FP64_SHAPES = {}


def fp64_shape(name):
    if name not in _FP64_SHAPES:
        s, n = SHAPES[name]
        _FP64_SHAPES[name] = run_energies(s, "fp64", n)
    return _FP64_SHAPES[name]


@pytest.mark.parametrize("name,prec", [("c2", "tf32x3"), ("c2", "bf16x3"), ("c2", "fp32"),
                                       ("c3", "tf32x3"), ("c3", "bf16x3"), ("c4", "tf32x3"),
                                       ("c4", "bf16x3"), ("c4", "fp32")])
def test_paired_energy_at_workload_shapes(name, prec):
    s, n = SHAPES[name]
    ref = fp64_shape(name)
    red = run_energies(s, prec, n)
    d = red - ref
    print(f"paired {name} {prec}: max |dE| = {np.max(np.abs(d)) / MHA:.5f} mHa over "
          f"{len(d)} measurements (E = {ref[-1]:.4f} Ha at step {n})")
    assert np.max(np.abs(d)) <= 0.5 * MHA


@pytest.mark.parametrize("prec", ["tf32x3", "fp32"])
def test_long_run_energy_matches_fp64(fp64_indep, prec):
    red = run_energies(INDEP, prec, INDEP_STEPS)
    a, b = fp64_indep[EQUIL:], red[EQUIL:]
    ea, eb = reblocked_error(a), reblocked_error(b)
    diff = float(np.mean(b) - np.mean(a))
    combined = float(np.hypot(ea, eb))
    print(f"long run c1 {prec}: E_fp64 = {np.mean(a):.6f} +- {ea:.6f}, E = {np.mean(b):.6f} "
          f"+- {eb:.6f}, diff = {diff / MHA:.4f} mHa, combined bar {combined / MHA:.4f} mHa")
    assert abs(diff) <= 2.0 * combined
