"""Pins of the FP64 oracle against things other than itself.

Each test fixes one piece of the oracle to an independent route: published
known-answer vectors, brute-force second quantisation in the full Fock space
(tests/fock.py), closed forms, invariants and textbook special cases. A
plausible slip in the oracle (a dropped term, a sign, a transposed Green's
function, a wrong exponent in the importance factor) fails at least one.
"""
import math
import os

import numpy as np
import pytest
from scipy.linalg import expm
from scipy import stats

from fock import FockSpace, eri_from_chol, mixed
from oracle import afqmc as O
from oracle import philox as P
from synth import small_system, make_system

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rand_walker(rng, M, N, scale=1.0):
    return (rng.normal(size=(M, N)) + 1j * rng.normal(size=(M, N))) * scale


# ---------------------------------------------------------------- Philox


def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        out = P.philox4x32_10(v[0], v[1], v[2], v[3], v[4], v[5])
        assert [int(o) for o in out] == v[6:10]


def test_gaussian_fields_statistics():
    x = P.gaussian_fields(seed=12345, run_id=3, step=7,
                          walkers=np.arange(2000), n_chol=101)
    assert x.shape == (2000, 101)
    flat = x.ravel()
    assert abs(flat.mean()) < 0.01
    assert abs(flat.var() - 1.0) < 0.01
    assert stats.kstest(flat, "norm").pvalue > 1e-3
    # distinct counters give uncorrelated draws
    y = P.gaussian_fields(seed=12345, run_id=3, step=8,
                          walkers=np.arange(2000), n_chol=101)
    assert abs(np.corrcoef(flat, y.ravel())[0, 1]) < 0.01
    # a walker's draws do not depend on which other walkers are drawn with it
    z = P.gaussian_fields(seed=12345, run_id=3, step=7, walkers=[5, 17],
                          n_chol=101)
    assert np.array_equal(z, x[[5, 17]])


def test_comb_uniform_range():
    us = [P.comb_uniform(9, 0, s) for s in range(500)]
    assert all(0.0 < u < 1.0 for u in us)
    assert stats.kstest(us, "uniform").pvalue > 1e-3


# ---------------------------------------------------------------- Fock space


@pytest.fixture(scope="module")
def fock4():
    return FockSpace(4)


@pytest.fixture(scope="module")
def sys4():
    return small_system(M=4, n_up=2, n_dn=1, n_chol=3, seed=5, l_sigma=0.3)


def test_slater_overlap_is_determinant(fock4):
    rng = np.random.default_rng(1)
    M = 4
    Pu, Pd = rand_walker(rng, M, 2), rand_walker(rng, M, 1)
    Du, Dd = rand_walker(rng, M, 2), rand_walker(rng, M, 1)
    a = np.vdot(fock4.slater(Du, Dd), fock4.slater(Pu, Pd))
    b = np.linalg.det(Du.conj().T @ Pu) * np.linalg.det(Dd.conj().T @ Pd)
    assert abs(a - b) < 1e-12 * abs(b)


def test_one_body_remainder_reproduces_hamiltonian(fock4, sys4):
    """H of Eq. 1 equals sum_s H1'(s) + 1/2 sum_g L_g^2 (operator identity)."""
    s = sys4
    H = fock4.hamiltonian(s.h1, eri_from_chol(s.L))
    h1p = O.one_body_remainder(s.h1, s.L)
    H2 = fock4.one_body(h1p.astype(complex))
    for g in range(s.n_chol):
        Lg = fock4.one_body(s.L[g].astype(complex))
        H2 = H2 + 0.5 * (Lg @ Lg)
    assert abs(H - H2).max() < 1e-12


@pytest.mark.parametrize("n_det", [1, 5])
def test_overlap_green_force_bias_energy_vs_fock(fock4, n_det):
    s = small_system(M=4, n_up=2, n_dn=1, n_chol=3, seed=7, l_sigma=0.3,
                     n_det=n_det)
    rng = np.random.default_rng(2)
    if n_det > 1:   # complex CI coefficients: the bra conjugates them
        s = s.replace(ci=s.ci * np.exp(1j * rng.uniform(0, 2 * np.pi, n_det)))
    trial = O.Trial.from_system(s)
    Pu, Pd = rand_walker(rng, 4, 2), rand_walker(rng, 4, 1)
    psi_t = fock4.multi_det(s.C_up, s.C_dn, s.occ_up, s.occ_dn, s.ci)
    phi = fock4.slater(Pu, Pd)
    # overlap
    logO, Gu, Gd, _ = O.mixed_green(trial, Pu[None], Pd[None])
    assert abs(np.exp(logO[0]) - np.vdot(psi_t, phi)) < 1e-12 * abs(np.vdot(psi_t, phi))
    # Green's function G_ij = <c+_i c_j>
    for spin, G in ((0, Gu), (1, Gd)):
        for i in range(4):
            for j in range(4):
                ref = mixed(fock4, psi_t, fock4.cdag(i, spin) @ fock4.c(j, spin), phi)
                assert abs(G[0, i, j] - ref) < 1e-11
    # force bias: X_g = <L_g hat>_mixed
    X, xbar = O.force_bias(s.L, Gu, Gd, dtau=0.01, cap=0.0)
    for g in range(s.n_chol):
        ref = mixed(fock4, psi_t, fock4.one_body(s.L[g].astype(complex)), phi)
        assert abs(X[0, g] - ref) < 1e-11
        assert abs(xbar[0, g] - (-1j * 0.1 * ref)) < 1e-12
    # local energy of Eq. 1
    H = fock4.hamiltonian(s.h1, eri_from_chol(s.L))
    ref = mixed(fock4, psi_t, H, phi)
    e = O.local_energy(s.h1, s.L, trial, Pu[None], Pd[None])[0]
    assert abs(e - ref) < 1e-10 * max(1.0, abs(ref))
    if n_det == 1:
        eg = O.local_energy_green(s.h1, s.L, Gu, Gd)[0]
        assert abs(eg - ref) < 1e-10 * max(1.0, abs(ref))
        _, Tu, _ = O.det_green(trial.D_up[0], Pu[None])
        _, Td, _ = O.det_green(trial.D_dn[0], Pd[None])
        ey = O.local_energy_y(s.h1, s.L, trial.D_up[0], trial.D_dn[0], Tu, Td)[0]
        assert abs(ey - ref) < 1e-10 * max(1.0, abs(ref))


def test_trial_energy_equals_variational_energy():
    """Closed form: with phi = Psi_T, E_L = E_var from Slater-Condon rules on
    the four-index integrals, E = sum h P + 1/2 sum (ij|kl)
    [P_ij P_kl - sum_s P^s_il P^s_kj], P^s = D^s D^s^T."""
    s = small_system(M=7, n_up=3, n_dn=2, n_chol=6, seed=3, l_sigma=0.2,
                     trial="random")
    Du, Dd = s.trial_up(), s.trial_dn()
    Pu_, Pd_ = Du @ Du.T, Dd @ Dd.T
    Ptot = Pu_ + Pd_
    eri = np.einsum("gij,gkl->ijkl", s.L, s.L)   # (ij|kl)
    e_var = np.sum(s.h1 * Ptot) + 0.5 * (
        np.einsum("ijkl,ij,kl->", eri, Ptot, Ptot)
        - np.einsum("ijkl,il,kj->", eri, Pu_, Pu_)
        - np.einsum("ijkl,il,kj->", eri, Pd_, Pd_))
    trial = O.Trial.from_system(s)
    e = O.local_energy(s.h1, s.L, trial, Du[None].astype(complex),
                       Dd[None].astype(complex))[0]
    assert abs(e - e_var) < 1e-12 * abs(e_var)
    assert abs(e.imag) < 1e-13


def test_hs_importance_factor_quadrature(fock4, sys4):
    """Eq. 2 with the force-bias shift: for one field, the Gaussian average of
    exp(x xbar - xbar^2/2) <Psi_T| exp(V(x - xbar)) |phi> equals
    <Psi_T| exp(-dt/2 L^2) |phi> for any shift xbar (Gauss-Hermite, exact for
    this entire integrand to quadrature accuracy)."""
    s = sys4
    rng = np.random.default_rng(4)
    dt = 0.05
    Pu, Pd = rand_walker(rng, 4, 2), rand_walker(rng, 4, 1)
    psi_t = fock4.slater(s.trial_up().astype(complex), s.trial_dn().astype(complex))
    phi = fock4.slater(Pu, Pd)
    L1 = s.L[:1]
    Lhat = fock4.one_body(L1[0].astype(complex)).toarray()
    target = np.vdot(psi_t, expm(-0.5 * dt * Lhat @ Lhat) @ phi)
    nodes, wts = np.polynomial.hermite_e.hermegauss(80)
    wts = wts / math.sqrt(2 * math.pi)
    for xbar in (0.0 + 0.0j, -0.3j, 0.2 - 0.1j):
        acc = 0.0
        for xq, wq in zip(nodes, wts):
            V = O.one_body_operator(L1, np.array([[xq]]), np.array([[xbar]]), dt)[0]
            Vhat = fock4.one_body(V).toarray()
            fac = np.exp(O.importance_log(np.array([[xq]]), np.array([[xbar]]))[0])
            acc += wq * fac * np.vdot(psi_t, expm(Vhat) @ phi)
        assert abs(acc - target) < 1e-10 * abs(target)


def test_propagation_is_thouless(fock4, sys4):
    """B_half exp(V) B_half Phi as a Slater determinant equals the Fock-space
    exponentials of the one-body operators applied to the determinant."""
    s = sys4
    rng = np.random.default_rng(8)
    dt = 0.05
    Pu, Pd = rand_walker(rng, 4, 2), rand_walker(rng, 4, 1)
    x = rng.normal(size=(1, s.n_chol))
    xbar = 0.1 * (rng.normal(size=(1, s.n_chol)) + 1j * rng.normal(size=(1, s.n_chol)))
    V = O.one_body_operator(s.L, x, xbar, dt)[0]
    h1p = O.one_body_remainder(s.h1, s.L)
    B = O.half_step_propagator(h1p, dt)
    nu = O.propagate(B, V[None], Pu[None], 40)[0]
    nd = O.propagate(B, V[None], Pd[None], 40)[0]
    Hh = fock4.one_body(h1p.astype(complex)).toarray()
    Vh = fock4.one_body(V).toarray()
    Eh = expm(-0.5 * dt * Hh)
    ref = Eh @ (expm(Vh) @ (Eh @ fock4.slater(Pu, Pd)))
    got = fock4.slater(nu, nd)
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


def test_mean_field_is_the_reference_expectation(fock4, sys4):
    """lbar_g = <D_0|L_g|D_0> / <D_0|D_0> for the reference determinant,
    by brute force in Fock space; at phi = D_0 the subtracted force bias
    vanishes, and the remainder with the mean field reproduces Eq. 1 with
    the constant E_0 (an operator identity on the whole Fock space)."""
    s = sys4
    trial = O.Trial.from_system(s)
    lbar = O.mean_field(s.L, trial.D_up[0], trial.D_dn[0])
    d0 = fock4.slater(trial.D_up[0], trial.D_dn[0])
    for g in range(s.n_chol):
        Lg = fock4.one_body(s.L[g].astype(complex))
        ref = np.vdot(d0, Lg @ d0) / np.vdot(d0, d0)
        assert abs(lbar[g] - ref) < 1e-12
    # a non-orthonormal determinant with the same span gives the same mean field
    T = np.array([[1.0, 0.3], [0.2, 2.0]])
    assert np.abs(O.mean_field(s.L, trial.D_up[0] @ T, 0.5 * trial.D_dn[0]) - lbar).max() < 1e-12
    _, Gu, Gd, _ = O.mixed_green(trial, trial.D_up[:1], trial.D_dn[:1])
    X, xbar = O.force_bias(s.L, Gu, Gd, 0.01, 0.0, lbar)
    assert np.abs(xbar).max() < 1e-13 and np.abs(X).max() > 0.1
    H = fock4.hamiltonian(s.h1, eri_from_chol(s.L)).toarray()
    H2 = fock4.one_body(O.one_body_remainder(s.h1, s.L, lbar).astype(complex)).toarray()
    eye = np.eye(fock4.dim)
    for g in range(s.n_chol):
        Lg = fock4.one_body(s.L[g].astype(complex)).toarray() - lbar[g] * eye
        H2 = H2 + 0.5 * (Lg @ Lg)
    assert np.abs(H - H2 - O.mean_field_constant(lbar) * eye).max() < 1e-12


def test_mean_field_hs_quadrature(fock4, sys4):
    """Eq. 2 for the subtracted operator: for one field, the Gaussian
    average of exp(x xbar - xbar^2/2) times the mean-field scalar times
    <Psi_T| exp(V(x - xbar)) |phi> equals <Psi_T| exp(-dt/2 (L - lbar)^2) |phi>
    for any shift xbar."""
    s = sys4
    rng = np.random.default_rng(14)
    dt = 0.05
    Pu, Pd = rand_walker(rng, 4, 2), rand_walker(rng, 4, 1)
    trial = O.Trial.from_system(s)
    lbar = O.mean_field(s.L[:1], trial.D_up[0], trial.D_dn[0])
    idx = fock4.sector(2, 1)          # the operators conserve both spins' counts
    psi_t = fock4.slater(trial.D_up[0], trial.D_dn[0])[idx]
    phi = fock4.slater(Pu, Pd)[idx]
    Lh = fock4.one_body(s.L[0].astype(complex)).toarray()[np.ix_(idx, idx)]
    Lh = Lh - lbar[0] * np.eye(len(idx))
    target = np.vdot(psi_t, expm(-0.5 * dt * Lh @ Lh) @ phi)
    nodes, wts = np.polynomial.hermite_e.hermegauss(80)
    wts = wts / math.sqrt(2 * math.pi)
    for xbar in (0.0 + 0.0j, -0.3j, 0.2 - 0.1j):
        acc = 0.0
        for xq, wq in zip(nodes, wts):
            x, xb = np.array([[xq]]), np.array([[xbar]])
            V = O.one_body_operator(s.L[:1], x, xb, dt)[0]
            Vhat = fock4.one_body(V).toarray()[np.ix_(idx, idx)]
            lnf = O.importance_log(x, xb)[0] + O.mean_field_log(x, xb, lbar, dt)[0]
            acc += wq * np.exp(lnf) * np.vdot(psi_t, expm(Vhat) @ phi)
        assert abs(acc - target) < 1e-10 * abs(target)


def _step_average(s, Pu, Pd, dt, mf, nodes, wts):
    """Gauss-Hermite average over the one field of the hybrid importance
    factor I(x) of one step from the walker (Pu, Pd), with the oracle's own
    force bias, propagation, overlaps and mean-field terms."""
    trial = O.Trial.from_system(s)
    lbar = O.mean_field(s.L, trial.D_up[0], trial.D_dn[0]) if mf else None
    e0 = 0.0 if lbar is None else O.mean_field_constant(lbar)
    B = O.half_step_propagator(O.one_body_remainder(s.h1, s.L, lbar), dt)
    lo, Gu, Gd, _ = O.mixed_green(trial, Pu[None], Pd[None])
    _, xb = O.force_bias(s.L, Gu, Gd, dt, 0.0, lbar)
    et = O.reference_energy(s.h1, s.L, trial)
    acc = 0.0
    for xq, wq in zip(nodes, wts):
        x = np.array([[xq]])
        V = O.one_body_operator(s.L, x, xb, dt)
        ln, _ = O.trial_overlap(trial, O.propagate(B, V, Pu[None], 30),
                                O.propagate(B, V, Pd[None], 30))
        lmf = 0.0 if lbar is None else O.mean_field_log(x, xb, lbar, dt)
        acc += wq * np.exp(O.log_importance(ln - lo + lmf, x, xb, dt, et, e0))[0]
    return acc, et, lbar


@pytest.mark.parametrize("mf", [0, 1])
def test_step_importance_factor_is_the_projected_overlap(fock4, mf):
    """One field, so the field integral is exact: the Gaussian average of the
    hybrid factor I(x) (overlap ratio, shift factor, mean-field scalar and
    both constants) equals <Psi_T| B_half exp(-dt/2 (L - lbar)^2) B_half
    |phi> / <Psi_T|phi> exp(dt (E_T - E_0)), with E_0 read off the Fock-space
    identity H = H1' + 1/2 (L - lbar)^2 + E_0 rather than from the oracle."""
    s = small_system(M=4, n_up=2, n_dn=1, n_chol=1, seed=5, l_sigma=0.3)
    rng = np.random.default_rng(4)
    Pu, Pd = rand_walker(rng, 4, 2), rand_walker(rng, 4, 1)
    dt = 0.05
    nodes, wts = np.polynomial.hermite_e.hermegauss(60)
    wts = wts / math.sqrt(2 * math.pi)
    got, et, lbar = _step_average(s, Pu, Pd, dt, mf, nodes, wts)
    lb = np.zeros(1) if lbar is None else lbar
    eye = np.eye(fock4.dim)
    H = fock4.hamiltonian(s.h1, eri_from_chol(s.L)).toarray()
    H1 = fock4.one_body(O.one_body_remainder(s.h1, s.L, lbar).astype(complex)).toarray()
    Lh = fock4.one_body(s.L[0].astype(complex)).toarray() - lb[0] * eye
    e0 = (H - H1 - 0.5 * Lh @ Lh)[0, 0]
    Bh = expm(-0.5 * dt * H1)
    trial = O.Trial.from_system(s)
    psi_t = fock4.slater(trial.D_up[0], trial.D_dn[0])
    phi = fock4.slater(Pu, Pd)
    target = (np.vdot(psi_t, Bh @ expm(-0.5 * dt * Lh @ Lh) @ Bh @ phi)
              / np.vdot(psi_t, phi) * np.exp(dt * (et - e0)))
    assert abs(got - target) < 1e-10 * abs(target)


@pytest.mark.parametrize("mf", [0, 1])
def test_local_energy_weight_is_the_mean_importance_factor(mf):
    """Sec. II's local-energy form: the factor exp(-dt (Re E_L - E_T)) that a
    step in that form gives a walker (its cut divided out) is the modulus of
    the Gaussian average of the hybrid factor up to O(dt^2): the gap falls
    by four when dt halves (one field, so the average is exact)."""
    s = small_system(M=4, n_up=2, n_dn=1, n_chol=1, seed=5, l_sigma=0.3)
    rng = np.random.default_rng(4)
    Pu, Pd = rand_walker(rng, 4, 2), rand_walker(rng, 4, 1)
    nodes, wts = np.polynomial.hermite_e.hermegauss(60)
    wts = wts / math.sqrt(2 * math.pi)
    gaps = []
    for dt in (0.02, 0.01):
        avg, _, _ = _step_average(s, Pu, Pd, dt, mf, nodes, wts)
        run = O.OracleRun(s.replace(dtau=dt, n_walkers=1, weight_mode=1, mf_subtract=mf,
                                    fb_cap=0.0, ortho_every=0, measure_every=0,
                                    pc_every=0))
        run.Phi_up, run.Phi_dn = Pu[None].copy(), Pd[None].copy()
        run.logO, _ = O.trial_overlap(run.trial, run.Phi_up, run.Phi_dn)
        run.step()
        cut = max(0.0, math.cos(run.last["lnR"][0].imag))
        assert cut > 0.5
        gaps.append(abs(run.weight[0] / cut - abs(avg)))
    assert gaps[1] < 3e-4 and 3.5 < gaps[0] / gaps[1] < 4.5


def test_mean_field_subtraction_shrinks_the_phase():
    """What the subtraction is for: with the mean field taken out, the
    overlap ratios' phases (the phaseless cut's argument) are smaller."""
    s = small_system(M=6, n_up=2, n_dn=2, n_chol=8, seed=3, n_walkers=64, dtau=0.02,
                     l_sigma=0.3, ortho_every=2, measure_every=0, pc_every=0, fb_cap=0.0)
    spread = []
    for mf in (0, 1):
        run = O.OracleRun(s.replace(mf_subtract=mf))
        ph = []
        for _ in range(4):
            run.step()
            ph.append(np.abs(run.last["lnR"].imag))
        spread.append(np.mean(ph))
    assert spread[1] < 0.5 * spread[0]


def test_taylor_truncation_bound():
    rng = np.random.default_rng(9)
    for scale in (0.05, 0.3, 0.8):
        V = scale * (rng.normal(size=(6, 6)) + 1j * rng.normal(size=(6, 6))) / 3
        Phi = rand_walker(rng, 6, 3)
        nv = np.linalg.norm(V, 2)
        err = np.linalg.norm(O.taylor_apply(V[None], Phi[None], 6)[0] - expm(V) @ Phi, 2)
        bound = nv ** 7 / math.factorial(7) * math.exp(nv) * np.linalg.norm(Phi, 2)
        assert err <= bound * (1 + 1e-9) + 1e-14


def test_half_step_propagator_matches_expm():
    s = small_system(M=7, n_up=2, n_dn=2, n_chol=4, seed=1)
    h1p = O.one_body_remainder(s.h1, s.L)
    assert np.abs(O.half_step_propagator(h1p, 0.03) - expm(-0.015 * h1p)).max() < 1e-14


# ---------------------------------------------------------------- closed forms


def test_zero_interaction_is_exact_free_propagation():
    """All L_g = 0: V = 0, the Taylor series is exact and the walkers follow
    exp(-n dt h1) Psi_0; with an eigenvector trial every weight stays 1 and
    E_L stays E_var = sum of occupied orbital energies."""
    s = make_system("free", M=8, n_up=3, n_dn=2, n_chol=4, ham_seed=21,
                    l_kind="zero", trial="random", dtau=0.02, n_walkers=3,
                    n_steps=10, seed=5, ortho_every=0, measure_every=0,
                    pc_every=0)
    run = O.OracleRun(s).run(10)
    U = expm(-10 * 0.02 * s.h1)
    assert np.abs(run.Phi_up[0] - U @ s.trial_up()).max() < 1e-13
    assert np.abs(run.Phi_dn[2] - U @ s.trial_dn()).max() < 1e-13
    s2 = s.replace(C_up=np.linalg.eigh(s.h1)[1], C_dn=np.linalg.eigh(s.h1)[1])
    run2 = O.OracleRun(s2).run(10)
    eps = np.linalg.eigh(s.h1)[0]
    assert abs(run2.e_shift - (eps[:3].sum() + eps[:2].sum())) < 1e-12
    assert np.abs(run2.weight - 1.0).max() < 1e-12
    assert np.abs(run2.local_energies() - run2.e_shift).max() < 1e-12


def test_green_invariants():
    s = small_system(M=9, n_up=4, n_dn=3, n_chol=5, seed=2, trial="random")
    rng = np.random.default_rng(3)
    D = s.trial_up().astype(complex)
    Phi = rand_walker(rng, 9, 4)[None]
    _, Th, G = O.det_green(D, Phi)
    GT = G[0].T
    assert np.abs(GT @ GT - GT).max() < 1e-12
    assert abs(np.trace(G[0]) - 4) < 1e-12
    assert np.abs(D.conj().T @ Th[0] - np.eye(4)).max() < 1e-12


def test_mgs_matches_householder():
    rng = np.random.default_rng(5)
    A = rand_walker(rng, 11, 5)
    Q, R = O.modified_gram_schmidt(A)
    assert np.abs(Q @ R - A).max() < 1e-13
    assert np.abs(Q.conj().T @ Q - np.eye(5)).max() < 1e-13
    assert np.abs(np.tril(R, -1)).max() == 0
    assert np.all(np.diag(R).real > 0) and np.abs(np.diag(R).imag).max() == 0
    Qh, Rh = np.linalg.qr(A)
    ph = np.diag(Rh) / np.abs(np.diag(Rh))
    assert np.abs(Qh * ph[None, :] - Q).max() < 1e-12


def test_orthonormalization_changes_nothing_observable():
    s = small_system(M=8, n_up=3, n_dn=3, n_chol=6, seed=4, n_walkers=5,
                     ortho_every=0, measure_every=0, pc_every=0, dtau=0.05,
                     l_sigma=0.15)
    a = O.OracleRun(s)
    b = O.OracleRun(s.replace(ortho_every=1))
    for _ in range(4):
        a.step()
        b.step()
    assert np.abs(a.weight - b.weight).max() < 1e-11 * np.abs(a.weight).max()
    assert np.abs(a.local_energies() - b.local_energies()).max() < 1e-10
    _, Gu_a, _, _ = O.mixed_green(a.trial, a.Phi_up, a.Phi_dn)
    _, Gu_b, _, _ = O.mixed_green(b.trial, b.Phi_up, b.Phi_dn)
    assert np.abs(Gu_a - Gu_b).max() < 1e-11
    # the overlaps differ exactly by the Gram-Schmidt factors: ratios agree
    assert np.abs(np.exp(a.logO - b.logO) -
                  np.exp(O.trial_overlap(a.trial, a.Phi_up, a.Phi_dn)[0]
                         - O.trial_overlap(b.trial, b.Phi_up, b.Phi_dn)[0])).max() < 1e-10


def test_weight_update_phaseless_cut():
    w = np.array([1.0, 2.0, 0.0, 1.0])
    lo = np.zeros(4, complex)
    ln = np.array([0.1 + 0.2j, -0.3 + 2.0j, 0.0, 0.5 + 0j])
    x = np.zeros((4, 2))
    xb = np.zeros((4, 2), complex)
    out = O.update_weights(w, lo, ln, x, xb, 0.01, -1.0)
    assert abs(out[0] - np.exp(0.1 - 0.01) * np.cos(0.2)) < 1e-15
    assert out[1] == 0.0                      # phase beyond pi/2: killed
    assert out[2] == 0.0                      # stays killed
    assert abs(out[3] - np.exp(0.5 - 0.01)) < 1e-15


def test_phaseless_cut_uses_overlap_phase_only():
    """Sec. II: the cut is max(0, cos dtheta) with dtheta the phase of the
    overlap ratio <Psi_T|phi'>/<Psi_T|phi> alone; the importance factor's
    phase enters the weight only through its modulus."""
    w = np.array([1.0, 1.0])
    lo = np.zeros(2, complex)
    ln = np.array([0.05 + 0.2j, 0.05 - 1.0j])
    x = np.array([[1.0], [1.0]])
    xb = np.array([[1.5j], [0.9j]])       # importance phase 1.5 and 0.9
    out = O.update_weights(w, lo, ln, x, xb, 0.01, -1.0)
    # |exp(x xbar - xbar^2/2)| = exp(Re(-xbar^2/2)) = exp(xbar_im^2 / 2)
    assert abs(out[0] - np.exp(0.05 + 1.5 ** 2 / 2 - 0.01) * np.cos(0.2)) < 1e-14
    assert abs(out[1] - np.exp(0.05 + 0.9 ** 2 / 2 - 0.01) * np.cos(1.0)) < 1e-14


def test_weight_cap_option():
    # the cap (an option beside the paper's step) clips at cap * w_ref and
    # changes nothing below it; an unbounded cap is the uncapped update
    w = np.array([1.0, 2.0, 0.0, 1.0])
    lo = np.zeros(4, complex)
    ln = np.array([0.1 + 0.2j, 1.5 + 0.1j, 0.0, 0.5 + 0j])
    x = np.zeros((4, 2))
    xb = np.zeros((4, 2), complex)
    free = O.update_weights(w, lo, ln, x, xb, 0.01, -1.0)
    capped = O.update_weights(w, lo, ln, x, xb, 0.01, -1.0, cap=2, w_ref=0.75)
    assert np.array_equal(capped, np.minimum(free, 1.5))
    assert capped[1] == 1.5 and capped[0] == free[0] and capped[2] == 0.0
    assert np.array_equal(O.update_weights(w, lo, ln, x, xb, 0.01, -1.0, cap=10 ** 9), free)
    # in a run the reference is the common weight of the last comb
    s = small_system(M=6, n_up=2, n_dn=2, n_chol=8, seed=3, n_walkers=16, dtau=0.05,
                     l_sigma=0.3, ortho_every=2, measure_every=0, pc_every=3)
    run = O.OracleRun(s.replace(weight_cap=1))
    ref = O.OracleRun(s)
    bound, differs = 1.0, False
    for k in range(1, 10):
        run.step()
        ref.step()
        assert np.all(run.weight <= bound * (1 + 1e-15)) or k % 3 == 0
        differs |= not np.array_equal(run.weight, ref.weight)
        bound = run.w_ref
    assert differs                              # the cap did bind in this run


# ---------------------------------------------------------------- comb


class _KeepScaleRun(O.OracleRun):
    """The run without the renormalisation: after a comb every walker keeps
    the common weight S/n."""

    def population_control(self):
        u = P.comb_uniform(self.s.seed, self.s.run_id, self.step_count)
        parent, wnew = O.comb(self.weight, u)
        self.w_ref = wnew
        self.Phi_up = self.Phi_up[parent].copy()
        self.Phi_dn = self.Phi_dn[parent].copy()
        self.logO = self.logO[parent].copy()
        self.weight = np.full(self.walker_ids.size, wnew)
        return parent


def test_renormalised_comb_changes_nothing_observable():
    """Dividing the common weight S/n out at each comb (and keeping its log)
    leaves the walkers and the mixed energies as they are: the weights times
    exp(log_scale) are the weights of the run that keeps S/n."""
    s = small_system(M=6, n_up=2, n_dn=2, n_chol=8, seed=3, n_walkers=32, dtau=0.05,
                     l_sigma=0.3, ortho_every=2, measure_every=3, pc_every=3)
    a = O.OracleRun(s, e_shift=-40.0)
    b = _KeepScaleRun(s, e_shift=-40.0)
    for _ in range(12):
        a.step()
        b.step()
    assert a.log_scale != 0.0
    assert np.abs(a.Phi_up - b.Phi_up).max() < 1e-12
    assert np.abs(a.weight * np.exp(a.log_scale) - b.weight).max() < 1e-11 * b.weight.max()
    for (sa, ea, _), (sb, eb, _) in zip(a.energies, b.energies):
        assert sa == sb and abs(ea - eb) < 1e-11 * abs(eb)


def test_blocked_prefix_sum_and_comb():
    rng = np.random.default_rng(6)
    for n in (1, 7, 32, 33, 100, 2048):
        w = rng.uniform(0, 2, size=n)
        w[rng.uniform(size=n) < 0.1] = 0.0
        if w.sum() == 0:
            w[0] = 1.0
        C, S = O.blocked_prefix_sum(w)
        assert np.abs(C - np.cumsum(w)).max() < 1e-12 * S
        parent, wn = O.comb(w, 0.37)
        counts = np.bincount(parent, minlength=n)
        exp = w * n / S
        assert np.all(counts >= np.floor(exp) - 1) and np.all(counts <= np.ceil(exp) + 1)
        assert np.all(counts[w == 0] == 0)
        assert abs(wn * n - S) < 1e-12 * S
    # equal weights: identity
    parent, _ = O.comb(np.full(64, 0.5), 0.5)
    assert np.array_equal(parent, np.arange(64))


def test_comb_brute_force_intervals():
    w = np.array([0.5, 0.0, 1.5, 1.0, 0.25, 0.75])
    parent, step = O.comb(w, 0.2)
    C = np.cumsum(w)
    for j, k in enumerate(parent):
        t = (j + 0.2) * step
        lo = C[k - 1] if k > 0 else 0.0
        assert lo <= t < C[k]


def test_all_zero_weights_raise():
    with pytest.raises(FloatingPointError):
        O.comb(np.zeros(4), 0.5)


# ---------------------------------------------------------------- 2e / 4o


def fci_trial_2e4o(fs, s):
    """Exact ground state of the 2-electron, 4-orbital problem as a 16-determinant
    trial over orbital pairs (i up, j down), reference (0, 0) first."""
    H = fs.hamiltonian(s.h1, eri_from_chol(s.L)).toarray()
    idx = fs.sector(1, 1)
    e, v = np.linalg.eigh(H[np.ix_(idx, idx)])
    psi = np.zeros(fs.dim, complex)
    psi[idx] = v[:, 0]
    C = s.C_up
    pairs = [(0, 0)] + [(i, j) for i in range(4) for j in range(4) if (i, j) != (0, 0)]
    pairs.sort(key=lambda p: (p[0] != 0) + (p[1] != 0))
    occ_up = np.array([[p[0]] for p in pairs], dtype=np.int32)
    occ_dn = np.array([[p[1]] for p in pairs], dtype=np.int32)
    ci = np.array([np.vdot(fs.slater(C[:, [i]], C[:, [j]]), psi) for i, j in pairs])
    return e[0], occ_up, occ_dn, ci


def test_zero_variance_exact_trial(fock4):
    s = small_system(M=4, n_up=1, n_dn=1, n_chol=4, seed=8, l_sigma=0.3,
                     n_walkers=6, dtau=0.02, ortho_every=2, measure_every=0,
                     pc_every=0)
    e0, ou, od, ci = fci_trial_2e4o(fock4, s)
    s = s.replace(occ_up=ou, occ_dn=od, ci=ci)
    run = O.OracleRun(s)
    for _ in range(5):
        run.step()
        E = run.local_energies()
        assert np.abs(E - e0).max() < 1e-10


@pytest.mark.slow
def test_long_run_2e4o_matches_exact(fock4):
    """Weak interaction, single-determinant trial: the mixed energy of a long
    run agrees with exact diagonalisation within the statistical error."""
    s = small_system(M=4, n_up=1, n_dn=1, n_chol=4, seed=8, l_sigma=0.05,
                     n_walkers=200, dtau=0.02, ortho_every=2,
                     measure_every=10, pc_every=10)
    H = fock4.hamiltonian(s.h1, eri_from_chol(s.L)).toarray()
    idx = fock4.sector(1, 1)
    e0 = np.linalg.eigvalsh(H[np.ix_(idx, idx)])[0]
    run = O.OracleRun(s).run(1500)
    es = np.array([e for (st, e, _) in run.energies if st > 300])
    nb = 10
    blocks = es[: len(es) // nb * nb].reshape(nb, -1).mean(axis=1)
    err = blocks.std(ddof=1) / math.sqrt(nb)
    assert abs(blocks.mean() - e0) < 4 * err + 2e-4, (blocks.mean(), e0, err)
