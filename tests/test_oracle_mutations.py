"""Mutation check of the oracle's pins.

Each case plants one plausible slip in the oracle (a sign, a dropped term, a
transposed Green's function, a wrong exponent, a missing conjugate, a wrong
constant) by replacing one oracle function or constant for the duration of
the case, then runs the pins of tests/test_oracle_pins.py. At least one pin
must fail for every slip; a slip that no pin catches would be a hole in the
oracle's independent checks. The slow pins (the Gauss-Hermite quadrature of
the field integral and the long 2e/4o run) run only for the slips they are
meant to catch.
"""
import numpy as np
import pytest

import test_oracle_pins as pins
from fock import FockSpace
from oracle import afqmc as O
from oracle import philox as P
from synth import small_system

_FOCK = FockSpace(4)
_SYS4 = small_system(M=4, n_up=2, n_dn=1, n_chol=3, seed=5, l_sigma=0.3)

FAST_PINS = [
    ("philox_kat", lambda: pins.test_philox_known_answers()),
    ("fields_statistics", lambda: pins.test_gaussian_fields_statistics()),
    ("comb_uniform", lambda: pins.test_comb_uniform_range()),
    ("slater_overlap", lambda: pins.test_slater_overlap_is_determinant(_FOCK)),
    ("remainder", lambda: pins.test_one_body_remainder_reproduces_hamiltonian(_FOCK, _SYS4)),
    ("fock_1det", lambda: pins.test_overlap_green_force_bias_energy_vs_fock(_FOCK, 1)),
    ("fock_5det", lambda: pins.test_overlap_green_force_bias_energy_vs_fock(_FOCK, 5)),
    ("trial_energy", lambda: pins.test_trial_energy_equals_variational_energy()),
    ("thouless", lambda: pins.test_propagation_is_thouless(_FOCK, _SYS4)),
    ("taylor_bound", lambda: pins.test_taylor_truncation_bound()),
    ("half_step", lambda: pins.test_half_step_propagator_matches_expm()),
    ("free_propagation", lambda: pins.test_zero_interaction_is_exact_free_propagation()),
    ("green_invariants", lambda: pins.test_green_invariants()),
    ("mgs", lambda: pins.test_mgs_matches_householder()),
    ("ortho_invariance", lambda: pins.test_orthonormalization_changes_nothing_observable()),
    ("phaseless_cut", lambda: pins.test_weight_update_phaseless_cut()),
    ("cut_phase_is_overlap_phase", lambda: pins.test_phaseless_cut_uses_overlap_phase_only()),
    ("weight_cap", lambda: pins.test_weight_cap_option()),
    ("comb", lambda: pins.test_blocked_prefix_sum_and_comb()),
    ("comb_intervals", lambda: pins.test_comb_brute_force_intervals()),
    ("zero_variance", lambda: pins.test_zero_variance_exact_trial(_FOCK)),
    ("mean_field", lambda: pins.test_mean_field_is_the_reference_expectation(_FOCK, _SYS4)),
    ("mf_hs_quadrature", lambda: pins.test_mean_field_hs_quadrature(_FOCK, _SYS4)),
    ("step_average", lambda: pins.test_step_importance_factor_is_the_projected_overlap(_FOCK, 0)),
    ("step_average_mf", lambda: pins.test_step_importance_factor_is_the_projected_overlap(_FOCK, 1)),
    ("local_weight", lambda: pins.test_local_energy_weight_is_the_mean_importance_factor(0)),
    ("local_weight_mf", lambda: pins.test_local_energy_weight_is_the_mean_importance_factor(1)),
    ("mf_phase", lambda: pins.test_mean_field_subtraction_shrinks_the_phase()),
    ("comb_renormalised", lambda: pins.test_renormalised_comb_changes_nothing_observable()),
]
SLOW_PINS = {
    "hs_quadrature": lambda: pins.test_hs_importance_factor_quadrature(_FOCK, _SYS4),
}


# ---------------------------------------------------------------- the slips

def exchange_sign(h1, L, D_up, D_dn, Theta_up, Theta_dn):
    e = 0.0
    X = 0.0
    ex = 0.0
    for D, Th in ((D_up, Theta_up), (D_dn, Theta_dn)):
        if D.shape[1] == 0:
            continue
        Dh = D.conj().T
        e = e + np.einsum("ak,wka->w", Dh @ h1, Th)
        Lt = np.einsum("ai,gik->gak", Dh, L)
        Pm = np.einsum("gak,wkb->wgab", Lt, Th)
        X = X + np.einsum("wgaa->wg", Pm)
        ex = ex + np.einsum("wgab,wgba->w", Pm, Pm)
    return e + 0.5 * np.sum(X * X, axis=1) + 0.5 * ex          # slip: + exchange


def importance_exponent(x, xbar):
    return np.sum(x * xbar + 0.5 * xbar * xbar, axis=1)         # slip: + xbar^2/2


def plus_force_bias_in_v(L, x, xbar, dtau):
    return 1j * np.sqrt(dtau) * np.einsum("wg,gij->wij", x + xbar, L)   # slip: x + xbar


def remainder_sign(h1, L, lbar=None):
    h = h1 + 0.5 * np.einsum("gik,gkj->ij", L, L)               # slip: + remainder
    return h if lbar is None else h + np.einsum("g,gij->ij", lbar, L)


def transposed_green(D, Phi):
    A = np.einsum("ka,wkb->wab", D.conj(), Phi)
    logdet = O.complex_logdet(A)
    Theta = Phi @ np.linalg.inv(A)
    GT = Theta @ D.conj().T
    return logdet, Theta, GT                                    # slip: G^T for G


def force_bias_sign(L, Gu, Gd, dtau, cap, lbar=None):
    X = np.einsum("gik,wik->wg", L, Gu + Gd)
    xbar = 1j * np.sqrt(dtau) * (X if lbar is None else X - lbar)   # slip: + i sqrt(dt)
    xbar = np.where(np.isfinite(xbar), xbar, 0.0)
    if cap > 0:
        a = np.abs(xbar)
        xbar = np.where(a > cap, xbar * (cap / np.where(a > 0, a, 1.0)), xbar)
    return X, xbar


def cut_on_importance_phase(weight, logO_old, logO_new, x, xbar, dtau, e_shift, cap=0,
                            w_ref=1.0, lmf=0.0, e0=0.0):
    lnR = logO_new - logO_old + lmf
    lnI = lnR + O.importance_log(x, xbar) + dtau * (e_shift - e0)
    with np.errstate(over="ignore", invalid="ignore"):
        w = weight * np.exp(lnI.real) * np.maximum(0.0, np.cos(lnI.imag))   # slip
    w = np.where(weight == 0.0, 0.0, w)
    w = np.where(np.isfinite(w), w, 0.0)
    if cap > 0 and w_ref > 0:
        w = np.minimum(w, cap * w_ref)
    return w


def no_ci_conjugate(trial, Phi_up, Phi_dn):
    terms = []
    for i in range(trial.n_det):
        lu = O.complex_logdet(np.einsum("ka,wkb->wab", trial.D_up[i].conj(), Phi_up))
        ld = O.complex_logdet(np.einsum("ka,wkb->wab", trial.D_dn[i].conj(), Phi_dn))
        terms.append(np.log(trial.ci[i]) + lu + ld)             # slip: c_i, not c_i^*
    terms = np.stack(terms, axis=1)
    m = np.max(terms.real, axis=1, keepdims=True)
    s = np.sum(np.exp(terms - m), axis=1)
    logO = m[:, 0] + np.log(s)
    return logO, np.exp(terms - logO[:, None])


def full_step_propagator(h1p, dtau):
    e, v = np.linalg.eigh(h1p)
    return (v * np.exp(-dtau * e)) @ v.T                        # slip: dt, not dt/2


def ln_det_r_sign(Phi_up, Phi_dn, logO):
    Pu, Pd, lo = Phi_up.copy(), Phi_dn.copy(), logO.copy()
    for w in range(Pu.shape[0]):
        for Pm in (Pu, Pd):
            if Pm.shape[2] == 0:
                continue
            Q, R = O.modified_gram_schmidt(Pm[w])
            Pm[w] = Q
            lo[w] += np.sum(np.log(np.diag(R).real))            # slip: += ln det R
    return Pu, Pd, lo


def no_factorial(V, Phi, order):
    t = Phi.copy()
    acc = Phi.copy()
    for n in range(1, order + 1):
        t = V @ t                                               # slip: no 1/n
        acc = acc + t
    return acc


def comb_offset_unscaled(weights, u):
    n = len(weights)
    C, S = O.blocked_prefix_sum(weights)
    if not S > 0.0:
        raise FloatingPointError("all walker weights are zero")
    step = S / n
    last = int(np.nonzero(np.asarray(weights) > 0)[0][-1])
    parent = np.zeros(n, dtype=np.int64)
    k = 0
    for j in range(n):
        t = j * step + u                                        # slip: u not scaled
        while k < n and C[k] <= t:
            k += 1
        parent[j] = min(k, last) if k < n else last
    return parent, step


def box_muller_radius(ra, rb):
    ua = P.uniform_open01(ra)
    ub = P.uniform_open01(rb)
    rad = np.sqrt(-np.log(ua))                                  # slip: missing factor 2
    return rad * np.cos(2.0 * np.pi * ub), rad * np.sin(2.0 * np.pi * ub)


def mgs_no_projection_update(Phi):
    M, N = Phi.shape
    Q = Phi.astype(np.complex128).copy()
    R = np.zeros((N, N), dtype=np.complex128)
    for j in range(N):
        for i in range(j):
            R[i, j] = np.vdot(Q[:, j], Q[:, i])                 # slip: conjugate on the wrong side
            Q[:, j] -= R[i, j] * Q[:, i]
        R[j, j] = np.linalg.norm(Q[:, j])
        Q[:, j] /= R[j, j]
    return Q, R


def mf_remainder_sign(h1, L, lbar=None):
    h = h1 - 0.5 * np.einsum("gik,gkj->ij", L, L)
    if lbar is not None:
        h = h - np.einsum("g,gij->ij", lbar, L)                 # slip: - lbar L
    return h


def mf_scalar_sign(x, xbar, lbar, dtau):
    return 1j * np.sqrt(dtau) * ((x - xbar) @ lbar)             # slip: + i


def mf_constant_sign(lbar):
    return 0.5 * float(np.sum(np.asarray(lbar) ** 2))           # slip: + 1/2


def mf_bias_sign(L, Gu, Gd, dtau, cap, lbar=None):
    X = np.einsum("gik,wik->wg", L, Gu + Gd)
    xbar = -1j * np.sqrt(dtau) * (X if lbar is None else X + lbar[None, :])   # slip: + lbar
    xbar = np.where(np.isfinite(xbar), xbar, 0.0)
    if cap > 0:
        a = np.abs(xbar)
        xbar = np.where(a > cap, xbar * (cap / np.where(a > 0, a, 1.0)), xbar)
    return X, xbar


def mean_field_up_only(L, D_up, D_dn):
    lbar = np.zeros(L.shape[0])
    Sinv = np.linalg.inv(D_up.conj().T @ D_up)
    for g in range(L.shape[0]):                                 # slip: one spin only
        lbar[g] += np.trace(Sinv @ (D_up.conj().T @ L[g] @ D_up)).real
    return lbar


def mf_constant_dropped(lnR, x, xbar, dtau, e_shift, e0=0.0):
    return lnR + O.importance_log(x, xbar) + dtau * e_shift    # slip: no E_0


def local_weight_sign(weight, eloc, lnR, dtau, e_shift, cap=0, w_ref=1.0):
    with np.errstate(over="ignore", invalid="ignore"):
        w = (weight * np.exp(dtau * (eloc.real - e_shift))       # slip: + dt
             * np.maximum(0.0, np.cos(lnR.imag)))
    return O._finish_weights(weight, w, cap, w_ref)


_STEP = O.OracleRun.step


def energy_after_move(self):
    """The step with the local-energy form reading E_L after the move."""
    if self.weight_mode != 1:
        return _STEP(self)
    s = self.s
    _, Gu, Gd, _ = O.mixed_green(self.trial, self.Phi_up, self.Phi_dn)
    X, xbar = O.force_bias(self.L, Gu, Gd, s.dtau, s.fb_cap, self.lbar)
    x = self.fields()
    V = O.one_body_operator(self.L, x, xbar, s.dtau)
    self.Phi_up = O.propagate(self.Bhalf, V, self.Phi_up, s.taylor_order)
    self.Phi_dn = O.propagate(self.Bhalf, V, self.Phi_dn, s.taylor_order)
    eloc = self.local_energies()                                 # slip: after the move
    logO_new, _ = O.trial_overlap(self.trial, self.Phi_up, self.Phi_dn)
    lmf = 0.0 if self.lbar is None else O.mean_field_log(x, xbar, self.lbar, s.dtau)
    lnR = logO_new - self.logO + lmf
    self.weight = O.update_weights_local(self.weight, eloc, lnR, s.dtau, self.e_shift)
    self.logO = logO_new
    self.last = dict(X=X, xbar=xbar, x=x, V=V, lnR=lnR, eloc=eloc)
    self.step_count += 1


def comb_scale_of_sum(self):
    u = P.comb_uniform(self.s.seed, self.s.run_id, self.step_count)
    parent, wnew = O.comb(self.weight, u)
    self.log_scale += float(np.log(wnew * len(self.weight)))   # slip: ln S, not ln(S/n)
    self.w_ref = 1.0
    self.Phi_up = self.Phi_up[parent].copy()
    self.Phi_dn = self.Phi_dn[parent].copy()
    self.logO = self.logO[parent].copy()
    self.weight = np.ones(self.walker_ids.size)
    return parent


SLIPS = {
    "exchange_sign": [(O, "local_energy_rotated", exchange_sign)],
    "importance_exponent": [(O, "importance_log", importance_exponent)],
    "x_plus_xbar": [(O, "one_body_operator", plus_force_bias_in_v)],
    "remainder_sign": [(O, "one_body_remainder", remainder_sign)],
    "transposed_green": [(O, "det_green", transposed_green)],
    "force_bias_sign": [(O, "force_bias", force_bias_sign)],
    "cut_phase": [(O, "update_weights", cut_on_importance_phase)],
    "ci_conjugate": [(O, "trial_overlap", no_ci_conjugate)],
    "half_step": [(O, "half_step_propagator", full_step_propagator)],
    "ln_det_r_sign": [(O, "orthonormalize", ln_det_r_sign)],
    "taylor_factorial": [(O, "taylor_apply", no_factorial)],
    "comb_offset": [(O, "comb", comb_offset_unscaled)],
    "philox_constants": [(P, "_M0", P._M1), (P, "_M1", P._M0)],
    "box_muller": [(P, "box_muller", box_muller_radius)],
    "mgs_conjugate": [(O, "modified_gram_schmidt", mgs_no_projection_update)],
    "mf_remainder_sign": [(O, "one_body_remainder", mf_remainder_sign)],
    "mf_scalar_sign": [(O, "mean_field_log", mf_scalar_sign)],
    "mf_constant_sign": [(O, "mean_field_constant", mf_constant_sign)],
    "mf_bias_sign": [(O, "force_bias", mf_bias_sign)],
    "mean_field_one_spin": [(O, "mean_field", mean_field_up_only)],
    "mf_constant_dropped": [(O, "log_importance", mf_constant_dropped)],
    "local_weight_sign": [(O, "update_weights_local", local_weight_sign)],
    "local_energy_after_move": [(O.OracleRun, "step", energy_after_move)],
    "comb_log_scale": [(O.OracleRun, "population_control", comb_scale_of_sum)],
}
# slips whose natural pin is one of the slow ones
NEEDS = {"importance_exponent": ["hs_quadrature"], "x_plus_xbar": ["hs_quadrature"]}


def run_pins(names_slow=()):
    failed = []
    for name, f in FAST_PINS + [(n, SLOW_PINS[n]) for n in names_slow]:
        try:
            f()
        except Exception as e:     # an assertion or a numerical breakdown
            failed.append((name, type(e).__name__))
    return failed


def test_pins_pass_on_the_unmodified_oracle():
    assert run_pins() == []


@pytest.mark.parametrize("slip", sorted(SLIPS))
def test_every_planted_slip_fails_a_pin(slip, monkeypatch):
    for mod, attr, value in SLIPS[slip]:
        monkeypatch.setattr(mod, attr, value)
    failed = run_pins(NEEDS.get(slip, ()))
    print(f"{slip}: caught by {failed}")
    assert failed, f"no pin catches the slip {slip}"
