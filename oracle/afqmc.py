"""Plain FP64 CPU ph-AFQMC walker step: the oracle.

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports, calls or
links this module: tests, the smoke check and the benchmark's CPU-baseline leg
are its only users. It shares no code with the CUDA library; the two meet only
in the seeded inputs of ``synth`` and in the published definition of the
Philox generator, which each side implements on its own.

Everything is numpy float64 / complex128, one walker per batch entry, and
every function follows one step of the method as the paper states it:

* Hamiltonian (Sec. II, Eq. 1): ``H = sum T_ij c+_i c_j + 1/2 sum V_ijkl
  c+_i c+_j c_l c_k`` with ``V_ijkl = sum_g L_g,ik L_g,jl`` (Sec. III, below
  Eq. 5). Writing the two-body part as ``-1/2 sum_g v_g^2`` with
  ``v_g = i L_g`` leaves the one-body remainder
  ``H1' = T - 1/2 sum_g L_g L_g`` (normal ordering of Eq. 1).
* Trotter split (Sec. II): ``exp(-dt H) ~ B_half exp(V(x)) B_half`` with
  ``B_half = exp(-dt/2 H1')``; the symmetric split is this code's reading.
* Hubbard-Stratonovich (Eq. 2) turns ``exp(dt/2 v_g^2)`` into a Gaussian
  integral over ``x_g``, so a walker moves by the one-body operator
  ``V = i sqrt(dt) sum_g (x_g - xbar_g) L_g`` (Eq. 3 and the Thouless
  theorem, Sec. II), applied by a truncated Taylor series.
* Force bias (Sec. II): ``xbar_g = -sqrt(dt) <v_g> = -i sqrt(dt) X_g`` with
  ``X_g = sum_sigma sum_ik L_g,ik G^sigma_ik`` the mixed estimate, optionally
  capped in modulus.
* Weight (Sec. II, hybrid form of Sec. IV.A): with
  ``R = <Psi_T|phi'> / <Psi_T|phi>`` the walker weight is multiplied by
  ``|R exp(sum_g x_g xbar_g - xbar_g^2/2) exp(dt E_T)|`` and by
  ``max(0, cos(Im ln R))``, the phaseless constraint. The local-energy form
  (Sec. II) multiplies it instead by ``exp(-dt (Re E_L - E_T))``, ``E_L`` the
  local energy of the walker before the move, and by the same cut.
* Mean-field subtraction (an option; Sec. II's propagator is unchanged by
  it): with ``lbar_g = <L_g>`` of the reference determinant,
  ``1/2 L_g^2 = 1/2 (L_g - lbar_g)^2 + lbar_g L_g - 1/2 lbar_g^2``, so the
  one-body remainder gains ``sum_g lbar_g L_g``, the force bias becomes
  ``-i sqrt(dt) (X_g - lbar_g)``, each walker's overlap ratio carries the
  scalar ``exp(-i sqrt(dt) sum_g (x_g - xbar_g) lbar_g)`` (inside the cut's
  phase), and the constant ``-1/2 sum_g lbar_g^2`` enters the weight's shift.
* Orthonormalisation every few steps (Sec. IV.A) by modified Gram-Schmidt;
  the log-overlap drops by ``ln det R``.
* Local energy ``<Psi_T|H|phi>/<Psi_T|phi>`` (Sec. II) from the mixed Green's
  function by Wick's theorem; an independent route through the precomputed
  four-index tensor of Eq. 5 checks the GPU's formula.
* Multi-determinant trials ``sum_i c_i |D_i>`` with orthonormal determinants
  (Sec. III): overlaps, Green's functions and energies are the plain
  weighted sums over determinants, each from a full inverse (no
  Sherman-Morrison-Woodbury shortcut here).
* Population control by simple combing (Sec. V, final comments) with a
  blocked FP64 prefix sum whose order is fixed below. After a comb every
  walker has the common weight S/n; the run divides it out (weights 1) and
  keeps ln(S/n) in a log scale, so that a population whose energy lies far
  below E_T cannot overflow. Every estimator is a ratio of weights, so
  nothing observable changes.

Green's function convention: ``G^sigma_ij = <c+_i c_j>`` (mixed), so for a
determinant trial D and walker Phi, ``G^T = Phi (D^H Phi)^-1 D^H``.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

from .philox import gaussian_fields, comb_uniform

# ---------------------------------------------------------------------------
# Setup (not part of the timed propagation, Sec. III "propagation time")
# ---------------------------------------------------------------------------


def one_body_remainder(h1, L, lbar=None):
    """H1' = T - 1/2 sum_g L_g L_g: the one-body part left after writing the
    two-body term of Eq. 1 as -1/2 sum_g v_g^2 (Sec. II). With the mean
    field lbar subtracted, H1' + sum_g lbar_g L_g."""
    h = h1 - 0.5 * np.einsum("gik,gkj->ij", L, L)
    if lbar is not None:
        h = h + np.einsum("g,gij->ij", lbar, L)
    return h


def mean_field(L, D_up, D_dn):
    """lbar_g = <D|L_g|D> / <D|D> for the determinant D (its spins' column
    blocks D_up, D_dn): sum_sigma tr((D^H D)^-1 D^H L_g D)."""
    lbar = np.zeros(L.shape[0])
    for D in (D_up, D_dn):
        if D.shape[1] == 0:
            continue
        Sinv = np.linalg.inv(D.conj().T @ D)
        for g in range(L.shape[0]):
            lbar[g] += np.trace(Sinv @ (D.conj().T @ L[g] @ D)).real
    return lbar


def mean_field_constant(lbar):
    """E_0 = -1/2 sum_g lbar_g^2, the constant of the rewritten two-body term."""
    return -0.5 * float(np.sum(np.asarray(lbar) ** 2))


def half_step_propagator(h1p, dtau):
    """B_half = exp(-dtau/2 H1') by eigendecomposition of the symmetric H1'."""
    e, v = np.linalg.eigh(h1p)
    return (v * np.exp(-0.5 * dtau * e)) @ v.T


@dataclasses.dataclass
class Trial:
    """Determinants D_i^sigma = C^sigma[:, occ_i^sigma] and coefficients c_i."""

    D_up: np.ndarray   # [n_det, M, n_up]
    D_dn: np.ndarray   # [n_det, M, n_dn]
    ci: np.ndarray     # [n_det] complex

    @classmethod
    def from_system(cls, s):
        D_up = np.stack([s.C_up[:, s.occ_up[i]] for i in range(s.n_det)])
        D_dn = np.stack([s.C_dn[:, s.occ_dn[i]] for i in range(s.n_det)])
        return cls(D_up.astype(np.complex128), D_dn.astype(np.complex128),
                   np.asarray(s.ci, dtype=np.complex128))

    @property
    def n_det(self):
        return self.ci.shape[0]


# ---------------------------------------------------------------------------
# Overlaps and Green's functions
# ---------------------------------------------------------------------------


def complex_logdet(A):
    """ln det A for a batch of complex matrices: ln|det| + i arg det."""
    sign, logabs = np.linalg.slogdet(A)
    return logabs + 1j * np.angle(sign)


def det_green(D, Phi):
    """For one trial determinant D [M,N] and walkers Phi [W,M,N]:
    returns (ln det(D^H Phi) [W], Theta = Phi (D^H Phi)^-1 [W,M,N],
    G [W,M,M] with G_ij = <c+_i c_j>)."""
    A = np.einsum("ka,wkb->wab", D.conj(), Phi)
    logdet = complex_logdet(A)
    Theta = Phi @ np.linalg.inv(A)
    GT = Theta @ D.conj().T
    return logdet, Theta, np.swapaxes(GT, 1, 2)


def trial_overlap(trial, Phi_up, Phi_dn):
    """ln <Psi_T|phi> = ln sum_i c_i^* det(D_i^up^H Phi^up) det(D_i^dn^H Phi^dn)
    and the normalised determinant weights w_i = c_i^* O_i / O_T."""
    terms = []
    for i in range(trial.n_det):
        lu = complex_logdet(np.einsum("ka,wkb->wab", trial.D_up[i].conj(), Phi_up))
        ld = complex_logdet(np.einsum("ka,wkb->wab", trial.D_dn[i].conj(), Phi_dn))
        terms.append(np.log(np.conj(trial.ci[i])) + lu + ld)
    terms = np.stack(terms, axis=1)              # [W, n_det]
    m = np.max(terms.real, axis=1, keepdims=True)
    s = np.sum(np.exp(terms - m), axis=1)
    logO = m[:, 0] + np.log(s)
    wdet = np.exp(terms - logO[:, None])
    return logO, wdet


def mixed_green(trial, Phi_up, Phi_dn):
    """Mixed Green's functions G^up, G^dn [W,M,M] and ln O_T [W].

    Single determinant: G from D^H Phi directly. Multi-determinant:
    G = sum_i w_i G_i with w_i = c_i^* O_i / O_T (Sec. III trial form)."""
    logO, wdet = trial_overlap(trial, Phi_up, Phi_dn)
    W, M = Phi_up.shape[0], Phi_up.shape[1]
    Gu = np.zeros((W, M, M), dtype=np.complex128)
    Gd = np.zeros((W, M, M), dtype=np.complex128)
    for i in range(trial.n_det):
        _, _, gu = det_green(trial.D_up[i], Phi_up)
        _, _, gd = det_green(trial.D_dn[i], Phi_dn)
        Gu += wdet[:, i, None, None] * gu
        Gd += wdet[:, i, None, None] * gd
    return logO, Gu, Gd, wdet


# ---------------------------------------------------------------------------
# One imaginary-time step pieces
# ---------------------------------------------------------------------------


def force_bias(L, Gu, Gd, dtau, cap, lbar=None):
    """X_g = sum_sigma sum_ik L_g,ik G^sigma_ik and xbar_g = -i sqrt(dt) X_g
    (-i sqrt(dt) (X_g - lbar_g) with the mean field subtracted), each xbar_g
    scaled down to modulus ``cap`` when larger (cap <= 0: none)."""
    X = np.einsum("gik,wik->wg", L, Gu + Gd)
    xbar = -1j * np.sqrt(dtau) * (X if lbar is None else X - lbar[None, :])
    xbar = np.where(np.isfinite(xbar), xbar, 0.0)   # a walker with no defined bias
    if cap > 0:
        a = np.abs(xbar)
        xbar = np.where(a > cap, xbar * (cap / np.where(a > 0, a, 1.0)), xbar)
    return X, xbar


def one_body_operator(L, x, xbar, dtau):
    """V = i sqrt(dt) sum_g (x_g - xbar_g) L_g for each walker [W,M,M]."""
    s = x - xbar
    return 1j * np.sqrt(dtau) * np.einsum("wg,gij->wij", s, L)


def taylor_apply(V, Phi, order):
    """sum_{n=0..order} V^n Phi / n!, by t_n = V t_{n-1} / n."""
    t = Phi.copy()
    acc = Phi.copy()
    for n in range(1, order + 1):
        t = (V @ t) / n
        acc = acc + t
    return acc


def propagate(Bhalf, V, Phi, order):
    """Phi <- B_half exp_T(V) B_half Phi (symmetric Trotter split)."""
    return Bhalf @ taylor_apply(V, Bhalf @ Phi, order)


def importance_log(x, xbar):
    """sum_g (x_g xbar_g - xbar_g^2 / 2): the log of the shift factor."""
    return np.sum(x * xbar - 0.5 * xbar * xbar, axis=1)


def mean_field_log(x, xbar, lbar, dtau):
    """-i sqrt(dt) sum_g (x_g - xbar_g) lbar_g: the log of the scalar factor
    that the subtracted mean field puts on each propagated walker."""
    return -1j * np.sqrt(dtau) * ((x - xbar) @ lbar)


def log_importance(lnR, x, xbar, dtau, e_shift, e0=0.0):
    """ln I = ln R + sum(x xbar - xbar^2/2) + dt (E_T - E_0): the complex
    importance factor of the hybrid form before the phaseless cut (E_0 the
    mean-field constant, 0 without the subtraction)."""
    return lnR + importance_log(x, xbar) + dtau * (e_shift - e0)


def _finish_weights(weight, w, cap, w_ref):
    w = np.where(weight == 0.0, 0.0, w)
    w = np.where(np.isfinite(w), w, 0.0)
    if cap > 0 and w_ref > 0:
        w = np.minimum(w, cap * w_ref)
    return w


def update_weights(weight, logO_old, logO_new, x, xbar, dtau, e_shift, cap=0,
                   w_ref=1.0, lmf=0.0, e0=0.0):
    """Hybrid weight with the phaseless cut (Sec. II):
    W <- W |I| max(0, cos(Im ln R)), ln I as in log_importance, ln R the
    overlap ratio's log plus the mean-field scalar lmf (0 without the
    subtraction). A walker at weight 0 stays there; non-finite results
    give 0. With cap > 0 (an option, not part of the paper's step) the
    result is capped at cap * w_ref, w_ref the common weight of the last
    comb."""
    lnR = logO_new - logO_old + lmf
    lnI = log_importance(lnR, x, xbar, dtau, e_shift, e0)
    with np.errstate(over="ignore", invalid="ignore"):
        w = weight * np.exp(lnI.real) * np.maximum(0.0, np.cos(lnR.imag))
    return _finish_weights(weight, w, cap, w_ref)


def update_weights_local(weight, eloc, lnR, dtau, e_shift, cap=0, w_ref=1.0):
    """Local-energy weight form with the phaseless cut (Sec. II):
    W <- W exp(-dt (Re E_L - E_T)) max(0, cos(Im ln R)), E_L the local
    energy before the move, ln R as for update_weights. Same handling of
    zero and non-finite weights and of the cap."""
    with np.errstate(over="ignore", invalid="ignore"):
        w = (weight * np.exp(-dtau * (eloc.real - e_shift))
             * np.maximum(0.0, np.cos(lnR.imag)))
    return _finish_weights(weight, w, cap, w_ref)


def modified_gram_schmidt(Phi):
    """Q, R of one complex M x N matrix by modified Gram-Schmidt (R's
    diagonal real and positive)."""
    M, N = Phi.shape
    Q = Phi.astype(np.complex128).copy()
    R = np.zeros((N, N), dtype=np.complex128)
    for j in range(N):
        for i in range(j):
            R[i, j] = np.vdot(Q[:, i], Q[:, j])
            Q[:, j] -= R[i, j] * Q[:, i]
        R[j, j] = np.linalg.norm(Q[:, j])
        Q[:, j] /= R[j, j]
    return Q, R


def orthonormalize(Phi_up, Phi_dn, logO):
    """Every walker: Phi^sigma <- Q^sigma, ln O_T -= sum_sigma ln det R^sigma."""
    Pu, Pd, lo = Phi_up.copy(), Phi_dn.copy(), logO.copy()
    for w in range(Pu.shape[0]):
        for P in (Pu, Pd):
            if P.shape[2] == 0:
                continue
            Q, R = modified_gram_schmidt(P[w])
            P[w] = Q
            lo[w] -= np.sum(np.log(np.diag(R).real))
    return Pu, Pd, lo


# ---------------------------------------------------------------------------
# Local energy (Sec. II definition; Sec. III Eq. 5 route)
# ---------------------------------------------------------------------------


def local_energy_green(h1, L, Gu, Gd):
    """E_L from the mixed Green's functions of one determinant pair by Wick's
    theorem on Eq. 1 with V_ijkl = sum_g L_g,ik L_g,jl:
    sum_sigma tr(T G^sigma^T) + 1/2 sum_g [(sum_sigma tr(L_g G^sigma^T))^2
    - sum_sigma tr(L_g G^sigma^T L_g G^sigma^T)]."""
    e1 = np.einsum("ij,wij->w", h1, Gu + Gd)
    X = np.einsum("gij,wij->wg", L, Gu + Gd)
    ex = 0.0
    for G in (Gu, Gd):
        LG = np.einsum("gik,wjk->wgij", L, G)        # (L_g G^T)_ij
        ex = ex + np.einsum("wgij,wgji->w", LG, LG)
    return e1 + 0.5 * np.sum(X * X, axis=1) - 0.5 * ex


def local_energy_rotated(h1, L, D_up, D_dn, Theta_up, Theta_dn):
    """Same quantity for one trial determinant, with G^T = Theta D^H inserted:
    tr(A G^T) = tr(D^H A Theta) and tr(L G^T L G^T) = tr((D^H L Theta)^2)."""
    e = 0.0
    X = 0.0
    ex = 0.0
    for D, Th in ((D_up, Theta_up), (D_dn, Theta_dn)):
        if D.shape[1] == 0:
            continue
        Dh = D.conj().T
        e = e + np.einsum("ak,wka->w", Dh @ h1, Th)
        Lt = np.einsum("ai,gik->gak", Dh, L)            # half-rotated L
        Pm = np.einsum("gak,wkb->wgab", Lt, Th)         # D^H L_g Theta
        X = X + np.einsum("wgaa->wg", Pm)
        ex = ex + np.einsum("wgab,wgba->w", Pm, Pm)
    return e + 0.5 * np.sum(X * X, axis=1) - 0.5 * ex


def y_tensor(L, D):
    """Eq. 5 for one spin: Y[i,j,a,b] = sum_kl sum_g L_g,ik L_g,jl
    (D^*_ka D^*_lb - D^*_la D^*_kb), i, j basis indices, a, b occupied."""
    Dc = D.conj()
    P = np.einsum("gik,ka->gia", L, Dc)   # sum_k L_ik D*_ka
    coul = np.einsum("gia,gjb->ijab", P, P)
    exch = np.einsum("gib,gja->ijab", P, P)
    return coul - exch


def local_energy_y(h1, L, D_up, D_dn, Theta_up, Theta_dn):
    """E_L through the precomputed tensor of Eq. 5: same-spin two-body part
    1/2 sum Theta_ia Theta_jb Y_ijab per spin, plus the opposite-spin Coulomb
    term X^up . X^dn, plus the one-body trace."""
    W = Theta_up.shape[0]
    e = np.zeros(W, dtype=np.complex128)
    Xs = []
    for D, Th in ((D_up, Theta_up), (D_dn, Theta_dn)):
        if D.shape[1] == 0:
            Xs.append(np.zeros((W, L.shape[0]), dtype=np.complex128))
            continue
        e = e + np.einsum("ak,wka->w", D.conj().T @ h1, Th)
        Y = y_tensor(L, D)
        e = e + 0.5 * np.einsum("wia,wjb,ijab->w", Th, Th, Y)
        P = np.einsum("gik,ka->gia", L, D.conj())
        Xs.append(np.einsum("gia,wia->wg", P, Th))
    return e + np.sum(Xs[0] * Xs[1], axis=1)


def local_energy(h1, L, trial, Phi_up, Phi_dn):
    """E_L = <Psi_T|H|phi>/<Psi_T|phi> per walker: sum_i w_i E_i over the
    trial's determinants (a single term for one determinant)."""
    logO, wdet = trial_overlap(trial, Phi_up, Phi_dn)
    E = np.zeros(Phi_up.shape[0], dtype=np.complex128)
    for i in range(trial.n_det):
        _, Tu, _ = det_green(trial.D_up[i], Phi_up)
        _, Td, _ = det_green(trial.D_dn[i], Phi_dn)
        E += wdet[:, i] * local_energy_rotated(h1, L, trial.D_up[i],
                                               trial.D_dn[i], Tu, Td)
    return E


def reference_energy(h1, L, trial):
    """E_T: the energy of the reference determinant alone, <D_0|H|D_0>
    (for a one-determinant trial, the trial's variational energy). At
    phi = D_0 the excited determinants have zero overlap, so the
    multi-determinant local energy there is a 0/0 limit; the reference
    energy is the well-defined shift used instead."""
    Du, Dd = trial.D_up[0], trial.D_dn[0]
    return float(local_energy_rotated(h1, L, Du, Dd, Du[None], Dd[None])[0].real)


# ---------------------------------------------------------------------------
# Population control (simple comb)
# ---------------------------------------------------------------------------

SCAN_BLOCK = 32


def blocked_prefix_sum(w):
    """Inclusive FP64 prefix sums in a fixed order: sequential inside blocks
    of 32 walkers, then a sequential sum of the block totals, each walker's
    sum being (total of earlier blocks) + (its running sum in its block)."""
    w = np.asarray(w, dtype=np.float64)
    n = w.size
    inside = np.zeros(n)
    totals = []
    for b0 in range(0, n, SCAN_BLOCK):
        run = 0.0
        for k in range(b0, min(n, b0 + SCAN_BLOCK)):
            run = run + w[k]
            inside[k] = run
        totals.append(run)
    base = 0.0
    C = np.zeros(n)
    for b, b0 in enumerate(range(0, n, SCAN_BLOCK)):
        for k in range(b0, min(n, b0 + SCAN_BLOCK)):
            C[k] = base + inside[k]
        base = base + totals[b]
    return C, base


def comb(weights, u):
    """Simple comb: teeth t_j = (j + u) * (S / n), j = 0..n-1; tooth j lands in
    [C_{k-1}, C_k) and copies walker k; every new weight is S / n. Returns the
    parent index of each new walker and the new weight. A tooth at or past
    C_{n-1} (rounding) goes to the last walker of nonzero weight."""
    n = len(weights)
    C, S = blocked_prefix_sum(weights)
    if not S > 0.0:
        raise FloatingPointError("all walker weights are zero")
    step = S / n
    last = int(np.nonzero(np.asarray(weights) > 0)[0][-1])
    parent = np.zeros(n, dtype=np.int64)
    k = 0
    for j in range(n):
        t = (j + u) * step
        while k < n and C[k] <= t:
            k += 1
        parent[j] = min(k, last) if k < n else last
    return parent, step


# ---------------------------------------------------------------------------
# A run: walkers, steps, cadence
# ---------------------------------------------------------------------------


class OracleRun:
    """W walkers of one system, propagated step by step in FP64.

    Step s (0-based counter, as drawn by Philox) does: mixed G and force bias
    at the current walkers (and, in the local-energy weight form, their local
    energies), field draw, propagation, new overlap, weight.
    After it, with n = s + 1 steps done: orthonormalise if n % ortho_every
    == 0, measure if n % measure_every == 0, comb if n % pc_every == 0.
    """

    def __init__(self, system, e_shift: Optional[float] = None,
                 walker_ids=None):
        s = system
        self.s = s
        # global walker indices (they key the Philox counters); a subset
        # reproduces those walkers exactly until the first comb
        self.walker_ids = (np.arange(s.n_walkers) if walker_ids is None
                           else np.asarray(walker_ids, dtype=np.int64))
        self.trial = Trial.from_system(s)
        self.h1 = np.asarray(s.h1, dtype=np.float64)
        self.L = np.asarray(s.L, dtype=np.float64)
        self.weight_mode = getattr(s, "weight_mode", 0)
        if self.weight_mode == 1 and s.n_det > 1:
            # the walkers start at the reference determinant, where the
            # other determinants' overlaps vanish and their energies are 0/0
            raise ValueError("the local-energy weight form needs a one-determinant trial")
        # mean field of the reference determinant (zero: no subtraction)
        self.lbar = (mean_field(self.L, self.trial.D_up[0], self.trial.D_dn[0])
                     if getattr(s, "mf_subtract", 0) else None)
        self.e0 = 0.0 if self.lbar is None else mean_field_constant(self.lbar)
        self.h1p = one_body_remainder(self.h1, self.L, self.lbar)
        self.Bhalf = half_step_propagator(self.h1p, s.dtau)
        W = self.walker_ids.size
        self.Phi_up = np.repeat(self.trial.D_up[0][None], W, axis=0).copy()
        self.Phi_dn = np.repeat(self.trial.D_dn[0][None], W, axis=0).copy()
        self.weight = np.ones(W)
        self.logO, _ = trial_overlap(self.trial, self.Phi_up, self.Phi_dn)
        if e_shift is None:
            e_shift = reference_energy(self.h1, self.L, self.trial)
        self.e_shift = e_shift
        self.step_count = 0
        self.w_ref = 1.0            # common weight of the last comb (weight cap)
        self.log_scale = 0.0        # sum of ln(S/n) divided out at the combs
        self.energies = []          # (step, mixed energy, E_L per walker)
        self.last = {}

    # -- single pieces, exposed for step-by-step parity ---------------------
    def fields(self, step=None):
        st = self.step_count if step is None else step
        return gaussian_fields(self.s.seed, self.s.run_id, st,
                               self.walker_ids, self.s.n_chol)

    def step(self):
        s = self.s
        logO_old, Gu, Gd, _ = mixed_green(self.trial, self.Phi_up, self.Phi_dn)
        X, xbar = force_bias(self.L, Gu, Gd, s.dtau, s.fb_cap, self.lbar)
        eloc = self.local_energies() if self.weight_mode == 1 else None
        x = self.fields()
        V = one_body_operator(self.L, x, xbar, s.dtau)
        self.Phi_up = propagate(self.Bhalf, V, self.Phi_up, s.taylor_order)
        self.Phi_dn = propagate(self.Bhalf, V, self.Phi_dn, s.taylor_order)
        logO_new, _ = trial_overlap(self.trial, self.Phi_up, self.Phi_dn)
        lmf = 0.0 if self.lbar is None else mean_field_log(x, xbar, self.lbar, s.dtau)
        cap = getattr(s, "weight_cap", 0)
        lnR = logO_new - self.logO + lmf
        if self.weight_mode == 1:
            self.weight = update_weights_local(self.weight, eloc, lnR, s.dtau,
                                               self.e_shift, cap, self.w_ref)
        else:
            self.weight = update_weights(self.weight, self.logO, logO_new, x,
                                         xbar, s.dtau, self.e_shift, cap,
                                         self.w_ref, lmf=lmf, e0=self.e0)
        self.logO = logO_new
        self.last = dict(X=X, xbar=xbar, x=x, V=V, lnR=lnR, eloc=eloc)
        self.step_count += 1
        n = self.step_count
        if s.ortho_every > 0 and n % s.ortho_every == 0:
            self.orthonormalize()
        if s.measure_every > 0 and n % s.measure_every == 0:
            self.measure()
        if s.pc_every > 0 and n % s.pc_every == 0:
            self.population_control()

    def orthonormalize(self):
        self.Phi_up, self.Phi_dn, self.logO = orthonormalize(
            self.Phi_up, self.Phi_dn, self.logO)

    def local_energies(self):
        return local_energy(self.h1, self.L, self.trial, self.Phi_up, self.Phi_dn)

    def measure(self):
        E = self.local_energies()
        w = self.weight
        sw = np.sum(w)
        live = w > 0
        emix = float(np.sum(w[live] * E.real[live]) / sw) if sw > 0 else float("nan")
        self.energies.append((self.step_count, emix, E))
        return emix, E

    def population_control(self):
        u = comb_uniform(self.s.seed, self.s.run_id, self.step_count)
        parent, wnew = comb(self.weight, u)
        self.log_scale += float(np.log(wnew))
        self.w_ref = 1.0
        self.Phi_up = self.Phi_up[parent].copy()
        self.Phi_dn = self.Phi_dn[parent].copy()
        self.logO = self.logO[parent].copy()
        self.weight = np.ones(self.walker_ids.size)
        self.last["parent"] = parent
        return parent

    def run(self, n_steps):
        for _ in range(n_steps):
            self.step()
        return self
