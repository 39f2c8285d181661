"""Seeded synthetic Hamiltonians and trial wavefunctions.

The paper's own systems (hydrogen chains and transition-metal atoms, Sec. IV
and Sec. V) need molecular integrals that are not available here. These
generators draw inputs with the same shapes and structure instead:

* ``h1``: a symmetric one-body matrix, ``0.1 * sym(N(0,1))`` plus a diagonal
  ramp from -2 to +1 Ha.
* ``L``: ``n_chol`` real symmetric Cholesky-like vectors ``L_g`` (Sec. II,
  ``V_ijkl = sum_g L_g,ik L_g,jl``), so the two-electron integrals they imply
  are positive semi-definite by construction.
* A trial made of orthonormal orbital sets ``C_up``/``C_dn`` (M x M, one
  orbital per column) plus occupation lists; a multi-determinant trial lists
  one occupation row per determinant and a CI coefficient per determinant
  (Sec. III, the multi-determinant trial).

Nothing here performs any part of the ph-AFQMC step.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np


@dataclasses.dataclass
class System:
    """One ph-AFQMC problem plus its run parameters.

    Arrays are float64 / int32 / complex128, C-contiguous:
      h1     [M, M]           symmetric one-body matrix T_ij
      L      [n_chol, M, M]   each L[g] symmetric
      C_up   [M, M]           orbitals for spin up (column = orbital)
      C_dn   [M, M]           orbitals for spin down
      occ_up [n_det, n_up]    orbital indices of each determinant, in column order
      occ_dn [n_det, n_dn]
      ci     [n_det]          CI coefficients (determinant 0 is the reference)
    """

    name: str
    h1: np.ndarray
    L: np.ndarray
    C_up: np.ndarray
    C_dn: np.ndarray
    occ_up: np.ndarray
    occ_dn: np.ndarray
    ci: np.ndarray
    dtau: float
    n_walkers: int
    n_steps: int
    seed: int
    ortho_every: int
    measure_every: int
    pc_every: int
    taylor_order: int = 6
    fb_cap: float = 1.0
    run_id: int = 0
    weight_cap: int = 0
    weight_mode: int = 0      # 0: hybrid weights, 1: local-energy form
    mf_subtract: int = 0      # 1: subtract the reference determinant's mean field

    @property
    def M(self) -> int:
        return self.h1.shape[0]

    @property
    def n_up(self) -> int:
        return self.occ_up.shape[1]

    @property
    def n_dn(self) -> int:
        return self.occ_dn.shape[1]

    @property
    def n_chol(self) -> int:
        return self.L.shape[0]

    @property
    def n_det(self) -> int:
        return self.ci.shape[0]

    def trial_up(self, det: int = 0) -> np.ndarray:
        return self.C_up[:, self.occ_up[det]]

    def trial_dn(self, det: int = 0) -> np.ndarray:
        return self.C_dn[:, self.occ_dn[det]]

    def replace(self, **kw) -> "System":
        return dataclasses.replace(self, **kw)


def sym(rng: np.random.Generator, n: int, scale: float = 1.0) -> np.ndarray:
    """Draw the upper triangle (diagonal included) from N(0, scale^2), then mirror."""
    a = np.zeros((n, n))
    iu = np.triu_indices(n)
    a[iu] = rng.normal(0.0, scale, size=iu[0].size)
    return a + np.triu(a, 1).T


def make_h1(rng: np.random.Generator, M: int) -> np.ndarray:
    return 0.1 * sym(rng, M) + np.diag(np.linspace(-2.0, 1.0, M))


def _chol_dense(rng, M, n_chol, sigma):
    return np.stack([sym(rng, M, sigma) for _ in range(n_chol)])


def _chol_banded(rng, M, n_chol, sigma, decay):
    i = np.arange(M)
    env = np.exp(-np.abs(i[:, None] - i[None, :]) / decay)
    return np.stack([sym(rng, M, sigma) * env for _ in range(n_chol)])


def shell_blocks(M: int, shells=(1, 3, 5, 7)) -> list:
    """Block sizes that repeat the angular shells, truncated to fill M."""
    blocks, used = [], 0
    while used < M:
        for s in shells:
            if used >= M:
                break
            b = min(s, M - used)
            blocks.append(b)
            used += b
    return blocks


def _chol_shells(rng, M, n_chol, sigma):
    blocks = shell_blocks(M)
    L = np.zeros((n_chol, M, M))
    for g in range(n_chol):
        o = 0
        for b in blocks:
            L[g, o:o + b, o:o + b] = sym(rng, b, sigma)
            o += b
    return L


def _eig_orbitals(h1):
    _, v = np.linalg.eigh(h1)
    return np.ascontiguousarray(v)


def _random_orbitals(rng, M):
    q, _ = np.linalg.qr(rng.normal(size=(M, M)))
    return np.ascontiguousarray(q)


def _single_det(n_up, n_dn):
    return (np.arange(n_up, dtype=np.int32)[None, :],
            np.arange(n_dn, dtype=np.int32)[None, :],
            np.ones(1, dtype=np.complex128))


def excitation_trial(rng: np.random.Generator, M: int, n_up: int, n_dn: int,
                     n_det: int, amp: float = 0.1, c0: float = 1.0):
    """Reference determinant plus random singles and doubles.

    Excited orbitals replace the holes in place (column order kept), and each
    determinant's coefficient is ``N(0,1) * amp**rank``; the reference gets
    ``c0``. The vector is normalised. Same-spin and opposite-spin doubles are
    both drawn.
    """
    ref_up = list(range(n_up))
    ref_dn = list(range(n_dn))
    seen = set()
    occ_up, occ_dn, ci = [ref_up], [ref_dn], [c0]
    seen.add((tuple(ref_up), tuple(ref_dn)))

    def excite(ref, n, k):
        holes = sorted(rng.choice(n, size=k, replace=False).tolist())
        parts = sorted(rng.choice(np.arange(n, M), size=k, replace=False).tolist())
        occ = list(ref)
        for h, p in zip(holes, parts):
            occ[h] = p
        return occ

    guard = 0
    while len(ci) < n_det:
        guard += 1
        if guard > 100 * n_det:
            raise ValueError("not enough distinct excitations for n_det")
        kind = rng.integers(0, 5)
        if kind == 0 and n_up > 0 and M > n_up:      # single up
            u, d, rank = excite(ref_up, n_up, 1), ref_dn, 1
        elif kind == 1 and n_dn > 0 and M > n_dn:    # single down
            u, d, rank = ref_up, excite(ref_dn, n_dn, 1), 1
        elif kind == 2 and n_up > 1 and M - n_up > 1:  # same-spin double up
            u, d, rank = excite(ref_up, n_up, 2), ref_dn, 2
        elif kind == 3 and n_dn > 1 and M - n_dn > 1:  # same-spin double down
            u, d, rank = ref_up, excite(ref_dn, n_dn, 2), 2
        elif kind == 4 and n_up > 0 and n_dn > 0 and M > max(n_up, n_dn):
            u, d, rank = excite(ref_up, n_up, 1), excite(ref_dn, n_dn, 1), 2
        else:
            continue
        key = (tuple(u), tuple(d))
        if key in seen:
            continue
        seen.add(key)
        occ_up.append(u)
        occ_dn.append(d)
        ci.append(rng.normal() * amp ** rank)
    ci = np.asarray(ci, dtype=np.complex128)
    ci /= np.linalg.norm(ci)
    return (np.asarray(occ_up, dtype=np.int32).reshape(n_det, n_up),
            np.asarray(occ_dn, dtype=np.int32).reshape(n_det, n_dn), ci)


def make_system(name, *, M, n_up, n_dn, n_chol, ham_seed, l_kind="dense",
                l_sigma=0.05, l_decay=4.0, trial="eig", n_det=1,
                dtau=0.01, n_walkers=64, n_steps=200, seed=0, ortho_every=5,
                measure_every=10, pc_every=10, taylor_order=6, fb_cap=1.0,
                run_id=0) -> System:
    rng = np.random.default_rng(ham_seed)
    h1 = make_h1(rng, M)
    if l_kind == "dense":
        L = _chol_dense(rng, M, n_chol, l_sigma)
    elif l_kind == "banded":
        L = _chol_banded(rng, M, n_chol, l_sigma, l_decay)
    elif l_kind == "shells":
        L = _chol_shells(rng, M, n_chol, l_sigma)
    elif l_kind == "zero":
        L = np.zeros((n_chol, M, M))
    else:
        raise ValueError(l_kind)
    if trial == "eig":
        C = _eig_orbitals(h1)
    elif trial == "random":
        C = _random_orbitals(rng, M)
    else:
        raise ValueError(trial)
    if n_det == 1:
        occ_up, occ_dn, ci = _single_det(n_up, n_dn)
    else:
        occ_up, occ_dn, ci = excitation_trial(rng, M, n_up, n_dn, n_det)
    return System(name=name, h1=np.ascontiguousarray(h1),
                  L=np.ascontiguousarray(L), C_up=C.copy(), C_dn=C.copy(),
                  occ_up=occ_up, occ_dn=occ_dn, ci=ci, dtau=dtau,
                  n_walkers=n_walkers, n_steps=n_steps, seed=seed,
                  ortho_every=ortho_every, measure_every=measure_every,
                  pc_every=pc_every, taylor_order=taylor_order, fb_cap=fb_cap,
                  run_id=run_id)


def config_c1(**kw) -> System:
    """Plain single determinant, M=10, N=5+5, 40 fields, 64 walkers."""
    args = dict(M=10, n_up=5, n_dn=5, n_chol=40, ham_seed=0, l_kind="dense",
                l_sigma=0.05, trial="eig", dtau=0.01, n_walkers=64,
                n_steps=200, seed=0, ortho_every=5, measure_every=10,
                pc_every=10)
    args.update(kw)
    return make_system("c1_plain_m10", **args)


def config_c2(**kw) -> System:
    """Hydrogen-chain shape: M=60, N=30+30, 300 banded fields, 1024 walkers."""
    args = dict(M=60, n_up=30, n_dn=30, n_chol=300, ham_seed=2,
                l_kind="banded", l_sigma=0.05, l_decay=4.0, trial="random",
                dtau=0.005, n_walkers=1024, n_steps=500, seed=2,
                ortho_every=2, measure_every=20, pc_every=20)
    args.update(kw)
    return make_system("c2_hchain_m60", **args)


def config_c3(**kw) -> System:
    """Transition-metal-atom shape: M=150, N=13+12, 900 shell-blocked fields."""
    args = dict(M=150, n_up=13, n_dn=12, n_chol=900, ham_seed=3,
                l_kind="shells", l_sigma=0.02, trial="eig", dtau=0.005,
                n_walkers=2048, n_steps=1000, seed=3, ortho_every=2,
                measure_every=20, pc_every=20)
    args.update(kw)
    return make_system("c3_tmatom_m150", **args)


def config_c4(**kw) -> System:
    """Multi-determinant trial: M=80, N=10+10, 400 fields, 200 determinants."""
    M = kw.pop("M", 80)
    args = dict(M=M, n_up=10, n_dn=10, n_chol=400, ham_seed=4,
                l_kind="dense", l_sigma=0.05 * math.sqrt(10.0 / M),
                trial="eig", n_det=200, dtau=0.005, n_walkers=1024,
                n_steps=300, seed=4, ortho_every=2, measure_every=20,
                pc_every=20)
    args.update(kw)
    return make_system("c4_multidet_m80", **args)


def serving_run(rng: np.random.Generator, run_id: int,
                m_range=(20, 200), w_range=(128, 2048)) -> System:
    """One request of the serving mix: sizes drawn as the serving workload states.
    Energy once per 50-step block; the comb every 10 steps. The entries of
    the dense Cholesky vectors have scale 0.5 / M, so that the exchange
    potential sum_g L_g P L_g (n_chol ~ 5M vectors, M/4 electrons per spin)
    stays near 0.3 Ha on the diagonal whatever M: with a scale falling only
    as M^-1/2 it grows linearly with M, the one-body eigenvector trial
    drifts out of reach (ln |<Psi_T|phi>| near -40 after 40 steps at M = 98)
    and the phaseless cut empties the population within 50 steps."""
    M = int(rng.integers(m_range[0], m_range[1] + 1))
    n = int(rng.integers(math.ceil(M / 5), M // 3 + 1))
    n_chol = int(rng.integers(4 * M, 6 * M + 1))
    W = int(rng.integers(w_range[0], w_range[1] + 1))
    ham_seed = int(rng.integers(0, 2**31 - 1))
    return make_system(f"serve_{run_id}", M=M, n_up=n, n_dn=n, n_chol=n_chol,
                       ham_seed=ham_seed, l_kind="dense",
                       l_sigma=0.5 / M, trial="eig",
                       dtau=0.005, n_walkers=W, n_steps=500, seed=ham_seed,
                       ortho_every=2, measure_every=50, pc_every=10,
                       run_id=run_id)


def small_system(M=6, n_up=2, n_dn=2, n_chol=5, *, seed=11, l_sigma=0.1,
                 n_det=1, trial="eig", dtau=0.01, n_walkers=8, l_kind="dense",
                 **kw) -> System:
    """Tiny problems for pins and ragged-size parity cases."""
    return make_system(f"small_m{M}", M=M, n_up=n_up, n_dn=n_dn,
                       n_chol=n_chol, ham_seed=seed, l_kind=l_kind,
                       l_sigma=l_sigma, trial=trial, n_det=n_det, dtau=dtau,
                       n_walkers=n_walkers, seed=seed, **kw)


CONFIGS = {"c1": config_c1, "c2": config_c2, "c3": config_c3, "c4": config_c4}
