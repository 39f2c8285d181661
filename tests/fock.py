"""Brute-force second quantisation in the full Fock space (test helper).

An independent route to the quantities the oracle computes with matrix
algebra: operators are built as explicit matrices over all 2**(2M)
occupation-number states, with Jordan-Wigner signs, and expectation values are
plain inner products. Only usable for M <= 5.

Mode ordering: spin-up orbitals 0..M-1, then spin-down orbitals M..2M-1.
A Slater determinant with orbital matrices Phi_up [M, N_up], Phi_dn [M, N_dn]
is the state (prod_a a+_a)(prod_b b+_b)|0>, with a+_a = sum_i Phi_up[i, a]
c+_{i up}, products written left to right in column order (leftmost applied
last).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.linalg import expm


class FockSpace:
    def __init__(self, M: int):
        self.M = M
        self.n_modes = 2 * M
        self.dim = 1 << self.n_modes
        self._cdag = [self._build_cdag(p) for p in range(self.n_modes)]
        self._c = [m.T.tocsr() for m in self._cdag]

    def _build_cdag(self, p):
        rows, cols, vals = [], [], []
        for n in range(self.dim):
            if (n >> p) & 1:
                continue
            sign = -1.0 if bin(n & ((1 << p) - 1)).count("1") % 2 else 1.0
            rows.append(n | (1 << p))
            cols.append(n)
            vals.append(sign)
        return sp.csr_matrix((vals, (rows, cols)), shape=(self.dim, self.dim))

    def mode(self, i, spin):
        return i + (self.M if spin else 0)

    def cdag(self, i, spin):
        return self._cdag[self.mode(i, spin)]

    def c(self, i, spin):
        return self._c[self.mode(i, spin)]

    # -- operators -----------------------------------------------------------
    def one_body(self, A, spins=(0, 1)):
        """sum_ij A_ij c+_{i s} c_{j s} over the given spins (A may be complex)."""
        M = self.M
        op = sp.csr_matrix((self.dim, self.dim), dtype=np.complex128)
        for s in spins:
            for i in range(M):
                for j in range(M):
                    if A[i, j] != 0:
                        op = op + A[i, j] * (self.cdag(i, s) @ self.c(j, s))
        return op

    def hamiltonian(self, T, V):
        """Eq. 1 written out term by term:
        sum_ij T_ij sum_s c+_is c_js
        + 1/2 sum_ijkl V_ijkl sum_{s,t} c+_is c+_jt c_lt c_ks."""
        M = self.M
        H = self.one_body(T.astype(np.complex128))
        for i in range(M):
            for j in range(M):
                for k in range(M):
                    for l in range(M):
                        v = V[i, j, k, l]
                        if v == 0:
                            continue
                        for s in (0, 1):
                            for t in (0, 1):
                                H = H + 0.5 * v * (self.cdag(i, s) @ self.cdag(j, t)
                                                   @ self.c(l, t) @ self.c(k, s))
        return H

    # -- states --------------------------------------------------------------
    def vacuum(self):
        v = np.zeros(self.dim, dtype=np.complex128)
        v[0] = 1.0
        return v

    def slater(self, Phi_up, Phi_dn):
        ops = []
        for a in range(Phi_up.shape[1]):
            ops.append(sum(Phi_up[i, a] * self.cdag(i, 0) for i in range(self.M)))
        for b in range(Phi_dn.shape[1]):
            ops.append(sum(Phi_dn[i, b] * self.cdag(i, 1) for i in range(self.M)))
        v = self.vacuum()
        for op in reversed(ops):
            v = op @ v
        return v

    def multi_det(self, C_up, C_dn, occ_up, occ_dn, ci):
        v = np.zeros(self.dim, dtype=np.complex128)
        for i in range(len(ci)):
            v = v + ci[i] * self.slater(C_up[:, occ_up[i]], C_dn[:, occ_dn[i]])
        return v

    def expm_op(self, op):
        return expm(op.toarray())

    def sector(self, n_up, n_dn):
        """Indices of basis states with the given particle numbers per spin."""
        M = self.M
        idx = []
        for n in range(self.dim):
            nu = bin(n & ((1 << M) - 1)).count("1")
            nd = bin(n >> M).count("1")
            if nu == n_up and nd == n_dn:
                idx.append(n)
        return np.asarray(idx)


def eri_from_chol(L):
    """V_ijkl = sum_g L_g,ik L_g,jl (the factorised integrals of Eq. 1)."""
    return np.einsum("gik,gjl->ijkl", L, L)


def mixed(fs: FockSpace, bra, op, ket):
    return np.vdot(bra, op @ ket) / np.vdot(bra, ket)
