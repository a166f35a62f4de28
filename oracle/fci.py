"""Brute-force Fock-space operators for tiny systems (pins for the oracle).

Test infrastructure only (see oracle/__init__.py).  Nothing here uses the
single-determinant formulas of oracle.afqmc: operators are built by applying
creation / annihilation operators to occupation bit strings, so quantities
computed here are exact many-body references for the Hamiltonian of Eqs. 2-3
and the operators of Eqs. 4-8.

Spin orbitals: alpha orbital p is bit p, beta orbital p is bit N + p.  A basis
state is a+_{i1} a+_{i2} ... |0> with i1 < i2 < ... ; a+_p and a_p carry the
sign (-1)^(number of occupied spin orbitals below p).
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.linalg


class Sector:
    """The (nalpha, nbeta) particle-number sector of N spatial orbitals."""

    def __init__(self, norb, nalpha, nbeta):
        self.norb, self.nalpha, self.nbeta = norb, nalpha, nbeta
        alpha = list(itertools.combinations(range(norb), nalpha))
        beta = list(itertools.combinations(range(norb), nbeta))
        self.occ = [(a, b) for a in alpha for b in beta]
        self.states = []
        for a, b in self.occ:
            s = 0
            for p in a:
                s |= 1 << p
            for p in b:
                s |= 1 << (norb + p)
            self.states.append(s)
        self.index = {s: i for i, s in enumerate(self.states)}
        self.dim = len(self.states)

    @staticmethod
    def _sign(state, bit):
        return -1.0 if bin(state & ((1 << bit) - 1)).count("1") % 2 else 1.0

    def apply_string(self, ops, state):
        """Apply ops = [(bit, dagger), ...] right to left to a basis state; returns (sign, state) or None."""
        sign = 1.0
        s = state
        for bit, dag in reversed(ops):
            occupied = (s >> bit) & 1
            if dag and occupied:
                return None
            if not dag and not occupied:
                return None
            sign *= self._sign(s, bit)
            s ^= 1 << bit
        return sign, s

    def operator(self, terms):
        """Matrix of sum_k coef_k * (operator string k) in this sector."""
        mat = np.zeros((self.dim, self.dim), dtype=np.complex128)
        for coef, ops in terms:
            if coef == 0:
                continue
            for j, s in enumerate(self.states):
                r = self.apply_string(ops, s)
                if r is None:
                    continue
                sign, t = r
                i = self.index.get(t)
                if i is not None:
                    mat[i, j] += coef * sign
        return mat

    def one_body(self, a):
        """sum_{pq, spin} a_pq a+_{p s} a_{q s}."""
        n = self.norb
        terms = []
        for p in range(n):
            for q in range(n):
                for off in (0, n):
                    terms.append((a[p, q], [(p + off, True), (q + off, False)]))
        return self.operator(terms)

    def one_body_spin(self, p, q, spin):
        off = 0 if spin == 0 else self.norb
        return self.operator([(1.0, [(p + off, True), (q + off, False)])])

    def hamiltonian(self, h1e, eri, ecore):
        """Eq. 2: sum h_pq a+_p a_q + 1/2 sum g_psqr a+_p a+_q a_r a_s (+ E0), spins summed."""
        n = self.norb
        terms = []
        for p in range(n):
            for q in range(n):
                for off in (0, n):
                    terms.append((h1e[p, q], [(p + off, True), (q + off, False)]))
        for p, s, q, r in itertools.product(range(n), repeat=4):
            g = eri[p, s, q, r]
            if g == 0.0:
                continue
            for o1 in (0, n):          # spin of the (p, s) electron
                for o2 in (0, n):      # spin of the (q, r) electron
                    terms.append((0.5 * g, [(p + o1, True), (q + o2, True), (r + o2, False), (s + o1, False)]))
        return self.operator(terms) + ecore * np.eye(self.dim)

    def determinant_vector(self, psi):
        """Amplitudes of the Slater determinant with orbitals psi [N, na+nb] (alpha columns first)."""
        na = self.nalpha
        pa, pb = psi[:, :na], psi[:, na:na + self.nbeta]
        v = np.zeros(self.dim, dtype=np.complex128)
        for i, (a, b) in enumerate(self.occ):
            da = np.linalg.det(pa[list(a), :]) if na else 1.0
            db = np.linalg.det(pb[list(b), :]) if self.nbeta else 1.0
            v[i] = da * db
        return v


def eri_from_cholesky(chol):
    """g_psqr = sum_gamma L^g_ps L^g_qr (Eq. 3)."""
    return np.einsum("gps,gqr->psqr", chol, chol)


def eri_from_complex_cholesky(chol):
    """g_psqr = (ps|qr) = sum_gamma L^g_ps conj(L^g_rq) for complex Cholesky vectors (the pair matrix
    (ps),(rq) is Hermitian positive semidefinite); equals eri_from_cholesky for real symmetric L."""
    return np.einsum("gps,grq->psqr", chol, np.conj(chol))


def expm(mat):
    return scipy.linalg.expm(mat)
