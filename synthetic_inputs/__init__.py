"""Seeded synthetic inputs for the phaseless-AFQMC hot path.

This module is shared by the oracle, the tests and the benchmark.  It holds
none of the method's arithmetic: it only draws the Hamiltonian (one-body
integrals h1e, Cholesky vectors L[naux, N, N], constant E0) and builds the
single-determinant trial that the method takes as input.

The paper's workloads are molecules (the S22 benzene dimer and [Cu2O2]2+,
Section "Distributed Hamiltonian" and "GPU accelerated MSD-AFQMC"); their
integrals are not available, so these generators produce inputs with the same
shapes (N orbitals, electron counts, naux, walker count) and the structure of
real Cholesky factorisations: symmetric L^gamma whose norms decay
geometrically, so that sum_gamma L^gamma (x) L^gamma is a positive
semidefinite ERI tensor (Eq. 3).

The trial determinant comes from a plain restricted / unrestricted Hartree-Fock
fixed-point iteration (a fixed number of Roothaan steps from the core guess, no
damping or DIIS).  It is an input-preparation step, not part of the AFQMC
method, and any determinant would do for parity.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BASE_SEED = 240616238


@dataclasses.dataclass
class Problem:
    """One synthetic Hamiltonian plus trial (all float64, C-contiguous)."""

    h1e: np.ndarray      # [N, N] real symmetric
    chol: np.ndarray     # [naux, N, N] real symmetric per gamma
    ecore: float
    nalpha: int
    nbeta: int
    psiT: np.ndarray     # [N, nalpha + nbeta], alpha columns first
    name: str = ""

    @property
    def norb(self) -> int:
        return self.h1e.shape[0]

    @property
    def naux(self) -> int:
        return self.chol.shape[0]


def _sym_gaussian(rng, n):
    a = rng.standard_normal((n, n))
    return 0.5 * (a + a.T)


def cholesky_vectors(rng, norb: int, naux: int, tau: float, orthogonalise: bool = True) -> np.ndarray:
    """L^gamma = exp(-gamma/tau) * S_gamma / ||S_gamma||_F with S_gamma random symmetric.

    With orthogonalise=True the vec(S_gamma) are Gram-Schmidt orthonormalised
    first (needs naux <= N(N+1)/2), so the singular values of the
    [naux, N*N] Cholesky matrix are exactly exp(-gamma/tau).
    """
    s = np.empty((naux, norb, norb))
    for g in range(naux):
        s[g] = _sym_gaussian(rng, norb)
    flat = s.reshape(naux, norb * norb)
    if orthogonalise:
        if naux > norb * (norb + 1) // 2:
            raise ValueError("naux exceeds the dimension of symmetric matrices")
        q, r = np.linalg.qr(flat.T)           # columns orthonormal
        q = q * np.sign(np.diag(r))[None, :]
        flat = q.T.copy()
    else:
        flat = flat / np.linalg.norm(flat, axis=1, keepdims=True)
    scale = np.exp(-np.arange(naux) / tau)
    chol = (flat * scale[:, None]).reshape(naux, norb, norb)
    # exact symmetry (Gram-Schmidt keeps it up to rounding)
    chol = 0.5 * (chol + chol.transpose(0, 2, 1))
    return np.ascontiguousarray(chol)


def one_body(rng, norb: int, ramp: float = 4.0, noise: float = 0.1) -> np.ndarray:
    """Diagonal ramp 0..ramp Ha plus symmetric N(0, noise^2) off-diagonal."""
    h = np.diag(np.linspace(0.0, ramp, norb))
    off = rng.standard_normal((norb, norb)) * noise
    off = np.triu(off, 1)
    return np.ascontiguousarray(h + off + off.T)


def _coulomb(chol, dm):
    return np.einsum("gpq,g->pq", chol, np.einsum("gpq,qp->g", chol, dm))


def _exchange(chol, dm):
    return np.einsum("gpr,rs,gsq->pq", chol, dm, chol, optimize=True)


def hartree_fock_trial(h1e, chol, nalpha, nbeta, iterations=20, unrestricted=False):
    """Trial orbitals [N, nalpha+nbeta] from plain Roothaan iterations.

    RHF: F = h + 2J[P] - K[P] with P the per-spin density of the nalpha lowest
    orbitals.  UHF: F^s = h + J[Pa+Pb] - K[P^s]; the beta guess mixes its HOMO
    and LUMO by pi/4 to break spin symmetry.
    """
    norb = h1e.shape[0]
    _, c = np.linalg.eigh(h1e)
    if not unrestricted:
        if nalpha != nbeta:
            raise ValueError("restricted trial needs nalpha == nbeta")
        for _ in range(iterations):
            occ = c[:, :nalpha]
            dm = occ @ occ.T
            fock = h1e + 2.0 * _coulomb(chol, dm) - _exchange(chol, dm)
            _, c = np.linalg.eigh(fock)
        occ = c[:, :nalpha]
        return np.ascontiguousarray(np.hstack([occ, occ]))
    ca = c.copy()
    cb = c.copy()
    if nbeta < norb and nbeta > 0:
        h, l = cb[:, nbeta - 1].copy(), cb[:, nbeta].copy()
        cb[:, nbeta - 1] = (h + l) / np.sqrt(2.0)
        cb[:, nbeta] = (l - h) / np.sqrt(2.0)
    for _ in range(iterations):
        da = ca[:, :nalpha] @ ca[:, :nalpha].T
        db = cb[:, :nbeta] @ cb[:, :nbeta].T
        j = _coulomb(chol, da + db)
        _, ca = np.linalg.eigh(h1e + j - _exchange(chol, da))
        _, cb = np.linalg.eigh(h1e + j - _exchange(chol, db))
    return np.ascontiguousarray(np.hstack([ca[:, :nalpha], cb[:, :nbeta]]))


def make_problem(norb, nalpha, nbeta, naux, tau, seed, unrestricted=False,
                 ecore=1.5, orthogonalise=None, scf_iterations=20, name="") -> Problem:
    rng = np.random.default_rng(seed)
    h1e = one_body(rng, norb)
    if orthogonalise is None:
        orthogonalise = norb <= 300 and naux <= norb * (norb + 1) // 2
    chol = cholesky_vectors(rng, norb, naux, tau, orthogonalise)
    psiT = hartree_fock_trial(h1e, chol, nalpha, nbeta, scf_iterations, unrestricted)
    return Problem(h1e, chol, float(ecore), nalpha, nbeta, psiT, name)


# Workload shapes (walker counts and step counts live with the runner).
def config_small(seed_offset=1):
    """N=8, 2a+2b, naux=24, tau=4, RHF (20 SCF iterations)."""
    return make_problem(8, 2, 2, 24, 4.0, BASE_SEED + seed_offset, name="N8_n2_X24")


def config_medium(seed_offset=2):
    """N=108, 21a+21b, naux=432, tau=40, RHF: the 108-orbital / 640-walker shape."""
    return make_problem(108, 21, 21, 432, 40.0, BASE_SEED + seed_offset, name="N108_n21_X432")


def config_cv(seed_offset=5):
    """N=300, 25a+25b, naux=1500, tau=150, RHF."""
    return make_problem(300, 25, 25, 1500, 150.0, BASE_SEED + seed_offset, name="N300_n25_X1500")


def tiny_problem(norb=4, nalpha=2, nbeta=2, naux=6, tau=3.0, seed=7, unrestricted=False, ecore=0.7):
    """4-orbital systems small enough for brute-force Fock-space checks."""
    return make_problem(norb, nalpha, nbeta, naux, tau, seed, unrestricted=unrestricted,
                        ecore=ecore, orthogonalise=True)


def make_complex_problem(norb, nalpha, nbeta, npairs, tau, seed, unrestricted=False, ecore=0.9, name=""):
    """A complex Hamiltonian (as with Bloch orbitals or a magnetic field): h1e complex Hermitian (the
    real ramp plus Hermitian complex noise) and 2 npairs complex Cholesky vectors, K_k and K_k^+ for
    random complex K_k scaled by exp(-k / tau) / ||K_k||_F.  A set closed under the conjugate transpose
    gives an ERI g_psqr = sum_g L^g_ps conj(L^g_rq) with the electron-exchange symmetry (ps|qr) = (qr|ps)
    of true integrals.  The trial is the core guess (lowest eigenvectors of h1e, complex), beta with its
    HOMO and LUMO mixed by pi/4 when unrestricted."""
    rng = np.random.default_rng(seed)
    h = np.diag(np.linspace(0.0, 4.0, norb)).astype(np.complex128)
    off = 0.1 * (rng.standard_normal((norb, norb)) + 1j * rng.standard_normal((norb, norb)))
    off = np.triu(off, 1)
    h1e = np.ascontiguousarray(h + off + off.conj().T)
    chol = np.empty((2 * npairs, norb, norb), dtype=np.complex128)
    for k in range(npairs):
        a = rng.standard_normal((norb, norb)) + 1j * rng.standard_normal((norb, norb))
        a *= math.exp(-k / tau) / np.linalg.norm(a)
        chol[2 * k] = a
        chol[2 * k + 1] = a.conj().T
    _, c = np.linalg.eigh(h1e)
    ca, cb = c[:, :nalpha].copy(), c.copy()
    if unrestricted and 0 < nbeta < norb:
        hh, ll = cb[:, nbeta - 1].copy(), cb[:, nbeta].copy()
        cb[:, nbeta - 1] = (hh + ll) / np.sqrt(2.0)
    psiT = np.ascontiguousarray(np.hstack([ca, cb[:, :nbeta]]))
    return Problem(h1e, np.ascontiguousarray(chol), float(ecore), nalpha, nbeta, psiT, name)


def random_walkers(rng, norb, ncols, nwalkers, spread=0.3, psiT=None):
    """Complex determinants near psiT (or random), for kernel-level parity cases."""
    base = psiT if psiT is not None else rng.standard_normal((norb, ncols))
    noise = rng.standard_normal((nwalkers, norb, ncols)) + 1j * rng.standard_normal((nwalkers, norb, ncols))
    return np.ascontiguousarray(base[None, :, :] + spread * noise)


def config_batched(nsys=32, seed_offset=4, nmin=50, nmax=300):
    """Uneven independent systems: N ~ U[nmin, nmax] (seeded), n = N // 6 per spin, naux = 4N,
    tau = naux / 10, RHF trial from the core guess (the lowest eigenvectors of h1e), L
    Frobenius-normalised only (no Gram-Schmidt, to keep generation fast at N = 300)."""
    rng = np.random.default_rng(BASE_SEED + seed_offset)
    sizes = rng.integers(nmin, nmax + 1, size=nsys)
    probs = []
    for i, n in enumerate(sizes):
        n = int(n)
        nocc = max(1, n // 6)
        probs.append(make_problem(n, nocc, nocc, 4 * n, 0.4 * n, BASE_SEED + 1000 + i, orthogonalise=False,
                                  scf_iterations=0, name=f"sys{i}_N{n}"))
    return probs


# --- the large system (1512 orbitals, 42 + 42 electrons, naux = 7560) ---------------------------
# Its Cholesky tensor (69 GB in binary32) is never materialised on the host.  Each entry comes from
# a counter-based integer hash of (gamma, min(p, q), max(p, q)), so any chunk of gammas can be drawn
# on its own, on the CPU (numpy) or on the GPU (torch), with identical bits:
#   u = (hash + 1/2) 2^-31 - 1 in (-1, 1),   L^g_pq = s_g u,   s_g = exp(-g / tau) sqrt(3) / N,
# s_g being exp(-g/tau) over the expected Frobenius norm (N / sqrt 3) of an N x N matrix of such u
# (so ||L^g||_F ~ exp(-g / tau), with no reduction needed).  The hash is 32-bit integer mixing
# (xor-shift and multiply by 0x45d9f3b, twice) in int64 arithmetic that never overflows.

_M32 = 0xFFFFFFFF
_MIX = 0x45D9F3B


def _mix32(x, xp):
    x = ((x >> 16) ^ x) * _MIX & _M32
    x = ((x >> 16) ^ x) * _MIX & _M32
    return (x >> 16) ^ x


def _chol_hash(key, seed, xp):
    """32-bit hash of the int64 entry keys (numpy or torch arrays)."""
    hi = _mix32((key >> 32) + (seed & _M32), xp)
    return _mix32((key & _M32) ^ hi, xp)


def large_chol_scales(naux, norb, tau):
    return [math.exp(-g / tau) * math.sqrt(3.0) / norb for g in range(naux)]


def large_chol_chunk(g0, ng, norb, tau, seed, dtype=np.float32, device=None):
    """Cholesky vectors g0 .. g0 + ng - 1 of the large synthetic system, [ng, norb, norb].

    device None: a numpy array (CPU); else a torch tensor drawn on that device (same bits)."""
    sc = large_chol_scales(g0 + ng, norb, tau)[g0:]
    if device is None:
        from concurrent.futures import ThreadPoolExecutor
        idx = np.arange(norb, dtype=np.int64)
        pair = np.minimum(idx[:, None], idx[None, :]) * norb + np.maximum(idx[:, None], idx[None, :])
        out = np.empty((ng, norb, norb), dtype=dtype)

        def one(k):   # numpy releases the GIL in these array operations
            key = np.int64(g0 + k) * (norb * norb) + pair
            h = _chol_hash(key, seed, np)
            u = (h.astype(np.float64) + 0.5) * 2.0 ** -31 - 1.0
            out[k] = (sc[k] * u).astype(dtype)

        with ThreadPoolExecutor(max_workers=min(16, max(1, ng))) as ex:
            list(ex.map(one, range(ng)))
        return out
    import torch
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    idx = torch.arange(norb, dtype=torch.int64, device=device)
    pair = torch.minimum(idx[:, None], idx[None, :]) * norb + torch.maximum(idx[:, None], idx[None, :])
    out = torch.empty((ng, norb, norb), dtype=tdt, device=device)
    scales = torch.tensor(sc, dtype=torch.float64, device=device)
    for k in range(ng):
        key = (g0 + k) * (norb * norb) + pair
        h = _chol_hash(key, seed, torch)
        u = (h.to(torch.float64) + 0.5) * 2.0 ** -31 - 1.0
        out[k] = (scales[k] * u).to(tdt)
    return out


@dataclasses.dataclass
class LargeProblem:
    """The large system without its Cholesky tensor: chunks come from large_chol_chunk."""

    h1e: np.ndarray
    ecore: float
    nalpha: int
    nbeta: int
    psiT: np.ndarray
    naux: int
    tau: float
    seed: int
    name: str = ""

    @property
    def norb(self) -> int:
        return self.h1e.shape[0]

    def chunks(self, size, dtype=np.float32, device=None, naux=None):
        """Iterator over [size, N, N] chunks of the first naux (default all) vectors."""
        total = self.naux if naux is None else naux
        for g0 in range(0, total, size):
            yield large_chol_chunk(g0, min(size, total - g0), self.norb, self.tau, self.seed, dtype, device)

    def dense(self, naux=None, dtype=np.float64):
        """The first naux vectors as one host array (small naux only)."""
        total = self.naux if naux is None else naux
        return large_chol_chunk(0, total, self.norb, self.tau, self.seed, dtype)


def config_large(naux=7560, seed_offset=3):
    """N=1512, 42a+42b, naux=7560 (tau = naux/10), UHF trial: the benzene-dimer aug-cc-pVQZ shape.

    The trial is the core guess (the 42 lowest eigenvectors of h1e; beta with its HOMO and LUMO
    mixed by pi/4, which breaks the spin symmetry): 20 Roothaan iterations would need exchange
    builds over the whole 69 GB tensor.  naux below 7560 gives the same system truncated to its
    first naux vectors (tau stays 756), for checks against the oracle."""
    norb, nocc, full = 1512, 42, 7560
    seed = BASE_SEED + seed_offset
    rng = np.random.default_rng(seed)
    h1e = one_body(rng, norb)
    _, c = np.linalg.eigh(h1e)
    ca, cb = c[:, :nocc].copy(), c[:, :nocc + 1].copy()
    h, l = cb[:, nocc - 1].copy(), cb[:, nocc].copy()
    cb[:, nocc - 1] = (h + l) / np.sqrt(2.0)
    psiT = np.ascontiguousarray(np.hstack([ca, cb[:, :nocc]]))
    return LargeProblem(h1e, 1.5, nocc, nocc, psiT, naux, full / 10.0, seed, name=f"N1512_n42_X{naux}")
