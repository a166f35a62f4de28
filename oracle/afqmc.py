"""Phaseless AFQMC with a Cholesky Hamiltonian and a single-determinant trial: FP64 CPU oracle.

Test infrastructure only (see oracle/__init__.py).  Plain NumPy / SciPy in
float64 / complex128, written for a reader to check against the paper by eye:
loops over walkers, no blocking or fusion.

Conventions (the paper's notation; readings where it is silent are marked R#):

* H = sum_pq h_pq a+_p a_q + 1/2 sum g_psqr a+_p a+_q a_r a_s with
  g_psqr = sum_gamma L^g_ps L^g_qr (Eqs. 2-3), written as
  H = v0 - 1/2 sum_g v_g^2 + E0 with v_g = i sum L^g_pq a+_p a_q (Eqs. 4-6).
* R1 mean-field subtraction: with vbar_g = <v_g>_T = i lbar_g (Eq. 12's
  "mean-field shift"), H = h_eff - 1/2 sum_g (v_g - vbar_g)^2 + E_c where
  h_eff = h - 1/2 sum_g L^g L^g + sum_g lbar_g L^g and E_c = E0 - 1/2 sum lbar^2.
* B(x) of Eq. 8 in that form: exp(-dt/2 h_eff) exp(-sqrt(dt) x.(v - vbar))
  exp(-dt/2 h_eff) exp(-dt E_c).  On a determinant, exp(-sqrt(dt) x.v) acts as
  the N x N matrix exp(VHS), VHS = -i sqrt(dt) sum_g x_g L^g (Thouless), and
  exp(+sqrt(dt) x.vbar) is the scalar exp(c_mf), c_mf = i sqrt(dt) x.lbar.
* R2 exp(VHS) is the Taylor series to order p (default 6); exp(-dt/2 h_eff)
  is exact (eigendecomposition).
* Overlap <Psi_T|psi> = prod_s det(Phi_s^+ psi_s) (Phi_s^+ = Phi_s^T for a real trial); the log is
  carried as log|det| + i arg(det), arg wrapped to (-pi, pi].
* Green's function G_pq = <a+_p a_q> = [Theta Phi^T]_qp with
  Theta = psi (Phi^T psi)^-1 (the trial's calc_greens_function, Section
  "Trial wavefunctions"); half-rotated tensors Ltilde^g = Phi^T L^g and
  htilde = Phi^T h ("half_rotate").
* Force bias (Eq. 12): xbar_g = -sqrt(dt) <v_g - vbar_g> = -i sqrt(dt)
  (vbias_g - lbar_g), vbias_g = sum_s Tr(Ltilde^{g s} Theta^s).
  R3 cap: if |xbar_g| > cap, xbar_g <- cap xbar_g / |xbar_g| (cap <= 0: off).
* Weights (Eqs. 11, 13-16): log S = log O' - log O + c_mf,
  I = S exp(x.xbar - xbar.xbar / 2), theta = arg S,
  w <- w |I| max(0, cos theta) exp(dt (E_T - E_c)).
  R4 E_T (energy shift) defaults to the trial's variational energy and is a
  common factor of all weights; optionally (TrialEnergy) it is replaced at
  each comb by the running mixed estimate sum ENumer / sum EDenom of the
  measurements made since the state was created; R5 walkers of weight 0 are
  frozen until the next comb.
* Local energy (Eq. 9), half-rotated: T^{g s} = Ltilde^{g s} Theta^s,
  E1 = sum_s Tr(htilde^s Theta^s), J = 1/2 sum_g (sum_s Tr T^{g s})^2,
  K = 1/2 sum_{g s} Tr(T^{g s} T^{g s}), E_L = E0 + E1 + J - K.
  Estimator sums as in the paper's energy estimator: ENumer = sum w Re E_L,
  EDenom = sum w, E1Body = sum w Re(E0 + E1), E2Body = sum w Re(J - K).
* R6 QR stabilisation: psi_s = Q R with diag(R) > 0, psi_s <- Q,
  log O -= sum log R_ii.
* R7 comb: ordered prefix sums c_i of the weights, teeth
  t_k = ((k + xi) W_tot) / N_w, walker i receives #{k : c_{i-1} <= t_k < c_i}
  copies in ascending i, all weights <- W_tot / N_w.
* R8 step order: [energy at psi_k] -> fields at step k -> propagate ->
  weights; after the step counter becomes k+1: QR if (k+1) % reortho == 0,
  then comb if (k+1) % comb == 0 (xi drawn with counter step = k+1).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.linalg

from . import philox


def wrap_phase(t):
    """Map an angle to (-pi, pi]."""
    return np.arctan2(np.sin(t), np.cos(t))


@dataclasses.dataclass
class Setup:
    norb: int
    naux: int
    nalpha: int
    nbeta: int
    dt: float
    h1e: np.ndarray
    chol: np.ndarray
    ecore: float
    phi_a: np.ndarray
    phi_b: np.ndarray
    lbar: np.ndarray        # [X]
    heff: np.ndarray        # [N, N]
    expm_half: np.ndarray   # exp(-dt/2 h_eff)
    ecore_mf: float         # E_c = E0 - 1/2 sum lbar^2
    lrot_a: np.ndarray      # [X, na, N]
    lrot_b: np.ndarray      # [X, nb, N]
    hrot_a: np.ndarray      # [na, N]
    hrot_b: np.ndarray      # [nb, N]
    evar: float


def hc(a):
    """Conjugate transpose (the plain transpose for real arrays)."""
    return np.conj(a).T


def trial_density(phi):
    """P = Phi (Phi^+ Phi)^-1 Phi^+, the trial's one-particle density (per spin)."""
    if phi.shape[1] == 0:
        return np.zeros((phi.shape[0], phi.shape[0]))
    return phi @ np.linalg.inv(hc(phi) @ phi) @ hc(phi)


def hermitian_fields(chol):
    """Complex Cholesky vectors (Section "Support of complex Cholesky vectors"): from X complex L^g with
    g_psqr = sum_g L^g_ps conj(L^g_rq), the 2X Hermitian one-body matrices of the auxiliary fields,
    A^g = (L^g + L^g+) / 2 and B^g = i (L^g - L^g+) / 2, in the order A^0, B^0, A^1, B^1, ...

    With the electron-exchange symmetry (ps|qr) = (qr|ps), sum_g L_g L_g+ = sum_g L_g+ L_g as Fock-space
    operators, so the two-body part 1/2 sum_g L_g L_g+ (less its one-body normal-ordering term) equals
    1/2 sum_g (A_g^2 + B_g^2): twice as many fields, each a Hermitian matrix that takes the place of a
    real symmetric L^g in every formula below."""
    chol = np.asarray(chol, dtype=np.complex128)
    out = np.empty((2 * chol.shape[0],) + chol.shape[1:], dtype=np.complex128)
    for g in range(chol.shape[0]):
        lh = hc(chol[g])
        out[2 * g] = 0.5 * (chol[g] + lh)
        out[2 * g + 1] = 0.5j * (chol[g] - lh)
    return out


def build_setup(h1e, chol, ecore, nalpha, nbeta, psiT, dt) -> Setup:
    """Set-up quantities of Eqs. 4-6 and the mean-field shift of Eq. 12 (reading R1).

    chol holds the fields' one-body matrices: real symmetric L^g, or (complex Hamiltonians) the
    Hermitian matrices of hermitian_fields; h1e and psiT may then be complex (h1e Hermitian)."""
    cplx = np.iscomplexobj(h1e) or np.iscomplexobj(chol) or np.iscomplexobj(psiT)
    dtype = np.complex128 if cplx else np.float64
    h1e = np.asarray(h1e, dtype=dtype)
    chol = np.asarray(chol, dtype=dtype)
    naux, norb, _ = chol.shape
    phi_a = np.asarray(psiT[:, :nalpha], dtype=dtype)
    phi_b = np.asarray(psiT[:, nalpha:nalpha + nbeta], dtype=dtype)
    p_tot = trial_density(phi_a) + trial_density(phi_b)
    # lbar_g = Tr(L^g (P_a + P_b)) (real: both Hermitian); <v_g>_T = i lbar_g
    lbar = np.array([np.sum(chol[g] * p_tot.T).real for g in range(naux)])
    # v0 = h - 1/2 sum_r (pr|rq) (Eq. 5); (pr|rq) = sum_g L^g_pr L^g_rq
    v0 = h1e - 0.5 * sum(chol[g] @ chol[g] for g in range(naux))
    heff = v0 + sum(lbar[g] * chol[g] for g in range(naux))
    evals, evecs = np.linalg.eigh(heff)
    expm_half = (evecs * np.exp(-0.5 * dt * evals)[None, :]) @ hc(evecs)
    ecore_mf = float(ecore - 0.5 * np.dot(lbar, lbar))
    lrot_a = np.stack([hc(phi_a) @ chol[g] for g in range(naux)]) if nalpha else np.zeros((naux, 0, norb), dtype)
    lrot_b = np.stack([hc(phi_b) @ chol[g] for g in range(naux)]) if nbeta else np.zeros((naux, 0, norb), dtype)
    st = Setup(norb, naux, nalpha, nbeta, float(dt), h1e, chol, float(ecore), phi_a, phi_b,
               lbar, heff, expm_half, ecore_mf, lrot_a, lrot_b, hc(phi_a) @ h1e, hc(phi_b) @ h1e, 0.0)
    psi0 = np.asarray(psiT, dtype=np.complex128)
    _, th_a, th_b = overlap_theta(st, psi0)
    st.evar = float(local_energy(st, th_a, th_b)[0].real)
    return st


def split_spins(st: Setup, psi):
    return psi[:, :st.nalpha], psi[:, st.nalpha:st.nalpha + st.nbeta]


def log_det(a):
    """log det(a) = sum log|u_ii| + i arg(det) from an LU factorisation with partial pivoting."""
    n = a.shape[0]
    if n == 0:
        return 0.0 + 0.0j
    lu, piv = scipy.linalg.lu_factor(a)
    d = np.diag(lu)
    swaps = int(np.sum(piv != np.arange(n)))
    re = float(np.sum(np.log(np.abs(d))))
    im = float(np.sum(np.angle(d)) + math.pi * (swaps % 2))
    return complex(re, float(wrap_phase(im)))


def overlap_theta(st: Setup, psi):
    """log <Psi_T|psi> and Theta^s = psi^s (Phi^s+ psi^s)^-1 for both spins."""
    pa, pb = split_spins(st, psi)
    out = []
    logo = 0.0 + 0.0j
    for phi, p in ((st.phi_a, pa), (st.phi_b, pb)):
        if p.shape[1] == 0:
            out.append(np.zeros_like(p))
            continue
        a = hc(phi) @ p
        ld = log_det(a)
        logo = logo + ld
        out.append(np.linalg.solve(a.T, p.T).T)
    return complex(logo.real, float(wrap_phase(logo.imag))), out[0], out[1]


def greens_function(phi, theta):
    """G_pq = <a+_p a_q> = [Theta Phi^+]_qp for one spin."""
    return (theta @ hc(phi)).T


def force_bias(st: Setup, th_a, th_b):
    """vbias_g = sum_s Tr(Ltilde^{g s} Theta^s) = <L_g> (the mixed estimate entering Eq. 12)."""
    vb = np.zeros(st.naux, dtype=np.complex128)
    for g in range(st.naux):
        vb[g] = np.trace(st.lrot_a[g] @ th_a) + np.trace(st.lrot_b[g] @ th_b)
    return vb


def field_shift(st: Setup, vbias, cap):
    """xbar of Eq. 12 in the mean-field-subtracted form, with the optional cap (R3)."""
    xbar = -1j * math.sqrt(st.dt) * (vbias - st.lbar)
    if cap is not None and cap > 0:
        mag = np.abs(xbar)
        big = mag > cap
        xbar = np.where(big, xbar * (cap / np.where(big, mag, 1.0)), xbar)
    return xbar


def taylor_exp_apply(vhs, psi, order):
    """sum_{k=0}^{order} VHS^k psi / k!  (recursive terms t_k = VHS t_{k-1} / k)."""
    out = psi.copy()
    t = psi
    for k in range(1, order + 1):
        t = (vhs @ t) / k
        out = out + t
    return out


def propagate_determinant(st: Setup, psi, xshift, order=6):
    """psi' = exp(-dt/2 h_eff) exp(VHS) exp(-dt/2 h_eff) psi (Eqs. 8, 10) and c_mf.

    xshift are the shifted fields x - xbar; VHS = -i sqrt(dt) sum_g xshift_g L^g;
    the scalar part of B is exp(c_mf - dt E_c), c_mf = i sqrt(dt) xshift.lbar.
    """
    sdt = math.sqrt(st.dt)
    vhs = -1j * sdt * np.tensordot(xshift, st.chol, axes=(0, 0))
    p = st.expm_half @ psi
    p = taylor_exp_apply(vhs, p, order)
    p = st.expm_half @ p
    cmf = 1j * sdt * np.dot(xshift, st.lbar)
    return p, complex(cmf)


def weight_update(st: Setup, w, logo_old, logo_new, cmf, x, xbar, e_trial):
    """Eqs. 13-16: returns (new weight, log I of the hybrid importance function, theta)."""
    log_s = logo_new - logo_old + cmf
    log_i = log_s + np.sum(x * xbar - 0.5 * xbar * xbar)
    theta = log_s.imag
    w_new = w * math.exp(log_i.real) * max(0.0, math.cos(theta)) * math.exp(st.dt * (e_trial - st.ecore_mf))
    return w_new, complex(log_i), float(theta)


def local_energy(st: Setup, th_a, th_b):
    """(E_L, E0 + E1, J - K) of Eq. 9 for one walker, half-rotated single-determinant form."""
    e1 = np.sum(st.hrot_a * th_a.T) + np.sum(st.hrot_b * th_b.T)
    vb = np.zeros(st.naux, dtype=np.complex128)
    exx = 0.0 + 0.0j
    for g in range(st.naux):
        ta = st.lrot_a[g] @ th_a
        tb = st.lrot_b[g] @ th_b
        vb[g] = np.trace(ta) + np.trace(tb)
        exx += np.sum(ta * ta.T) + np.sum(tb * tb.T)
    e2 = 0.5 * np.sum(vb * vb) - 0.5 * exx
    return complex(st.ecore + e1 + e2), complex(st.ecore + e1), complex(e2)


def local_energy_full_g(st: Setup, psi):
    """Same estimate from the full Green's function (independent cross-check of the half rotation)."""
    _, th_a, th_b = overlap_theta(st, psi)
    ga = greens_function(st.phi_a, th_a) if st.nalpha else np.zeros((st.norb, st.norb))
    gb = greens_function(st.phi_b, th_b) if st.nbeta else np.zeros((st.norb, st.norb))
    e1 = np.sum(st.h1e * ga) + np.sum(st.h1e * gb)
    j = 0.0 + 0.0j
    k = 0.0 + 0.0j
    for g in range(st.naux):
        lg = st.chol[g]
        j += 0.5 * (np.sum(lg * ga) + np.sum(lg * gb)) ** 2
        k += 0.5 * (np.trace(lg @ ga.T @ lg @ ga.T) + np.trace(lg @ gb.T @ lg @ gb.T))
    return complex(st.ecore + e1 + j - k)


@dataclasses.dataclass
class Walkers:
    psi: np.ndarray     # [W, N, na+nb] complex128
    logo: np.ndarray    # [W] complex128
    w: np.ndarray       # [W] float64
    step: int = 0

    def copy(self):
        return Walkers(self.psi.copy(), self.logo.copy(), self.w.copy(), self.step)


def init_walkers(st: Setup, psiT, nwalkers) -> Walkers:
    psi = np.repeat(np.asarray(psiT, dtype=np.complex128)[None], nwalkers, axis=0)
    logo, _, _ = overlap_theta(st, psi[0])
    return Walkers(psi, np.full(nwalkers, logo), np.ones(nwalkers))


def energy_sums(st: Setup, wk: Walkers):
    """(ENumer, EDenom, E1Body, E2Body) and per-walker (E, E1, E2)."""
    nw = wk.psi.shape[0]
    eloc = np.zeros((nw, 3), dtype=np.complex128)
    sums = np.zeros(4)
    for i in range(nw):
        if wk.w[i] == 0.0:
            continue
        _, th_a, th_b = overlap_theta(st, wk.psi[i])
        eloc[i] = local_energy(st, th_a, th_b)
        sums += wk.w[i] * np.array([eloc[i, 0].real, 1.0, eloc[i, 1].real, eloc[i, 2].real])
    return sums, eloc


def phaseless_step(st: Setup, wk: Walkers, seed, e_trial, fb_cap=1.0, order=6, record=None):
    """One step of Eqs. 10-11 for every walker; fields drawn with counter step = wk.step."""
    nw = wk.psi.shape[0]
    x = philox.normals(seed, wk.step, nw, st.naux)
    for i in range(nw):
        if wk.w[i] == 0.0:
            continue
        _, th_a, th_b = overlap_theta(st, wk.psi[i])
        vb = force_bias(st, th_a, th_b)
        xbar = field_shift(st, vb, fb_cap)
        xs = x[i] - xbar
        psi_new, cmf = propagate_determinant(st, wk.psi[i], xs, order)
        logo_new, _, _ = overlap_theta(st, psi_new)
        w_new, log_i, theta = weight_update(st, wk.w[i], wk.logo[i], logo_new, cmf, x[i], xbar, e_trial)
        if record is not None:
            record.append(dict(walker=i, vbias=vb, xbar=xbar, x=x[i].copy(), cmf=cmf, logo_new=logo_new,
                               log_i=log_i, theta=theta))
        wk.psi[i] = psi_new
        wk.logo[i] = logo_new
        wk.w[i] = w_new
    wk.step += 1
    return x


def reorthogonalise(st: Setup, wk: Walkers):
    """QR stabilisation (R6): psi^s <- Q with diag(R) > 0, log O -= sum log R_ii."""
    for i in range(wk.psi.shape[0]):
        shift = 0.0
        for lo, hi in ((0, st.nalpha), (st.nalpha, st.nalpha + st.nbeta)):
            if hi == lo:
                continue
            q, r = np.linalg.qr(wk.psi[i][:, lo:hi])
            d = np.diag(r)
            ph = d / np.abs(d)
            wk.psi[i][:, lo:hi] = q * ph[None, :]
            shift += float(np.sum(np.log(np.abs(d))))
        wk.logo[i] = wk.logo[i] - shift


def comb_assignment(weights, xi):
    """Comb (R7): source walker of every new slot and the common new weight."""
    nw = len(weights)
    cum = np.empty(nw)
    total = 0.0
    for i in range(nw):
        total = total + float(weights[i])
        cum[i] = total
    if not total > 0.0:
        raise ValueError("all walker weights are zero")
    last_alive = max(i for i in range(nw) if weights[i] > 0.0)
    src = np.empty(nw, dtype=np.int64)
    for k in range(nw):
        tooth = ((float(k) + xi) * total) / float(nw)
        i = int(np.searchsorted(cum, tooth, side="right"))
        src[k] = i if i < nw else last_alive
    return src, total / float(nw)


def population_control(wk: Walkers, seed):
    xi = philox.comb_uniform(seed, wk.step)
    src, wnew = comb_assignment(wk.w, xi)
    wk.psi = wk.psi[src].copy()
    wk.logo = wk.logo[src].copy()
    wk.w = np.full(len(src), wnew)
    return src, xi


@dataclasses.dataclass
class TrialEnergy:
    """E_T that follows the estimate (R4): the shift in use and the running sums it is taken from.

    The paper leaves the constant factor of Eq. 14 out; in this reading E_T starts at a given value
    (E_var by default) and, at each comb, becomes the mixed estimate accumulated so far,
    num / den = sum ENumer / sum EDenom over every measurement made while this state was in use.
    Before the first measurement (den = 0) E_T keeps its value.
    """
    et: float
    num: float = 0.0
    den: float = 0.0

    def measured(self, sums):
        self.num += float(sums[0])
        self.den += float(sums[1])

    def at_comb(self):
        if self.den > 0.0:
            self.et = self.num / self.den


def run_phaseless(st: Setup, psiT, nwalkers, nsteps, seed, e_trial=None, fb_cap=1.0, order=6,
                  reortho_every=5, comb_every=10, energy_every=1, walkers=None, trial_energy=None):
    """The block loop (R8).  Returns per-measurement estimator sums and the final walkers.

    trial_energy (a TrialEnergy, updated in place): E_T is taken from it and updated at each comb
    (e_trial is then unused); without it E_T stays at e_trial (E_var by default).
    """
    wk = walkers if walkers is not None else init_walkers(st, psiT, nwalkers)
    et = st.evar if e_trial is None else e_trial
    history = []
    for _ in range(nsteps):
        if energy_every and wk.step % energy_every == 0:
            sums, _ = energy_sums(st, wk)
            history.append(sums)
            if trial_energy is not None:
                trial_energy.measured(sums)
        if trial_energy is not None:
            et = trial_energy.et
        phaseless_step(st, wk, seed, et, fb_cap, order)
        if reortho_every and wk.step % reortho_every == 0:
            reorthogonalise(st, wk)
        if comb_every and wk.step % comb_every == 0:
            population_control(wk, seed)
            if trial_energy is not None:
                trial_energy.at_comb()
    return np.array(history), wk


# --- free projection (Section "Free projection AFQMC") ---------------------------------

def free_projection_step(st: Setup, psi, logo, wc, seed, step, order=6, e_trial=0.0):
    """Unbiased step: x ~ N(0,1) with no force bias, mean-field subtraction kept, no comb.

    Complex weights: w <- w O'/O exp(c_mf) exp(dt (E_T - E_c)).
    """
    nw = psi.shape[0]
    x = philox.normals(seed, step, nw, st.naux)
    for i in range(nw):
        psi_new, cmf = propagate_determinant(st, psi[i], x[i], order)
        logo_new, _, _ = overlap_theta(st, psi_new)
        wc[i] = wc[i] * np.exp(logo_new - logo[i] + cmf + st.dt * (e_trial - st.ecore_mf))
        psi[i] = psi_new
        logo[i] = logo_new
    return x


def free_projection_energy(st: Setup, psi, wc):
    num = 0.0 + 0.0j
    den = 0.0 + 0.0j
    for i in range(psi.shape[0]):
        _, th_a, th_b = overlap_theta(st, psi[i])
        e = local_energy(st, th_a, th_b)[0]
        num += wc[i] * e
        den += wc[i]
    return num / den
