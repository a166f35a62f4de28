"""The large single system (1512 orbitals, 42 + 42 electrons, UHF trial; the benzene-dimer
aug-cc-pVQZ shape of Section "Distributed Hamiltonian for limited memory") through the chunked
set-up, against the FP64 oracle.

* With its first 240 Cholesky vectors (every kernel at N = 1512 and two spin blocks of 42, the
  oracle finishing in about a minute): the whole trajectory, 2 steps with a QR, against the
  oracle on identical fields.
* At full size (naux = 7560, 128 walkers, L drawn on the GPU in binary32 chunks: the benchmark's
  configuration): the force-bias shift x-bar of sampled walkers and Cholesky vectors after one
  step, which the oracle forms one vector at a time from the walker's determinant.
* Chunked construction against afqmc_create on a small system (host / device chunks, binary64 /
  binary32, uneven chunk sizes).
"""
import numpy as np
import pytest

import paper_2406_16238_b300 as pkg
from oracle import afqmc as orc
from synthetic_inputs import config_large, config_medium, large_chol_chunk, make_problem

pytestmark = pytest.mark.gpu

TOL = {"bf16x3": 1e-4, "bf16": 1e-3}


@pytest.fixture(scope="module")
def reduced_large():
    """config_large truncated to its first 240 vectors, with the oracle's 2-step trajectory (4 walkers,
    dt = 0.005, energy every step, QR after step 2, no comb)."""
    prob = config_large(naux=240)
    chol = prob.dense(dtype=np.float32).astype(np.float64)   # the values the library receives in binary32
    st = orc.build_setup(prob.h1e, chol, prob.ecore, prob.nalpha, prob.nbeta, prob.psiT, 0.005)
    hist, wk = orc.run_phaseless(st, prob.psiT, 4, 2, 8191, reortho_every=2, comb_every=0, energy_every=1)
    e_final, _ = orc.energy_sums(st, wk)
    return prob, st, np.vstack([hist, e_final[None]])


@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
def test_large_system_truncated_tracks_the_oracle(reduced_large, prec):
    prob, st, ref = reduced_large
    ctx = pkg.Afqmc(prob.h1e, prob.chunks(48), prob.ecore, prob.nalpha, prob.nbeta, prob.psiT, nwalkers=4,
                    dt=0.005, seed=8191, prec=prec, naux=240)
    info = ctx.info()
    assert info["restricted"] == 0 and info["norb"] == 1512
    assert abs(info["e_var"] - st.evar) < TOL[prec]
    assert abs(info["e_core_mf"] - st.ecore_mf) < 1e-9 * max(1.0, abs(st.ecore_mf))   # binary64 lbar sums
    e = ctx.run(2, energy_every=1, reortho_every=2, comb_every=0)
    e = np.vstack([e, ctx.local_energy()[None]])
    ctx.close()
    d = np.abs(e[:, 0] / e[:, 1] - ref[:, 0] / ref[:, 1])
    assert np.max(d) <= TOL[prec], d


def test_large_system_full_size_sampled_force_bias():
    """naux = 7560, 128 walkers, bf16x3, L drawn on the GPU: x-bar of walkers 0 and 77 at four
    Cholesky vectors, formed by the oracle from the walkers after the first step."""
    import torch
    prob = config_large()
    dev = torch.device("cuda", 0)
    nw, seed = 128, 99
    ctx = pkg.Afqmc(prob.h1e, prob.chunks(120, device=dev), prob.ecore, prob.nalpha, prob.nbeta, prob.psiT,
                    nwalkers=nw, dt=0.005, seed=seed, prec="bf16x3", naux=prob.naux, device=dev)
    assert np.isfinite(ctx.info()["e_var"])
    ctx.propagate(1)
    psi1, _, w1, _ = ctx.get_walkers()
    e = ctx.local_energy()   # the tensor-core exchange also forms the force bias the next step uses
    ctx.propagate(1)         # its fields are formed at psi1
    _, xbar = ctx.get_fields()
    ctx.close()
    assert np.all(np.isfinite(e)) and np.all(w1 > 0)
    gam = np.array([0, 1, 3001, 7559])
    sub = np.concatenate([large_chol_chunk(int(g), 1, prob.norb, prob.tau, prob.seed) for g in gam]).astype(np.float64)
    st = orc.build_setup(prob.h1e, sub, prob.ecore, prob.nalpha, prob.nbeta, prob.psiT, 0.005)
    for w in (0, 77):
        _, th_a, th_b = orc.overlap_theta(st, psi1[w])
        ref = orc.field_shift(st, orc.force_bias(st, th_a, th_b), 1.0)
        got = xbar[w, gam]
        # split bf16 keeps ~2^-16 of each product: |dx| << 1e-4 |x| + 1e-6
        assert np.all(np.abs(got - ref) <= 1e-4 * np.abs(ref) + 1e-6), (w, got, ref)


@pytest.mark.parametrize("prec,rtol,atol", [("fp64", 1e-9, 1e-12), ("bf16x3", 0, 1e-6)])
def test_chunked_creation_matches_afqmc_create(prec, rtol, atol):
    """Host binary64 chunks of uneven sizes, device binary32 chunks and one device tensor give the
    energies and walkers of afqmc_create (binary32 inputs compared with afqmc_create of the same
    binary32-rounded values).  The chunks change only the order of the set-up's binary64 sums, so
    FP64 agrees to rounding; in BF16x3 such a difference can move a bf16 rounding of E_h or L."""
    import torch
    prob = make_problem(20, 4, 3, 50, 6.0, 314, unrestricted=True)
    dev = torch.device("cuda", 0)
    kw = dict(nwalkers=16, dt=0.01, seed=4, prec=prec)

    def run(chol, **extra):
        c = pkg.Afqmc(prob.h1e, chol, prob.ecore, prob.nalpha, prob.nbeta, prob.psiT, **kw, **extra)
        e = c.run(6, energy_every=1, reortho_every=3, comb_every=0)
        psi, _, w, _ = c.get_walkers()
        c.close()
        return e, psi, w

    ref = run(prob.chol)
    host = run([prob.chol[:7], prob.chol[7:8], prob.chol[8:50]], naux=50)
    for a, b in zip(ref, host):
        assert np.allclose(a, b, rtol=rtol, atol=atol)
    c32 = prob.chol.astype(np.float32)
    ref32 = run(c32.astype(np.float64))
    dev32 = run([torch.from_numpy(c32[:25]).to(dev), torch.from_numpy(c32[25:]).to(dev)], naux=50)
    one = run(torch.from_numpy(c32).to(dev))
    for a, b, c in zip(ref32, dev32, one):
        assert np.allclose(a, b, rtol=rtol, atol=atol)
        assert np.allclose(a, c, rtol=rtol, atol=atol)


def test_chunked_creation_rejects_bad_sequences():
    import torch
    prob = config_medium()
    lib = pkg.load()
    with pytest.raises(pkg.AfqmcError, match="outside"):
        pkg.Afqmc(prob.h1e, iter([prob.chol[:10], prob.chol[5:]]), prob.ecore, prob.nalpha, prob.nbeta,
                  prob.psiT, nwalkers=8, naux=prob.naux, prec="bf16x3")
    with pytest.raises(pkg.AfqmcError, match="of 432"):
        pkg.Afqmc(prob.h1e, iter([prob.chol[:10]]), prob.ecore, prob.nalpha, prob.nbeta, prob.psiT, nwalkers=8,
                  naux=prob.naux, prec="bf16x3")
    bad = torch.from_numpy(prob.chol.copy()).cuda()
    bad[5, 1, 2] += 1e-3
    with pytest.raises(pkg.AfqmcError, match="not symmetric"):
        pkg.Afqmc(prob.h1e, bad, prob.ecore, prob.nalpha, prob.nbeta, prob.psiT, nwalkers=8, prec="bf16x3")
    assert lib.afqmc_add_cholesky(None, 0, 1, None, 0, 0) == 1
