"""ctypes binding of libafqmc.so (the C ABI declared in include/afqmc.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  PyTorch provides the device workspace and the stream.  There
is no fallback: if the library is missing or cannot be loaded, importing the
binding raises.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libafqmc.so")

PREC = {"fp64": 0, "fp32": 1, "bf16": 2, "bf16x3": 3}
STATUS = {0: "AFQMC_OK", 1: "AFQMC_EINVAL", 2: "AFQMC_ENOMEM", 3: "AFQMC_ECUDA", 4: "AFQMC_ESINGULAR",
          5: "AFQMC_ENONFINITE", 6: "AFQMC_ENOWALKERS", 7: "AFQMC_ETIMEOUT"}


STAGES = ["overlap", "force_bias", "exchange", "energy", "fields", "vhs", "propagate", "qr", "comb"]


class AfqmcError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status
        self.name = STATUS.get(status, str(status))


class Params(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("nwalkers", ctypes.c_int32), ("taylor_order", ctypes.c_int32),
                ("fb_cap", ctypes.c_double), ("seed", ctypes.c_uint64), ("prec", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("e_trial", ctypes.c_double), ("stream", ctypes.c_void_p)]


class Info(ctypes.Structure):
    _fields_ = [("norb", ctypes.c_int32), ("naux", ctypes.c_int32), ("nalpha", ctypes.c_int32),
                ("nbeta", ctypes.c_int32), ("nwalkers", ctypes.c_int32), ("restricted", ctypes.c_int32),
                ("prec", ctypes.c_int32), ("reserved", ctypes.c_int32), ("step", ctypes.c_uint64),
                ("e_var", ctypes.c_double), ("e_trial", ctypes.c_double), ("e_core_mf", ctypes.c_double),
                ("workspace_bytes", ctypes.c_size_t)]


class Tuning(ctypes.Structure):
    _fields_ = [("tile_cap", ctypes.c_int32), ("prop_path", ctypes.c_int32), ("exch_groups", ctypes.c_int32),
                ("prop_tile", ctypes.c_int32), ("exch_form", ctypes.c_int32), ("ms_per_step", ctypes.c_float)]


_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_u64 = ctypes.c_uint64

# name -> (restype, argtypes); every symbol include/afqmc.h declares
SIGNATURES = {
    "afqmc_workspace_size": (_i32, [_i32, _i32, _i32, _i32, _dp, ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_size_t)]),
    "afqmc_create": (_i32, [_dp, _dp, ctypes.c_double, _i32, _i32, _i32, _i32, _dp, ctypes.POINTER(Params), _vp,
                            ctypes.c_size_t, ctypes.POINTER(_vp)]),
    "afqmc_create_begin": (_i32, [_dp, ctypes.c_double, _i32, _i32, _i32, _i32, _dp, ctypes.POINTER(Params), _vp,
                                  ctypes.c_size_t, ctypes.POINTER(_vp)]),
    "afqmc_add_cholesky": (_i32, [_vp, _i32, _i32, _vp, _i32, _i32]),
    "afqmc_create_end": (_i32, [_vp]),
    "afqmc_workspace_size_complex": (_i32, [_i32, _i32, _i32, _i32, _dp, ctypes.POINTER(Params),
                                            ctypes.POINTER(ctypes.c_size_t)]),
    "afqmc_create_begin_complex": (_i32, [_dp, ctypes.c_double, _i32, _i32, _i32, _i32, _dp, ctypes.POINTER(Params),
                                          _vp, ctypes.c_size_t, ctypes.POINTER(_vp)]),
    "afqmc_propagate": (_i32, [_vp, _i32]),
    "afqmc_local_energy": (_i32, [_vp, _dp, _dp]),
    "afqmc_local_energy_async": (_i32, [_vp, _dp]),
    "afqmc_reortho": (_i32, [_vp]),
    "afqmc_popcontrol": (_i32, [_vp]),
    "afqmc_run": (_i32, [_vp, _i32, _i32, _i32, _i32, _dp, ctypes.POINTER(_i32)]),
    "afqmc_run_async": (_i32, [_vp, _i32, _i32, _i32, _i32, _dp, ctypes.POINTER(_i32)]),
    "afqmc_get_walkers": (_i32, [_vp, _dp, _dp, _dp, ctypes.POINTER(_u64)]),
    "afqmc_set_walkers": (_i32, [_vp, _dp, _dp, _u64]),
    "afqmc_get_fields": (_i32, [_vp, _dp, _dp]),
    "afqmc_draw_normals": (_i32, [_u64, _u64, ctypes.c_uint32, _i32, _i32, _vp, _vp]),
    "afqmc_get_info": (_i32, [_vp, ctypes.POINTER(Info)]),
    "afqmc_set_etrial": (_i32, [_vp, ctypes.c_double]),
    "afqmc_set_etrial_update": (_i32, [_vp, _i32]),
    "afqmc_set_graphs": (_i32, [_vp, _i32]),
    "afqmc_set_free_projection": (_i32, [_vp, _i32]),
    "afqmc_get_weight_phases": (_i32, [_vp, _dp]),
    "afqmc_autotune": (_i32, [_vp, _i32, ctypes.POINTER(Tuning)]),
    "afqmc_set_tuning": (_i32, [_vp, ctypes.POINTER(Tuning)]),
    "afqmc_batch_create": (_i32, [_i32, ctypes.POINTER(_vp), ctypes.POINTER(_vp)]),
    "afqmc_batch_run": (_i32, [_vp, _i32, _i32, _i32, _i32, _dp, ctypes.POINTER(_i32)]),
    "afqmc_batch_destroy": (None, [_vp]),
    "afqmc_batch_set_mode": (_i32, [_vp, _i32, _i32, _i32]),
    "afqmc_batch_get_mode": (_i32, [_vp, ctypes.POINTER(_i32)]),
    "afqmc_batch_profile": (_i32, [_vp, _i32]),
    "afqmc_batch_describe": (_i32, [_vp, ctypes.c_char_p, ctypes.c_size_t]),
    "afqmc_batch_stage_times": (_i32, [_vp, _dp, ctypes.POINTER(ctypes.c_int64)]),
    "afqmc_cv_workspace_size": (_i32, [_vp, _i32, _i32, ctypes.POINTER(ctypes.c_size_t)]),
    "afqmc_cv_attach": (_i32, [_vp, _i32, _i32, ctypes.c_double, _u64, _vp, ctypes.c_size_t]),
    "afqmc_cv_collect": (_i32, [_vp, _i32, _i32, _i32, ctypes.POINTER(_i32)]),
    "afqmc_cv_train": (_i32, [_vp, _i32, ctypes.c_double, _dp]),
    "afqmc_cv_enable": (_i32, [_vp, _i32]),
    "afqmc_cv_params": (_i32, [_vp, _i32, _fp]),
    "afqmc_cv_eval": (_i32, [_vp, _fp, _fp, _i32, _fp, _fp, _fp]),
    "afqmc_cv_info": (_i32, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_u64), ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "afqmc_synchronize": (_i32, [_vp, ctypes.c_double]),
    "afqmc_destroy": (None, [_vp]),
    "afqmc_launch_count": (_u64, [_vp]),
    "afqmc_profile": (_i32, [_vp, _i32]),
    "afqmc_stage_times": (_i32, [_vp, _dp, ctypes.POINTER(ctypes.c_int64)]),
    "afqmc_last_error": (ctypes.c_char_p, []),
    "afqmc_comb_plan_noalloc": (_i32, [_vp, _i32, _u64, _u64, _vp, _vp, _vp]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libafqmc.so (raises if it is missing: there is no CPU fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing; build it with `python -m paper_2406_16238_b300.build` "
                          "(or __graft_entry__.build())")
    try:
        import torch  # noqa: F401  (loads the CUDA runtime the library links against)
    except ImportError:
        pass
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status):
    if status != 0:
        raise AfqmcError(status, load().afqmc_last_error().decode(errors="replace"))


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None and a.shape != tuple(shape):
        raise ValueError(f"expected shape {tuple(shape)}, got {a.shape}")
    return a


def _ptr(a):
    return a.ctypes.data_as(_dp)


class Afqmc:
    """One walker batch of phaseless AFQMC on the current CUDA device (afqmc_create ... afqmc_destroy).

    chol is either the whole [naux, norb, norb] array (afqmc_create) or an iterable of Cholesky
    chunks (then naux must be given): each chunk a [ngamma, norb, norb] float64 / float32 array
    (host: numpy or a CPU torch tensor) or a CUDA torch tensor on the context's device, passed in
    gamma order through afqmc_create_begin / afqmc_add_cholesky / afqmc_create_end.
    """

    def __init__(self, h1e, chol, ecore, nalpha, nbeta, psiT, *, nwalkers, dt=0.005, taylor_order=6, fb_cap=1.0,
                 seed=0, prec="fp64", e_trial=None, device=None, stream=None, naux=None):
        import torch
        lib = load()
        # complex Hamiltonian (complex h1e, psiT or Cholesky vectors): the complex entry points
        self.cplx = (np.iscomplexobj(h1e) or np.iscomplexobj(psiT) or
                     (isinstance(chol, np.ndarray) and np.iscomplexobj(chol)) or
                     (isinstance(chol, torch.Tensor) and chol.is_complex()))
        if self.cplx:
            self._init_complex(lib, h1e, chol, ecore, nalpha, nbeta, psiT, nwalkers, dt, taylor_order, fb_cap,
                               seed, prec, e_trial, device, stream, naux)
            return
        self.h1e = _f64(h1e)
        norb = self.h1e.shape[0]
        if isinstance(chol, torch.Tensor):   # one chunk holding every vector
            naux = int(chol.shape[0]) if naux is None else naux
            chol = [chol]
        chunked = not isinstance(chol, np.ndarray)
        if chunked:
            if naux is None:
                raise ValueError("naux is required when chol is given in chunks")
            self.chol = None
        else:
            self.chol = _f64(chol)
            naux = self.chol.shape[0]
            if self.chol.shape != (naux, norb, norb):
                raise ValueError("chol must be [naux, norb, norb]")
        self.psiT = _f64(psiT, (norb, nalpha + nbeta))
        self.norb, self.naux, self.nalpha, self.nbeta, self.nwalkers = norb, naux, nalpha, nbeta, int(nwalkers)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.prec = prec
        self.params = Params(float(dt), int(nwalkers), int(taylor_order), float(fb_cap), int(seed) & (2 ** 64 - 1),
                             PREC[prec], 0, math.nan if e_trial is None else float(e_trial),
                             ctypes.c_void_p(self.stream.cuda_stream))
        nbytes = ctypes.c_size_t()
        _check(lib.afqmc_workspace_size(norb, naux, nalpha, nbeta, _ptr(self.psiT), ctypes.byref(self.params),
                                        ctypes.byref(nbytes)))
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(nbytes.value, dtype=torch.uint8, device=self.device)
        ctx = ctypes.c_void_p()
        self._lib = lib
        if not chunked:
            _check(lib.afqmc_create(_ptr(self.h1e), _ptr(self.chol), float(ecore), norb, naux, nalpha, nbeta,
                                    _ptr(self.psiT), ctypes.byref(self.params),
                                    ctypes.c_void_p(self.workspace.data_ptr()), nbytes.value, ctypes.byref(ctx)))
            self._ctx = ctx
            return
        with torch.cuda.device(self.device):
            _check(lib.afqmc_create_begin(_ptr(self.h1e), float(ecore), norb, naux, nalpha, nbeta, _ptr(self.psiT),
                                          ctypes.byref(self.params), ctypes.c_void_p(self.workspace.data_ptr()),
                                          nbytes.value, ctypes.byref(ctx)))
            self._ctx = ctx
            g0 = 0
            for chunk in chol:
                g0 += self._add_cholesky(g0, chunk, norb)
            _check(lib.afqmc_create_end(self._ctx))

    def _init_complex(self, lib, h1e, chol, ecore, nalpha, nbeta, psiT, nwalkers, dt, taylor_order, fb_cap, seed,
                      prec, e_trial, device, stream, naux):
        """afqmc_create_begin_complex + afqmc_add_cholesky (complex chunks) + afqmc_create_end."""
        import torch
        h = np.asarray(h1e, dtype=np.complex128)
        norb = h.shape[0]
        pt = np.asarray(psiT, dtype=np.complex128)
        if pt.shape != (norb, nalpha + nbeta):
            raise ValueError(f"psiT must be [{norb}, {nalpha + nbeta}]")
        self.h1e = np.ascontiguousarray(np.stack([h.real, h.imag], axis=-1))
        self.psiT = np.ascontiguousarray(np.stack([pt.real, pt.imag], axis=-1))
        if isinstance(chol, (np.ndarray, torch.Tensor)):
            naux = int(chol.shape[0]) if naux is None else naux
            chol = [chol]
        if naux is None:
            raise ValueError("naux is required when chol is given in chunks")
        self.chol = None
        self.norb, self.nalpha, self.nbeta, self.nwalkers = norb, nalpha, nbeta, int(nwalkers)
        self.naux = 2 * naux   # auxiliary fields
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.prec = prec
        self.params = Params(float(dt), int(nwalkers), int(taylor_order), float(fb_cap), int(seed) & (2 ** 64 - 1),
                             PREC[prec], 0, math.nan if e_trial is None else float(e_trial),
                             ctypes.c_void_p(self.stream.cuda_stream))
        nbytes = ctypes.c_size_t()
        _check(lib.afqmc_workspace_size_complex(norb, naux, nalpha, nbeta, _ptr(self.psiT), ctypes.byref(self.params),
                                                ctypes.byref(nbytes)))
        self._lib = lib
        ctx = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(nbytes.value, dtype=torch.uint8, device=self.device)
            _check(lib.afqmc_create_begin_complex(_ptr(self.h1e), float(ecore), norb, naux, nalpha, nbeta,
                                                  _ptr(self.psiT), ctypes.byref(self.params),
                                                  ctypes.c_void_p(self.workspace.data_ptr()), nbytes.value,
                                                  ctypes.byref(ctx)))
            self._ctx = ctx
            g0 = 0
            for chunk in chol:
                g0 += self._add_cholesky(g0, chunk, norb)
            _check(lib.afqmc_create_end(self._ctx))

    def _add_cholesky(self, g0, chunk, norb):
        import torch
        codes = {torch.float64: 0, torch.float32: 1, torch.complex128: 2, torch.complex64: 3}
        if isinstance(chunk, torch.Tensor):
            t = chunk.contiguous()
            if self.cplx and not t.is_complex():
                t = t.to(torch.complex128)
            if t.dtype not in codes:
                raise ValueError("Cholesky chunks must be float64 / float32 (complex128 / complex64 if complex)")
            if t.is_cuda and t.device != self.device:
                raise ValueError(f"chunk is on {t.device}, the context on {self.device}")
            dtype = codes[t.dtype]
            loc = 1 if t.is_cuda else 0
            ptr, shape = t.data_ptr(), tuple(t.shape)
            keep = t
        else:
            a = np.asarray(chunk)
            if self.cplx:
                if a.dtype not in (np.complex128, np.complex64):
                    a = a.astype(np.complex128)
            elif a.dtype not in (np.float64, np.float32):
                a = a.astype(np.float64)
            a = np.ascontiguousarray(a)
            dtype = {np.dtype(np.float64): 0, np.dtype(np.float32): 1, np.dtype(np.complex128): 2,
                     np.dtype(np.complex64): 3}[a.dtype]
            loc, ptr, shape, keep = 0, a.ctypes.data, a.shape, a
        if len(shape) != 3 or shape[1:] != (norb, norb):
            raise ValueError(f"a Cholesky chunk must be [ngamma, {norb}, {norb}] (got {shape})")
        _check(self._lib.afqmc_add_cholesky(self._ctx, int(g0), int(shape[0]), ctypes.c_void_p(ptr), dtype, loc))
        del keep
        return shape[0]

    # --- the hot path -------------------------------------------------------------------
    def propagate(self, nsteps=1):
        _check(self._lib.afqmc_propagate(self._ctx, int(nsteps)))

    def local_energy(self, per_walker=False):
        sums = np.zeros(4)
        eloc = np.zeros((self.nwalkers, 3, 2)) if per_walker else None
        _check(self._lib.afqmc_local_energy(self._ctx, _ptr(sums), _ptr(eloc) if per_walker else None))
        if per_walker:
            return sums, eloc[..., 0] + 1j * eloc[..., 1]
        return sums

    def local_energy_async(self, out):
        """Enqueue the four estimator sums' copy into `out` (a contiguous float64 host array of at least
        4 entries, page-locked for an asynchronous copy); valid after synchronize()."""
        if out.dtype != np.float64 or out.size < 4 or not out.flags["C_CONTIGUOUS"]:
            raise ValueError("out must be a contiguous float64 array with at least 4 entries")
        _check(self._lib.afqmc_local_energy_async(self._ctx, _ptr(out)))

    def reortho(self):
        _check(self._lib.afqmc_reortho(self._ctx))

    def popcontrol(self):
        _check(self._lib.afqmc_popcontrol(self._ctx))

    def run(self, nsteps, energy_every=1, reortho_every=5, comb_every=10):
        nmax = (nsteps + energy_every - 1) // energy_every + 1 if energy_every > 0 else 1
        out = np.zeros((nmax, 4))
        nmeas = ctypes.c_int32()
        _check(self._lib.afqmc_run(self._ctx, int(nsteps), int(energy_every), int(reortho_every), int(comb_every),
                                   _ptr(out), ctypes.byref(nmeas)))
        return out[: nmeas.value]

    def run_async(self, nsteps, out, energy_every=1, reortho_every=5, comb_every=10):
        """The driver loop without synchronising: measurement k's four sums land in out[4k:4k+4] (a
        contiguous float64 host array, page-locked for asynchronous copies) once the stream gets there
        (synchronize()).  Returns the number of measurements."""
        need = 4 * ((nsteps + energy_every - 1) // energy_every) if energy_every > 0 else 0   # at most
        if energy_every > 0 and (out.dtype != np.float64 or not out.flags["C_CONTIGUOUS"] or out.size < need):
            raise ValueError("out must be a contiguous float64 array with 4 entries per measurement")
        nmeas = ctypes.c_int32()
        _check(self._lib.afqmc_run_async(self._ctx, int(nsteps), int(energy_every), int(reortho_every),
                                         int(comb_every), _ptr(out) if energy_every > 0 else None,
                                         ctypes.byref(nmeas)))
        return nmeas.value

    # --- state --------------------------------------------------------------------------
    def get_walkers(self):
        nt = self.nalpha + self.nbeta
        psi = np.zeros((self.nwalkers, self.norb, nt, 2))
        logo = np.zeros((self.nwalkers, 2))
        w = np.zeros(self.nwalkers)
        step = ctypes.c_uint64()
        _check(self._lib.afqmc_get_walkers(self._ctx, _ptr(psi), _ptr(logo), _ptr(w), ctypes.byref(step)))
        return psi[..., 0] + 1j * psi[..., 1], logo[:, 0] + 1j * logo[:, 1], w, int(step.value)

    def set_walkers(self, psi, w, step):
        psi = np.asarray(psi, dtype=np.complex128)
        buf = _f64(np.stack([psi.real, psi.imag], axis=-1))
        ww = _f64(w, (self.nwalkers,))
        _check(self._lib.afqmc_set_walkers(self._ctx, _ptr(buf), _ptr(ww), int(step)))

    def get_fields(self):
        x = np.zeros((self.nwalkers, self.naux))
        xb = np.zeros((self.nwalkers, self.naux, 2))
        _check(self._lib.afqmc_get_fields(self._ctx, _ptr(x), _ptr(xb)))
        return x, xb[..., 0] + 1j * xb[..., 1]

    def info(self):
        inf = Info()
        _check(self._lib.afqmc_get_info(self._ctx, ctypes.byref(inf)))
        return {k: getattr(inf, k) for k, _ in Info._fields_}

    # --- learned control variate -------------------------------------------------------
    def cv_attach(self, capacity=100000, batch=1024, sample_frac=0.125, seed=1):
        import torch
        nbytes = ctypes.c_size_t()
        _check(self._lib.afqmc_cv_workspace_size(self._ctx, int(capacity), int(batch), ctypes.byref(nbytes)))
        self.cv_workspace = torch.empty(nbytes.value, dtype=torch.uint8, device=self.device)
        _check(self._lib.afqmc_cv_attach(self._ctx, int(capacity), int(batch), float(sample_frac), int(seed),
                                         ctypes.c_void_p(self.cv_workspace.data_ptr()), nbytes.value))
        dim, npar, npairs, nsample = ctypes.c_int32(), ctypes.c_uint64(), ctypes.c_int32(), ctypes.c_int32()
        _check(self._lib.afqmc_cv_info(self._ctx, ctypes.byref(dim), ctypes.byref(npar), ctypes.byref(npairs),
                                       ctypes.byref(nsample)))
        self.cv_dim, self.cv_nparams, self.cv_batch, self.cv_nsample = dim.value, npar.value, int(batch), nsample.value

    def cv_collect(self, nsteps, reortho_every=5, comb_every=10):
        n = ctypes.c_int32()
        _check(self._lib.afqmc_cv_collect(self._ctx, int(nsteps), int(reortho_every), int(comb_every), ctypes.byref(n)))
        return n.value

    def cv_train(self, epochs, lr=1e-3):
        losses = np.zeros(max(1, epochs))
        _check(self._lib.afqmc_cv_train(self._ctx, int(epochs), float(lr), _ptr(losses)))
        return losses[:epochs]

    def cv_enable(self, enable=True):
        _check(self._lib.afqmc_cv_enable(self._ctx, 1 if enable else 0))

    def cv_get_params(self):
        p = np.zeros(self.cv_nparams, dtype=np.float32)
        _check(self._lib.afqmc_cv_params(self._ctx, 0, p.ctypes.data_as(_fp)))
        return p

    def cv_set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.cv_nparams
        _check(self._lib.afqmc_cv_params(self._ctx, 1, p.ctypes.data_as(_fp)))

    def cv_eval(self, x, y=None):
        """Forward (and, with y, loss + gradients) of the network on host rows x [rows][dim]."""
        x = np.ascontiguousarray(x, dtype=np.float32)
        rows = x.shape[0]
        out = np.zeros(rows, dtype=np.float32)
        loss = np.zeros(1, dtype=np.float32)
        grads = np.zeros(self.cv_nparams, dtype=np.float32)
        yy = None if y is None else np.ascontiguousarray(y, dtype=np.float32)
        _check(self._lib.afqmc_cv_eval(self._ctx, x.ctypes.data_as(_fp), None if yy is None else yy.ctypes.data_as(_fp),
                                       rows, out.ctypes.data_as(_fp), loss.ctypes.data_as(_fp),
                                       grads.ctypes.data_as(_fp)))
        return (out, float(loss[0]), grads) if y is not None else out

    def autotune(self, steps=3):
        t = Tuning()
        _check(self._lib.afqmc_autotune(self._ctx, int(steps), ctypes.byref(t)))
        return {k: getattr(t, k) for k, _ in Tuning._fields_}

    def set_tuning(self, tile_cap=4, prop_path=0, exch_groups=0, prop_tile=0, exch_form=0):
        t = Tuning(int(tile_cap), int(prop_path), int(exch_groups), int(prop_tile), int(exch_form), 0.0)
        _check(self._lib.afqmc_set_tuning(self._ctx, ctypes.byref(t)))

    def set_graphs(self, enable=True):
        _check(self._lib.afqmc_set_graphs(self._ctx, 1 if enable else 0))

    def set_free_projection(self, enable=True):
        """Free projection (unshifted fields, complex weights w e^{i phi}, no comb) or back to phaseless."""
        _check(self._lib.afqmc_set_free_projection(self._ctx, 1 if enable else 0))

    def weight_phases(self):
        ph = np.zeros(self.nwalkers)
        _check(self._lib.afqmc_get_weight_phases(self._ctx, _ptr(ph)))
        return ph

    def set_etrial(self, e):
        _check(self._lib.afqmc_set_etrial(self._ctx, float(e)))

    def set_etrial_update(self, enable=True):
        """E_T replaced at each comb by the running mixed estimate of the run's measurements (or fixed again)."""
        _check(self._lib.afqmc_set_etrial_update(self._ctx, 1 if enable else 0))

    @property
    def e_trial(self):
        """The energy shift E_T in use (read from the device while it follows the estimate)."""
        return self.info()["e_trial"]

    def synchronize(self, timeout_s=60.0):
        _check(self._lib.afqmc_synchronize(self._ctx, float(timeout_s)))

    def profile(self, enable=True):
        _check(self._lib.afqmc_profile(self._ctx, 1 if enable else 0))

    def stage_times(self):
        """{stage name: (milliseconds, timed executions)} since profile(True)."""
        ms = np.zeros(len(STAGES))
        cnt = (ctypes.c_int64 * len(STAGES))()
        _check(self._lib.afqmc_stage_times(self._ctx, _ptr(ms), cnt))
        return {name: (float(ms[i]), int(cnt[i])) for i, name in enumerate(STAGES)}

    def launch_count(self):
        return int(self._lib.afqmc_launch_count(self._ctx))

    def close(self):
        if getattr(self, "_ctx", None):
            self.stream.synchronize()
            self._lib.afqmc_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def draw_normals(seed, step, nwalkers, naux, stream_id=0, device="cuda"):
    """Philox fields x[w, gamma] on the device (afqmc_draw_normals); returns a float64 torch tensor."""
    import torch
    lib = load()
    out = torch.empty((nwalkers, naux), dtype=torch.float64, device=device)
    s = torch.cuda.current_stream(out.device)
    _check(lib.afqmc_draw_normals(int(seed), int(step), int(stream_id), int(nwalkers), int(naux),
                                  ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(s.cuda_stream)))
    return out


NOALLOC_MAX_WALKERS = 65536


def comb_plan_noalloc(w, seed, step, src, neww, stream=None):
    """afqmc_comb_plan_noalloc on caller-owned device tensors (w float64 [W], src int32 [W], neww float64 [1]).

    For callers that cannot allocate device memory: the library uses a static
    device array for its scratch and allocates nothing; the caller owns every
    buffer passed here.  The three tensors must be contiguous and on one CUDA
    device (ValueError otherwise); the call is made with that device current.
    Enqueued on `stream` (default: that device's current stream).  neww = -1
    reports a weight total that is not positive and finite (src is then the
    identity).
    """
    import torch
    lib = load()
    for name, t, dt in (("w", w, torch.float64), ("src", src, torch.int32), ("neww", neww, torch.float64)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.dtype != dt:
            raise ValueError(f"{name} must be {dt} (got {t.dtype})")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if t.device != w.device:
            raise ValueError(f"{name} is on {t.device}, w on {w.device}: all three must share one device")
    if w.numel() < 1 or w.numel() > NOALLOC_MAX_WALKERS:
        raise ValueError(f"w must hold 1 to {NOALLOC_MAX_WALKERS} weights (got {w.numel()})")
    if src.numel() < w.numel():
        raise ValueError(f"src holds {src.numel()} entries, fewer than the {w.numel()} weights")
    if neww.numel() < 1:
        raise ValueError("neww must hold one entry")
    with torch.cuda.device(w.device):
        s = stream if stream is not None else torch.cuda.current_stream(w.device)
        _check(lib.afqmc_comb_plan_noalloc(ctypes.c_void_p(w.data_ptr()), int(w.numel()), int(seed) & (2 ** 64 - 1),
                                           int(step), ctypes.c_void_p(src.data_ptr()),
                                           ctypes.c_void_p(neww.data_ptr()), ctypes.c_void_p(s.cuda_stream)))


BATCH_MODES = {"auto": 0, "grouped": 1, "graphs": 2}


class Batch:
    """Independent contexts advanced in lockstep, one CUDA graph launch per step (afqmc_batch_*):
    mode "grouped" (one launch per stage over every system), "graphs" (one child graph per system)
    or "auto" (grouped where the contexts allow it)."""

    def __init__(self, contexts, mode="auto", exch_groups=0, branches=0):
        self._lib = load()
        self.contexts = list(contexts)
        arr = (ctypes.c_void_p * len(self.contexts))(*[c._ctx.value for c in self.contexts])
        b = ctypes.c_void_p()
        _check(self._lib.afqmc_batch_create(len(self.contexts), arr, ctypes.byref(b)))
        self._b = b
        self.set_mode(mode, exch_groups, branches)

    def set_mode(self, mode="auto", exch_groups=0, branches=0):
        if mode not in BATCH_MODES:
            raise ValueError(f"mode must be one of {sorted(BATCH_MODES)}")
        _check(self._lib.afqmc_batch_set_mode(self._b, BATCH_MODES[mode], int(exch_groups), int(branches)))

    def profile(self, enable=True):
        _check(self._lib.afqmc_batch_profile(self._b, 1 if enable else 0))

    def stage_times(self):
        """{stage: (ms, launches)} of the grouped stages traced since profile(True)."""
        ms = np.zeros(len(STAGES))
        n = (ctypes.c_int64 * len(STAGES))()
        _check(self._lib.afqmc_batch_stage_times(self._b, _ptr(ms), n))
        return {name: (float(ms[i]), int(n[i])) for i, name in enumerate(STAGES)}

    def describe(self):
        """The grouped launches' plan as text (after the first grouped run)."""
        buf = ctypes.create_string_buffer(8192)
        _check(self._lib.afqmc_batch_describe(self._b, buf, len(buf)))
        return buf.value.decode()

    def mode(self):
        """The form the next run takes: "grouped" or "graphs"."""
        m = ctypes.c_int32()
        _check(self._lib.afqmc_batch_get_mode(self._b, ctypes.byref(m)))
        return {1: "grouped", 2: "graphs"}[m.value]

    def run(self, nsteps, energy_every=1, reortho_every=5, comb_every=10):
        start = self.contexts[0].info()["step"]
        nm = sum(1 for k in range(nsteps) if energy_every > 0 and (start + k) % energy_every == 0)
        out = np.zeros((len(self.contexts), max(nm, 1), 4))
        n = ctypes.c_int32()
        _check(self._lib.afqmc_batch_run(self._b, int(nsteps), int(energy_every), int(reortho_every), int(comb_every),
                                         _ptr(out), ctypes.byref(n)))
        return out[:, : n.value]

    def close(self):
        if getattr(self, "_b", None):
            self._lib.afqmc_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
