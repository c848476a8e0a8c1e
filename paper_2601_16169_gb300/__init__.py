"""Python binding of libsqd (include/sqd.h): the GB300 (sm_103a) hot path of
sample-based quantum diagonalisation, arXiv 2601.16169.

Argument marshalling only.  Every step -- string filtering, excitation
tables, sigma = H C, the Davidson iteration, the RDMs -- runs in the CUDA
kernels of ``libsqd.so``; PyTorch supplies device memory and the stream.
There is no CPU fallback: without a built library or a CUDA device every
call raises.

The functions carry the C names without the ``sqd_`` prefix:
``build_strings``, ``excitation_tables``, ``sigma``, ``davidson``, ``rdm``
(plus ``diagonal`` and the ``Tables`` object's ``info``/``export``).
Strings travel as ``torch.int64`` tensors holding the uint64 bit patterns.
"""

from __future__ import annotations

import ctypes
import os
from typing import Optional

import torch

__all__ = [
    "SQDError", "lib", "library_path", "Context", "Tables", "Options",
    "build_strings", "excitation_tables", "sigma", "davidson", "diagonal", "rdm",
    "orbital_gradient", "SQDEnergy", "davidson_batched", "batched_tuning",
    "build_strings_noalloc", "stored_h_build", "sigma_stored", "string_weights",
    "select_strings", "map_vector",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libsqd.so")
_LIB = None

SQD_OK = 0
SQD_EINVAL = -1
SQD_ENOMEM = -2
SQD_ECUDA = -3
SQD_ENOTCONVERGED = -4
SQD_EBREAKDOWN = -5
_NAMES = {0: "SQD_OK", -1: "SQD_EINVAL", -2: "SQD_ENOMEM", -3: "SQD_ECUDA",
          -4: "SQD_ENOTCONVERGED", -5: "SQD_EBREAKDOWN", -6: "SQD_ETIMEOUT"}

EXPORTED = [
    "sqd_create", "sqd_set_stream", "sqd_destroy", "sqd_last_error", "sqd_version",
    "sqd_build_strings", "sqd_excitation_tables", "sqd_free_tables", "sqd_tables_info",
    "sqd_tables_export", "sqd_diagonal", "sqd_sigma", "sqd_davidson", "sqd_rdm",
    "sqd_profile_enable", "sqd_profile_read", "sqd_launch_count", "sqd_orbital_gradient",
    "sqd_build_strings_noalloc", "sqd_davidson_batched", "sqd_batched_tuning",
    "sqd_batched_tuning_buckets", "sqd_batched_set_tile",
    "sqd_stored_h_build", "sqd_sigma_stored", "sqd_string_weights", "sqd_select_strings",
    "sqd_map_vector", "sqd_tables_set_sigma_mode", "sqd_measure_fp64_peaks",
    "sqd_tables_set_spin_flip",
]

PROFILE_CLASSES = ["same_spin_alpha", "same_spin_beta", "alpha_beta", "transpose", "tables",
                   "strings", "davidson", "rdm", "stored", "ortho", "eigh", "batched",
                   "batched_sigma", "batched_vector", "batched_eigh", "gcols", "ortho_block",
                   "batched_sigma_ab"]


class SQDError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (_NAMES.get(code, str(code)), msg))
        self.code = code


class Options(ctypes.Structure):
    """sqd_options (see include/sqd.h)."""
    _fields_ = [("nroots", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("max_subspace", ctypes.c_int), ("tol_energy", ctypes.c_double),
                ("tol_residual", ctypes.c_double), ("precond_floor", ctypes.c_double),
                ("use_guess", ctypes.c_int), ("use_stored_h", ctypes.c_int),
                ("correction", ctypes.c_int)]


def library_path() -> str:
    return _LIB_PATH


def lib():
    """Load libsqd.so.  Raises if it has not been built (no fallback)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(
            "libsqd.so is not built (%s); run `python -c 'import __graft_entry__ as g; "
            "g.build()'` or `python paper_2601_16169_gb300/build.py`" % _LIB_PATH)
    L = ctypes.CDLL(_LIB_PATH)
    vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    L.sqd_create.argtypes = [ctypes.POINTER(vp), i32, vp]
    L.sqd_set_stream.argtypes = [vp, vp]
    L.sqd_destroy.argtypes = [vp]
    L.sqd_destroy.restype = None
    L.sqd_last_error.argtypes = [vp]
    L.sqd_last_error.restype = ctypes.c_char_p
    L.sqd_version.restype = ctypes.c_char_p
    L.sqd_build_strings.argtypes = [vp, vp, i64, i32, i32, vp, ctypes.POINTER(i64)]
    L.sqd_excitation_tables.argtypes = [vp, i32, vp, i64, i32, vp, i64, i32, vp, vp, dbl,
                                        ctypes.POINTER(vp)]
    L.sqd_free_tables.argtypes = [vp]
    L.sqd_free_tables.restype = None
    L.sqd_tables_info.argtypes = [vp, vp]
    L.sqd_tables_export.argtypes = [vp, vp, i32, i32, vp, vp, vp, vp, vp]
    L.sqd_diagonal.argtypes = [vp, vp, vp]
    L.sqd_sigma.argtypes = [vp, vp, vp, vp, i32]
    L.sqd_davidson.argtypes = [vp, vp, ctypes.POINTER(Options), vp, vp,
                               ctypes.POINTER(i32), vp]
    L.sqd_rdm.argtypes = [vp, vp, vp, vp, vp]
    L.sqd_profile_enable.argtypes = [vp, i32]
    L.sqd_profile_read.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_char_p),
                                   ctypes.POINTER(i64), ctypes.POINTER(dbl),
                                   ctypes.POINTER(dbl), ctypes.POINTER(dbl)]
    L.sqd_launch_count.argtypes = [vp, ctypes.POINTER(i64)]
    L.sqd_orbital_gradient.argtypes = [vp, vp, vp, vp, vp]
    L.sqd_build_strings_noalloc.argtypes = [vp, vp, i64, i32, i32, vp, ctypes.POINTER(i64)]
    L.sqd_davidson_batched.argtypes = [vp, i32, vp, ctypes.POINTER(Options), vp, vp, vp, vp]
    L.sqd_batched_tuning.argtypes = [vp, ctypes.POINTER(dbl), ctypes.POINTER(i32)]
    L.sqd_batched_tuning_buckets.argtypes = [vp, i32, ctypes.POINTER(i32), vp, vp, vp]
    L.sqd_batched_set_tile.argtypes = [vp, i32, dbl]
    L.sqd_stored_h_build.argtypes = [vp, vp, i64, ctypes.POINTER(i64)]
    L.sqd_sigma_stored.argtypes = [vp, vp, vp, vp, i32]
    L.sqd_string_weights.argtypes = [vp, vp, vp, vp, vp]
    L.sqd_select_strings.argtypes = [vp, vp, vp, i64, dbl, vp, ctypes.POINTER(i64)]
    L.sqd_map_vector.argtypes = [vp, vp, i64, vp, i64, vp, vp, i64, vp, i64, vp,
                                 ctypes.POINTER(dbl)]
    L.sqd_tables_set_sigma_mode.argtypes = [vp, i32]
    L.sqd_tables_set_spin_flip.argtypes = [vp, i32]
    L.sqd_measure_fp64_peaks.argtypes = [vp, ctypes.POINTER(dbl), ctypes.POINTER(dbl)]
    _LIB = L
    return L


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _need_cuda(t: torch.Tensor, name: str, dtype):
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise ValueError("%s must have dtype %s" % (name, dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)


class Context:
    """An sqd_ctx bound to one device and (by default) torch's current stream."""

    def __init__(self, device: Optional[int] = None, stream: Optional[torch.cuda.Stream] = None):
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the SQD library has no CPU path")
        self.device = torch.cuda.current_device() if device is None else int(device)
        self._lib = lib()
        st = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._stream = st
        h = ctypes.c_void_p()
        rc = self._lib.sqd_create(ctypes.byref(h), self.device, ctypes.c_void_p(st.cuda_stream))
        if rc != SQD_OK:
            raise SQDError(rc, self._lib.sqd_last_error(None).decode())
        self.handle = h

    def set_stream(self, stream: torch.cuda.Stream):
        self._stream = stream
        self._check(self._lib.sqd_set_stream(self.handle, ctypes.c_void_p(stream.cuda_stream)))

    @property
    def stream(self):
        return self._stream

    def _check(self, rc, allow=()):
        if rc != SQD_OK and rc not in allow:
            raise SQDError(rc, self._lib.sqd_last_error(self.handle).decode())
        return rc

    def profile(self, enable: bool = True):
        """sqd_profile_enable: reset the counters; time kernel regions if enable."""
        self._check(self._lib.sqd_profile_enable(self.handle, 1 if enable else 0))

    def profile_read(self) -> dict:
        """sqd_profile_read for every class: {name: dict(regions, ms, flops, bytes)}."""
        out = {}
        for c in range(len(PROFILE_CLASSES)):
            nm = ctypes.c_char_p()
            reg = ctypes.c_int64()
            ms, fl, by = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
            self._check(self._lib.sqd_profile_read(self.handle, c, ctypes.byref(nm),
                                                   ctypes.byref(reg), ctypes.byref(ms),
                                                   ctypes.byref(fl), ctypes.byref(by)))
            out[nm.value.decode()] = dict(regions=reg.value, ms=ms.value, flops=fl.value,
                                          bytes=by.value)
        return out

    def launch_count(self) -> int:
        """sqd_launch_count: kernels launched since the last profile() call."""
        n = ctypes.c_int64()
        self._check(self._lib.sqd_launch_count(self.handle, ctypes.byref(n)))
        return n.value

    def measure_fp64_peaks(self):
        """sqd_measure_fp64_peaks: (FP64 FMA pipe, FP64 tensor MMA) TFLOP/s."""
        a, b = ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.sqd_measure_fp64_peaks(self.handle, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def close(self):
        if getattr(self, "handle", None):
            self._lib.sqd_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Tables:
    """Owner of an sqd_tables object (excitation lists, diagonal, scratch)."""

    def __init__(self, ctx: Context, handle, norb: int, na: int, nb: int):
        self.ctx, self.handle, self.norb, self.na, self.nb = ctx, handle, norb, na, nb

    @property
    def ndet(self) -> int:
        return self.na * self.nb

    def info(self) -> dict:
        buf = (ctypes.c_int64 * 12)()
        self.ctx._check(self.ctx._lib.sqd_tables_info(self.handle, buf))
        keys = ["norb", "n_alpha", "n_beta", "nnz1_alpha", "nnz2_alpha", "nnz1_beta",
                "nnz2_beta", "shared", "device_bytes", "max_singles", "max_doubles",
                "ab_groups"]
        return {k: int(buf[i]) for i, k in enumerate(keys)}

    def set_sigma_mode(self, mode: int):
        """sqd_tables_set_sigma_mode: 0 native FP64, 1 double-float on the
        FP32 pipe (sigma and Davidson on these tables)."""
        self.ctx._check(self.ctx._lib.sqd_tables_set_sigma_mode(self.handle, int(mode)))

    def set_spin_flip(self, sector: int):
        """sqd_tables_set_spin_flip: +1 / -1 for vectors with C^T = sector * C
        (sigma with one same-spin pass, Davidson in that sector); 0 for
        general vectors.  Shared string sets only."""
        self.ctx._check(self.ctx._lib.sqd_tables_set_spin_flip(self.handle, int(sector)))

    def export(self, spin: int, kind: int) -> dict:
        """Host (numpy) copy of one excitation table: off, tgt, orb, sign, val."""
        import numpy as np
        n = self.na if spin == 0 else self.nb
        inf = self.info()
        nnz = inf[("nnz%d_%s" % (kind, "alpha" if spin == 0 else "beta"))]
        off = np.zeros(n + 1, dtype=np.int64)
        tgt = np.zeros(max(nnz, 1), dtype=np.int32)
        orb = np.zeros((max(nnz, 1), 2 * kind), dtype=np.uint8)
        sign = np.zeros(max(nnz, 1), dtype=np.int8)
        val = np.zeros(max(nnz, 1), dtype=np.float64)
        c = ctypes.c_void_p
        self.ctx._check(self.ctx._lib.sqd_tables_export(
            self.ctx.handle, self.handle, spin, kind, c(off.ctypes.data), c(tgt.ctypes.data),
            c(orb.ctypes.data), c(sign.ctypes.data), c(val.ctypes.data)))
        return dict(off=off, tgt=tgt[:nnz], orb=orb[:nnz], sign=sign[:nnz], val=val[:nnz])

    def close(self):
        if getattr(self, "handle", None):
            self.ctx._lib.sqd_free_tables(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def build_strings(ctx: Context, raw: torch.Tensor, norb: int, nelec: int) -> torch.Tensor:
    """sqd_build_strings: filter raw samples into the sorted set of distinct
    strings with ``nelec`` electrons in ``norb`` orbitals."""
    _need_cuda(raw, "raw", torch.int64)
    out = torch.empty_like(raw)
    n = ctypes.c_int64(0)
    ctx._check(ctx._lib.sqd_build_strings(ctx.handle, _ptr(raw), raw.numel(), norb, nelec,
                                          _ptr(out), ctypes.byref(n)))
    return out[:n.value]


def build_strings_noalloc(ctx: Context, raw: torch.Tensor, norb: int, nelec: int,
                          out: torch.Tensor) -> int:
    """sqd_build_strings_noalloc: the filter of build_strings for callers
    that cannot allocate device memory (the library uses a fixed scratch
    array instead).  ``out`` (caller-allocated, at least raw.numel() int64
    elements) receives the strings; returns their count.  At most 2**18 raw
    strings; calls that overlap on the GPU race on the shared scratch."""
    _need_cuda(raw, "raw", torch.int64)
    _need_cuda(out, "out", torch.int64)
    if out.numel() < raw.numel():
        raise ValueError("out is smaller than raw")
    n = ctypes.c_int64(0)
    ctx._check(ctx._lib.sqd_build_strings_noalloc(ctx.handle, _ptr(raw), raw.numel(), norb,
                                                  nelec, _ptr(out), ctypes.byref(n)))
    return n.value


def excitation_tables(ctx: Context, norb: int, alpha: torch.Tensor, nalpha_e: int,
                      beta: torch.Tensor, nbeta_e: int, h: torch.Tensor, V: torch.Tensor,
                      ecore: float = 0.0) -> Tables:
    """sqd_excitation_tables.  Pass the same tensor for alpha and beta to
    share one table between the spins."""
    _need_cuda(alpha, "alpha", torch.int64)
    _need_cuda(beta, "beta", torch.int64)
    _need_cuda(h, "h", torch.float64)
    _need_cuda(V, "V", torch.float64)
    if h.numel() != norb * norb or V.numel() != norb ** 4:
        raise ValueError("h must have norb^2 and V norb^4 elements")
    t = ctypes.c_void_p()
    ctx._check(ctx._lib.sqd_excitation_tables(
        ctx.handle, norb, _ptr(alpha), alpha.numel(), nalpha_e,
        _ptr(beta), beta.numel(), nbeta_e, _ptr(h), _ptr(V), float(ecore), ctypes.byref(t)))
    return Tables(ctx, t, norb, alpha.numel(), beta.numel())


def diagonal(ctx: Context, tables: Tables) -> torch.Tensor:
    """sqd_diagonal: H_II of every determinant, shape (n_alpha, n_beta)."""
    out = torch.empty((tables.na, tables.nb), dtype=torch.float64,
                      device="cuda:%d" % ctx.device)
    ctx._check(ctx._lib.sqd_diagonal(ctx.handle, tables.handle, _ptr(out)))
    return out


def sigma(ctx: Context, tables: Tables, C: torch.Tensor,
          out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """sqd_sigma: sigma = H C.  C has shape (n_alpha, n_beta) or
    (nvec, n_alpha, n_beta), float64, contiguous, on the device."""
    _need_cuda(C, "C", torch.float64)
    if C.numel() % tables.ndet != 0 or C.numel() == 0:
        raise ValueError("C size is not a multiple of n_alpha * n_beta")
    nvec = C.numel() // tables.ndet
    if out is None:
        out = torch.empty_like(C)
    _need_cuda(out, "out", torch.float64)
    ctx._check(ctx._lib.sqd_sigma(ctx.handle, tables.handle, _ptr(C), _ptr(out), nvec))
    return out


def davidson(ctx: Context, tables: Tables, nroots: int = 1, tol_residual: float = 1e-8,
             tol_energy: float = 1e-8, max_iter: int = 200, max_subspace: int = 0,
             precond_floor: float = 1e-8, guess: Optional[torch.Tensor] = None,
             raise_on_nonconvergence: bool = True, use_stored_h: bool = False,
             correction: str = "davidson"):
    """sqd_davidson.  Returns (energies (numpy), C (nroots, n_alpha, n_beta)
    tensor, iterations, residual norms (numpy), status code).  correction:
    "davidson" (t = r / (theta - H_II)) or "olsen" (t orthogonal to x)."""
    import numpy as np
    C = torch.zeros((nroots, tables.na, tables.nb), dtype=torch.float64,
                    device="cuda:%d" % ctx.device)
    use_guess = 0
    if guess is not None:
        C.copy_(guess.reshape(C.shape))
        use_guess = 1
    o = Options(nroots=nroots, max_iter=max_iter, max_subspace=max_subspace,
                tol_energy=tol_energy, tol_residual=tol_residual, precond_floor=precond_floor,
                use_guess=use_guess, use_stored_h=1 if use_stored_h else 0,
                correction={"davidson": 0, "olsen": 1}[correction])
    e = np.zeros(nroots)
    r = np.zeros(nroots)
    it = ctypes.c_int(0)
    allow = () if raise_on_nonconvergence else (SQD_ENOTCONVERGED, SQD_EBREAKDOWN)
    rc = ctx._check(ctx._lib.sqd_davidson(ctx.handle, tables.handle, ctypes.byref(o),
                                          ctypes.c_void_p(e.ctypes.data), _ptr(C),
                                          ctypes.byref(it), ctypes.c_void_p(r.ctypes.data)),
                    allow=allow)
    return e, C, it.value, r, rc


def davidson_batched(ctx: Context, tables, tol_residual: float = 1e-8,
                     tol_energy: float = 1e-8, max_iter: int = 200, max_subspace: int = 0,
                     precond_floor: float = 1e-8, want_vectors: bool = True,
                     raise_on_nonconvergence: bool = True):
    """sqd_davidson_batched: ground states of many subspaces in one solve.
    Returns (energies, list of C tensors or None, iterations, statuses, rc)."""
    import numpy as np
    nb = len(tables)
    handles = (ctypes.c_void_p * nb)(*[t.handle.value for t in tables])
    Cs = [torch.empty((t.na, t.nb), dtype=torch.float64, device="cuda:%d" % ctx.device)
          for t in tables] if want_vectors else None
    ptrs = (ctypes.c_void_p * nb)(*([c.data_ptr() for c in Cs] if Cs else [0] * nb))
    o = Options(nroots=1, max_iter=max_iter, max_subspace=max_subspace, tol_energy=tol_energy,
                tol_residual=tol_residual, precond_floor=precond_floor, use_guess=0,
                use_stored_h=0)
    e = np.zeros(nb)
    it = np.zeros(nb, dtype=np.int32)
    st = np.zeros(nb, dtype=np.int32)
    allow = () if raise_on_nonconvergence else (SQD_ENOTCONVERGED, SQD_EBREAKDOWN)
    rc = ctx._check(ctx._lib.sqd_davidson_batched(
        ctx.handle, nb, handles, ctypes.byref(o), ctypes.c_void_p(e.ctypes.data),
        ptrs if Cs else None, ctypes.c_void_p(it.ctypes.data), ctypes.c_void_p(st.ctypes.data)),
        allow=allow)
    return e, Cs, it, st, rc


def stored_h_build(ctx: Context, tables: Tables, max_bytes: int = 0) -> int:
    """sqd_stored_h_build: assemble P H P once (the stored-H method); returns
    the nonzero count.  Raises SQDError(SQD_ENOMEM) if it would not fit."""
    n = ctypes.c_int64()
    ctx._check(ctx._lib.sqd_stored_h_build(ctx.handle, tables.handle, int(max_bytes),
                                           ctypes.byref(n)))
    return n.value


def sigma_stored(ctx: Context, tables: Tables, C: torch.Tensor,
                 out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """sqd_sigma_stored: sigma = H C with the stored matrix."""
    _need_cuda(C, "C", torch.float64)
    nvec = C.numel() // tables.ndet
    if out is None:
        out = torch.empty_like(C)
    ctx._check(ctx._lib.sqd_sigma_stored(ctx.handle, tables.handle, _ptr(C), _ptr(out), nvec))
    return out


def string_weights(ctx: Context, tables: Tables, C: torch.Tensor):
    """sqd_string_weights: (w_alpha, w_beta), the squared-norm weight of every
    alpha and beta string in the state C."""
    _need_cuda(C, "C", torch.float64)
    dev = "cuda:%d" % ctx.device
    wa = torch.empty(tables.na, dtype=torch.float64, device=dev)
    wb = torch.empty(tables.nb, dtype=torch.float64, device=dev)
    ctx._check(ctx._lib.sqd_string_weights(ctx.handle, tables.handle, _ptr(C), _ptr(wa), _ptr(wb)))
    return wa, wb


def select_strings(ctx: Context, strings: torch.Tensor, weights: torch.Tensor,
                   threshold: float) -> torch.Tensor:
    """sqd_select_strings: the strings whose weight is >= threshold."""
    _need_cuda(strings, "strings", torch.int64)
    _need_cuda(weights, "weights", torch.float64)
    out = torch.empty_like(strings)
    n = ctypes.c_int64()
    ctx._check(ctx._lib.sqd_select_strings(ctx.handle, _ptr(strings), _ptr(weights),
                                           strings.numel(), float(threshold), _ptr(out),
                                           ctypes.byref(n)))
    return out[:n.value]


def map_vector(ctx: Context, old_a: torch.Tensor, old_b: torch.Tensor, C: torch.Tensor,
               new_a: torch.Tensor, new_b: torch.Tensor):
    """sqd_map_vector: warm-start guess on (new_a, new_b) from the state C on
    (old_a, old_b).  Returns (vector (n_new_a, n_new_b), norm before
    normalisation)."""
    for x, nm in ((old_a, "old_a"), (old_b, "old_b"), (new_a, "new_a"), (new_b, "new_b")):
        _need_cuda(x, nm, torch.int64)
    _need_cuda(C, "C", torch.float64)
    out = torch.empty((new_a.numel(), new_b.numel()), dtype=torch.float64, device=C.device)
    nrm = ctypes.c_double()
    ctx._check(ctx._lib.sqd_map_vector(ctx.handle, _ptr(old_a), old_a.numel(), _ptr(old_b),
                                       old_b.numel(), _ptr(C), _ptr(new_a), new_a.numel(),
                                       _ptr(new_b), new_b.numel(), _ptr(out), ctypes.byref(nrm)))
    return out, nrm.value


def batched_tuning(ctx: Context, with_loop: bool = False):
    """sqd_batched_tuning: alpha-group scale chosen by the last batched solve
    (and, with_loop=True, whether its iteration loop ran inside one graph)."""
    v = ctypes.c_double()
    dl = ctypes.c_int()
    ctx._check(ctx._lib.sqd_batched_tuning(ctx.handle, ctypes.byref(v), ctypes.byref(dl)))
    return (v.value, bool(dl.value)) if with_loop else v.value


def batched_set_tile(ctx: Context, entries_per_thread: int = 0, group_scale: float = 1.0):
    """sqd_batched_set_tile: fix the paired-singles tile of later batched
    solves (16 or 8 entries per thread, group scale 0.5 / 1 / 2 / 4); 0 restores
    autotuning."""
    ctx._check(ctx._lib.sqd_batched_set_tile(ctx.handle, int(entries_per_thread),
                                             float(group_scale)))


def batched_tuning_buckets(ctx: Context):
    """sqd_batched_tuning_buckets: the paired-singles tile chosen per size
    bucket by the last batched solve, as a list of dicts (max_det, scale,
    entries_per_thread) in increasing bucket size."""
    import numpy as np
    n = ctypes.c_int(0)
    md = np.zeros(16, dtype=np.int64)
    sc = np.zeros(16)
    ep = np.zeros(16, dtype=np.int32)
    ctx._check(ctx._lib.sqd_batched_tuning_buckets(
        ctx.handle, 16, ctypes.byref(n), ctypes.c_void_p(md.ctypes.data),
        ctypes.c_void_p(sc.ctypes.data), ctypes.c_void_p(ep.ctypes.data)))
    return [dict(max_det=int(md[q]), scale=float(sc[q]), entries_per_thread=int(ep[q]))
            for q in range(min(n.value, 16))]


def rdm(ctx: Context, tables: Tables, C: torch.Tensor, two_body: bool = True):
    """sqd_rdm: spin-summed 1-RDM (norb, norb) and 2-RDM (norb,)*4 of C."""
    _need_cuda(C, "C", torch.float64)
    n = tables.norb
    dev = "cuda:%d" % ctx.device
    g1 = torch.empty((n, n), dtype=torch.float64, device=dev)
    g2 = torch.empty((n, n, n, n), dtype=torch.float64, device=dev) if two_body else None
    ctx._check(ctx._lib.sqd_rdm(ctx.handle, tables.handle, _ptr(C), _ptr(g1), _ptr(g2)))
    return g1, g2


def orbital_gradient(ctx: Context, tables: Tables, g1: torch.Tensor,
                     g2: torch.Tensor) -> torch.Tensor:
    """sqd_orbital_gradient: dE/dkappa_pq = 2 (F_pq - F_qp) from the RDMs."""
    _need_cuda(g1, "rdm1", torch.float64)
    _need_cuda(g2, "rdm2", torch.float64)
    g = torch.empty_like(g1)
    ctx._check(ctx._lib.sqd_orbital_gradient(ctx.handle, tables.handle, _ptr(g1), _ptr(g2),
                                             _ptr(g)))
    return g


class SQDEnergy(torch.autograd.Function):
    """E(h, V) = lowest eigenvalue of P H P on the given string sets, with
    the Hellmann-Feynman backward dE/dh = rdm1, dE/dV = rdm2 / 2 (C is an
    exact eigenvector of P H P and P does not depend on the integrals).
    Only the converged state C is kept for backward, no Davidson history.

    Usage: E = SQDEnergy.apply(h, V, ctx, alpha, nalpha_e, beta, nbeta_e,
    ecore, tol_residual)."""

    @staticmethod
    def forward(fctx, h, V, ctx, alpha, nalpha_e, beta, nbeta_e, ecore=0.0,
                tol_residual=1e-9):
        norb = h.shape[0]
        t = excitation_tables(ctx, norb, alpha, nalpha_e, beta, nbeta_e,
                              h.detach().contiguous(), V.detach().contiguous(), ecore)
        e, C, it, res, rc = davidson(ctx, t, nroots=1, tol_residual=tol_residual,
                                     tol_energy=1e-12, max_iter=500)
        fctx.sqd = (ctx, t)
        fctx.save_for_backward(C)
        return torch.tensor(e[0], dtype=torch.float64, device=h.device)

    @staticmethod
    def backward(fctx, grad):
        (C,) = fctx.saved_tensors
        ctx, t = fctx.sqd
        g1, g2 = rdm(ctx, t, C[0].contiguous())
        t.close()
        return (grad * g1, 0.5 * grad * g2, None, None, None, None, None, None, None)
