"""CPU oracle for the SQD Hamiltonian on a selected alpha x beta subspace.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` import this package.  It shares no code
with the CUDA path (``paper_2601_16169_gb300``) and never imports it.

Plain and slow on purpose.  Every function states the passage of arXiv
2601.16169 it follows and the reading taken where the paper is silent:

* the Hamiltonian and the Slater-Condon elements (Sections I-II, the paper's
  Hij/OneExcite/TwoExcite of Table I) are in ``sqd_oracle.c``: the generic
  element of two full 2*norb-bit determinants, no alpha/beta factorisation;
* ``build_strings``: the filtering of sampled configurations into a sorted
  set of distinct strings (Sections I, V-A);
* ``dense_h`` + ``eigh``: full diagonalisation of P H P for tiny cases;
* ``sigma``: matrix-free sigma = (P H P) C recomputing every H_IJ
  (Section II, method 1);
* ``davidson`` and ``correction_vector``: the Davidson eigensolver
  (Section I, Davidson 1975) with the readings listed in its docstring, and
  the correction of one root (Davidson's, or Olsen's as an option);
* ``rdm1`` / ``rdm2`` / ``orbital_gradient``: the reduced density matrices
  of the converged state and the derivatives of E they give (not in the
  paper; the Hellmann-Feynman adjoint of the subspace energy);
* ``string_weights`` / ``select_strings`` / ``map_vector``: the carry-over of
  configurations between SQD rounds (Section I; weights, selection by
  threshold, warm-start vector on the new sets).

Every function is pinned by ``tests/test_oracle_pins.py`` against something
other than itself (Jordan-Wigner operator sums, LAPACK, closed forms,
invariants, finite differences); ``tests/golden/`` holds values it wrote.

Conventions: strings are uint64 (bit k = spatial orbital k); determinant
index I = ia * nb + ib; a vector C is stored as an na x nb row-major matrix.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

__all__ = [
    "lib", "build_strings", "hij", "dense_h", "sigma", "diag", "excitations",
    "string_energy", "expect", "rdm1", "rdm2", "energy_from_rdms",
    "orbital_gradient", "rotate_integrals", "davidson", "eigh_lowest",
    "string_weights", "select_strings", "map_vector", "correction_vector",
]

_LIB = None

_u64p = ctypes.POINTER(ctypes.c_uint64)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_i8p = ctypes.POINTER(ctypes.c_int8)
_dp = ctypes.POINTER(ctypes.c_double)


def lib():
    """Load (building first if needed) the oracle's C library."""
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.oracle_hij.restype = ctypes.c_double
        L.oracle_hij.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_double,
                                 ctypes.c_uint64, ctypes.c_uint64,
                                 ctypes.c_uint64, ctypes.c_uint64]
        L.oracle_dense_h.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_double,
                                     _u64p, ctypes.c_int64, _u64p, ctypes.c_int64, _dp]
        L.oracle_sigma.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_double,
                                   _u64p, ctypes.c_int64, _u64p, ctypes.c_int64,
                                   _dp, ctypes.c_int, _dp, _i64p, ctypes.c_int64]
        L.oracle_diag.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_double,
                                  _u64p, ctypes.c_int64, _u64p, ctypes.c_int64, _dp]
        L.oracle_excitations.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_int,
                                         _u64p, ctypes.c_int64, _i64p, _i32p,
                                         _u8p, _i8p, _dp]
        L.oracle_string_energy.argtypes = [ctypes.c_int, _dp, _dp, _u64p,
                                           ctypes.c_int64, _dp]
        L.oracle_neighbours.argtypes = [_u64p, ctypes.c_int64, _i64p, _i32p]
        L.oracle_expect.argtypes = [ctypes.c_int, _u64p, ctypes.c_int64, _u64p,
                                    ctypes.c_int64, _dp, ctypes.c_int, _i32p,
                                    ctypes.c_int64, _dp]
        _LIB = L
    return _LIB


def _p(a, t):
    return a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _u64(a):
    return np.ascontiguousarray(a, dtype=np.uint64)


# ----------------------------------------------------------------- strings --

def build_strings(raw, norb: int, nelec: int) -> np.ndarray:
    """The set of distinct raw strings that have exactly ``nelec`` bits set,
    all below bit ``norb``, sorted ascending (the filtering of sampled
    configurations into the alpha or beta string set, Sections I and V-A)."""
    keep = []
    for x in np.asarray(raw, dtype=np.uint64).tolist():
        x = int(x)
        if norb < 64 and (x >> norb) != 0:
            continue
        if bin(x).count("1") != nelec:
            continue
        keep.append(x)
    return np.array(sorted(set(keep)), dtype=np.uint64)


# ------------------------------------------------------ Hamiltonian access --

def hij(norb, h, V, ecore, ia, ib, ja, jb) -> float:
    """<I_a I_b|H|J_a J_b> from the generic Slater-Condon element."""
    h, V = _f64(h), _f64(V)
    return lib().oracle_hij(norb, _p(h, _dp), _p(V, _dp), float(ecore),
                            int(ia), int(ib), int(ja), int(jb))


def dense_h(norb, h, V, ecore, sa, sb) -> np.ndarray:
    """Dense P H P over the product set sa x sb (index ia * nb + ib)."""
    h, V, sa, sb = _f64(h), _f64(V), _u64(sa), _u64(sb)
    N = len(sa) * len(sb)
    out = np.empty((N, N))
    lib().oracle_dense_h(norb, _p(h, _dp), _p(V, _dp), float(ecore),
                         _p(sa, _u64p), len(sa), _p(sb, _u64p), len(sb), _p(out, _dp))
    return out


def sigma(norb, h, V, ecore, sa, sb, C, rows=None) -> np.ndarray:
    """Matrix-free sigma = (P H P) C (Section II, the recompute-every-H_ij
    method).  C is (N,) or (nvec, N); with ``rows`` only those determinant
    rows are returned, shape (nvec, len(rows)) or (len(rows),)."""
    h, V, sa, sb = _f64(h), _f64(V), _u64(sa), _u64(sb)
    C = _f64(C)
    single = C.ndim == 1
    C2 = C.reshape(1, -1) if single else C
    nvec, N = C2.shape
    assert N == len(sa) * len(sb)
    if rows is None:
        R, rp = N, None
    else:
        rr = np.ascontiguousarray(rows, dtype=np.int64)
        R, rp = len(rr), _p(rr, _i64p)
    out = np.empty((nvec, R))
    for v0 in range(0, nvec, 64):
        nv = min(64, nvec - v0)
        blk = np.ascontiguousarray(C2[v0:v0 + nv])
        o = np.empty((nv, R))
        rc = lib().oracle_sigma(norb, _p(h, _dp), _p(V, _dp), float(ecore),
                                _p(sa, _u64p), len(sa), _p(sb, _u64p), len(sb),
                                _p(blk, _dp), nv, _p(o, _dp), rp, R if rp else 0)
        if rc != 0:
            raise RuntimeError("oracle_sigma failed: %d" % rc)
        out[v0:v0 + nv] = o
    return out[0] if single else out


def diag(norb, h, V, ecore, sa, sb) -> np.ndarray:
    """H_II for every determinant, (na * nb,)."""
    h, V, sa, sb = _f64(h), _f64(V), _u64(sa), _u64(sb)
    out = np.empty(len(sa) * len(sb))
    lib().oracle_diag(norb, _p(h, _dp), _p(V, _dp), float(ecore),
                      _p(sa, _u64p), len(sa), _p(sb, _u64p), len(sb), _p(out, _dp))
    return out


def excitations(norb, h, V, s, kind: int) -> dict:
    """Same-spin single (kind 1) or double (kind 2) excitation table of the
    string set ``s`` by brute-force pair scan (the paper's excitation lists,
    Sections II and V-A, flattened as offset + entries).

    Entries of row I are ordered by ascending target index.  Fields:
    ``off`` (n+1), ``tgt``, ``orb`` ((nnz,2) = p, q for kind 1: J = I - q + p;
    (nnz,4) = i, j, a, b for kind 2: J = I - i - j + a + b, i<j, a<b),
    ``sign`` (<J|a+_p a_q|I>, resp. <J|a+_a a+_b a_j a_i|I>) and ``val``
    (<I|H_s|J>, the one-spin Hamiltonian element)."""
    h, V, s = _f64(h), _f64(V), _u64(s)
    n = len(s)
    off = np.zeros(n + 1, dtype=np.int64)
    L = lib()
    L.oracle_excitations(norb, _p(h, _dp), _p(V, _dp), kind, _p(s, _u64p), n,
                         _p(off, _i64p), None, None, None, None)
    nnz = int(off[-1])
    tgt = np.zeros(max(nnz, 1), dtype=np.int32)
    orb = np.zeros((max(nnz, 1), 2 * kind), dtype=np.uint8)
    sign = np.zeros(max(nnz, 1), dtype=np.int8)
    val = np.zeros(max(nnz, 1))
    L.oracle_excitations(norb, _p(h, _dp), _p(V, _dp), kind, _p(s, _u64p), n,
                         _p(off, _i64p), _p(tgt, _i32p), _p(orb, _u8p),
                         _p(sign, _i8p), _p(val, _dp))
    return dict(off=off, tgt=tgt[:nnz], orb=orb[:nnz], sign=sign[:nnz], val=val[:nnz])


def string_energy(norb, h, V, s) -> np.ndarray:
    """One-spin diagonal energy <I|H_s|I> of every string (no E_core)."""
    h, V, s = _f64(h), _f64(V), _u64(s)
    out = np.empty(len(s))
    lib().oracle_string_energy(norb, _p(h, _dp), _p(V, _dp), _p(s, _u64p), len(s),
                               _p(out, _dp))
    return out


# ------------------------------------------------------------------ RDMs ---

def expect(norb, sa, sb, C, ops) -> np.ndarray:
    """<C|op|C> for a list of spin-orbital operator strings: rows of 2
    (a+_k a_l) or 4 (a+_k a+_l a_m a_n) spin-orbital indices."""
    sa, sb, C = _u64(sa), _u64(sb), _f64(C).reshape(-1)
    ops = np.ascontiguousarray(ops, dtype=np.int32)
    nent, nops = ops.shape
    out = np.empty(nent)
    lib().oracle_expect(norb, _p(sa, _u64p), len(sa), _p(sb, _u64p), len(sb),
                        _p(C, _dp), nops, _p(ops, _i32p), nent, _p(out, _dp))
    return out


def rdm1(norb, sa, sb, C, entries=None) -> np.ndarray:
    """Spin-summed 1-RDM gamma_pq = sum_s <a+_{ps} a_{qs}>.  With ``entries``
    (list of (p, q)) only those values are returned."""
    pairs = entries if entries is not None else [(p, q) for p in range(norb)
                                                 for q in range(norb)]
    ops = []
    for p, q in pairs:
        for s in (0, 1):
            ops.append((p + s * norb, q + s * norb))
    v = expect(norb, sa, sb, C, np.array(ops)).reshape(-1, 2).sum(1)
    if entries is not None:
        return v
    return v.reshape(norb, norb)


def rdm2(norb, sa, sb, C, entries=None) -> np.ndarray:
    """Spin-summed 2-RDM Gamma_pqrs = sum_{s,t} <a+_{ps} a+_{rt} a_{st} a_{qs}>
    (so that E = E_core + sum h_pq gamma_pq + 1/2 sum (pq|rs) Gamma_pqrs)."""
    quads = entries if entries is not None else [
        (p, q, r, s) for p in range(norb) for q in range(norb)
        for r in range(norb) for s in range(norb)]
    ops = []
    for p, q, r, s in quads:
        for a in (0, 1):
            for b in (0, 1):
                ops.append((p + a * norb, r + b * norb, s + b * norb, q + a * norb))
    v = expect(norb, sa, sb, C, np.array(ops)).reshape(-1, 4).sum(1)
    if entries is not None:
        return v
    return v.reshape(norb, norb, norb, norb)


def energy_from_rdms(h, V, ecore, g1, g2) -> float:
    """E = E_core + sum_pq h_pq gamma_pq + 1/2 sum_pqrs (pq|rs) Gamma_pqrs."""
    return float(ecore + np.einsum("pq,pq->", h, g1)
                 + 0.5 * np.einsum("pqrs,pqrs->", V, g2))


def orbital_gradient(h, V, g1, g2) -> np.ndarray:
    """dE/dkappa_pq at kappa = 0 for orbitals rotated by U = expm(kappa),
    kappa antisymmetric, h' = U^T h U and V rotated on all four indices:
    g_pq = 2 (F_pq - F_qp) with F_pq = sum_r h_pr gamma_qr
    + sum_rst (pr|st) Gamma_qrst (generalized Fock matrix)."""
    F = np.einsum("pr,qr->pq", h, g1) + np.einsum("prst,qrst->pq", V, g2)
    return 2.0 * (F - F.T)


def rotate_integrals(h, V, U):
    """h' = U^T h U, V'_pqrs = sum U_ap U_bq U_cr U_ds V_abcd."""
    h2 = U.T @ h @ U
    V2 = np.einsum("abcd,ap,bq,cr,ds->pqrs", V, U, U, U, U, optimize=True)
    return h2, V2


# ------------------------------------------------------------ outer loop --

def string_weights(C, na, nb):
    """w_a[i] = sum_j C(i,j)^2, w_b[j] = sum_i C(i,j)^2 (probability of each
    alpha / beta string in the state; the carry-over criterion of the SQD
    loop, Section I)."""
    M = np.asarray(C, dtype=np.float64).reshape(na, nb)
    return (M * M).sum(axis=1), (M * M).sum(axis=0)


def select_strings(s, w, threshold):
    """The strings with weight >= threshold, in their order."""
    return np.array([x for x, v in zip(np.asarray(s, np.uint64).tolist(), w) if v >= threshold],
                    dtype=np.uint64)


def map_vector(old_a, old_b, C, new_a, new_b):
    """C' on the new sets: C'(I,J) = C(I,J) where both strings are in the old
    sets, else 0, then normalised; returns (C', norm before normalisation)."""
    ia = {int(x): i for i, x in enumerate(np.asarray(old_a, np.uint64).tolist())}
    ib = {int(x): i for i, x in enumerate(np.asarray(old_b, np.uint64).tolist())}
    M = np.asarray(C, dtype=np.float64).reshape(len(old_a), len(old_b))
    out = np.zeros((len(new_a), len(new_b)))
    for i, x in enumerate(np.asarray(new_a, np.uint64).tolist()):
        if int(x) not in ia:
            continue
        for j, y in enumerate(np.asarray(new_b, np.uint64).tolist()):
            if int(y) in ib:
                out[i, j] = M[ia[int(x)], ib[int(y)]]
    nrm = float(np.sqrt((out * out).sum()))
    if nrm > 0:
        out /= nrm
    return out, nrm


# ----------------------------------------------------------- eigensolvers --

def eigh_lowest(H: np.ndarray, k: int = 1):
    """Lowest k eigenpairs of a dense symmetric matrix (LAPACK via scipy)."""
    import scipy.linalg
    w, v = scipy.linalg.eigh(H, subset_by_index=[0, k - 1])
    return w, v


def _fix_phase(X):
    # Largest-|.| component positive (ties to the lower index).
    for k in range(X.shape[1]):
        i = int(np.argmax(np.abs(X[:, k])))
        if X[i, k] < 0:
            X[:, k] = -X[:, k]
    return X


def correction_vector(r, x, theta, hdiag, precond_floor=1e-8, correction="davidson"):
    """The Davidson correction of one root: t = r / D with D = theta - H_II
    clamped to sign * max(|D|, precond_floor) (sign + for D = 0); with
    correction="olsen", t = (r - eps x) / D, eps = (x^T D^-1 r) / (x^T D^-1 x),
    which makes x^T t = 0 (Olsen, Jorgensen, Simons 1990; not in the paper)."""
    den = theta - hdiag
    den = np.where(np.abs(den) < precond_floor,
                   np.where(den < 0, -precond_floor, precond_floor), den)
    if correction == "olsen":
        b = x @ (x / den)
        eps = (x @ (r / den)) / b if b != 0.0 else 0.0
        r = r - eps * x
    elif correction != "davidson":
        raise ValueError(correction)
    return r / den


def davidson(matvec, hdiag, nroots=1, tol_residual=1e-8, tol_energy=1e-8,
             max_iter=200, max_subspace=None, precond_floor=1e-8, guess=None,
             drop_tol=1e-12, correction="davidson"):
    """Block Davidson for the lowest ``nroots`` eigenpairs (Davidson 1975,
    cited in Section I; one matrix-vector product per iteration and vector,
    diagonal preconditioner and Gram-Schmidt, Section VI).

    Readings where the paper is silent (its "specified convergence
    criterion", Section VI):
    * guess: unit vectors on the nroots smallest H_II (ties: lower index),
      unless ``guess`` (N, k) is given;
    * correction t = r / (theta - H_II), the denominator clamped to
      sign * max(|.|, precond_floor) (sign + for a zero denominator);
      correction="olsen" (not in the paper: J. Olsen, P. Jorgensen and
      J. Simons, Chem. Phys. Lett. 169, 463 (1990)) takes instead
      t = (r - eps x) / (theta - H_II) with eps = (x^T D^-1 r) / (x^T D^-1 x),
      D the same clamped denominator, so that x^T t = 0;
    * classical Gram-Schmidt applied twice; a vector whose norm after the
      two passes is below ``drop_tol`` is dropped;
    * subspace limit max(6 * nroots, 16); on reaching it, restart from the
      2 * nroots lowest Ritz vectors plus the nroots Ritz vectors of the
      previous iteration, orthonormalised against them (the GD+k restart of
      Stathopoulos and Saad, 1998); a previous direction whose norm after
      two Gram-Schmidt passes is below 1e-8 is left out;
    * converged when every root has ||r||_2 <= tol_residual and
      |theta - theta_previous| <= tol_energy.
    Returns (theta, X, iterations, residual_norms, converged).
    """
    N = len(hdiag)
    if max_subspace is None:
        max_subspace = max(6 * nroots, 16)
    max_subspace = min(max_subspace, N)
    if guess is None:
        order = np.argsort(hdiag, kind="stable")[:nroots]
        Vb = np.zeros((N, nroots))
        Vb[order, np.arange(nroots)] = 1.0
    else:
        Vb = np.array(guess, dtype=np.float64).reshape(N, -1)
        Vb, _ = np.linalg.qr(Vb)
    Wb = matvec(Vb)
    theta_old = np.full(nroots, np.inf)
    it = 0
    converged = False
    Yprev = None  # previous Ritz coefficients, in the basis of that iteration
    while True:
        G = Vb.T @ Wb
        G = 0.5 * (G + G.T)
        w, Y = np.linalg.eigh(G)
        theta = w[:nroots]
        X = Vb @ Y[:, :nroots]
        R = Wb @ Y[:, :nroots] - X * theta
        rn = np.linalg.norm(R, axis=0)
        conv = (rn <= tol_residual) & (np.abs(theta - theta_old) <= tol_energy)
        if conv.all():
            converged = True
            break
        if it >= max_iter:
            break
        it += 1
        theta_old = theta.copy()
        T = []
        for k in np.nonzero(~conv)[0]:
            T.append(correction_vector(R[:, k], X[:, k], theta[k], hdiag, precond_floor,
                                       correction))
        nkeep = Vb.shape[1]
        if nkeep + len(T) > max_subspace:
            m = min(2 * nroots, Vb.shape[1])
            Z = Y[:, :m]
            if Yprev is not None:
                cols = []
                for j in range(Yprev.shape[1]):
                    p = np.zeros(Vb.shape[1])
                    p[:Yprev.shape[0]] = Yprev[:, j]
                    for _ in range(2):
                        p = p - Z @ (Z.T @ p)
                        for c in cols:
                            p = p - c * (c @ p)
                    nrm = np.linalg.norm(p)
                    if nrm > 1e-8:
                        cols.append(p / nrm)
                if cols:
                    Z = np.concatenate([Z, np.stack(cols, axis=1)], axis=1)
            Vb = Vb @ Z
            Wb = Wb @ Z
            Yprev = np.eye(Z.shape[1])[:, :nroots]
        else:
            Yprev = Y[:, :nroots].copy()
        new = []
        for t in T:
            for _ in range(2):
                t = t - Vb @ (Vb.T @ t)
                for u in new:
                    t = t - u * (u @ t)
            nt = np.linalg.norm(t)
            if nt < drop_tol:
                continue
            new.append(t / nt)
        if not new:
            break
        Nw = np.stack(new, axis=1)
        Vb = np.concatenate([Vb, Nw], axis=1)
        Wb = np.concatenate([Wb, matvec(Nw)], axis=1)
    return theta, _fix_phase(X), it, rn, converged
