"""Seeded synthetic inputs for the SQD sigma / Davidson path.

This module only draws random numbers and shapes them into the two inputs the
method consumes: integrals (h, V) and raw alpha/beta occupation bit-strings.
It holds none of the Hamiltonian arithmetic.  Both the CPU oracle (tests and
the CPU baseline) and the CUDA path take their inputs from here, so that the
two sides see identical data; nothing else is shared between them.

The paper's workloads are H2O/cc-pVDZ and N2 configuration sets produced by
PySCF full CI plus a coefficient cutoff (Section II) that are not available
here.  The five workloads below stand in for them with the same shapes: a
full-space check (norb 8), an H2O-like space (29 orbitals, 5+5 electrons),
a 4e8-determinant space at the paper's 1e8-1e9 scale (Section VI), a batch
of uneven subspaces, and a 2.5e7-determinant adjoint case.

Conventions
-----------
* A string is a ``uint64``; bit k set means spatial orbital k is occupied.
* ``h`` is a (norb, norb) float64 array, ``V`` a (norb, norb, norb, norb)
  float64 array in chemist notation, V[p, q, r, s] = (pq|rs), row-major.
* Every generator takes an explicit seed and uses
  ``numpy.random.Generator(PCG64(seed))``.
"""

from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

__all__ = [
    "WORKLOADS",
    "Workload",
    "make_integrals",
    "hubbard_chain_integrals",
    "weights_exp",
    "weights_fermi",
    "sample_strings",
    "full_strings",
    "workload",
    "batched_workload",
    "random_vectors",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def make_integrals(norb: int, rank: int, seed: int):
    """Random symmetric one- and two-electron integrals.

    h: diagonal linearly spaced in [-2, 2] (orbital energies), off-diagonal
    N(0, 0.05) drawn for the upper triangle and mirrored.
    V: V_pqrs = sum_L L^L_pq L^L_rs with each L^L symmetric, N(0, 0.1) drawn
    for the upper triangle (diagonal included) and mirrored.  The result is
    exactly 8-fold symmetric and positive semidefinite as a (pq),(rs) matrix.
    """
    rng = _rng(seed)
    h = np.zeros((norb, norb))
    iu = np.triu_indices(norb, 1)
    h[iu] = rng.normal(0.0, 0.05, size=len(iu[0]))
    h = h + h.T
    h[np.diag_indices(norb)] = np.linspace(-2.0, 2.0, norb)
    iu0 = np.triu_indices(norb, 0)
    L = np.zeros((rank, norb, norb))
    for l in range(rank):
        m = np.zeros((norb, norb))
        m[iu0] = rng.normal(0.0, 0.1, size=len(iu0[0]))
        m = m + np.triu(m, 1).T
        L[l] = m
    Lm = L.reshape(rank, norb * norb)
    V = (Lm.T @ Lm).reshape(norb, norb, norb, norb)
    # Exact symmetrisation against any BLAS summation-order asymmetry.
    V = 0.5 * (V + V.transpose(2, 3, 0, 1))
    V = 0.5 * (V + V.transpose(1, 0, 2, 3))
    V = 0.5 * (V + V.transpose(0, 1, 3, 2))
    return np.ascontiguousarray(h), np.ascontiguousarray(V)


def hubbard_chain_integrals(L: int, t: float, U: float):
    """Open Hubbard chain in the site basis: h_{i,i+1} = h_{i+1,i} = -t and
    (pp|pp) = U, every other integral zero."""
    h = np.zeros((L, L))
    for i in range(L - 1):
        h[i, i + 1] = h[i + 1, i] = -t
    V = np.zeros((L, L, L, L))
    for p in range(L):
        V[p, p, p, p] = U
    return h, V


def weights_exp(norb: int, scale: float = 6.0) -> np.ndarray:
    """Occupation weights w_k = exp(-k / scale)."""
    return np.exp(-np.arange(norb) / scale)


def weights_fermi(norb: int, mu: float = 15.0, width: float = 2.5) -> np.ndarray:
    """Occupation weights w_k = 1 / (1 + exp((k - mu) / width))."""
    return 1.0 / (1.0 + np.exp((np.arange(norb) - mu) / width))


def _bits_from_orbitals(occ: np.ndarray) -> np.ndarray:
    # occ: (ndraw, nelec) int array of orbital indices
    out = np.zeros(occ.shape[0], dtype=np.uint64)
    for c in range(occ.shape[1]):
        out |= np.left_shift(np.uint64(1), occ[:, c].astype(np.uint64))
    return out


def sample_strings(norb: int, nelec: int, n_unique: int, weights: np.ndarray,
                   seed: int, batch: int = 4096, max_draws: int = 50_000_000):
    """Draw occupation strings until ``n_unique`` distinct ones have been seen.

    Each draw picks ``nelec`` distinct orbitals without replacement, orbital k
    with weight ``weights[k]`` (successive draws renormalised over the
    remaining orbitals).  It is done with the Gumbel-top-k construction: the
    ``nelec`` largest of log(w_k) + G_k with G_k i.i.d. standard Gumbel, which
    has exactly that distribution.

    Returns ``raw`` (uint64, every draw in order up to and including the one
    that produced the ``n_unique``-th distinct string, duplicates kept) and
    ``unique`` (the distinct strings, sorted ascending).
    """
    if not (0 <= nelec <= norb <= 64):
        raise ValueError("need 0 <= nelec <= norb <= 64")
    rng = _rng(seed)
    logw = np.log(np.asarray(weights, dtype=np.float64))
    seen = set()
    raw: List[np.ndarray] = []
    drawn = 0
    while len(seen) < n_unique:
        if drawn > max_draws:
            raise RuntimeError("string space too small for the requested size")
        g = rng.gumbel(size=(batch, norb))
        keys = logw[None, :] + g
        occ = np.argpartition(-keys, nelec - 1, axis=1)[:, :nelec] if nelec > 0 \
            else np.zeros((batch, 0), dtype=np.int64)
        bits = _bits_from_orbitals(occ)
        take = batch
        for i, b in enumerate(bits.tolist()):
            seen.add(b)
            if len(seen) == n_unique:
                take = i + 1
                break
        raw.append(bits[:take])
        drawn += take
    raw_all = np.concatenate(raw) if raw else np.zeros(0, dtype=np.uint64)
    unique = np.array(sorted(seen), dtype=np.uint64)
    return raw_all, unique


def full_strings(norb: int, nelec: int) -> np.ndarray:
    """All C(norb, nelec) strings, sorted ascending (the full CI string set)."""
    from itertools import combinations
    out = []
    for occ in combinations(range(norb), nelec):
        b = 0
        for k in occ:
            b |= 1 << k
        out.append(b)
    return np.array(sorted(out), dtype=np.uint64)


@dataclasses.dataclass
class Workload:
    name: str
    norb: int
    nelec_a: int
    nelec_b: int
    h: np.ndarray
    V: np.ndarray
    raw_a: np.ndarray
    raw_b: np.ndarray
    strings_a: np.ndarray
    strings_b: np.ndarray
    ecore: float = 0.0
    nroots: int = 1

    @property
    def ndet(self) -> int:
        return int(len(self.strings_a) * len(self.strings_b))


# name -> (norb, nelec, n_unique or None for the full set, weight kind, rank, nroots)
WORKLOADS = {
    "full8": dict(norb=8, nelec=4, n_unique=None, weights=None, rank=16, nroots=1,
                  seed=1000),
    "h2o29": dict(norb=29, nelec=5, n_unique=2000, weights="exp", rank=58, nroots=8,
                  seed=1001),
    "scale36": dict(norb=36, nelec=15, n_unique=20000, weights="fermi", rank=72,
                    nroots=1, seed=1002),
    "adjoint29": dict(norb=29, nelec=5, n_unique=5000, weights="exp", rank=58,
                      nroots=1, seed=1004),
}


def _weights(kind: Optional[str], norb: int):
    if kind == "exp":
        return weights_exp(norb)
    if kind == "fermi":
        return weights_fermi(norb)
    raise ValueError(kind)


def workload(name: str, n_unique: Optional[int] = None) -> Workload:
    """One of the named synthetic workloads (seeded, deterministic).

    ``n_unique`` overrides the string-set size (same distribution and seed),
    which gives smaller cases of the same shape for tests.
    """
    spec = WORKLOADS[name]
    norb, ne = spec["norb"], spec["nelec"]
    # Integrals of the 29-orbital workloads are shared (one Hamiltonian).
    iseed = 1001 if norb == 29 else spec["seed"]
    h, V = make_integrals(norb, spec["rank"], iseed)
    n = spec["n_unique"] if n_unique is None else n_unique
    if n is None:
        s = full_strings(norb, ne)
        raw = s.copy()
    else:
        raw, s = sample_strings(norb, ne, n, _weights(spec["weights"], norb),
                                spec["seed"])
    return Workload(name=name, norb=norb, nelec_a=ne, nelec_b=ne, h=h, V=V,
                    raw_a=raw, raw_b=raw, strings_a=s, strings_b=s,
                    nroots=spec["nroots"])


def batched_workload(nbatch: int = 64, lo: int = 200, hi: int = 3000,
                     size_seed: int = 3000, sizes: Optional[List[int]] = None):
    """Many independent subspaces over the 29-orbital, 5+5-electron Hamiltonian.

    Subspace b draws its own string set (shared by alpha and beta) with the
    exp(-k/6) weights and seed 2000 + b; its size is uniform in [lo, hi] from
    the ``size_seed`` stream unless ``sizes`` is given.
    """
    h, V = make_integrals(29, 58, 1001)
    if sizes is None:
        sizes = _rng(size_seed).integers(lo, hi + 1, size=nbatch).tolist()
    out = []
    for b, n in enumerate(sizes):
        raw, s = sample_strings(29, 5, int(n), weights_exp(29), 2000 + b)
        out.append(Workload(name=f"batch{b}", norb=29, nelec_a=5, nelec_b=5, h=h, V=V,
                            raw_a=raw, raw_b=raw, strings_a=s, strings_b=s))
    return out


def random_vectors(nvec: int, ndet: int, seed: int) -> np.ndarray:
    """nvec random float64 vectors of length ndet, N(0, 1) entries."""
    return _rng(seed).standard_normal((nvec, ndet))
