"""Spin-flip sectors (sqd_tables_set_spin_flip) against the oracle.

With one string set for both spins, exchanging the alpha and beta strings
commutes with H, and on a vector of one sector (C^T = s C, s = +1 or -1) the
library forms the beta side of sigma as s times the transposed alpha side.
The references here are independent of that shortcut:
* sigma of a sector vector against the oracle's sigma (every H_IJ from the
  generic Slater-Condon element), relative L2 <= 1e-12, on small cases with
  ragged 32 x 32 tiles and on sampled rows at full size;
* Davidson in a sector against LAPACK on the oracle's dense H restricted to
  that sector (basis e_II and (e_IJ + s e_JI)/sqrt(2)), |dE| <= 1e-9 Ha; the
  Ritz vectors must lie exactly in the sector;
* the ground state of h2o29 from the general solve is the lower of the two
  sector ground states (the sectors span the space).
"""
import numpy as np
import pytest
import torch

import oracle
import sqd_inputs as si

pytestmark = pytest.mark.gpu

SIGMA_TOL = 1e-12


@pytest.fixture(scope="module")
def sqd():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2601_16169_gb300 as m
    return m


@pytest.fixture(scope="module")
def ctx(sqd):
    torch.cuda.set_device(0)
    return sqd.Context(0)


def _tables(sqd, ctx, w, shared=True):
    da = torch.tensor(np.ascontiguousarray(w.strings_a, dtype=np.uint64).view(np.int64),
                      device="cuda")
    db = da if shared else da.clone()
    h = torch.tensor(w.h, dtype=torch.float64, device="cuda")
    V = torch.tensor(w.V, dtype=torch.float64, device="cuda")
    return sqd.excitation_tables(ctx, w.norb, da, w.nelec_a, db, w.nelec_b, h, V, 0.0)


def _sector_vector(n, seed, s):
    R = np.random.default_rng(seed).standard_normal((n, n))
    return R + s * R.T


def _rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _sector_basis(n, s):
    """Columns: the orthonormal unit vectors of sector s of an n x n matrix."""
    cols = []
    for i in range(n):
        for j in range(i if s > 0 else i + 1, n):
            q = np.zeros((n, n))
            if i == j:
                q[i, i] = 1.0
            else:
                q[i, j] = np.sqrt(0.5)
                q[j, i] = s * np.sqrt(0.5)
            cols.append(q.reshape(-1))
    return np.array(cols).T


CASES = {
    "full8": lambda: si.workload("full8"),
    "h2o29_120": lambda: si.workload("h2o29", n_unique=120),
    "scale36_90": lambda: si.workload("scale36", n_unique=90),
}


@pytest.mark.parametrize("sector", [1, -1])
@pytest.mark.parametrize("name", sorted(CASES))
def test_spin_flip_sigma_matches_oracle(sqd, ctx, name, sector):
    w = CASES[name]()
    n = w.strings_a.size
    assert w.strings_b is w.strings_a or np.array_equal(w.strings_a, w.strings_b)
    t = _tables(sqd, ctx, w)
    Ch = _sector_vector(n, 4, sector)
    C = torch.tensor(Ch, device="cuda")
    general = sqd.sigma(ctx, t, C).cpu().numpy()
    t.set_spin_flip(sector)
    S = sqd.sigma(ctx, t, C).cpu().numpy()
    ref = oracle.sigma(w.norb, w.h, w.V, 0.0, w.strings_a, w.strings_b, Ch.reshape(-1))
    assert _rel_l2(S.reshape(-1), ref) <= SIGMA_TOL
    assert _rel_l2(S, general) <= SIGMA_TOL
    t.set_spin_flip(0)  # back to the general product
    assert _rel_l2(sqd.sigma(ctx, t, C).cpu().numpy(), general) <= 1e-14
    t.close()


@pytest.mark.parametrize("name,sector", [("h2o29", 1), ("scale36", -1)])
def test_spin_flip_sigma_full_size_sampled_rows(sqd, ctx, name, sector):
    w = si.workload(name)
    n = w.strings_a.size
    t = _tables(sqd, ctx, w)
    t.set_spin_flip(sector)
    R = torch.tensor(si.random_vectors(1, w.ndet, 13)[0].reshape(n, n), device="cuda")
    C = R + sector * R.T
    del R
    S = sqd.sigma(ctx, t, C).cpu().numpy().reshape(-1)
    Ch = C.cpu().numpy().reshape(-1)
    del C
    rows = np.sort(np.random.default_rng(1).choice(w.ndet, size=400, replace=False))
    ref = oracle.sigma(w.norb, w.h, w.V, 0.0, w.strings_a, w.strings_b, Ch, rows=rows)
    assert _rel_l2(S[rows], ref) <= SIGMA_TOL
    t.close()


def test_spin_flip_needs_a_shared_string_set(sqd, ctx):
    w = si.workload("full8")
    t = _tables(sqd, ctx, w, shared=False)
    for sector in (1, -1):
        with pytest.raises(RuntimeError):
            t.set_spin_flip(sector)
    t.set_spin_flip(0)
    t.close()
    t = _tables(sqd, ctx, w)
    with pytest.raises(RuntimeError):
        t.set_spin_flip(2)
    t.close()


@pytest.mark.parametrize("name,nroots,sector", [
    ("full8", 1, 1), ("full8", 3, 1), ("full8", 2, -1), ("h2o29_70", 4, 1),
    ("h2o29_70", 4, -1), ("scale36_60", 1, -1), ("scale36_60", 2, 1)])
def test_spin_flip_davidson_vs_lapack_in_the_sector(sqd, ctx, name, nroots, sector):
    w = {"full8": lambda: si.workload("full8"),
         "h2o29_70": lambda: si.workload("h2o29", n_unique=70),
         "scale36_60": lambda: si.workload("scale36", n_unique=60)}[name]()
    n = w.strings_a.size
    H = oracle.dense_h(w.norb, w.h, w.V, 0.0, w.strings_a, w.strings_b)
    Q = _sector_basis(n, sector)
    ref = np.linalg.eigvalsh(Q.T @ H @ Q)[:nroots]
    t = _tables(sqd, ctx, w)
    t.set_spin_flip(sector)
    e, X, it, res, rc = sqd.davidson(ctx, t, nroots=nroots, tol_residual=1e-8, tol_energy=1e-11)
    assert np.max(np.abs(e - ref)) <= 1e-9
    Xh = X.cpu().numpy()
    for k in range(nroots):
        assert np.array_equal(Xh[k].T, sector * Xh[k])  # exactly in the sector
    Xf = Xh.reshape(nroots, -1)
    assert np.allclose(Xf @ Xf.T, np.eye(nroots), atol=1e-10)
    assert np.all(np.linalg.norm(Xf @ H - e[:, None] * Xf, axis=1) <= 1e-7)
    t.close()


def test_spin_flip_ground_state_h2o29_matches_general_solve(sqd, ctx):
    w = si.workload("h2o29")
    t = _tables(sqd, ctx, w)
    # the general solve starts on the lowest H_II at (Ia, Ib) = (0, 3), which
    # has a part in each sector; its lowest singlet and triplet lie close, so
    # it converges slowly: residual 1e-7 (energy error ~ |r|^2 / gap)
    opts = dict(nroots=1, tol_residual=1e-7, tol_energy=1e-10, max_iter=600)
    e0, X0, it0, _, _ = sqd.davidson(ctx, t, **opts)
    best = None
    for sector in (1, -1):
        t.set_spin_flip(sector)
        e1, X1, it1, r1, _ = sqd.davidson(ctx, t, **opts)
        assert r1[0] <= 1e-7
        if best is None or e1[0] < best[0]:
            best = (e1[0], X1[0].reshape(-1))
    assert abs(best[0] - e0[0]) <= 1e-9
    assert abs(abs(float(X0[0].reshape(-1) @ best[1])) - 1.0) <= 1e-8
    t.close()
