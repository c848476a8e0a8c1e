"""Reduced density matrices, the orbital gradient and the autograd adjoint
on the GPU, against the oracle and against finite differences.

The oracle receives only seeded inputs: RDM parity uses random normalised
vectors from sqd_inputs (an RDM is defined for any state).  Properties that
need an eigenvector (energy from the RDMs, Hellmann-Feynman) compare the GPU
path with itself through independent routes (Davidson energies, finite
differences of re-solved energies).
Bars: RDM entries |d| <= 1e-12 (sums of ~1e4-1e7 products of O(1) numbers);
FD |FD - analytic| <= 1e-6 max(1, |analytic|) (step 1e-5).
"""
import numpy as np
import pytest
import torch

import oracle
import sqd_inputs as si

pytestmark = pytest.mark.gpu


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


def dev_s(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64), device="cuda")


def dev_f(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def tables(sqd, ctx, norb, sa, na_e, sb, nb_e, h, V, ecore=0.0):
    da = dev_s(sa)
    db = da if sa is sb else dev_s(sb)
    return sqd.excitation_tables(ctx, norb, da, na_e, db, nb_e, dev_f(h), dev_f(V), ecore)


def unit_vector(n, seed):
    c = si.random_vectors(1, n, seed)[0]
    return c / np.linalg.norm(c)


CASES = {
    "full8": lambda: (si.workload("full8"), None),
    "uneven": lambda: (None, "uneven"),
}


def small(name):
    if name == "full8":
        w = si.workload("full8")
        return w.norb, w.strings_a, 4, w.strings_b, 4, w.h, w.V
    h, V = si.make_integrals(7, 14, 71)
    _, sa = si.sample_strings(7, 3, 25, si.weights_exp(7), 4)
    _, sb = si.sample_strings(7, 2, 15, si.weights_exp(7), 5)
    return 7, sa, 3, sb, 2, h, V


@pytest.mark.parametrize("name", ["full8", "uneven"])
def test_rdm_matches_oracle_full(sqd, ctx, name):
    norb, sa, na_e, sb, nb_e, h, V = small(name)
    t = tables(sqd, ctx, norb, sa, na_e, sb, nb_e, h, V)
    c = unit_vector(len(sa) * len(sb), 31)
    g1, g2 = sqd.rdm(ctx, t, dev_f(c.reshape(len(sa), len(sb))))
    r1 = oracle.rdm1(norb, sa, sb, c)
    r2 = oracle.rdm2(norb, sa, sb, c)
    assert np.max(np.abs(g1.cpu().numpy() - r1)) <= 1e-12
    assert np.max(np.abs(g2.cpu().numpy() - r2)) <= 1e-12
    t.close()


def _entries(rng, norb, k):
    quads = [tuple(int(x) for x in rng.integers(0, norb, 4)) for _ in range(k)]
    quads += [(0, 0, 1, 1), (1, 0, 0, 1), (2, 3, 3, 2), (0, 1, 0, 1), (4, 4, 4, 4)]
    return quads


@pytest.mark.parametrize("name", ["h2o29", "adjoint29"])
def test_rdm_sampled_entries_full_size(sqd, ctx, name):
    w = si.workload(name)
    t = tables(sqd, ctx, w.norb, w.strings_a, 5, w.strings_b, 5, w.h, w.V)
    n = w.strings_a.size
    c = unit_vector(w.ndet, 41)
    g1, g2 = sqd.rdm(ctx, t, dev_f(c.reshape(n, n)))
    g1, g2 = g1.cpu().numpy(), g2.cpu().numpy()
    rng = np.random.default_rng(7)
    k1 = 12 if name == "adjoint29" else 30
    pairs = [tuple(int(x) for x in rng.integers(0, w.norb, 2)) for _ in range(k1)] + [(0, 0), (3, 5)]
    r1 = oracle.rdm1(w.norb, w.strings_a, w.strings_b, c, entries=pairs)
    assert np.max(np.abs(np.array([g1[p] for p in pairs]) - r1)) <= 1e-12
    quads = _entries(rng, w.norb, 12 if name == "adjoint29" else 30)
    r2 = oracle.rdm2(w.norb, w.strings_a, w.strings_b, c, entries=quads)
    assert np.max(np.abs(np.array([g2[q] for q in quads]) - r2)) <= 1e-12
    # identities that hold for any normalised state with 10 electrons
    assert abs(np.trace(g1) - 10.0) <= 1e-10
    assert np.allclose(np.einsum("pqrr->pq", g2), 9.0 * g1, atol=1e-10)
    assert np.allclose(g2, g2.transpose(2, 3, 0, 1), atol=1e-12)
    t.close()


def _energy(sqd, ctx, norb, sa, na_e, sb, nb_e, h, V, tol=1e-10, guess=None):
    t = tables(sqd, ctx, norb, sa, na_e, sb, nb_e, h, V)
    e, C, it, res, rc = sqd.davidson(ctx, t, nroots=1, tol_residual=tol, tol_energy=1e-13,
                                     max_iter=500, guess=guess)
    return e[0], C, t


def test_energy_from_rdms_and_hellmann_feynman(sqd, ctx):
    w = si.workload("h2o29", n_unique=150)
    norb, sa, sb = w.norb, w.strings_a, w.strings_b
    e0, C, t = _energy(sqd, ctx, norb, sa, 5, sb, 5, w.h, w.V)
    g1, g2 = sqd.rdm(ctx, t, C[0].contiguous())
    g1, g2 = g1.cpu().numpy(), g2.cpu().numpy()
    assert abs(oracle.energy_from_rdms(w.h, w.V, 0.0, g1, g2) - e0) <= 1e-9
    rng = np.random.default_rng(3)
    step = 1e-5
    for _ in range(3):
        p, q = (int(x) for x in rng.integers(0, norb, 2))
        d = np.zeros_like(w.h)
        d[p, q] = d[q, p] = 1.0
        ep, _, tp = _energy(sqd, ctx, norb, sa, 5, sb, 5, w.h + step * d, w.V)
        em, _, tm = _energy(sqd, ctx, norb, sa, 5, sb, 5, w.h - step * d, w.V)
        tp.close(); tm.close()
        an = g1[p, q] + (g1[q, p] if p != q else 0.0)
        assert abs((ep - em) / (2 * step) - an) <= 1e-6 * max(1.0, abs(an))
    t.close()


def test_orbital_gradient_matches_oracle_formula(sqd, ctx):
    norb, sa, na_e, sb, nb_e, h, V = small("uneven")
    t = tables(sqd, ctx, norb, sa, na_e, sb, nb_e, h, V)
    c = unit_vector(len(sa) * len(sb), 51)
    g1, g2 = sqd.rdm(ctx, t, dev_f(c.reshape(len(sa), len(sb))))
    g = sqd.orbital_gradient(ctx, t, g1, g2).cpu().numpy()
    ref = oracle.orbital_gradient(h, V, oracle.rdm1(norb, sa, sb, c), oracle.rdm2(norb, sa, sb, c))
    assert np.max(np.abs(g - ref)) <= 1e-11
    t.close()


def test_orbital_gradient_finite_differences(sqd, ctx):
    import scipy.linalg
    w = si.workload("h2o29", n_unique=60)
    norb, sa, sb = w.norb, w.strings_a, w.strings_b
    e0, C, t = _energy(sqd, ctx, norb, sa, 5, sb, 5, w.h, w.V)
    g1, g2 = sqd.rdm(ctx, t, C[0].contiguous())
    g = sqd.orbital_gradient(ctx, t, g1, g2).cpu().numpy()
    step = 1e-5
    for p, q in [(0, 5), (3, 11), (7, 2)]:
        K = np.zeros((norb, norb))
        K[p, q], K[q, p] = 1.0, -1.0
        es = []
        for sgn in (1, -1):
            U = scipy.linalg.expm(sgn * step * K)
            h2, V2 = oracle.rotate_integrals(w.h, w.V, U)
            V2 = 0.5 * (V2 + V2.transpose(1, 0, 2, 3))
            V2 = 0.5 * (V2 + V2.transpose(0, 1, 3, 2))
            V2 = 0.5 * (V2 + V2.transpose(2, 3, 0, 1))
            h2 = 0.5 * (h2 + h2.T)
            e, _, tt = _energy(sqd, ctx, norb, sa, 5, sb, 5, h2, V2)
            tt.close()
            es.append(e)
        fd = (es[0] - es[1]) / (2 * step)
        assert abs(fd - g[p, q]) <= 1e-6 * max(1.0, abs(g[p, q]))
    t.close()


def test_autograd_function(sqd, ctx):
    w = si.workload("h2o29", n_unique=80)
    s = dev_s(w.strings_a)
    h = dev_f(w.h).requires_grad_(True)
    V = dev_f(w.V).requires_grad_(True)
    E = sqd.SQDEnergy.apply(h, V, ctx, s, 5, s, 5)
    E.backward()
    t = tables(sqd, ctx, w.norb, w.strings_a, 5, w.strings_a, 5, w.h, w.V)
    e, C, it, res, rc = sqd.davidson(ctx, t, nroots=1, tol_residual=1e-9, tol_energy=1e-12)
    g1, g2 = sqd.rdm(ctx, t, C[0].contiguous())
    assert abs(float(E.detach()) - e[0]) <= 1e-9
    assert torch.allclose(h.grad, g1, atol=1e-8)
    assert torch.allclose(V.grad, 0.5 * g2, atol=1e-8)
    t.close()


def test_adjoint29_finite_differences_20_entries(sqd, ctx):
    # converged ground state of the 2.5e7-determinant space, then dE/dh and
    # dE/dV by central differences (step 1e-5) on 20 random integral entries
    # (symmetry orbits moved together) against the RDMs
    w = si.workload("adjoint29")
    norb, sa = w.norb, w.strings_a
    # ||r|| <= 1e-8 keeps the RDM error near 1e-8; the perturbed energies need
    # only ||r|| <= 1e-7 (energy error ~ ||r||^2 / gap, far below 1e-12)
    e0, C, t = _energy(sqd, ctx, norb, sa, 5, sa, 5, w.h, w.V, tol=1e-8)
    g1, g2 = sqd.rdm(ctx, t, C[0].contiguous())
    g1, g2 = g1.cpu().numpy(), g2.cpu().numpy()
    t.close()
    assert abs(oracle.energy_from_rdms(w.h, w.V, 0.0, g1, g2) - e0) <= 1e-9
    rng = np.random.default_rng(20)
    step = 1e-5
    for i in range(20):
        if i < 10:
            p, q = (int(x) for x in rng.integers(0, norb, 2))
            D = np.zeros_like(w.h)
            D[p, q] = D[q, p] = 1.0
            an = g1[p, q] + (g1[q, p] if p != q else 0.0)
            args = lambda s_: (w.h + s_ * D, w.V)
        else:
            p, q, r, s = (int(x) for x in rng.integers(0, norb, 4))
            orbit = set()
            for a, b, c2, d in [(p, q, r, s), (q, p, r, s), (p, q, s, r), (q, p, s, r)]:
                orbit.add((a, b, c2, d))
                orbit.add((c2, d, a, b))
            D = np.zeros_like(w.V)
            for o in orbit:
                D[o] = 1.0
            an = 0.5 * sum(g2[o] for o in orbit)
            args = lambda s_: (w.h, w.V + s_ * D)
        # warm start from the unperturbed ground state
        ep, _, tp = _energy(sqd, ctx, norb, sa, 5, sa, 5, *args(step), tol=1e-7, guess=C)
        tp.close()
        em, _, tm = _energy(sqd, ctx, norb, sa, 5, sa, 5, *args(-step), tol=1e-7, guess=C)
        tm.close()
        fd = (ep - em) / (2 * step)
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (i, fd, an)
