"""Stored-H variant (the paper's second method: H assembled once and
re-used) against the matrix-free sigma and the oracle.  Bars: sigma relative
L2 <= 1e-12, energies |dE| <= 1e-9."""
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


def _tables(sqd, ctx, norb, sa, na_e, sb, nb_e, h, V, ecore=0.0):
    da = torch.tensor(sa.view(np.int64), device="cuda")
    db = da if sa is sb else torch.tensor(sb.view(np.int64), device="cuda")
    return sqd.excitation_tables(ctx, norb, da, na_e, db, nb_e, torch.tensor(h, device="cuda"),
                                 torch.tensor(V, device="cuda"), ecore)


@pytest.mark.parametrize("name", ["uneven", "h2o29_300"])
def test_stored_sigma_matches_oracle_and_matrix_free(sqd, ctx, name):
    if name == "uneven":
        h, V = si.make_integrals(12, 24, 77)
        _, sa = si.sample_strings(12, 5, 90, si.weights_exp(12), 5)
        _, sb = si.sample_strings(12, 3, 70, si.weights_exp(12), 6)
        norb, na_e, nb_e, ecore = 12, 5, 3, 0.5
    else:
        w = si.workload("h2o29", n_unique=300)
        norb, sa, sb, na_e, nb_e, h, V, ecore = 29, w.strings_a, w.strings_b, 5, 5, w.h, w.V, 0.0
    t = _tables(sqd, ctx, norb, sa, na_e, sb, nb_e, h, V, ecore)
    nnz = sqd.stored_h_build(ctx, t)
    N = len(sa) * len(sb)
    # nonzero count = sum over rows of 1 + |H_a row| + |H_b row| + k1_a k1_b
    ta1, ta2 = oracle.excitations(norb, h, V, sa, 1), oracle.excitations(norb, h, V, sa, 2)
    tb1, tb2 = oracle.excitations(norb, h, V, sb, 1), oracle.excitations(norb, h, V, sb, 2)
    expect = (N + (ta1["off"][-1] + ta2["off"][-1]) * len(sb)
              + (tb1["off"][-1] + tb2["off"][-1]) * len(sa) + ta1["off"][-1] * tb1["off"][-1])
    assert nnz == expect
    C = si.random_vectors(2, N, 17)
    Cd = torch.tensor(C.reshape(2, len(sa), len(sb)), device="cuda")
    got = sqd.sigma_stored(ctx, t, Cd).cpu().numpy().reshape(2, N)
    mf = sqd.sigma(ctx, t, Cd).cpu().numpy().reshape(2, N)
    rows = np.arange(N) if N <= 20000 else np.sort(np.random.default_rng(0).choice(N, 3000, replace=False))
    ref = oracle.sigma(norb, h, V, ecore, sa, sb, C, rows=rows)
    for v in range(2):
        assert np.linalg.norm(got[v][rows] - ref[v]) <= 1e-12 * np.linalg.norm(ref[v])
        assert np.linalg.norm(got[v] - mf[v]) <= 1e-12 * np.linalg.norm(mf[v])
    t.close()


def test_stored_davidson_matches_matrix_free(sqd, ctx):
    w = si.workload("h2o29", n_unique=400)
    t = _tables(sqd, ctx, 29, w.strings_a, 5, w.strings_b, 5, w.h, w.V)
    sqd.stored_h_build(ctx, t)
    e1, X1, it1, _, _ = sqd.davidson(ctx, t, nroots=3, tol_residual=1e-8, tol_energy=1e-10,
                                     use_stored_h=True)
    e2, X2, it2, _, _ = sqd.davidson(ctx, t, nroots=3, tol_residual=1e-8, tol_energy=1e-10)
    assert np.max(np.abs(e1 - e2)) <= 1e-9
    t.close()


def test_stored_refuses_when_too_large(sqd, ctx):
    w = si.workload("h2o29", n_unique=300)
    t = _tables(sqd, ctx, 29, w.strings_a, 5, w.strings_b, 5, w.h, w.V)
    with pytest.raises(sqd.SQDError) as e:
        sqd.stored_h_build(ctx, t, max_bytes=1 << 20)
    assert e.value.code == sqd.SQD_ENOMEM
    with pytest.raises(sqd.SQDError):
        sqd.sigma_stored(ctx, t, torch.zeros((300, 300), dtype=torch.float64, device="cuda"))
    t.close()
