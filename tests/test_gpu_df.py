"""Double-float sigma mode (FP64 operands as float pairs, exact products,
error-free sums on the FP32 pipe) against the oracle and the native FP64
kernels.  Bars: sigma relative L2 <= 1e-12 against the oracle (the build's
sigma tolerance), <= 1e-13 against the FP64 kernels; energies |dE| <= 1e-10."""
import numpy as np
import pytest
import torch

import oracle
import sqd_inputs as si
from tests.test_gpu_parity import CASES, case, make_tables, dev_f64, rel_l2

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


@pytest.mark.parametrize("name", CASES)
def test_df_sigma_matches_oracle(sqd, ctx, name):
    norb, sa, na_e, sb, nb_e, h, V, ecore = case(name)
    t = make_tables(sqd, ctx, norb, sa, na_e, sb, nb_e, h, V, ecore)
    N = len(sa) * len(sb)
    C = si.random_vectors(2, N, 11)
    Cd = dev_f64(C.reshape(2, len(sa), len(sb)))
    s64 = sqd.sigma(ctx, t, Cd).cpu().numpy().reshape(2, N)
    t.set_sigma_mode(1)
    sdf = sqd.sigma(ctx, t, Cd).cpu().numpy().reshape(2, N)
    ref = oracle.sigma(norb, h, V, ecore, sa, sb, C)
    for v in range(2):
        assert rel_l2(sdf[v], ref[v]) <= 1e-12
        assert rel_l2(sdf[v], s64[v]) <= 1e-13
    t.close()


@pytest.mark.parametrize("name", ["h2o29", "scale36"])
def test_df_sigma_full_size_sampled_rows(sqd, ctx, name):
    w = si.workload(name)
    t = make_tables(sqd, ctx, w.norb, w.strings_a, w.nelec_a, w.strings_b, w.nelec_b, w.h, w.V)
    t.set_sigma_mode(1)
    N = w.ndet
    Ch = si.random_vectors(1, N, 13)[0]
    C = dev_f64(Ch.reshape(w.strings_a.size, -1))
    S = sqd.sigma(ctx, t, C).cpu().numpy().reshape(-1)
    del C
    rows = np.sort(np.random.default_rng(1).choice(N, size=400, replace=False))
    ref = oracle.sigma(w.norb, w.h, w.V, 0.0, w.strings_a, w.strings_b, Ch, rows=rows)
    assert rel_l2(S[rows], ref) <= 1e-12
    t.close()


def test_df_davidson_energies(sqd, ctx):
    w = si.workload("h2o29", n_unique=400)
    t = make_tables(sqd, ctx, 29, w.strings_a, 5, w.strings_b, 5, w.h, w.V)
    e64, _, _, _, _ = sqd.davidson(ctx, t, nroots=3, tol_residual=1e-8, tol_energy=1e-11)
    t.set_sigma_mode(1)
    edf, X, _, res, _ = sqd.davidson(ctx, t, nroots=3, tol_residual=1e-8, tol_energy=1e-11)
    assert np.max(np.abs(edf - e64)) <= 1e-10
    # residuals against the FP64 kernels
    t.set_sigma_mode(0)
    S = sqd.sigma(ctx, t, X)
    r = (S - torch.tensor(edf, device="cuda")[:, None, None] * X).reshape(3, -1).norm(dim=1)
    assert float(r.max()) <= 2e-8
    t.close()
