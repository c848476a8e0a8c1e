"""SQD outer-loop support on the GPU: string weights, carry-over selection
and warm-start mapping against the oracle, and a two-round SQD run.
Bars: weights and mapped vectors |d| <= 1e-13; selections bit-exact."""
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
    return torch.tensor(np.ascontiguousarray(a, np.uint64).view(np.int64), device="cuda")


def host_s(t):
    return t.cpu().numpy().view(np.uint64)


def test_weights_selection_mapping_match_oracle(sqd, ctx):
    w = si.workload("h2o29", n_unique=300)
    sa = dev_s(w.strings_a)
    t = sqd.excitation_tables(ctx, 29, sa, 5, sa, 5, torch.tensor(w.h, device="cuda"),
                              torch.tensor(w.V, device="cuda"))
    C = si.random_vectors(1, w.ndet, 3)[0]
    Cd = torch.tensor(C.reshape(300, 300), device="cuda")
    wa, wb = sqd.string_weights(ctx, t, Cd)
    ra, rb = oracle.string_weights(C, 300, 300)
    assert np.max(np.abs(wa.cpu().numpy() - ra)) <= 1e-13 * ra.max()
    assert np.max(np.abs(wb.cpu().numpy() - rb)) <= 1e-13 * rb.max()
    thr = float(np.quantile(ra, 0.6))
    keep = sqd.select_strings(ctx, sa, torch.tensor(ra, device="cuda"), thr)
    assert np.array_equal(host_s(keep), oracle.select_strings(w.strings_a, ra, thr))
    # map onto a different, overlapping set
    other = si.workload("h2o29", n_unique=450).strings_a
    M, nrm = sqd.map_vector(ctx, sa, sa, Cd, dev_s(other), dev_s(other))
    Mr, nr = oracle.map_vector(w.strings_a, w.strings_a, C, other, other)
    assert abs(nrm - nr) <= 1e-12 * nr
    assert np.max(np.abs(M.cpu().numpy() - Mr)) <= 1e-13
    t.close()


def test_two_sqd_rounds_with_carry_over(sqd, ctx):
    h, V = torch.tensor(si.workload("h2o29", n_unique=10).h, device="cuda"), None
    w1 = si.workload("h2o29", n_unique=250)
    V = torch.tensor(w1.V, device="cuda")
    # first SQD iteration
    s1 = sqd.build_strings(ctx, dev_s(w1.raw_a), 29, 5)
    t1 = sqd.excitation_tables(ctx, 29, s1, 5, s1, 5, h, V)
    e1, X1, it1, _, _ = sqd.davidson(ctx, t1, nroots=1, tol_residual=1e-7, tol_energy=1e-10)
    # carry every string (threshold 0) plus a fresh sample of 20 distinct
    # strings (a modest change of the set: the previous ground state is then a
    # good start; after a large extension it can be a worse start than the
    # lowest-diagonal determinant, which the CPU oracle's Davidson shows too)
    wa, _ = sqd.string_weights(ctx, t1, X1[0])
    carried = sqd.select_strings(ctx, s1, wa, 0.0)
    raw_new, _ = si.sample_strings(29, 5, 20, si.weights_exp(29), 77)
    raw2 = torch.cat([carried, dev_s(raw_new)])
    s2 = sqd.build_strings(ctx, raw2, 29, 5)
    assert np.all(np.isin(host_s(s1), host_s(s2)))  # old set kept
    t2 = sqd.excitation_tables(ctx, 29, s2, 5, s2, 5, h, V)
    guess, nrm = sqd.map_vector(ctx, s1, s1, X1[0].contiguous(), s2, s2)
    assert abs(nrm - 1.0) <= 1e-12  # every old determinant is in the new space
    e2w, _, it_w, _, _ = sqd.davidson(ctx, t2, nroots=1, tol_residual=1e-7, tol_energy=1e-10,
                                      guess=guess)
    e2c, _, it_c, _, _ = sqd.davidson(ctx, t2, nroots=1, tol_residual=1e-7, tol_energy=1e-10)
    assert abs(e2w - e2c)[0] <= 1e-9
    assert e2w[0] <= e1[0] + 1e-10  # a larger subspace cannot raise the energy
    assert it_w < it_c  # the carried state is a better start
    t1.close()
    t2.close()
