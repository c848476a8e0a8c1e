"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bars (stated here, used below):
* strings and excitation-table integer fields: bit-exact;
* excitation-table values and the diagonal: |d| <= 1e-13 (1 + |v|) -- the
  same Slater-Condon sums taken in another order;
* sigma: relative L2 error <= 1e-12 (the sigma tolerance of the build);
* energies: |dE| <= 1e-10 Ha against LAPACK on the full 8-orbital space,
  <= 1e-9 Ha elsewhere.
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


def dev_strings(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64), device="cuda")


def dev_f64(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def make_tables(sqd, ctx, norb, sa, na_e, sb, nb_e, h, V, ecore=0.0, shared=None):
    da = dev_strings(sa)
    db = da if (shared if shared is not None else sa is sb) else dev_strings(sb)
    return sqd.excitation_tables(ctx, norb, da, na_e, db, nb_e, dev_f64(h), dev_f64(V), ecore)


def case(name):
    """Small cases of every workload shape (the oracle finishes them in
    seconds) plus uneven alpha/beta sets."""
    if name == "full8":
        w = si.workload("full8")
        return w.norb, w.strings_a, 4, w.strings_b, 4, w.h, w.V, 0.0
    if name == "h2o29_small":
        w = si.workload("h2o29", n_unique=260)
        return w.norb, w.strings_a, 5, w.strings_b, 5, w.h, w.V, -3.5
    if name == "scale36_small":
        w = si.workload("scale36", n_unique=180)
        return w.norb, w.strings_a, 15, w.strings_b, 15, w.h, w.V, 0.0
    if name == "uneven":
        h, V = si.make_integrals(12, 24, 77)
        _, sa = si.sample_strings(12, 5, 90, si.weights_exp(12), 5)
        _, sb = si.sample_strings(12, 3, 70, si.weights_exp(12), 6)
        return 12, sa, 5, sb, 3, h, V, 1.25
    if name == "norb64":
        h, V = si.make_integrals(64, 4, 3)
        _, sa = si.sample_strings(64, 3, 40, si.weights_exp(64, 20.0), 8)
        return 64, sa, 3, sa, 3, h, V, 0.0
    raise KeyError(name)


CASES = ["full8", "h2o29_small", "scale36_small", "uneven", "norb64"]


# ------------------------------------------------------------------ a1 ---

@pytest.mark.parametrize("which", ["h2o29", "scale36", "junk", "tiny", "empty", "big"])
def test_build_strings_bit_exact(sqd, ctx, which):
    rng = np.random.default_rng(3)
    if which in ("h2o29", "scale36"):
        w = si.workload(which)
        raw, norb, ne = w.raw_a, w.norb, w.nelec_a
    elif which == "junk":
        norb, ne = 20, 6
        raw = rng.integers(0, 1 << 22, size=5000, dtype=np.uint64)  # wrong counts, high bits
        raw = np.concatenate([raw, si.sample_strings(20, 6, 300, si.weights_exp(20), 2)[0]])
    elif which == "tiny":
        norb, ne = 6, 3
        raw = np.array([0b000111], dtype=np.uint64)
    elif which == "empty":
        norb, ne = 6, 3
        raw = np.array([0b1, 0b11, 0b1111], dtype=np.uint64)  # none valid
    else:
        norb, ne = 40, 12
        raw, _ = si.sample_strings(40, 12, 150000, si.weights_fermi(40, 12.0, 3.0), 9)
    got = sqd.build_strings(ctx, dev_strings(raw), norb, ne).cpu().numpy().view(np.uint64)
    ref = oracle.build_strings(raw, norb, ne)
    assert np.array_equal(got, ref)


# -------------------------------------------------------------- a2-a4 ---

@pytest.mark.parametrize("name", CASES)
def test_tables_bit_exact(sqd, ctx, name):
    norb, sa, na_e, sb, nb_e, h, V, ecore = case(name)
    t = make_tables(sqd, ctx, norb, sa, na_e, sb, nb_e, h, V, ecore)
    for spin, s in ((0, sa), (1, sb)):
        for kind in (1, 2):
            g = t.export(spin, kind)
            r = oracle.excitations(norb, h, V, s, kind)
            assert np.array_equal(g["off"], r["off"])
            assert np.array_equal(g["tgt"], r["tgt"])
            assert np.array_equal(g["orb"], r["orb"])
            assert np.array_equal(g["sign"], r["sign"])
            assert np.all(np.abs(g["val"] - r["val"]) <= 1e-13 * (1 + np.abs(r["val"])))
    d = sqd.diagonal(ctx, t).cpu().numpy().reshape(-1)
    dr = oracle.diag(norb, h, V, ecore, sa, sb)
    assert np.all(np.abs(d - dr) <= 1e-13 * (1 + np.abs(dr)))
    t.close()


def test_tables_match_golden_digest(sqd, ctx):
    # the full-size h2o29 lists against the stored oracle digest
    from tests.golden import make_golden as mg
    ref = mg.read_tables()
    w = si.workload("h2o29")
    t = make_tables(sqd, ctx, w.norb, w.strings_a, 5, w.strings_b, 5, w.h, w.V)
    for kind, name in ((1, "singles"), (2, "doubles")):
        g = t.export(0, kind)
        orb = np.asarray(g["orb"], dtype=np.int64).reshape(len(g["tgt"]), -1)
        got = {"nnz": int(g["off"][-1]), "max_per_string": int(np.diff(g["off"]).max()),
               "sum_target": int(np.sum(g["tgt"], dtype=np.int64)),
               "sum_sign": int(np.sum(g["sign"], dtype=np.int64)),
               "sum_orbital_code": int(np.sum(orb * np.arange(1, orb.shape[1] + 1),
                                              dtype=np.int64))}
        for key, val in got.items():
            assert ref["%s.%s" % (name, key)] == val, (name, key)
    t.close()


def test_tables_info_counts(sqd, ctx):
    norb, sa, na_e, sb, nb_e, h, V, ecore = case("uneven")
    t = make_tables(sqd, ctx, norb, sa, na_e, sb, nb_e, h, V, ecore)
    info = t.info()
    assert info["shared"] == 0
    assert info["nnz1_alpha"] == oracle.excitations(norb, h, V, sa, 1)["off"][-1]
    assert info["nnz2_beta"] == oracle.excitations(norb, h, V, sb, 2)["off"][-1]


# ------------------------------------------------------------- sigma -----

def rel_l2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("name", CASES)
def test_sigma_matches_oracle(sqd, ctx, name):
    norb, sa, na_e, sb, nb_e, h, V, ecore = case(name)
    t = make_tables(sqd, ctx, norb, sa, na_e, sb, nb_e, h, V, ecore)
    N = len(sa) * len(sb)
    C = si.random_vectors(2, N, 11)
    got = sqd.sigma(ctx, t, dev_f64(C.reshape(2, len(sa), len(sb)))).cpu().numpy().reshape(2, N)
    ref = oracle.sigma(norb, h, V, ecore, sa, sb, C)
    for v in range(2):
        assert rel_l2(got[v], ref[v]) <= SIGMA_TOL
    t.close()


def test_sigma_columns_are_hamiltonian_columns(sqd, ctx):
    # sigma(e_J) = H[:, J] for a few unit vectors, against the dense oracle H
    norb, sa, na_e, sb, nb_e, h, V, ecore = case("uneven")
    t = make_tables(sqd, ctx, norb, sa, na_e, sb, nb_e, h, V, ecore)
    H = oracle.dense_h(norb, h, V, ecore, sa, sb)
    N = H.shape[0]
    for J in (0, 17, N // 2, N - 1):
        e = np.zeros(N)
        e[J] = 1.0
        got = sqd.sigma(ctx, t, dev_f64(e.reshape(len(sa), len(sb)))).cpu().numpy().reshape(-1)
        assert np.max(np.abs(got - H[:, J])) <= 1e-13
    t.close()


@pytest.mark.parametrize("name", ["h2o29", "adjoint29", "scale36"])
def test_sigma_full_size_sampled_rows(sqd, ctx, name):
    w = si.workload(name)
    t = make_tables(sqd, ctx, w.norb, w.strings_a, w.nelec_a, w.strings_b, w.nelec_b, w.h, w.V)
    N = w.ndet
    Ch = si.random_vectors(1, N, 13)[0]
    C = dev_f64(Ch.reshape(w.strings_a.size, -1))
    S = sqd.sigma(ctx, t, C).cpu().numpy().reshape(-1)
    del C
    rows = np.sort(np.random.default_rng(1).choice(N, size=400, replace=False))
    ref = oracle.sigma(w.norb, w.h, w.V, 0.0, w.strings_a, w.strings_b, Ch, rows=rows)
    assert rel_l2(S[rows], ref) <= SIGMA_TOL
    t.close()


def test_sigma_hermitian_full_size(sqd, ctx):
    w = si.workload("h2o29")
    t = make_tables(sqd, ctx, w.norb, w.strings_a, 5, w.strings_b, 5, w.h, w.V)
    shape = (w.strings_a.size, w.strings_b.size)
    x = dev_f64(si.random_vectors(1, w.ndet, 21).reshape(shape))
    y = dev_f64(si.random_vectors(1, w.ndet, 22).reshape(shape))
    Hx, Hy = sqd.sigma(ctx, t, x), sqd.sigma(ctx, t, y)
    a = float((x * Hy).sum())
    b = float((Hx * y).sum())
    assert abs(a - b) <= 1e-12 * float(Hx.norm() * y.norm())
    t.close()


# ----------------------------------------------------------- Davidson ----

def test_davidson_full8_vs_lapack(sqd, ctx):
    norb, sa, na_e, sb, nb_e, h, V, ecore = case("full8")
    t = make_tables(sqd, ctx, norb, sa, na_e, sb, nb_e, h, V, ecore)
    H = oracle.dense_h(norb, h, V, ecore, sa, sb)
    ref = np.linalg.eigvalsh(H)
    e, X, it, res, rc = sqd.davidson(ctx, t, nroots=1, tol_residual=1e-8, tol_energy=1e-12)
    assert abs(e[0] - ref[0]) <= 1e-10
    x = X.cpu().numpy().reshape(-1)
    assert abs(np.linalg.norm(x) - 1) <= 1e-12
    assert np.linalg.norm(H @ x - e[0] * x) <= 1e-8
    e3, X3, _, _, _ = sqd.davidson(ctx, t, nroots=3, tol_residual=1e-8, tol_energy=1e-12)
    assert np.max(np.abs(e3 - ref[:3])) <= 1e-10
    t.close()


@pytest.mark.parametrize("name", ["uneven", "h2o29_70"])
def test_davidson_multiroot_vs_lapack(sqd, ctx, name):
    if name == "h2o29_70":
        w = si.workload("h2o29", n_unique=70)
        norb, sa, na_e, sb, nb_e, h, V, ecore = w.norb, w.strings_a, 5, w.strings_b, 5, w.h, w.V, 0.0
    else:
        norb, sa, na_e, sb, nb_e, h, V, ecore = case(name)
    t = make_tables(sqd, ctx, norb, sa, na_e, sb, nb_e, h, V, ecore)
    H = oracle.dense_h(norb, h, V, ecore, sa, sb)
    ref = np.linalg.eigvalsh(H)[:4]
    e, X, it, res, rc = sqd.davidson(ctx, t, nroots=4, tol_residual=1e-8, tol_energy=1e-11)
    assert np.max(np.abs(e - ref)) <= 1e-9
    Xh = X.cpu().numpy().reshape(4, -1)
    assert np.allclose(Xh @ Xh.T, np.eye(4), atol=1e-10)
    assert np.all(np.linalg.norm(Xh @ H - e[:, None] * Xh, axis=1) <= 1e-7)
    t.close()


def test_davidson_full8_golden(sqd, ctx):
    from tests.golden import make_golden as mg
    w = si.workload("full8")
    t = make_tables(sqd, ctx, w.norb, w.strings_a, 4, w.strings_b, 4, w.h, w.V)
    e, X, it, res, rc = sqd.davidson(ctx, t, nroots=4, tol_residual=1e-8, tol_energy=1e-12)
    assert np.max(np.abs(e - mg.read_full8())) <= 1e-10
    t.close()


def test_davidson_exhausts_tiny_space(sqd, ctx):
    # 36 determinants, 6 roots, a subspace as large as the space: the new
    # blocks become linearly dependent on the basis and vectors are dropped
    # inside a block; the energies must still be the exact lowest six
    norb = 4
    s = si.full_strings(norb, 2)
    h, V = si.make_integrals(norb, 8, 77)
    t = make_tables(sqd, ctx, norb, s, 2, s, 2, h, V)
    H = oracle.dense_h(norb, h, V, 0.0, s, s)
    ref = np.linalg.eigvalsh(H)[:6]
    e, X, it, res, rc = sqd.davidson(ctx, t, nroots=6, tol_residual=1e-9, tol_energy=1e-12,
                                     max_subspace=36)
    assert np.max(np.abs(e - ref)) <= 1e-10
    Xh = X.cpu().numpy().reshape(6, -1)
    assert np.allclose(Xh @ Xh.T, np.eye(6), atol=1e-10)
    t.close()


def test_davidson_guess_block_dependent(sqd, ctx):
    # a guess block with two equal vectors is rejected; an exact eigenvector
    # guess converges at once to the same energy
    w = si.workload("full8")
    t = make_tables(sqd, ctx, w.norb, w.strings_a, 4, w.strings_b, 4, w.h, w.V)
    H = oracle.dense_h(w.norb, w.h, w.V, 0.0, w.strings_a, w.strings_b)
    ev, U = np.linalg.eigh(H)
    g = np.stack([U[:, 0], U[:, 0]]).reshape(2, 70, 70)
    with pytest.raises(sqd.SQDError):
        sqd.davidson(ctx, t, nroots=2, guess=dev_f64(g))
    g = np.stack([U[:, 0], U[:, 1]]).reshape(2, 70, 70)
    e, X, it, res, rc = sqd.davidson(ctx, t, nroots=2, guess=dev_f64(g), tol_residual=1e-8,
                                     tol_energy=1e-10)
    assert np.max(np.abs(e - ev[:2])) <= 1e-10 and it <= 2
    t.close()


def test_davidson_outputs_consistent_when_stopped_early(sqd, ctx):
    # stopped by max_iter: the returned vectors, energies and residual norms
    # must still belong together (Ritz pairs of the final basis)
    w = si.workload("h2o29", n_unique=70)
    t = make_tables(sqd, ctx, w.norb, w.strings_a, 5, w.strings_b, 5, w.h, w.V)
    H = oracle.dense_h(w.norb, w.h, w.V, 0.0, w.strings_a, w.strings_b)
    for iters in (2, 7, 15):
        e, X, it, res, rc = sqd.davidson(ctx, t, nroots=4, tol_residual=1e-12, tol_energy=1e-14,
                                         max_iter=iters, raise_on_nonconvergence=False)
        assert rc == sqd.SQD_ENOTCONVERGED and it == iters
        Xh = X.cpu().numpy().reshape(4, -1)
        assert np.allclose(Xh @ Xh.T, np.eye(4), atol=1e-10)
        r = np.linalg.norm(Xh @ H - e[:, None] * Xh, axis=1)
        assert np.allclose(r, res, rtol=1e-6, atol=1e-12)
        assert np.allclose(np.einsum("ij,jk,ik->i", Xh, H, Xh), e, rtol=0, atol=1e-10)
    t.close()


@pytest.mark.parametrize("name", ["uneven", "h2o29_70"])
def test_davidson_olsen_vs_lapack_and_oracle(sqd, ctx, name):
    if name == "h2o29_70":
        w = si.workload("h2o29", n_unique=70)
        norb, sa, na_e, sb, nb_e, h, V, ecore = w.norb, w.strings_a, 5, w.strings_b, 5, w.h, w.V, 0.0
    else:
        norb, sa, na_e, sb, nb_e, h, V, ecore = case(name)
    t = make_tables(sqd, ctx, norb, sa, na_e, sb, nb_e, h, V, ecore)
    H = oracle.dense_h(norb, h, V, ecore, sa, sb)
    ref = np.linalg.eigvalsh(H)[:4]
    e, X, it, res, rc = sqd.davidson(ctx, t, nroots=4, tol_residual=1e-8, tol_energy=1e-11,
                                     correction="olsen")
    assert rc == 0 and np.max(np.abs(e - ref)) <= 1e-9
    Xh = X.cpu().numpy().reshape(4, -1)
    assert np.all(np.linalg.norm(Xh @ H - e[:, None] * Xh, axis=1) <= 1e-7)
    hd = oracle.diag(norb, h, V, ecore, sa, sb)
    th, _, _, _, conv = oracle.davidson(lambda Y: H @ Y, hd, nroots=4, tol_residual=1e-8,
                                        tol_energy=1e-11, correction="olsen")
    assert conv and np.max(np.abs(e - th)) <= 1e-9
    t.close()


def test_davidson_matches_oracle_davidson(sqd, ctx):
    # same algorithm on the oracle side (matrix-free oracle sigma)
    w = si.workload("h2o29", n_unique=120)
    norb, sa, sb = w.norb, w.strings_a, w.strings_b
    t = make_tables(sqd, ctx, norb, sa, 5, sb, 5, w.h, w.V)
    hd = oracle.diag(norb, w.h, w.V, 0.0, sa, sb)
    th, Xo, _, _, conv = oracle.davidson(
        lambda X: oracle.sigma(norb, w.h, w.V, 0.0, sa, sb, X.T).T, hd, nroots=2,
        tol_residual=1e-8, tol_energy=1e-10)
    assert conv
    e, X, it, res, rc = sqd.davidson(ctx, t, nroots=2, tol_residual=1e-8, tol_energy=1e-10)
    assert np.max(np.abs(e - th)) <= 1e-9
    t.close()


def test_davidson_h2o29_eight_roots(sqd, ctx):
    w = si.workload("h2o29")
    t = make_tables(sqd, ctx, w.norb, w.strings_a, 5, w.strings_b, 5, w.h, w.V)
    e, X, it, res, rc = sqd.davidson(ctx, t, nroots=8, tol_residual=1e-8, tol_energy=1e-8)
    assert rc == 0 and np.all(res <= 1e-8)
    assert np.all(np.diff(e) >= -1e-12)
    # residuals recomputed independently through sigma, orthonormality
    S = sqd.sigma(ctx, t, X)
    Xf, Sf = X.reshape(8, -1), S.reshape(8, -1)
    r = (Sf - torch.tensor(e, device="cuda")[:, None] * Xf).norm(dim=1).cpu().numpy()
    assert np.all(r <= 2e-8)
    G = (Xf @ Xf.T).cpu().numpy()
    assert np.allclose(G, np.eye(8), atol=1e-10)
    # variational: every Ritz value lies above the exact eigenvalue it
    # approximates, which is above the lowest diagonal element's bound
    assert e[0] <= float(sqd.diagonal(ctx, t).min())
    t.close()


# ------------------------------------------------------------- errors ----

def test_fp64_probes(sqd, ctx):
    # the FP64 rates the roofline is read against: positive, and not above
    # the nominal 4 flop/clk/SM of the FP64 pipe at the highest SM clock
    dfma, dmma = ctx.measure_fp64_peaks()
    props = torch.cuda.get_device_properties(0)
    bound = props.multi_processor_count * 4 * 2.2e9 / 1e12
    assert 0.0 < dfma <= bound and 0.0 < dmma <= 4 * bound


def test_errors_are_status_codes(sqd, ctx):
    norb, sa, na_e, sb, nb_e, h, V, ecore = case("uneven")
    bad_count = np.unique(np.append(sa, np.uint64(0b111111)))  # a 6-electron string
    with pytest.raises(sqd.SQDError) as ei:
        make_tables(sqd, ctx, norb, bad_count, na_e, sb, nb_e, h, V, ecore)
    assert ei.value.code == sqd.SQD_EINVAL
    with pytest.raises(sqd.SQDError):  # unsorted
        make_tables(sqd, ctx, norb, sa[::-1].copy(), na_e, sb, nb_e, h, V, ecore)
    Vb = V.copy()
    Vb[0, 1, 2, 3] += 1e-3
    with pytest.raises(sqd.SQDError):  # asymmetric integrals
        make_tables(sqd, ctx, norb, sa, na_e, sb, nb_e, h, Vb, ecore)
    hb = h.copy()
    hb[1, 1] = np.nan
    with pytest.raises(sqd.SQDError):
        make_tables(sqd, ctx, norb, sa, na_e, sb, nb_e, hb, V, ecore)
    with pytest.raises(sqd.SQDError):
        sqd.build_strings(ctx, dev_strings(sa), 65, 3)
    with pytest.raises(sqd.SQDError):
        sqd.build_strings(ctx, dev_strings(sa), 12, 13)
    t = make_tables(sqd, ctx, norb, sa, na_e, sb, nb_e, h, V, ecore)
    e, X, it, res, rc = sqd.davidson(ctx, t, nroots=2, max_iter=1,
                                     raise_on_nonconvergence=False)
    assert rc == sqd.SQD_ENOTCONVERGED and np.all(np.isfinite(e))
    with pytest.raises(sqd.SQDError):
        sqd.davidson(ctx, t, nroots=2, max_iter=1)
    with pytest.raises(sqd.SQDError):
        sqd.davidson(ctx, t, nroots=0)
    t.close()


def test_single_determinant_space(sqd, ctx):
    h, V = si.make_integrals(6, 6, 1)
    s = np.array([0b000111], dtype=np.uint64)
    t = make_tables(sqd, ctx, 6, s, 3, s, 3, h, V, 0.5)
    e, X, it, res, rc = sqd.davidson(ctx, t, nroots=1)
    assert abs(e[0] - oracle.diag(6, h, V, 0.5, s, s)[0]) <= 1e-13
    assert float(X.abs().sum()) == 1.0
    t.close()


def test_sigma_run_to_run_spread(sqd, ctx):
    # the paired-singles term adds its entry sums into sigma with FP64
    # atomics, so the summation order (not the terms) varies between runs:
    # two products of the same vector agree to a few units of rounding
    w = si.workload("adjoint29")
    t = make_tables(sqd, ctx, w.norb, w.strings_a, 5, w.strings_b, 5, w.h, w.V)
    C = dev_f64(si.random_vectors(1, w.ndet, 31).reshape(w.strings_a.size, -1))
    S1 = sqd.sigma(ctx, t, C)
    S2 = sqd.sigma(ctx, t, C)
    d = float((S1 - S2).abs().max())
    assert d <= 1e-14 * float(S1.abs().max())
    assert float((S1 - S2).norm()) <= 1e-14 * float(S1.norm())
    t.close()
