"""Pins of the CPU oracle against what the mathematics fixes.

None of these compares the oracle with itself: each reference is a closed
form, an operator construction that uses no excitation rules (Jordan-Wigner,
tests/_jw.py), a LAPACK routine, an identity of the reduced density
matrices, or a finite difference.  The paper (arXiv 2601.16169) prints no
worked numeric example, so there is no printed value to pin to; its
validation criterion is agreement to 1e-10 relative (Sections I and VI),
which every tolerance below is tighter than or equal to.
"""
import itertools

import numpy as np
import pytest

import oracle
import sqd_inputs as si
from tests import _jw

pytestmark = pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")


def _rand_strings(rng, norb, ne, k):
    full = si.full_strings(norb, ne)
    pick = rng.choice(len(full), size=min(k, len(full)), replace=False)
    return np.sort(full[pick])


def _nonsym_integrals(rng, norb):
    h = rng.normal(size=(norb, norb))
    V = rng.normal(size=(norb,) * 4)
    return h, V


# ------------------------------------------------------------ strings ------

def test_build_strings_definition():
    # norb 6, 3 electrons: keep distinct strings with 3 bits, all below bit 6.
    raw = np.array([0b000111, 0b101010, 0b000111, 0b1000011,  # last: bit 6 set
                    0b001111, 0b110001, 0b101010, 0b000011, 0b110001], dtype=np.uint64)
    got = oracle.build_strings(raw, 6, 3)
    assert got.tolist() == [0b000111, 0b101010, 0b110001]
    assert oracle.build_strings(np.zeros(0, np.uint64), 6, 3).size == 0


# ------------------------------------------------- Slater-Condon vs JW -----

@pytest.mark.parametrize("case", ["sym_full", "nonsym_full", "nonsym_sampled", "uneven"])
def test_dense_h_equals_jordan_wigner(case):
    rng = np.random.default_rng(11)
    if case == "sym_full":
        norb, na_e, nb_e = 4, 2, 2
        h, V = si.make_integrals(norb, 8, 5)
        sa, sb = si.full_strings(norb, na_e), si.full_strings(norb, nb_e)
    elif case == "nonsym_full":
        norb, na_e, nb_e = 4, 2, 2
        h, V = _nonsym_integrals(rng, norb)
        sa, sb = si.full_strings(norb, na_e), si.full_strings(norb, nb_e)
    elif case == "nonsym_sampled":
        norb, na_e, nb_e = 5, 3, 2
        h, V = _nonsym_integrals(rng, norb)
        sa, sb = _rand_strings(rng, norb, na_e, 7), _rand_strings(rng, norb, nb_e, 6)
    else:
        norb, na_e, nb_e = 5, 1, 3
        h, V = _nonsym_integrals(rng, norb)
        sa, sb = si.full_strings(norb, na_e), _rand_strings(rng, norb, nb_e, 8)
    ecore = 0.375
    Hf = _jw.hamiltonian(norb, h, V, ecore)
    ref = _jw.subspace_matrix(Hf, norb, sa, sb)
    got = oracle.dense_h(norb, h, V, ecore, sa, sb)
    assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_jw_pin_detects_transposed_integrals():
    # The pin is sensitive: the oracle fed V with two indices swapped (a
    # plausible transposition bug) must disagree with the true operator sum.
    rng = np.random.default_rng(3)
    norb = 4
    h, V = _nonsym_integrals(rng, norb)
    sa = sb = si.full_strings(norb, 2)
    ref = _jw.subspace_matrix(_jw.hamiltonian(norb, h, V), norb, sa, sb)
    bad = oracle.dense_h(norb, h, np.ascontiguousarray(V.transpose(1, 0, 2, 3)), 0.0, sa, sb)
    assert np.max(np.abs(bad - ref)) > 1e-3
    badh = oracle.dense_h(norb, np.ascontiguousarray(h.T), V, 0.0, sa, sb)
    assert np.max(np.abs(badh - ref)) > 1e-3


def test_sigma_equals_jordan_wigner_matvec():
    rng = np.random.default_rng(5)
    norb = 5
    h, V = si.make_integrals(norb, 10, 9)
    sa, sb = _rand_strings(rng, norb, 2, 8), _rand_strings(rng, norb, 3, 9)
    Hs = _jw.subspace_matrix(_jw.hamiltonian(norb, h, V, -1.25), norb, sa, sb)
    C = rng.normal(size=(3, len(sa) * len(sb)))
    got = oracle.sigma(norb, h, V, -1.25, sa, sb, C)
    ref = C @ Hs.T
    assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)
    rows = np.array([0, 5, 17, len(sa) * len(sb) - 1])
    got_r = oracle.sigma(norb, h, V, -1.25, sa, sb, C, rows=rows)
    assert np.allclose(got_r, ref[:, rows], rtol=0, atol=1e-13)


def test_diag_equals_jordan_wigner_diagonal():
    norb = 4
    h, V = si.make_integrals(norb, 8, 21)
    sa, sb = si.full_strings(norb, 2), si.full_strings(norb, 1)
    Hs = _jw.subspace_matrix(_jw.hamiltonian(norb, h, V, 0.5), norb, sa, sb)
    assert np.allclose(oracle.diag(norb, h, V, 0.5, sa, sb), np.diag(Hs), rtol=0, atol=1e-13)


# --------------------------------------------------- excitation tables -----

@pytest.mark.parametrize("kind", [1, 2])
def test_excitation_tables_vs_jordan_wigner(kind):
    rng = np.random.default_rng(kind)
    norb, ne = 6, 3
    h, V = si.make_integrals(norb, 12, 4)
    s = _rand_strings(rng, norb, ne, 14)
    t = oracle.excitations(norb, h, V, s, kind)
    # one-spin Hamiltonian from the alpha modes alone
    Hf = _jw.hamiltonian(norb, h, V, 0.0, spins=(0,))
    Hs = Hf[np.array(s, dtype=np.int64)][:, np.array(s, dtype=np.int64)].toarray()
    n = len(s)
    for i in range(n):
        row = range(t["off"][i], t["off"][i + 1])
        tg = [t["tgt"][e] for e in row]
        assert tg == sorted(tg)
        # completeness: every string at that excitation level is listed
        exp = [j for j in range(n) if bin(int(s[i]) ^ int(s[j])).count("1") == 2 * kind]
        assert tg == exp
        for e in row:
            j = t["tgt"][e]
            o = [int(x) for x in t["orb"][e]]
            if kind == 1:
                p, q = o
                op = _jw.operator_matrix(norb, [("c", p), ("a", q)])
                assert int(s[j]) == int(s[i]) - (1 << q) + (1 << p)
            else:
                i1, j1, a1, b1 = o
                assert i1 < j1 and a1 < b1
                op = _jw.operator_matrix(norb, [("c", a1), ("c", b1), ("a", j1), ("a", i1)])
                assert int(s[j]) == int(s[i]) - (1 << i1) - (1 << j1) + (1 << a1) + (1 << b1)
            sign = op[int(s[j]), int(s[i])]
            assert t["sign"][e] == sign and abs(sign) == 1
            assert abs(t["val"][e] - Hs[i, j]) <= 1e-13


def test_table_sizes_full_space():
    # Full string set: every string has n(norb-n) singles, C(n,2)C(norb-n,2) doubles.
    norb, ne = 7, 3
    h, V = si.make_integrals(norb, 4, 1)
    s = si.full_strings(norb, ne)
    t1 = oracle.excitations(norb, h, V, s, 1)
    t2 = oracle.excitations(norb, h, V, s, 2)
    assert np.all(np.diff(t1["off"]) == ne * (norb - ne))
    assert np.all(np.diff(t2["off"]) == 3 * 6)


# ---------------------------------------------------------- closed forms ---

def _ground(norb, h, V, sa, sb, ecore=0.0):
    H = oracle.dense_h(norb, h, V, ecore, sa, sb)
    return np.linalg.eigvalsh(H)[0], H


def test_free_fermions_general_h():
    # V = 0: the full-space ground energy is the sum of the lowest n_a and
    # n_b eigenvalues of h (non-interacting fermions).
    rng = np.random.default_rng(2)
    norb, na_e, nb_e = 6, 3, 2
    A = rng.normal(size=(norb, norb))
    h = 0.5 * (A + A.T)
    V = np.zeros((norb,) * 4)
    e0, _ = _ground(norb, h, V, si.full_strings(norb, na_e), si.full_strings(norb, nb_e))
    eps = np.linalg.eigvalsh(h)
    assert abs(e0 - (eps[:na_e].sum() + eps[:nb_e].sum())) <= 1e-12


def test_diagonal_h_no_two_body_is_diagonal():
    norb = 6
    eps = np.linspace(-2, 2, norb)
    h = np.diag(eps)
    V = np.zeros((norb,) * 4)
    sa = sb = si.full_strings(norb, 2)
    e0, H = _ground(norb, h, V, sa, sb)
    assert np.count_nonzero(H - np.diag(np.diag(H))) == 0
    assert abs(e0 - 2 * (eps[0] + eps[1])) <= 1e-13


def test_hubbard_chain_u0_closed_form():
    L, n, t = 6, 3, 1.0
    h, V = si.hubbard_chain_integrals(L, t, 0.0)
    e0, _ = _ground(L, h, V, si.full_strings(L, n), si.full_strings(L, n))
    eps = -2 * t * np.cos(np.arange(1, L + 1) * np.pi / (L + 1))
    assert abs(e0 - 2 * np.sort(eps)[:n].sum()) <= 1e-12


@pytest.mark.parametrize("U", [0.0, 1.0, 4.0, 10.0])
def test_two_site_hubbard_closed_form(U):
    t = 1.0
    h, V = si.hubbard_chain_integrals(2, t, U)
    e0, _ = _ground(2, h, V, si.full_strings(2, 1), si.full_strings(2, 1))
    assert abs(e0 - (U / 2 - np.sqrt(U * U / 4 + 4 * t * t))) <= 1e-13


def test_hermitian():
    rng = np.random.default_rng(8)
    norb = 6
    h, V = si.make_integrals(norb, 12, 3)
    sa, sb = _rand_strings(rng, norb, 3, 12), _rand_strings(rng, norb, 2, 10)
    H = oracle.dense_h(norb, h, V, 0.0, sa, sb)
    assert np.max(np.abs(H - H.T)) <= 1e-15
    x, y = rng.normal(size=(2, H.shape[0]))
    Hx = oracle.sigma(norb, h, V, 0.0, sa, sb, x)
    Hy = oracle.sigma(norb, h, V, 0.0, sa, sb, y)
    assert abs(x @ Hy - Hx @ y) <= 1e-13 * np.linalg.norm(Hx) * np.linalg.norm(y)


def _random_rotation(rng, n, scale=0.3):
    import scipy.linalg
    K = rng.normal(scale=scale, size=(n, n))
    return scipy.linalg.expm(K - K.T)


def test_full_space_energy_invariant_under_orbital_rotation():
    rng = np.random.default_rng(13)
    norb, ne = 6, 3
    h, V = si.make_integrals(norb, 12, 17)
    s = si.full_strings(norb, ne)
    e0, _ = _ground(norb, h, V, s, s)
    U = _random_rotation(rng, norb)
    h2, V2 = oracle.rotate_integrals(h, V, U)
    e1, _ = _ground(norb, h2, V2, s, s)
    assert abs(e0 - e1) <= 1e-10
    # ... while a truncated subspace is not invariant (the check has teeth)
    sub = s[::2]
    ea, _ = _ground(norb, h, V, sub, sub)
    eb, _ = _ground(norb, h2, V2, sub, sub)
    assert abs(ea - eb) > 1e-6


def test_subspace_energy_interlaces_full_ci():
    rng = np.random.default_rng(4)
    norb, ne = 6, 3
    h, V = si.make_integrals(norb, 12, 2)
    full = si.full_strings(norb, ne)
    e_fci, _ = _ground(norb, h, V, full, full)
    order = rng.permutation(len(full))
    prev = np.inf
    for k in (4, 8, 12, 16, 20):
        sub = np.sort(full[order[:k]])
        e, _ = _ground(norb, h, V, sub, sub)
        assert e >= e_fci - 1e-12
        assert e <= prev + 1e-12  # adding strings can only lower it
        prev = e
    assert abs(prev - e_fci) <= 1e-11


# ------------------------------------------------------------- Davidson ----

def test_davidson_matches_lapack_full8():
    w = si.workload("full8")
    sa = sb = w.strings_a
    H = oracle.dense_h(w.norb, w.h, w.V, 0.0, sa, sb)
    ref = np.linalg.eigvalsh(H)[:3]
    hd = oracle.diag(w.norb, w.h, w.V, 0.0, sa, sb)

    def mv(X):
        return oracle.sigma(w.norb, w.h, w.V, 0.0, sa, sb, X.T).T

    th, X, it, rn, conv = oracle.davidson(mv, hd, nroots=1, tol_residual=1e-7,
                                          tol_energy=1e-12)
    assert conv and abs(th[0] - ref[0]) <= 1e-10
    th3, X3, _, rn3, conv3 = oracle.davidson(mv, hd, nroots=3, tol_residual=1e-7,
                                             tol_energy=1e-12)
    assert conv3 and np.max(np.abs(th3 - ref)) <= 1e-10
    # Ritz vectors are eigenvectors of the dense matrix
    assert np.linalg.norm(H @ X3 - X3 * th3) <= 1e-6


def test_olsen_correction_pins():
    # the correction of one root, from its definition: Davidson's t solves
    # D t = r; Olsen's t is orthogonal to x and differs from Davidson's by a
    # multiple of D^-1 x
    rng = np.random.default_rng(5)
    n = 50
    hd = np.sort(rng.normal(size=n)) * 3.0
    x = rng.normal(size=n)
    x /= np.linalg.norm(x)
    r = rng.normal(size=n)
    theta = hd[0] - 0.1
    td = oracle.correction_vector(r, x, theta, hd)
    assert np.allclose((theta - hd) * td, r, rtol=1e-14, atol=1e-14)
    to = oracle.correction_vector(r, x, theta, hd, correction="olsen")
    assert abs(x @ to) <= 1e-12 * np.linalg.norm(to)
    dx = x / (theta - hd)
    c = (td - to) @ dx / (dx @ dx)
    assert np.allclose(td - to, c * dx, rtol=0, atol=1e-12 * np.linalg.norm(td))


def test_davidson_olsen_matches_lapack():
    w = si.workload("full8")
    sa = sb = w.strings_a
    H = oracle.dense_h(w.norb, w.h, w.V, 0.0, sa, sb)
    ref = np.linalg.eigvalsh(H)[:3]
    hd = oracle.diag(w.norb, w.h, w.V, 0.0, sa, sb)

    def mv(X):
        return oracle.sigma(w.norb, w.h, w.V, 0.0, sa, sb, X.T).T

    th, X, it, rn, conv = oracle.davidson(mv, hd, nroots=3, tol_residual=1e-7,
                                          tol_energy=1e-12, correction="olsen")
    assert conv and np.max(np.abs(th - ref)) <= 1e-10
    assert np.linalg.norm(H @ X - X * th) <= 1e-6


# ---------------------------------------------------------------- RDMs -----

def _tiny_state(seed=0, norb=4, na_e=2, nb_e=2, k=None):
    rng = np.random.default_rng(seed)
    h, V = si.make_integrals(norb, 8, 30 + seed)
    sa = si.full_strings(norb, na_e)
    sb = si.full_strings(norb, nb_e)
    if k is not None:
        sa, sb = _rand_strings(rng, norb, na_e, k), _rand_strings(rng, norb, nb_e, k)
    H = oracle.dense_h(norb, h, V, 0.0, sa, sb)
    w, v = np.linalg.eigh(H)
    return norb, h, V, sa, sb, w[0], v[:, 0]


def test_rdm_vs_jordan_wigner_expectations():
    norb, h, V, sa, sb, e, c = _tiny_state(1, k=5)
    dim = 2 ** (2 * norb)
    psi = np.zeros(dim)
    psi[[_jw.fock_index(norb, a, b) for a in sa for b in sb]] = c
    g1 = oracle.rdm1(norb, sa, sb, c)
    g2 = oracle.rdm2(norb, sa, sb, c)
    P = np.zeros(dim)
    P[[_jw.fock_index(norb, a, b) for a in sa for b in sb]] = 1.0
    rng = np.random.default_rng(0)
    for _ in range(25):
        p, q, r, s = rng.integers(0, norb, size=4)
        ref1 = 0.0
        ref2 = 0.0
        for a in (0, 1):
            op = _jw.operator_matrix(norb, [("c", p + a * norb), ("a", q + a * norb)])
            ref1 += psi @ (P * (op @ psi))
            for b in (0, 1):
                op2 = _jw.operator_matrix(norb, [("c", p + a * norb), ("c", r + b * norb),
                                                 ("a", s + b * norb), ("a", q + a * norb)])
                ref2 += psi @ (P * (op2 @ psi))
        assert abs(g1[p, q] - ref1) <= 1e-13
        assert abs(g2[p, q, r, s] - ref2) <= 1e-13


def test_rdm_identities():
    norb, h, V, sa, sb, e, c = _tiny_state(2)
    g1 = oracle.rdm1(norb, sa, sb, c)
    g2 = oracle.rdm2(norb, sa, sb, c)
    ne = 4
    assert abs(np.trace(g1) - ne) <= 1e-12
    assert np.allclose(np.einsum("pqrr->pq", g2), (ne - 1) * g1, atol=1e-12)
    assert np.allclose(g2, g2.transpose(2, 3, 0, 1), atol=1e-13)
    assert np.allclose(g1, g1.T, atol=1e-13)
    assert abs(oracle.energy_from_rdms(h, V, 0.0, g1, g2) - e) <= 1e-11


def test_rdm_wick_factorisation_free_fermions():
    # V = 0 full space: the ground state is a Slater determinant and
    # Gamma_pqrs = g_pq g_rs - sum_s g^s_ps g^s_rq (Wick).
    rng = np.random.default_rng(6)
    norb = 4
    A = rng.normal(size=(norb, norb))
    h = 0.5 * (A + A.T)
    V = np.zeros((norb,) * 4)
    sa = sb = si.full_strings(norb, 2)
    H = oracle.dense_h(norb, h, V, 0.0, sa, sb)
    w, v = np.linalg.eigh(H)
    assert w[1] - w[0] > 1e-6  # nondegenerate
    c = v[:, 0]
    g1 = oracle.rdm1(norb, sa, sb, c)
    g2 = oracle.rdm2(norb, sa, sb, c)
    gs = 0.5 * g1  # per-spin 1-RDM (closed shell)
    wick = np.einsum("pq,rs->pqrs", g1, g1) - 2 * np.einsum("ps,rq->pqrs", gs, gs)
    assert np.allclose(g2, wick, atol=1e-11)


def test_hellmann_feynman_finite_differences():
    # dE/dh_pq (moving h_pq and h_qp together) = gamma_pq + gamma_qp and
    # dE/d(pq|rs) over a symmetry orbit = 1/2 sum over the orbit of Gamma.
    norb, h, V, sa, sb, e, c = _tiny_state(3, k=5)
    g1 = oracle.rdm1(norb, sa, sb, c)
    g2 = oracle.rdm2(norb, sa, sb, c)
    step = 1e-5

    def energy(h_, V_):
        return np.linalg.eigvalsh(oracle.dense_h(norb, h_, V_, 0.0, sa, sb))[0]

    for p, q in [(0, 1), (2, 2), (1, 3)]:
        d = np.zeros_like(h)
        d[p, q] = d[q, p] = 1.0
        fd = (energy(h + step * d, V) - energy(h - step * d, V)) / (2 * step)
        an = g1[p, q] + (g1[q, p] if p != q else 0.0)
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))
    for p, q, r, s in [(0, 1, 2, 3), (1, 1, 0, 0), (0, 2, 0, 2)]:
        orbit = set()
        for a, b, cc, dd in [(p, q, r, s), (q, p, r, s), (p, q, s, r), (q, p, s, r)]:
            orbit.add((a, b, cc, dd))
            orbit.add((cc, dd, a, b))
        D = np.zeros_like(V)
        for o in orbit:
            D[o] = 1.0
        fd = (energy(h, V + step * D) - energy(h, V - step * D)) / (2 * step)
        an = 0.5 * sum(g2[o] for o in orbit)
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))


def test_orbital_gradient_finite_differences():
    import scipy.linalg
    norb, h, V, sa, sb, e, c = _tiny_state(4, k=5)
    g1 = oracle.rdm1(norb, sa, sb, c)
    g2 = oracle.rdm2(norb, sa, sb, c)
    g = oracle.orbital_gradient(h, V, g1, g2)
    assert np.max(np.abs(g)) > 1e-3  # a truncated space has a nonzero gradient
    step = 1e-5

    def energy_k(K):
        U = scipy.linalg.expm(K)
        h2, V2 = oracle.rotate_integrals(h, V, U)
        return np.linalg.eigvalsh(oracle.dense_h(norb, h2, V2, 0.0, sa, sb))[0]

    for p, q in [(0, 1), (1, 3), (2, 0)]:
        K = np.zeros((norb, norb))
        K[p, q], K[q, p] = 1.0, -1.0
        fd = (energy_k(step * K) - energy_k(-step * K)) / (2 * step)
        assert abs(fd - g[p, q]) <= 1e-6 * max(1.0, abs(g[p, q]))


def test_orbital_gradient_vanishes_at_full_ci():
    norb, h, V, sa, sb, e, c = _tiny_state(5)
    g = oracle.orbital_gradient(h, V, oracle.rdm1(norb, sa, sb, c),
                                oracle.rdm2(norb, sa, sb, c))
    assert np.max(np.abs(g)) <= 1e-10


# ------------------------------------------------------------ outer loop ---

def test_outer_loop_helpers_invariants():
    rng = np.random.default_rng(12)
    sa = _rand_strings(rng, 8, 3, 20)
    sb = _rand_strings(rng, 8, 2, 15)
    C = rng.normal(size=len(sa) * len(sb))
    wa, wb = oracle.string_weights(C, len(sa), len(sb))
    assert abs(wa.sum() - C @ C) <= 1e-12 and abs(wb.sum() - C @ C) <= 1e-12
    # mapping onto the same sets is normalisation
    M, nrm = oracle.map_vector(sa, sb, C, sa, sb)
    assert abs(nrm - np.linalg.norm(C)) <= 1e-12
    assert np.allclose(M.reshape(-1), C / np.linalg.norm(C), atol=1e-15)
    # onto a superset: old values kept in place, zeros elsewhere; and back
    full_a, full_b = si.full_strings(8, 3), si.full_strings(8, 2)
    M2, _ = oracle.map_vector(sa, sb, C, full_a, full_b)
    ia = np.searchsorted(full_a, sa)
    ib = np.searchsorted(full_b, sb)
    assert np.count_nonzero(M2) == np.count_nonzero(C)
    assert np.allclose(M2[np.ix_(ia, ib)].reshape(-1), C / np.linalg.norm(C))
    back, _ = oracle.map_vector(full_a, full_b, M2, sa, sb)
    assert np.allclose(back.reshape(-1), C / np.linalg.norm(C))
    # disjoint sets: nothing carried
    other = np.setdiff1d(full_a, sa)
    Z, z = oracle.map_vector(sa, sb, C, other, sb)
    assert z == 0.0 and not Z.any()
    assert len(oracle.select_strings(sa, wa, -1.0)) == len(sa)
    assert len(oracle.select_strings(sa, wa, wa.max() + 1)) == 0
    keep = oracle.select_strings(sa, wa, np.median(wa))
    assert set(keep.tolist()) == {int(x) for x, v in zip(sa, wa) if v >= np.median(wa)}


# ------------------------------------------- elementary oracle functions ----

def test_hij_equals_jordan_wigner_elements():
    # the generic Slater-Condon element of two determinants, against the
    # Jordan-Wigner operator matrix, with non-symmetric integrals
    rng = np.random.default_rng(11)
    norb = 4
    h, V = _nonsym_integrals(rng, norb)
    Hf = _jw.hamiltonian(norb, h, V, 0.75)
    sa, sb = si.full_strings(norb, 2), si.full_strings(norb, 1)
    for _ in range(60):
        ia, ja = rng.choice(sa, size=2)
        ib, jb = rng.choice(sb, size=2)
        ref = Hf[_jw.fock_index(norb, ia, ib), _jw.fock_index(norb, ja, jb)]
        got = oracle.hij(norb, h, V, 0.75, ia, ib, ja, jb)
        assert abs(got - ref) <= 1e-12 * (1.0 + abs(ref))


def test_string_energy_equals_one_spin_diagonal():
    rng = np.random.default_rng(12)
    norb = 5
    h, V = _nonsym_integrals(rng, norb)
    Hf = _jw.hamiltonian(norb, h, V, 0.0, spins=(0,))
    s = si.full_strings(norb, 3)
    got = oracle.string_energy(norb, h, V, s)
    ref = np.array([Hf[_jw.fock_index(norb, x, 0), _jw.fock_index(norb, x, 0)] for x in s])
    assert np.allclose(got, ref, rtol=1e-13, atol=1e-13)


def test_expect_equals_jordan_wigner():
    # <C| P op P |C> for one- and two-body spin-orbital operator strings
    rng = np.random.default_rng(13)
    norb = 3
    sa, sb = si.full_strings(norb, 2), si.full_strings(norb, 1)
    C = rng.normal(size=len(sa) * len(sb))
    dim = 2 ** (2 * norb)
    idx = [_jw.fock_index(norb, a, b) for a in sa for b in sb]
    psi = np.zeros(dim)
    psi[idx] = C
    P = np.zeros(dim)
    P[idx] = 1.0
    ops2 = rng.integers(0, 2 * norb, size=(12, 2))
    ops4 = rng.integers(0, 2 * norb, size=(12, 4))
    for ops, kinds in ((ops2, "ca"), (ops4, "ccaa")):
        got = oracle.expect(norb, sa, sb, C, ops)
        for row, g in zip(ops, got):
            op = _jw.operator_matrix(norb, list(zip(kinds, row.tolist())))
            ref = psi @ (P * (op @ psi))
            assert abs(g - ref) <= 1e-12 * (1.0 + abs(ref))


def test_eigh_lowest_is_the_lowest_eigenpairs():
    rng = np.random.default_rng(14)
    A = rng.normal(size=(40, 40))
    H = A + A.T
    w, v = oracle.eigh_lowest(H, 3)
    assert np.allclose(w, np.sort(np.linalg.eigvalsh(H))[:3], rtol=0, atol=1e-11)
    assert np.allclose(H @ v, v * w, atol=1e-10)
    assert np.allclose(v.T @ v, np.eye(3), atol=1e-12)
