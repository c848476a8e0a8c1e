"""The spin-flip sectors of the library's shared-string-set mode, pinned on
the oracle's dense Hamiltonian (no GPU).

With the alpha-first determinant ordering an eigenstate of total spin S has
C^T = (-1)^S C whatever the electron count.  The half-filled Hubbard chain
with open ends has a singlet ground state (Lieb and Mattis, 1962), which
must therefore be symmetric for n = 1, 2 and 3 electrons per spin; on two
sites the Ms = 0 triplet (energy 0) must be antisymmetric.
"""
import numpy as np
import pytest

import oracle
import sqd_inputs as si


@pytest.mark.parametrize("L,n", [(2, 1), (4, 2), (6, 3)])
def test_singlet_ground_state_is_symmetric(L, n):
    h, V = si.hubbard_chain_integrals(L, 1.0, 4.0)
    s = si.full_strings(L, n)
    H = oracle.dense_h(L, h, V, 0.0, s, s)
    e, X = np.linalg.eigh(H)
    assert e[1] - e[0] > 1e-6  # a single ground state
    C = X[:, 0].reshape(len(s), len(s))
    assert np.max(np.abs(C - C.T)) <= 1e-12


def test_two_site_triplet_is_antisymmetric():
    h, V = si.hubbard_chain_integrals(2, 1.0, 4.0)
    s = si.full_strings(2, 1)
    H = oracle.dense_h(2, h, V, 0.0, s, s)
    e, X = np.linalg.eigh(H)
    k = int(np.argmin(np.abs(e)))  # the Ms = 0 triplet has energy 0
    assert abs(e[k]) <= 1e-12
    C = X[:, k].reshape(2, 2)
    assert np.max(np.abs(C + C.T)) <= 1e-12 and np.max(np.abs(C)) > 0.5


@pytest.mark.parametrize("name,nu", [("h2o29", 40), ("scale36", 30)])
def test_oracle_sigma_commutes_with_the_spin_flip(name, nu):
    # a shared string set: sigma(C^T) = sigma(C)^T for any C, the identity the
    # sector products rest on (a sign convention that treated the spins
    # differently would break it)
    w = si.workload(name, n_unique=nu)
    n = w.strings_a.size
    C = np.random.default_rng(6).standard_normal((n, n))
    s1 = oracle.sigma(w.norb, w.h, w.V, 0.0, w.strings_a, w.strings_b, C.reshape(-1))
    s2 = oracle.sigma(w.norb, w.h, w.V, 0.0, w.strings_a, w.strings_b, C.T.reshape(-1))
    a, b = s1.reshape(n, n).T, s2.reshape(n, n)
    assert np.linalg.norm(a - b) <= 1e-13 * np.linalg.norm(b)
