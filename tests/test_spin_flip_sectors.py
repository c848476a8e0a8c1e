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
