"""The seeded synthetic inputs follow their stated recipe: integrals with the
symmetries the Hamiltonian needs, string sets of the stated sizes and
electron counts, deterministic for a seed, and raw draws that filter to the
stored set."""
import numpy as np
import pytest

import oracle
import sqd_inputs as si


@pytest.mark.parametrize("norb,rank", [(8, 16), (29, 58)])
def test_integrals_symmetric_and_positive(norb, rank):
    h, V = si.make_integrals(norb, rank, 1001)
    assert np.array_equal(h, h.T)
    assert np.allclose(np.diag(h), np.linspace(-2, 2, norb), atol=1e-12)
    for perm in ((1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1)):
        assert np.array_equal(V, V.transpose(perm))
    # sum of squares of symmetric factors: positive semidefinite as a matrix
    # over the (pq) pairs
    M = V.reshape(norb * norb, norb * norb)
    assert np.linalg.eigvalsh(M).min() >= -1e-10


def test_integrals_deterministic():
    a = si.make_integrals(12, 24, 7)
    b = si.make_integrals(12, 24, 7)
    c = si.make_integrals(12, 24, 8)
    assert np.array_equal(a[1], b[1]) and not np.array_equal(a[1], c[1])


@pytest.mark.parametrize("name,norb,ne,n", [("h2o29", 29, 5, 2000), ("adjoint29", 29, 5, 5000)])
def test_workload_string_sets(name, norb, ne, n):
    w = si.workload(name)
    s = w.strings_a
    assert len(s) == n and np.all(np.diff(s.astype(np.int64)) > 0)
    bits = np.array([bin(int(x)).count("1") for x in s])
    assert np.all(bits == ne) and int(s.max()) < (1 << norb)
    # the raw draws (duplicates kept) filter to exactly the stored set
    assert np.array_equal(oracle.build_strings(w.raw_a, norb, ne), s)
    assert len(w.raw_a) >= n


def test_full_strings_count():
    from math import comb
    for norb, ne in ((8, 4), (6, 3), (10, 1)):
        assert len(si.full_strings(norb, ne)) == comb(norb, ne)


def test_batched_workload_sizes():
    subs = si.batched_workload(nbatch=6)
    sizes = [len(w.strings_a) for w in subs]
    assert all(200 <= k <= 3000 for k in sizes)
    # one Hamiltonian for every subspace
    for w in subs[1:]:
        assert np.array_equal(w.V, subs[0].V) and np.array_equal(w.h, subs[0].h)
