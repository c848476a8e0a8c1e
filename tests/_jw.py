"""Jordan-Wigner construction of the second-quantised Hamiltonian.

An independent check of the oracle's Slater-Condon elements: creation and
annihilation operators are built as Kronecker products of Pauli matrices,
the Hamiltonian as the literal operator sum

    H = E_core + sum_{pq,s} h_pq a+_{ps} a_{qs}
        + 1/2 sum_{pqrs,st} (pq|rs) a+_{ps} a+_{rt} a_{st} a_{qs}

by sparse matrix products, with no excitation rules at all.  Mode k < norb is
alpha orbital k, mode norb + k beta orbital k; the Fock basis index has bit k
set when mode k is occupied, and a_k = Z x ... x Z x sigma^- x I x ... with
the Z string on the modes below k.
"""
import numpy as np
import scipy.sparse as sp

_I = sp.identity(2, format="csr")
_Z = sp.csr_matrix(np.diag([1.0, -1.0]))
_SM = sp.csr_matrix(np.array([[0.0, 1.0], [0.0, 0.0]]))  # |0><1|


def annihilators(nmodes):
    ops = []
    for k in range(nmodes):
        m = None
        for j in range(nmodes - 1, -1, -1):  # most significant factor first
            f = _I if j > k else (_SM if j == k else _Z)
            m = f if m is None else sp.kron(m, f, format="csr")
        ops.append(m.tocsr())
    return ops


def hamiltonian(norb, h, V, ecore=0.0, spins=(0, 1)):
    """Sparse Fock-space H on 2*norb modes (or only the listed spin blocks)."""
    n = 2 * norb
    a = annihilators(n)
    c = [x.T.tocsr() for x in a]
    dim = 2 ** n
    H = sp.csr_matrix((dim, dim))
    H = H + ecore * sp.identity(dim, format="csr")
    for s in spins:
        for p in range(norb):
            for q in range(norb):
                if h[p, q] != 0.0:
                    H = H + h[p, q] * (c[p + s * norb] @ a[q + s * norb])
    cc = {}
    aa = {}
    for s in spins:
        for t in spins:
            for p in range(norb):
                for r in range(norb):
                    cc[(p + s * norb, r + t * norb)] = c[p + s * norb] @ c[r + t * norb]
                    aa[(r + t * norb, p + s * norb)] = a[r + t * norb] @ a[p + s * norb]
    for s in spins:
        for t in spins:
            for p in range(norb):
                for q in range(norb):
                    for r in range(norb):
                        for u in range(norb):
                            v = V[p, q, r, u]
                            if v == 0.0:
                                continue
                            P, Q, R, U = p + s * norb, q + s * norb, r + t * norb, u + t * norb
                            H = H + (0.5 * v) * (cc[(P, R)] @ aa[(U, Q)])
    return H.tocsr()


def fock_index(norb, ia, ib):
    return int(ia) | (int(ib) << norb)


def subspace_matrix(Hf, norb, sa, sb):
    idx = np.array([fock_index(norb, a, b) for a in sa for b in sb], dtype=np.int64)
    return Hf[idx][:, idx].toarray()


def operator_matrix(norb, ops_list):
    """Dense-able sparse matrix of a product of mode operators, given as a
    list of (kind, mode) with kind 'c' (creation) or 'a' (annihilation),
    applied right to left like the written product."""
    a = annihilators(2 * norb)
    M = None
    for kind, k in ops_list:
        f = a[k].T.tocsr() if kind == "c" else a[k]
        M = f if M is None else M @ f
    return M
