"""Write the stored expected values under tests/golden/ from the CPU oracle
alone (python tests/golden/make_golden.py from the repository root).

* full8_lowest4.txt -- the four lowest eigenvalues of P H P on the full
  8-orbital, 4+4-electron space of the seeded full8 integrals: the dense
  determinant Hamiltonian assembled element by element from the
  Slater-Condon rules, diagonalised by LAPACK (the paper's Davidson target,
  Sections I and VI, on a space small enough to solve exactly).
* h2o29_tables.txt -- sizes and checksums of the same-spin single and
  double excitation lists of the 2000-string h2o29 set (the per-string
  excitation lists of Table I and Section V-A), found by brute-force pair
  scan.

Nothing here reads the CUDA path."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import sqd_inputs as si  # noqa: E402


def full8_lowest4():
    w = si.workload("full8")
    H = oracle.dense_h(w.norb, w.h, w.V, 0.0, w.strings_a, w.strings_b)
    return np.linalg.eigvalsh(H)[:4]


def table_digest(norb, h, V, s, kind):
    t = oracle.excitations(norb, h, V, s, kind)
    off = t["off"]
    per = np.diff(off)
    orb = np.asarray(t["orb"], dtype=np.int64).reshape(len(t["tgt"]), -1)
    weights = np.arange(1, orb.shape[1] + 1, dtype=np.int64)
    return {
        "nnz": int(off[-1]),
        "max_per_string": int(per.max()),
        "sum_target": int(np.sum(t["tgt"], dtype=np.int64)),
        "sum_sign": int(np.sum(t["sign"], dtype=np.int64)),
        "sum_orbital_code": int(np.sum(orb * weights, dtype=np.int64)),
    }


def h2o29_tables():
    w = si.workload("h2o29")
    return {kind: table_digest(w.norb, w.h, w.V, w.strings_a, kind) for kind in (1, 2)}


def write():
    e = full8_lowest4()
    with open(os.path.join(HERE, "full8_lowest4.txt"), "w") as f:
        f.write("# four lowest eigenvalues (Ha) of the dense full8 P H P, oracle + LAPACK\n")
        for v in e:
            f.write("%.17g\n" % v)
    d = h2o29_tables()
    with open(os.path.join(HERE, "h2o29_tables.txt"), "w") as f:
        f.write("# h2o29 same-spin excitation lists (2000 strings), oracle brute force\n")
        f.write("# sum_orbital_code = sum over entries of sum_c (c+1) * orbital_c\n")
        for kind, name in ((1, "singles"), (2, "doubles")):
            for key, val in d[kind].items():
                f.write("%s.%s = %d\n" % (name, key, val))


def read_full8():
    with open(os.path.join(HERE, "full8_lowest4.txt")) as f:
        return np.array([float(x) for x in f if not x.startswith("#")])


def read_tables():
    out = {}
    with open(os.path.join(HERE, "h2o29_tables.txt")) as f:
        for line in f:
            if line.startswith("#") or "=" not in line:
                continue
            k, v = line.split("=")
            out[k.strip()] = int(v)
    return out


if __name__ == "__main__":
    write()
