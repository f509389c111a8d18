"""Write the FP64 oracle's top eigenvalues of the normalised symmetrised R-MAT
graph (largest component, scale 18) to eigs_symrmat_lcc18_top8.json.

The eigenproblem is Section 4.2's: the largest algebraic eigenvalues of
S = D^-1/2 A D^-1/2.  The values come from the oracle's Lanczos with full
reorthogonalisation (basis 1000; its projection is diagonalised by Householder
tridiagonalisation, Sturm bisection and inverse iteration); the file records
the graph's size and a SHA-256 of its CSR arrays, so a reader can tell when
the generator no longer produces the same matrix.  Run from the repository
root: python tests/golden/make_eigs_reference.py"""
import hashlib
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "eigs_symrmat_lcc18_top8.json")
SCALE, SEED, NEV, BASIS, START_SEED = 18, 0, 8, 1000, 9


def csr_digest(S) -> str:
    h = hashlib.sha256()
    for a in (np.ascontiguousarray(S.row_ptr, dtype=np.int64), np.ascontiguousarray(S.col_idx, dtype=np.int32),
              np.ascontiguousarray(S.values, dtype=np.float32)):
        h.update(a.tobytes())
    return h.hexdigest()


def main():
    S = synth.sym_rmat_lcc(SCALE, seed=SEED)
    Q0 = synth.dense(S.n_rows, NEV, seed=START_SEED).astype(np.float64)
    ev, V, m = oracle.lanczos(S.n_rows, S.row_ptr, S.col_idx, S.values, Q0, NEV, BASIS)
    SV = oracle.spmm(S.n_rows, S.n_cols, S.row_ptr, S.col_idx, S.values, V)
    res = np.linalg.norm(SV - V * ev[None, :], axis=0)
    rec = {
        "what": "top 8 eigenvalues (largest algebraic) of D^-1/2 A D^-1/2, A the symmetrised R-MAT graph's "
                "largest connected component (lognormal weights), Section 4.2",
        "graph": {"generator": "synth.sym_rmat_lcc", "scale": SCALE, "seed": SEED, "n": int(S.n_rows),
                  "nnz": int(S.nnz), "csr_sha256": csr_digest(S)},
        "method": {"routine": "oracle.lanczos (FP64, full reorthogonalisation)", "basis": BASIS, "basis_used": int(m),
                   "start": f"synth.dense(n, {NEV}, seed={START_SEED})"},
        "evals": [float(x) for x in ev],
        "residuals": [float(x) for x in res],   # ||S v - lambda v||_2 through oracle.spmm
    }
    with open(OUT, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print(json.dumps(rec["evals"]))


if __name__ == "__main__":
    main()
