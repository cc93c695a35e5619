"""Writes cd3d64_nd.json: the FP64 oracle's factorization and GMRES(30) on the 64^3 benchmark
matrix (3D upwind convection-diffusion, seed 1, blocks of 64) after the block nested
dissection of Sec. 3.3 (the oracle's reference dissection, oracle/nd_oracle.py).  Calls only
oracle/ and the seeded input generator; about half a minute of CPU time.

    python tests/golden/computed/make_cd3d64_nd.py
"""
import json
import os
import sys

import numpy as np
import scipy.sparse as sp

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(HERE))))

import oracle as O  # noqa: E402
from oracle import nd_oracle as N  # noqa: E402
from paper_1908_10169_gb300 import workloads as W  # noqa: E402


def main():
    w = W.cd3d(side=64, seed=1, block=64)
    bs = O.partition_fixed(w.A.n, 64)
    perm, nbs, _ = N.nd_order(w.A, bs)
    A = sp.csr_matrix((w.A.val, w.A.colind, w.A.rowptr), shape=(w.A.n, w.A.n))
    Ap = A[perm][:, perm].tocsr()
    Ap.sort_indices()
    Aw = W.CSR(w.A.n, Ap.indptr.astype(np.int64), Ap.indices.astype(np.int32), Ap.data.copy())
    F = O.bilu_factor(Aw, nbs, w.droptol)
    r = O.gmres(Aw, F, w.b[perm], tol=w.gmres_tol, restart=w.restart)
    parent = N.block_etree(Aw, nbs)
    depth = np.zeros(len(parent), dtype=np.int64)
    for K in range(len(parent) - 1, -1, -1):
        depth[K] = depth[parent[K]] + 1 if parent[K] >= 0 else 1
    out = {"source": "oracle (FP64 Crout BILU, Sec. 2.2; GMRES(30), Sec. 4) on the 64^3 upwind "
                     "convection-diffusion matrix after block nested dissection (Sec. 3.3)",
           "script": "tests/golden/computed/make_cd3d64_nd.py", "droptol": w.droptol, "nblocks": int(len(nbs) - 1),
           "gmres_iters": int(r.iters), "kept_rows": int(F.Lrow.size), "kept_cols": int(F.Ucol.size),
           "nnz_l": int(F.Lval.size), "nnz_u": int(F.Uval.size), "tree_height": int(depth.max()),
           "relres_true": float(np.linalg.norm(w.b[perm] - Aw.matvec(r.x)) / np.linalg.norm(w.b))}
    F.free()
    with open(os.path.join(HERE, "cd3d64_nd.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(out)


if __name__ == "__main__":
    main()
