"""Work counts of the oracle on the full-size Darcy + transport workload
(64^3 jittered hex, four fractures, lognormal anisotropic Lambda_m, ratio 1e4,
Jacobi-PCG to 1e-10, 200 transport steps).

TEST INFRASTRUCTURE: the CPU-baseline leg of bench.py times the oracle on a
bounded sample (the same recipe at 32^3, run end to end) and scales every
phase to the full size by these exact work counts (cells, nonzeros times CG
iterations, control volumes).  This script calls only the oracle and the input
generators; run it to regenerate cpu_baseline_counts.json.
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import vag_inputs as vi  # noqa: E402
from oracle import vag_oracle as vo  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cpu_baseline_counts.json")


def counts(n):
    pb = vi.config_scale64(n)
    m = vo.Mesh(pb)
    cms = vo._all_cell_matrices(pb, m)
    fm = vo.fracture_local_matrices(pb, m)
    A = vo.assemble_full(pb, m, cms, fm)
    S, b, R = vo.schur_system(pb, A)
    _, it = vo.pcg_jacobi(S, b, rtol=1e-10, maxit=100000)
    return dict(n=n, n_cells=pb.n_cells, n_ff=pb.n_ff, n_rows=int(S.shape[0]), nnz=int(S.nnz),
                n_cv=pb.n_nodes + pb.n_ff + pb.n_cells, oracle_pcg_iterations=int(it))


if __name__ == "__main__":
    data = {"scale64": counts(64), "scale32": counts(32)}
    with open(OUT, "w") as f:
        json.dump(data, f, indent=1)
    print(json.dumps(data, indent=1))
