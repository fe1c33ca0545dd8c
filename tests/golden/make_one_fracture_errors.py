"""Writes one_fracture_l1_errors.txt: the oracle's L1 errors against the
paper's one-fracture solution (Sec. 5.1) at t_f = 1/2 on n x n meshes, with
the time stepping of Sec. 4.3 (the CFL maximum, the last step shortened).
Calls the oracle only; run from the repository root:

    python tests/golden/make_one_fracture_errors.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import vag_inputs as vi  # noqa: E402
from oracle import analytic as an  # noqa: E402
from oracle import vag_oracle as vo  # noqa: E402

T_F = 0.5


def main():
    s = an.OneFracture()
    rows = []
    for n in (64, 128, 256):
        pb = vi.one_fracture_problem(n)
        d = vo.DarcyTransport(pb)
        c, dt, steps = d.run_to_time(T_F)
        m = vo.Mesh(pb)
        vol = vo.cell_local_matrices(pb, m)["vol"]
        area = vo.fracture_local_matrices(pb, m)["area"]
        nv, nf = pb.n_nodes, pb.n_ff
        ex_k = s.c_m(m.xK[:, 0], m.xK[:, 1], T_F)
        em = np.sum(vol * np.abs(c[nv + nf:] - ex_k)) / np.sum(vol * np.abs(ex_k))
        ex_f = s.c_f(m.xS[pb.ff_faces][:, 0], T_F)
        ef = np.sum(area * np.abs(c[nv:nv + nf] - ex_f)) / np.sum(area * np.abs(ex_f))
        rows.append((n, steps, dt, em, ef))
        print(n, steps, dt, em, ef, flush=True)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "one_fracture_l1_errors.txt")
    with open(out, "w") as f:
        f.write("# Oracle L1 errors vs the Sec. 5.1 one-fracture solution at t_f = 1/2\n")
        f.write("# written by tests/golden/make_one_fracture_errors.py (oracle only)\n")
        f.write("# n  steps  dt  err_matrix  err_fracture\n")
        for n, steps, dt, em, ef in rows:
            f.write(f"{n} {steps} {dt:.17g} {em:.17g} {ef:.17g}\n")


if __name__ == "__main__":
    main()
