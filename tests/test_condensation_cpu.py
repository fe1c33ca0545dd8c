"""The fracture-face static condensation variant, evaluated on the oracle's
eliminated system (CPU only; the variant is not built on the GPU path).

After the cells are eliminated (Eq. eqschur) the Krylov unknowns are the
non-Dirichlet nodes and the fracture faces.  A fracture face that shares no
cell with another fracture face has a 1x1 diagonal block in the fracture-face
rows, so it could be eliminated exactly too:
    S_c = S_KK - S_KE D_E^-1 S_EK,   b_c = b_K - S_KE D_E^-1 b_E,
    u_E = D_E^-1 (b_E - S_EK u_K).
These tests check that this second Schur step is exact (the condensed solve
equals the full one) and measure what it saves: the rows it removes, the
nonzeros it removes net of the fill it adds between the far nodes of the two
cells of each condensed face, and the bytes of one FP64 sliced-ELL product
(12 per stored entry, 20 per row).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import vag_inputs as vi
from oracle import vag_oracle as vo


def condense(pb):
    S, b, R = vo.schur_system(pb)
    S = S.tocsr()
    isf = R >= pb.n_nodes                       # fracture-face rows of S
    fidx = np.nonzero(isf)[0]
    Sff = S[fidx][:, fidx].tocsr()
    offdiag = np.diff(Sff.indptr) - (Sff.diagonal() != 0)
    E = fidx[offdiag == 0]                      # faces with a diagonal block
    keep = np.ones(S.shape[0], bool)
    keep[E] = False
    K = np.nonzero(keep)[0]
    dE = S.diagonal()[E]
    S_KE, S_EK = S[K][:, E], S[E][:, K]
    Sc = (S[K][:, K] - S_KE @ sp.diags(1.0 / dE) @ S_EK).tocsr()
    Sc.eliminate_zeros()
    bc = b[K] - S_KE @ (b[E] / dE)
    return dict(S=S, b=b, K=K, E=E, dE=dE, S_EK=S_EK, Sc=Sc, bc=bc, n_ff_rows=len(fidx))


def spmv_bytes(A):
    return 12 * A.nnz + 20 * A.shape[0]


# local node quads of the six faces of a lattice hexahedron
HEX_FACES = ((0, 1, 3, 2), (4, 5, 7, 6), (0, 1, 5, 4), (2, 3, 7, 6), (0, 2, 6, 4), (1, 3, 7, 5))


def condensable_by_topology(pb):
    """Fracture faces whose adjacent cells carry no other fracture face (the
    cell elimination couples every unknown of a cell, and the fracture-face
    matrices couple a face only to its own nodes, so this is when the face's
    block in the eliminated system is diagonal).  Hexahedral lattice meshes."""
    cn = pb.cell_nodes.reshape(-1, 8)
    M = np.int64(pb.n_nodes)

    def keys(quads):
        q = np.sort(quads, axis=1).astype(np.int64)
        return np.rec.fromarrays([q[:, 0] * M + q[:, 1], q[:, 2] * M + q[:, 3]])

    kf = keys(pb.ff_nodes.reshape(-1, 4))
    order = np.argsort(kf, kind="stable")
    kfs = kf[order]
    per_cell = np.zeros(len(cn), np.int32)
    hits = []
    for q in HEX_FACES:
        kc = keys(cn[:, list(q)])
        pos = np.minimum(np.searchsorted(kfs, kc), len(kfs) - 1)
        hit = kfs[pos] == kc
        per_cell += hit
        hits.append((np.nonzero(hit)[0], order[pos[hit]]))
    ok = np.ones(len(kf), bool)
    for cells, faces in hits:
        ok[faces[per_cell[cells] > 1]] = False
    return int(ok.sum()), len(kf)


def test_condensation_is_exact():
    for pb in (vi.config_mixed128(16, 1e4), vi.config_scale64(16)):
        c = condense(pb)
        u = spla.spsolve(c["S"].tocsc(), c["b"])
        uk = spla.spsolve(c["Sc"].tocsc(), c["bc"])
        ue = (c["b"][c["E"]] - c["S_EK"] @ uk) / c["dE"]
        scale = np.abs(u).max()
        assert len(c["E"]) > 0
        assert np.abs(uk - u[c["K"]]).max() <= 1e-11 * scale
        assert np.abs(ue - u[c["E"]]).max() <= 1e-11 * scale
        # the condensed matrix stays symmetric (and SPD: the solve succeeded)
        d = c["Sc"] - c["Sc"].T
        assert abs(d).max() <= 1e-12 * abs(c["Sc"]).max()


def test_topological_count_equals_the_algebraic_one():
    for pb in (vi.config_mixed128(16, 1e4), vi.config_mixed128(24, 1e4), vi.config_scale64(16)):
        assert condensable_by_topology(pb) == (len(condense(pb)["E"]), pb.n_ff)


def test_condensable_faces_of_the_128_workload():
    """The 128^3 benchmark recipe itself: 83 987 of its 97 542 fracture faces
    would condense, 3.8 % of the 2 210 949 Krylov rows."""
    pb = vi.config_mixed128(128, 1e4)
    assert condensable_by_topology(pb) == (83987, 97542)


def test_what_condensation_saves_on_the_dfn_recipe():
    """The 50-rectangle DFN recipe of the 128^3 workload at 24^3: about half
    of the fracture faces condense (the others share a cell with another
    fracture face, at intersections and on adjacent parallel planes); each
    condensed face removes one row and, net of its fill, about four stored
    entries, so the product's bytes fall by only a few per cent."""
    c = condense(vi.config_mixed128(24, 1e4))
    S, Sc = c["S"], c["Sc"]
    frac_faces = len(c["E"]) / c["n_ff_rows"]
    rows = len(c["E"]) / S.shape[0]
    nnz = (S.nnz - Sc.nnz) / S.nnz
    per_face = (S.nnz - Sc.nnz) / len(c["E"])
    saved = 1.0 - spmv_bytes(Sc) / spmv_bytes(S)
    print(f"condensed faces {len(c['E'])} of {c['n_ff_rows']} ({frac_faces:.3f}); rows -{rows:.4f}; "
          f"nonzeros -{nnz:.4f} ({per_face:.2f} a face); product bytes -{saved:.4f}")
    assert 0.35 < frac_faces < 0.65
    assert 0.0 < nnz < 0.03
    assert 2.0 < per_face < 8.0
    assert 0.0 < saved < 0.04
