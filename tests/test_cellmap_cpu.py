"""The general polyhedral mesh descriptor of Sec. 3.1 turned into the
padded per-shape numbering the kernels run on (csrc/vag_cellmap.h and
csrc/vag_topo.h, the code the assembly kernel and the server run, compiled
here with g++).

* On a hexahedral lattice it returns the lattice numbering itself, whatever
  the order of a cell's faces and of each face's nodes: the canonical
  numbering depends on node ids and edges only.
* After a random relabelling of the nodes it still returns a numbering whose
  edges are edges of the cell and whose faces, through the shape's table,
  are exactly the cell's faces: hexahedra, tetrahedra, prisms (also mixed
  with hexahedra) and pyramids.
* Cells of none of the shapes (a face listed out of cyclic order, a repeated
  face, a missing face, a pentagon) are rejected, and so are ids out of
  range.  CPU only."""
import os
import subprocess
import tempfile

import numpy as np
import pytest

import vag_inputs as vi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1602_03641_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include <vector>
#include "vag_cellmap.h"
int main() {
  int nn, nf; std::scanf("%d %d", &nn, &nf);
  std::vector<int32_t> fptr(nf + 1);
  for (auto &v : fptr) std::scanf("%d", &v);
  std::vector<int32_t> fidx(fptr[nf] > 0 ? fptr[nf] : 1);
  for (int i = 0; i < fptr[nf]; ++i) std::scanf("%d", &fidx[i]);
  int nc; std::scanf("%d", &nc);
  std::vector<int32_t> cptr(nc + 1);
  for (auto &v : cptr) std::scanf("%d", &v);
  std::vector<int32_t> cidx(cptr[nc] > 0 ? cptr[nc] : 1);
  for (int i = 0; i < cptr[nc]; ++i) std::scanf("%d", &cidx[i]);
  for (int K = 0; K < nc; ++K) {
    int32_t out[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int sh = -1;
    const int e = vag::cell_from_faces(fptr.data(), fidx.data(), fptr[nf], cptr.data(), cidx.data(), cptr[nc], nf,
                                       nn, K, out, &sh);
    std::printf("%d %d", e, sh);
    for (int l = 0; l < 8; ++l) std::printf(" %d", out[l]);
    std::printf("\n");
  }
  int nq; std::scanf("%d", &nq);
  for (int i = 0; i < nq; ++i) {
    int f; std::scanf("%d", &f);
    int32_t out[4] = {0, 0, 0, 0};
    const int e = vag::face_nodes_of(fptr.data(), fidx.data(), fptr[nf], nf, nn, f, out);
    std::printf("%d %d %d %d %d\n", e, out[0], out[1], out[2], out[3]);
  }
  // the shape tables: n_nodes, n_faces, then each face's nodes
  for (int sh = 0; sh < vag::topo::N_SHAPES; ++sh) {
    std::printf("%d %d", vag::topo::n_nodes(sh), vag::topo::n_faces(sh));
    for (int lf = 0; lf < vag::topo::n_faces(sh); ++lf) {
      std::printf(" |");
      for (int t = 0; t < vag::topo::face_size(sh, lf); ++t) std::printf(" %d", vag::topo::face(sh, lf, t));
    }
    std::printf("\n");
  }
  return 0;
}
"""

OK, BAD_INDEX, UNSUPPORTED = 0, 1, 3
HEX, TET, PRISM, PYRAMID = 0, 1, 2, 3

CUBE_EDGES = [(0, 1), (0, 2), (0, 4), (1, 3), (1, 5), (2, 3), (2, 6), (3, 7), (4, 5), (4, 6), (5, 7), (6, 7)]
CUBE_FACES = [{0, 2, 4, 6}, {1, 3, 5, 7}, {0, 1, 4, 5}, {2, 3, 6, 7}, {0, 1, 2, 3}, {4, 5, 6, 7}]


@pytest.fixture(scope="module")
def run():
    d = tempfile.mkdtemp()
    src = os.path.join(d, "h.cpp")
    exe = os.path.join(d, "h")
    open(src, "w").write(HARNESS)
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, src, "-o", exe], check=True)

    def call(n_nodes, faces, cells, quads=(), tables=False):
        faces = [[v for v in f if v >= 0] for f in faces]
        cells = [[c for c in cl if c >= 0] for cl in cells]
        fptr = np.concatenate([[0], np.cumsum([len(f) for f in faces])])
        cptr = np.concatenate([[0], np.cumsum([len(c) for c in cells])])
        toks = [n_nodes, len(faces), *fptr, *[v for f in faces for v in f], len(cells), *cptr,
                *[v for c in cells for v in c], len(quads), *quads]
        out = subprocess.run([exe], input=" ".join(str(int(t)) for t in toks) + "\n", capture_output=True, text=True,
                             check=True).stdout.split("\n")
        res = [list(map(int, l.split())) for l in out[:len(cells)]]
        qs = [list(map(int, l.split())) for l in out[len(cells):len(cells) + len(quads)]]
        if tables:
            tab = []
            for l in out[len(cells) + len(quads):len(cells) + len(quads) + 4]:
                head, *fs = l.split("|")
                nn, nfc = map(int, head.split())
                tab.append((nn, [tuple(map(int, f.split())) for f in fs]))
            return tab
        return [(r[0], r[1], r[2:]) for r in res], [(q[0], q[1:]) for q in qs]
    return call


def _lattice(dims=(3, 2, 2)):
    pb = vi.build_problem(dims, [(0, 1, 0, dims[1], 0, dims[2])])
    return pb


def test_lattice_gives_the_lattice_numbering(run):
    pb = _lattice()
    res, qs = run(pb.n_nodes, pb.faces.tolist(), pb.cell_faces.tolist(), pb.ff_faces.tolist())
    for K, (e, sh, out) in enumerate(res):
        assert e == 0 and sh == HEX and out == pb.cell_nodes[K].tolist(), K
    for i, (e, out) in enumerate(qs):
        assert e == 0 and out == pb.ff_nodes[i].tolist(), i


def test_face_order_and_cycles_do_not_matter(run):
    pb = _lattice((2, 3, 2))
    rng = np.random.default_rng(4)
    faces = []
    for f in pb.faces.tolist():
        k = int(rng.integers(0, 4))
        f = f[k:] + f[:k]
        faces.append(f[::-1] if rng.random() < 0.5 else f)
    cells = [list(rng.permutation(c)) for c in pb.cell_faces.tolist()]
    res, _ = run(pb.n_nodes, faces, cells)
    for K, (e, sh, out) in enumerate(res):
        assert e == 0 and sh == HEX and out == pb.cell_nodes[K].tolist(), K


def test_relabelled_nodes_give_a_valid_cube_numbering(run):
    pb = _lattice((3, 3, 2))
    rng = np.random.default_rng(8)
    perm = rng.permutation(pb.n_nodes)
    faces = [[int(perm[v]) for v in f] for f in pb.faces.tolist()]
    res, _ = run(pb.n_nodes, faces, pb.cell_faces.tolist())
    for K, (e, sh, out) in enumerate(res):
        assert e == 0 and sh == HEX, K
        cell_faces = [faces[f] for f in pb.cell_faces[K]]
        edges = {frozenset((f[t], f[(t + 1) % 4])) for f in cell_faces for t in range(4)}
        assert all(frozenset((out[a], out[b])) in edges for a, b in CUBE_EDGES), K
        assert sorted(map(sorted, ({out[l] for l in s} for s in CUBE_FACES))) == \
            sorted(map(sorted, (set(f) for f in cell_faces))), K
        assert out[0] == min(out) and out[1] < out[2] < out[4], K
        assert set(out) == {int(perm[v]) for v in pb.cell_nodes[K]}, K


def test_bad_cells_and_bad_ids_are_rejected(run):
    pb = _lattice((1, 1, 1))
    faces = pb.faces.tolist()
    cf = pb.cell_faces[0].tolist()
    # a face listed out of cyclic order (its diagonal as an edge)
    bad = [list(f) for f in faces]
    f0 = bad[cf[0]]
    bad[cf[0]] = [f0[0], f0[2], f0[1], f0[3]]
    res, _ = run(pb.n_nodes, bad, [cf])
    assert res[0][0] == UNSUPPORTED
    # a repeated face
    res, _ = run(pb.n_nodes, faces, [[cf[0], cf[0], cf[2], cf[3], cf[4], cf[5]]])
    assert res[0][0] == UNSUPPORTED
    # five quadrilaterals (a hexahedron missing a face)
    res, _ = run(pb.n_nodes, faces, [cf[:5]])
    assert res[0][0] == UNSUPPORTED
    # a face id or a node id out of range
    res, _ = run(pb.n_nodes, faces, [[cf[0], cf[1], cf[2], cf[3], cf[4], len(faces)]])
    assert res[0][0] == BAD_INDEX
    res, _ = run(pb.n_nodes - 1, faces, [cf])
    assert res[0][0] == BAD_INDEX
    # three faces folded onto a repeated node ((0,1,0,2) for the bottom face,
    # and two more that restore every node's count): eight nodes, each in
    # three faces, and the cube's twelve edges, but not the cube's faces
    cube = [[0, 2, 6, 4], [1, 3, 7, 5], [0, 1, 5, 4], [2, 3, 7, 6], [0, 1, 3, 2], [4, 5, 7, 6]]
    res, _ = run(8, cube, [[0, 1, 2, 3, 4, 5]])
    assert res[0][0] == OK
    folded = [[6, 2, 6, 4], [1, 3, 7, 5], [0, 1, 5, 4], [3, 2, 3, 7], [0, 1, 0, 2], [4, 5, 7, 6]]
    res, _ = run(8, folded, [[0, 1, 2, 3, 4, 5]])
    assert res[0][0] == UNSUPPORTED
    # a prism with a lateral face whose nodes do not join its triangles
    prism_faces = [[0, 1, 2], [3, 4, 5], [0, 1, 4, 3], [1, 2, 5, 4], [2, 0, 3, 5]]
    twisted = [list(f) for f in prism_faces]
    twisted[2] = [0, 1, 5, 3]
    res, _ = run(6, twisted, [[0, 1, 2, 3, 4]])
    assert res[0][0] == UNSUPPORTED
    # a pentagonal face; a tetrahedron with a face listed twice
    res, _ = run(6, [[0, 1, 2, 3, 4], [0, 1, 5], [1, 2, 5], [2, 3, 5], [3, 4, 5], [4, 0, 5]], [[0, 1, 2, 3, 4, 5]])
    assert res[0][0] == UNSUPPORTED
    res, _ = run(4, [[1, 2, 3], [0, 3, 2], [0, 1, 3], [0, 2, 1]], [[0, 0, 2, 3]])
    assert res[0][0] == UNSUPPORTED
    # fracture faces: triangles and quadrilaterals; a repeated node; out-of-range id
    _, qs = run(6, prism_faces + [[0, 1, 1]], [], [0, 2, 5, 7])
    assert [q[0] for q in qs] == [OK, OK, UNSUPPORTED, BAD_INDEX]
    assert qs[0][1] == [0, 1, 2, -1] and qs[1][1] == [0, 1, 4, 3]


def _check_numbering(tab, sh, out, cell_faces_nodes):
    """The shape's faces through the numbering are the cell's faces, each
    consecutive pair of a listed face an edge of the shape."""
    nn, tfaces = tab[sh]
    assert all(v >= 0 for v in out[:nn]) and all(v == -1 for v in out[nn:])
    got = sorted(sorted(out[l] for l in f) for f in tfaces)
    want = sorted(sorted(f) for f in cell_faces_nodes)
    assert got == want
    edges = {frozenset((f[t], f[(t + 1) % len(f)])) for f in cell_faces_nodes for t in range(len(f))}
    assert all(frozenset((out[f[t]], out[f[(t + 1) % len(f)]])) in edges for f in tfaces for t in range(len(f)))


def test_shape_tables(run):
    tab = run(1, [[0, 0, 0]], [], tables=True)
    assert [t[0] for t in tab] == [8, 4, 6, 5]
    assert [len(t[1]) for t in tab] == [6, 4, 5, 5]
    assert [sorted(len(f) for f in t[1]) for t in tab] == [[4] * 6, [3] * 4, [3, 3, 4, 4, 4], [3, 3, 3, 3, 4]]
    # every edge of a shape lies on exactly two of its faces (closed surface)
    for nn, fs in tab:
        cnt = {}
        for f in fs:
            for t in range(len(f)):
                e = frozenset((f[t], f[(t + 1) % len(f)]))
                cnt[e] = cnt.get(e, 0) + 1
        assert set(cnt.values()) == {2}
        assert len(cnt) - nn - len(fs) == -2        # Euler: V - E + F = 2
    assert tab[HEX][1] == [(0, 2, 6, 4), (1, 3, 7, 5), (0, 1, 5, 4), (2, 3, 7, 6), (0, 1, 3, 2), (4, 5, 7, 6)]


@pytest.mark.parametrize("kind", ["tet", "prism", "prism_half", "pyramid"])
def test_other_shapes_are_numbered_canonically(run, kind):
    if kind == "tet":
        pb = vi.tet_problem((2, 2, 1))
        want_shape = {TET}
    elif kind == "prism":
        pb = vi.prism_problem((2, 2), 2)
        want_shape = {PRISM}
    elif kind == "prism_half":
        pb = vi.prism_problem((4, 2), 2, split="half")
        want_shape = {PRISM, HEX}
    else:
        pb = vi.pyramid_problem((2, 1, 1))
        want_shape = {PYRAMID}
    tab = run(1, [[0, 0, 0]], [], tables=True)
    rng = np.random.default_rng(11)
    perm = rng.permutation(pb.n_nodes)
    faces = [[int(perm[v]) for v in f if v >= 0] for f in pb.faces.tolist()]
    # rotate and reverse each face, shuffle each cell's faces: same numbering
    faces2 = []
    for f in faces:
        k = int(rng.integers(0, len(f)))
        g = f[k:] + f[:k]
        faces2.append(g[::-1] if rng.random() < 0.5 else g)
    cells = [[c for c in cl if c >= 0] for cl in pb.cell_faces.tolist()]
    cells2 = [list(rng.permutation(c)) for c in cells]
    res, _ = run(pb.n_nodes, faces, cells)
    res2, _ = run(pb.n_nodes, faces2, cells2)
    shapes = set()
    for K, ((e, sh, out), (e2, sh2, out2)) in enumerate(zip(res, res2)):
        assert e == 0 and e2 == 0, K
        assert (sh, out) == (sh2, out2), K
        shapes.add(sh)
        _check_numbering(tab, sh, out, [faces[f] for f in cells[K]])
        nn = tab[sh][0] if sh != PYRAMID else 4    # a pyramid starts its base at the base's smallest id
        assert out[0] == min(out[:nn]), K
        if sh == TET:
            assert out[:4] == sorted(out[:4])
        if sh == PRISM:
            assert out[1] < out[2]
    assert shapes == want_shape


def test_binding_tables_match_the_library(run):
    """The Python binding's SHAPE_FACES (used to read exported fluxes) is
    the library's table."""
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "vagbind", os.path.join(ROOT, "paper_1602_03641_gb300", "vag.py"))
    tab = run(1, [[0, 0, 0]], [], tables=True)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    for sh in range(4):
        assert mod.SHAPE_FACES[sh] == tab[sh][1]
