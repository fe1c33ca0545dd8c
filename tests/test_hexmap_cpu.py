"""The general polyhedral mesh descriptor of Sec. 3.1 turned into the
hexahedral numbering the kernels run on (csrc/vag_hexmap.h, the code the
assembly kernel and the server run, compiled here with g++).

* On a lattice it returns the lattice numbering itself, whatever the order of
  a cell's faces and of each face's nodes: the canonical numbering depends on
  node ids and edges only.
* After a random relabelling of the nodes it still returns a numbering whose
  twelve cube edges are edges of the cell and whose six cube faces are its
  faces.
* Cells that are not hexahedra (a prism, a face listed out of cyclic order,
  a repeated face) are rejected, and so are ids out of range.  CPU only."""
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
#include "vag_hexmap.h"
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
    const int e = vag::hex_from_faces(fptr.data(), fidx.data(), fptr[nf], cptr.data(), cidx.data(), cptr[nc], nf, nn,
                                      K, out);
    std::printf("%d", e);
    for (int l = 0; l < 8; ++l) std::printf(" %d", out[l]);
    std::printf("\n");
  }
  int nq; std::scanf("%d", &nq);
  for (int i = 0; i < nq; ++i) {
    int f; std::scanf("%d", &f);
    int32_t out[4] = {0, 0, 0, 0};
    const int e = vag::quad_of_face(fptr.data(), fidx.data(), fptr[nf], nf, nn, f, out);
    std::printf("%d %d %d %d %d\n", e, out[0], out[1], out[2], out[3]);
  }
  return 0;
}
"""

CUBE_EDGES = [(0, 1), (0, 2), (0, 4), (1, 3), (1, 5), (2, 3), (2, 6), (3, 7), (4, 5), (4, 6), (5, 7), (6, 7)]
CUBE_FACES = [{0, 2, 4, 6}, {1, 3, 5, 7}, {0, 1, 4, 5}, {2, 3, 6, 7}, {0, 1, 2, 3}, {4, 5, 6, 7}]


@pytest.fixture(scope="module")
def run():
    d = tempfile.mkdtemp()
    src = os.path.join(d, "h.cpp")
    exe = os.path.join(d, "h")
    open(src, "w").write(HARNESS)
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, src, "-o", exe], check=True)

    def call(n_nodes, faces, cells, quads=()):
        fptr = np.concatenate([[0], np.cumsum([len(f) for f in faces])])
        cptr = np.concatenate([[0], np.cumsum([len(c) for c in cells])])
        toks = [n_nodes, len(faces), *fptr, *[v for f in faces for v in f], len(cells), *cptr,
                *[v for c in cells for v in c], len(quads), *quads]
        out = subprocess.run([exe], input=" ".join(str(int(t)) for t in toks) + "\n", capture_output=True, text=True,
                             check=True).stdout.split("\n")
        res = [list(map(int, l.split())) for l in out[:len(cells)]]
        qs = [list(map(int, l.split())) for l in out[len(cells):len(cells) + len(quads)]]
        return [(r[0], r[1:]) for r in res], [(q[0], q[1:]) for q in qs]
    return call


def _lattice(dims=(3, 2, 2)):
    pb = vi.build_problem(dims, [(0, 1, 0, dims[1], 0, dims[2])])
    return pb


def test_lattice_gives_the_lattice_numbering(run):
    pb = _lattice()
    res, qs = run(pb.n_nodes, pb.faces.tolist(), pb.cell_faces.tolist(), pb.ff_faces.tolist())
    for K, (e, out) in enumerate(res):
        assert e == 0 and out == pb.cell_nodes[K].tolist(), K
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
    for K, (e, out) in enumerate(res):
        assert e == 0 and out == pb.cell_nodes[K].tolist(), K


def test_relabelled_nodes_give_a_valid_cube_numbering(run):
    pb = _lattice((3, 3, 2))
    rng = np.random.default_rng(8)
    perm = rng.permutation(pb.n_nodes)
    faces = [[int(perm[v]) for v in f] for f in pb.faces.tolist()]
    res, _ = run(pb.n_nodes, faces, pb.cell_faces.tolist())
    for K, (e, out) in enumerate(res):
        assert e == 0, K
        cell_faces = [faces[f] for f in pb.cell_faces[K]]
        edges = {frozenset((f[t], f[(t + 1) % 4])) for f in cell_faces for t in range(4)}
        assert all(frozenset((out[a], out[b])) in edges for a, b in CUBE_EDGES), K
        assert sorted(map(sorted, ({out[l] for l in s} for s in CUBE_FACES))) == \
            sorted(map(sorted, (set(f) for f in cell_faces))), K
        assert out[0] == min(out) and out[1] < out[2] < out[4], K
        assert set(out) == {int(perm[v]) for v in pb.cell_nodes[K]}, K


def test_non_hexahedra_and_bad_ids_are_rejected(run):
    pb = _lattice((1, 1, 1))
    faces = pb.faces.tolist()
    cf = pb.cell_faces[0].tolist()
    # a triangular prism: nodes 0..5, two triangles and three quads
    prism_faces = [[0, 1, 2], [3, 4, 5], [0, 1, 4, 3], [1, 2, 5, 4], [2, 0, 3, 5]]
    res, _ = run(6, prism_faces, [[0, 1, 2, 3, 4]])
    assert res[0][0] == 2
    # a face listed out of cyclic order (its diagonal as an edge)
    bad = [list(f) for f in faces]
    f0 = bad[cf[0]]
    bad[cf[0]] = [f0[0], f0[2], f0[1], f0[3]]
    res, _ = run(pb.n_nodes, bad, [cf])
    assert res[0][0] == 2
    # a repeated face
    res, _ = run(pb.n_nodes, faces, [[cf[0], cf[0], cf[2], cf[3], cf[4], cf[5]]])
    assert res[0][0] == 2
    # five faces
    res, _ = run(pb.n_nodes, faces, [cf[:5]])
    assert res[0][0] == 2
    # a face id or a node id out of range
    res, _ = run(pb.n_nodes, faces, [[cf[0], cf[1], cf[2], cf[3], cf[4], len(faces)]])
    assert res[0][0] == 1
    res, _ = run(pb.n_nodes - 1, faces, [cf])
    assert res[0][0] == 1
    # fracture faces: a triangle is not a quadrilateral; out-of-range id
    _, qs = run(6, prism_faces, [], [0, 2, 7])
    assert [q[0] for q in qs] == [2, 0, 1]
    assert qs[1][1] == [0, 1, 4, 3]
