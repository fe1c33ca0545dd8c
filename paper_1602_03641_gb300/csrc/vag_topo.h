// Local numbering of the cell shapes the kernels take (the library's own
// tables).  Sec. 3.1 admits any polyhedral cell; the kernels take the four
// shapes of the paper's meshes and their usual mixes: hexahedra (Cartesian
// and corner-point grids), tetrahedra (Sec. 5.4), triangular prisms (the
// extruded triangular mesh of Sec. 5.5) and pyramids (the transition between
// hexahedra and tetrahedra).  A cell keeps 8 node slots and 6 face slots
// whatever its shape; unused slots hold -1.
//
// Every face lists its nodes cyclically, so that consecutive entries share an
// edge e of the face (the triangles T_{sigma,e} and the tetrahedra
// T_{K,sigma,e} of Sec. 3.1 are built on those edges).
//
//   HEX      node l at the lattice offset (l & 1, (l >> 1) & 1, (l >> 2) & 1);
//            faces -x, +x, -y, +y, -z, +z.
//   TET      nodes 0..3; face l is the one opposite node l.
//   PRISM    nodes 0 1 2 the bottom triangle, 3 4 5 the top one with node
//            3 + i joined to node i by a lateral edge; faces bottom, top and
//            the quadrilaterals on the bottom edges 01, 12, 20.
//   PYRAMID  nodes 0 1 2 3 the base in cyclic order, 4 the apex; faces the
//            base and the triangles on the base edges 01, 12, 23, 30.
//
// Host and device code (a CPU test compiles it with g++).
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define VAG_TOPO_HD __host__ __device__
#else
#define VAG_TOPO_HD
#endif

namespace vag {
namespace topo {

enum : int { HEX = 0, TET = 1, PRISM = 2, PYRAMID = 3, N_SHAPES = 4 };
constexpr int kMaxNodes = 8, kMaxFaces = 6, kMaxFaceNodes = 4;

VAG_TOPO_HD constexpr int n_nodes(int sh) { return sh == HEX ? 8 : sh == TET ? 4 : sh == PRISM ? 6 : 5; }
VAG_TOPO_HD constexpr int n_faces(int sh) { return sh == HEX ? 6 : sh == TET ? 4 : 5; }

// four 4-bit node entries, 0xF = no node
VAG_TOPO_HD constexpr unsigned pk(unsigned a, unsigned b, unsigned c, unsigned d = 0xFu) {
  return a | (b << 4) | (c << 8) | (d << 12);
}

VAG_TOPO_HD constexpr unsigned face_packed(int sh, int lf) {
  return sh == HEX ? (lf == 0 ? pk(0, 2, 6, 4) : lf == 1 ? pk(1, 3, 7, 5) : lf == 2 ? pk(0, 1, 5, 4)
                      : lf == 3 ? pk(2, 3, 7, 6) : lf == 4 ? pk(0, 1, 3, 2) : lf == 5 ? pk(4, 5, 7, 6) : 0xFFFFu)
       : sh == TET ? (lf == 0 ? pk(1, 2, 3) : lf == 1 ? pk(0, 3, 2) : lf == 2 ? pk(0, 1, 3)
                      : lf == 3 ? pk(0, 2, 1) : 0xFFFFu)
       : sh == PRISM ? (lf == 0 ? pk(0, 1, 2) : lf == 1 ? pk(3, 4, 5) : lf == 2 ? pk(0, 1, 4, 3)
                        : lf == 3 ? pk(1, 2, 5, 4) : lf == 4 ? pk(2, 0, 3, 5) : 0xFFFFu)
                     : (lf == 0 ? pk(0, 1, 2, 3) : lf == 1 ? pk(0, 1, 4) : lf == 2 ? pk(1, 2, 4)
                        : lf == 3 ? pk(2, 3, 4) : lf == 4 ? pk(3, 0, 4) : 0xFFFFu);
}

// node at position t (0..3) of local face lf, or -1
VAG_TOPO_HD constexpr int face(int sh, int lf, int t) {
  return ((face_packed(sh, lf) >> (4 * t)) & 0xFu) == 0xFu ? -1 : (int)((face_packed(sh, lf) >> (4 * t)) & 0xFu);
}

// number of nodes of local face lf (3 or 4; 0 past the last face)
VAG_TOPO_HD constexpr int face_size(int sh, int lf) {
  return face(sh, lf, 0) < 0 ? 0 : face(sh, lf, 3) < 0 ? 3 : 4;
}

// position of local node a on local face lf, or -1
VAG_TOPO_HD constexpr int pos_on_face(int sh, int lf, int a) {
  return face(sh, lf, 0) == a ? 0 : face(sh, lf, 1) == a ? 1 : face(sh, lf, 2) == a ? 2
       : (face(sh, lf, 3) == a && a >= 0) ? 3 : -1;
}

// packed upper-triangle index of (i, j) in a symmetric 9x9 matrix over
// (K, node slots 0..7)
VAG_TOPO_HD constexpr int pidx(int i, int j) {
  return i <= j ? i * 9 - (i * (i - 1)) / 2 + (j - i) : j * 9 - (j * (j - 1)) / 2 + (i - j);
}
constexpr int kPacked = 45;

}  // namespace topo
}  // namespace vag
