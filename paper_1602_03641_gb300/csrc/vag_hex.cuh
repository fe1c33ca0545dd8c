// Local numbering of a hexahedral cell (the library's own table).
// Node l sits at lattice offset (l & 1, (l >> 1) & 1, (l >> 2) & 1).  The six
// faces, in the order -x, +x, -y, +y, -z, +z, list their nodes cyclically so
// that consecutive entries share an edge e (the triangles T_{sigma,e} and the
// tetrahedra T_{K,sigma,e} of Sec. 3.1 are built on those edges).
#pragma once

namespace vag {
namespace hex {

__host__ __device__ constexpr unsigned pack4(unsigned a, unsigned b, unsigned c, unsigned d) {
  return a | (b << 3) | (c << 6) | (d << 9);
}

__host__ __device__ constexpr unsigned face_packed(int lf) {
  return lf == 0 ? pack4(0, 2, 6, 4)
       : lf == 1 ? pack4(1, 3, 7, 5)
       : lf == 2 ? pack4(0, 1, 5, 4)
       : lf == 3 ? pack4(2, 3, 7, 6)
       : lf == 4 ? pack4(0, 1, 3, 2)
                 : pack4(4, 5, 7, 6);
}

// node (0..7) at position t (0..3) of local face lf (0..5)
__host__ __device__ constexpr int face(int lf, int t) { return (int)((face_packed(lf) >> (3 * t)) & 7u); }

// position of local node a on local face lf, or -1
__host__ __device__ constexpr int pos_on_face(int lf, int a) {
  return face(lf, 0) == a ? 0 : face(lf, 1) == a ? 1 : face(lf, 2) == a ? 2 : face(lf, 3) == a ? 3 : -1;
}

// packed upper-triangle index of (i, j), i <= j, in a 9x9 symmetric matrix
// over (K, n0..n7)
__host__ __device__ constexpr int pidx(int i, int j) {
  return i <= j ? i * 9 - (i * (i - 1)) / 2 + (j - i) : j * 9 - (j * (j - 1)) / 2 + (i - j);
}
constexpr int kPacked = 45;

}  // namespace hex
}  // namespace vag
