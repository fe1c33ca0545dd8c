// From the general polyhedral mesh descriptor of Sec. 3.1 (faces as cyclic
// node lists, cells as face lists, fracture faces as face ids) to the padded
// per-shape numbering the kernels run on (vag_topo.h).
//
// A cell is recognised from its faces: six quadrilaterals form a hexahedron,
// four triangles a tetrahedron, two triangles and three quadrilaterals a
// prism, one quadrilateral and four triangles a pyramid; any other cell is
// rejected.  The local numbering is canonical, independent of the order in
// which faces and their nodes are listed:
//   hexahedron  node 0 is the smallest node id; 1, 2, 4 are its edge
//               neighbours in increasing id; 3 is the other common neighbour
//               of 1 and 2, 5 of 1 and 4, 6 of 2 and 4; 7 is the last node.
//               Node l then sits at the lattice offset (l & 1, (l >> 1) & 1,
//               (l >> 2) & 1), and on a lattice whose node ids grow with x,
//               then y, then z it is exactly the lattice numbering.
//   tetrahedron the four nodes in increasing id.
//   prism       node 0 is the smallest id, 1 and 2 the rest of its triangle
//               in increasing id, 3 + i the node joined to node i by a
//               lateral edge.
//   pyramid     0..3 the base from its smallest id towards its smaller
//               neighbour, 4 the apex.
// (The local matrices use |det| of every sub-tetrahedron, so a mirror-image
// numbering gives the same matrix.)
//
// Host and device code: the assembly converts device descriptors with a
// kernel, the server converts host descriptors on the host, and a CPU test
// compiles this header with g++.
#pragma once

#include <stdint.h>

#include "vag_topo.h"

#ifdef __CUDACC__
#define VAG_HEXMAP_HD __host__ __device__
#else
#define VAG_HEXMAP_HD
#endif

namespace vag {

enum : int { HEXMAP_OK = 0, HEXMAP_BAD_INDEX = 1, HEXMAP_NOT_HEX = 2, CELLMAP_UNSUPPORTED = 3 };

VAG_HEXMAP_HD inline int hexmap_popc(unsigned x) {
  int c = 0;
  for (; x; x &= x - 1) ++c;
  return c;
}

// the common edge neighbour of local nodes a and b other than k0, or -1
VAG_HEXMAP_HD inline int hexmap_common(const unsigned (&adj)[8], int a, int b, int k0) {
  const unsigned c = adj[a] & adj[b] & ~(1u << k0);
  if (hexmap_popc(c) != 1) return -1;
  for (int k = 0; k < 8; ++k)
    if (c & (1u << k)) return k;
  return -1;
}

// Canonical hexahedral numbering of cell K into out[8].
//   fptr [n_faces+1], fidx [fidx_len]: nodes of face f are fidx[fptr[f]..fptr[f+1])
//   cptr [n_cells+1], cidx [cidx_len]: faces of cell K are cidx[cptr[K]..cptr[K+1])
// Returns HEXMAP_OK, HEXMAP_BAD_INDEX (an offset or id out of range) or
// HEXMAP_NOT_HEX (the cell is not a hexahedron).
VAG_HEXMAP_HD inline int hex_from_faces(const int32_t *fptr, const int32_t *fidx, int64_t fidx_len,
                                        const int32_t *cptr, const int32_t *cidx, int64_t cidx_len, int32_t n_faces,
                                        int32_t n_nodes, int32_t K, int32_t out[8]) {
  const int64_t c0 = cptr[K], c1 = cptr[K + 1];
  if (c0 < 0 || c1 > cidx_len || c1 < c0) return HEXMAP_BAD_INDEX;
  if (c1 - c0 != 6) return HEXMAP_NOT_HEX;
  int32_t q[6][4];
  for (int f = 0; f < 6; ++f) {
    const int32_t fid = cidx[c0 + f];
    if (fid < 0 || fid >= n_faces) return HEXMAP_BAD_INDEX;
    const int64_t p0 = fptr[fid], p1 = fptr[fid + 1];
    if (p0 < 0 || p1 > fidx_len || p1 < p0) return HEXMAP_BAD_INDEX;
    if (p1 - p0 != 4) return HEXMAP_NOT_HEX;
    for (int t = 0; t < 4; ++t) {
      const int32_t v = fidx[p0 + t];
      if (v < 0 || v >= n_nodes) return HEXMAP_BAD_INDEX;
      q[f][t] = v;
    }
  }
  // the distinct nodes and how many faces carry each
  int32_t node[8];
  int cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int nn = 0;
  int loc[6][4];
  for (int f = 0; f < 6; ++f)
    for (int t = 0; t < 4; ++t) {
      int k = 0;
      while (k < nn && node[k] != q[f][t]) ++k;
      if (k == nn) {
        if (nn == 8) return HEXMAP_NOT_HEX;
        node[nn++] = q[f][t];
      }
      ++cnt[k];
      loc[f][t] = k;
    }
  if (nn != 8) return HEXMAP_NOT_HEX;
  for (int k = 0; k < 8; ++k)
    if (cnt[k] != 3) return HEXMAP_NOT_HEX;
  // edge graph: consecutive nodes of a face share an edge
  unsigned adj[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int f = 0; f < 6; ++f)
    for (int t = 0; t < 4; ++t) {
      const int a = loc[f][t], b = loc[f][(t + 1) & 3];
      if (a == b) return HEXMAP_NOT_HEX;
      adj[a] |= 1u << b;
      adj[b] |= 1u << a;
    }
  for (int k = 0; k < 8; ++k)
    if (hexmap_popc(adj[k]) != 3) return HEXMAP_NOT_HEX;
  // node 0: the smallest id; 1, 2, 4: its neighbours in increasing id
  int k0 = 0;
  for (int k = 1; k < 8; ++k)
    if (node[k] < node[k0]) k0 = k;
  int nb[3], m = 0;
  for (int k = 0; k < 8; ++k)
    if (adj[k0] & (1u << k)) nb[m++] = k;
  for (int i = 0; i < 3; ++i)
    for (int j = i + 1; j < 3; ++j)
      if (node[nb[j]] < node[nb[i]]) {
        const int tmp = nb[i];
        nb[i] = nb[j];
        nb[j] = tmp;
      }
  int L[8];
  L[0] = k0;
  L[1] = nb[0];
  L[2] = nb[1];
  L[4] = nb[2];
  L[3] = hexmap_common(adj, L[1], L[2], k0);
  L[5] = hexmap_common(adj, L[1], L[4], k0);
  L[6] = hexmap_common(adj, L[2], L[4], k0);
  if (L[3] < 0 || L[5] < 0 || L[6] < 0) return HEXMAP_NOT_HEX;
  unsigned used = 0;
  for (int l = 0; l < 8; ++l)
    if (l != 7) used |= 1u << L[l];
  if (hexmap_popc(used) != 7) return HEXMAP_NOT_HEX;
  L[7] = -1;
  for (int k = 0; k < 8; ++k)
    if (!(used & (1u << k))) L[7] = k;
  if ((adj[L[7]] & ((1u << L[3]) | (1u << L[5]) | (1u << L[6]))) !=
      ((1u << L[3]) | (1u << L[5]) | (1u << L[6])))
    return HEXMAP_NOT_HEX;
  // every face is one of the six faces of the cube numbering, as a node set
  int lof[8];
  for (int l = 0; l < 8; ++l) lof[L[l]] = l;
  for (int f = 0; f < 6; ++f) {
    unsigned set = 0;
    for (int t = 0; t < 4; ++t) set |= 1u << lof[loc[f][t]];
    const bool ok = set == 0x55u /* 0 2 4 6 */ || set == 0xAAu /* 1 3 5 7 */ || set == 0x33u /* 0 1 4 5 */ ||
                    set == 0xCCu /* 2 3 6 7 */ || set == 0x0Fu /* 0 1 2 3 */ || set == 0xF0u /* 4 5 6 7 */;
    if (!ok) return HEXMAP_NOT_HEX;
  }
  for (int l = 0; l < 8; ++l) out[l] = node[L[l]];
  return HEXMAP_OK;
}

// The nodes of fracture face `fid` in the face's cyclic order: 3 or 4 of
// them, out[3] = -1 for a triangle.
VAG_HEXMAP_HD inline int face_nodes_of(const int32_t *fptr, const int32_t *fidx, int64_t fidx_len, int32_t n_faces,
                                       int32_t n_nodes, int32_t fid, int32_t out[4]) {
  if (fid < 0 || fid >= n_faces) return HEXMAP_BAD_INDEX;
  const int64_t p0 = fptr[fid], p1 = fptr[fid + 1];
  if (p0 < 0 || p1 > fidx_len || p1 < p0) return HEXMAP_BAD_INDEX;
  if (p1 - p0 != 3 && p1 - p0 != 4) return CELLMAP_UNSUPPORTED;
  out[3] = -1;
  for (int t = 0; t < (int)(p1 - p0); ++t) {
    const int32_t v = fidx[p0 + t];
    if (v < 0 || v >= n_nodes) return HEXMAP_BAD_INDEX;
    out[t] = v;
  }
  for (int t = 0; t < (int)(p1 - p0); ++t)
    for (int u = t + 1; u < (int)(p1 - p0); ++u)
      if (out[t] == out[u]) return CELLMAP_UNSUPPORTED;
  return HEXMAP_OK;
}

// Any of the four shapes: writes the canonical numbering into out[8] (-1 in
// the unused slots) and the shape (topo::HEX ...) into *shape.  Same
// arguments and return values as hex_from_faces, plus CELLMAP_UNSUPPORTED
// for a cell of none of the shapes.
VAG_HEXMAP_HD inline int cell_from_faces(const int32_t *fptr, const int32_t *fidx, int64_t fidx_len,
                                         const int32_t *cptr, const int32_t *cidx, int64_t cidx_len, int32_t n_faces,
                                         int32_t n_nodes, int32_t K, int32_t out[8], int *shape) {
  for (int l = 0; l < 8; ++l) out[l] = -1;
  *shape = -1;
  const int64_t c0 = cptr[K], c1 = cptr[K + 1];
  if (c0 < 0 || c1 > cidx_len || c1 < c0) return HEXMAP_BAD_INDEX;
  const int nfc = (int)(c1 - c0);
  if (nfc < 4 || nfc > 6) return CELLMAP_UNSUPPORTED;
  int32_t q[6][4];
  int sz[6], n3 = 0, n4 = 0;
  for (int f = 0; f < nfc; ++f) {
    const int e = face_nodes_of(fptr, fidx, fidx_len, n_faces, n_nodes, cidx[c0 + f], q[f]);
    if (e != HEXMAP_OK) return e;
    sz[f] = q[f][3] < 0 ? 3 : 4;
    (sz[f] == 3 ? n3 : n4) += 1;
  }
  if (nfc == 6 && n4 == 6) {
    const int e = hex_from_faces(fptr, fidx, fidx_len, cptr, cidx, cidx_len, n_faces, n_nodes, K, out);
    if (e == HEXMAP_OK) *shape = topo::HEX;
    return e == HEXMAP_NOT_HEX ? CELLMAP_UNSUPPORTED : e;
  }
  // distinct nodes, the faces each lies on, and the edge graph
  int32_t node[8];
  unsigned onf[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int nn = 0;
  int loc[6][4];
  for (int f = 0; f < nfc; ++f)
    for (int t = 0; t < sz[f]; ++t) {
      int k = 0;
      while (k < nn && node[k] != q[f][t]) ++k;
      if (k == nn) {
        if (nn == 8) return CELLMAP_UNSUPPORTED;
        node[nn++] = q[f][t];
      }
      onf[k] |= 1u << f;
      loc[f][t] = k;
    }
  unsigned adj[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int f = 0; f < nfc; ++f)
    for (int t = 0; t < sz[f]; ++t) {
      const int a = loc[f][t], b = loc[f][(t + 1) % sz[f]];
      adj[a] |= 1u << b;
      adj[b] |= 1u << a;
    }
  int L[8];
  int sh = -1;
  if (nfc == 4 && n3 == 4 && nn == 4) {
    // tetrahedron: four nodes, each face misses a different one
    for (int k = 0; k < 4; ++k) L[k] = k;
    for (int i = 0; i < 4; ++i)
      for (int j = i + 1; j < 4; ++j)
        if (node[L[j]] < node[L[i]]) { const int t = L[i]; L[i] = L[j]; L[j] = t; }
    unsigned missed = 0;
    for (int f = 0; f < 4; ++f) {
      unsigned set = 0;
      for (int t = 0; t < 3; ++t) set |= 1u << loc[f][t];
      if (hexmap_popc(set) != 3) return CELLMAP_UNSUPPORTED;
      missed |= 0xFu & ~set;
    }
    if (missed != 0xFu) return CELLMAP_UNSUPPORTED;
    sh = topo::TET;
  } else if (nfc == 5 && n3 == 2 && n4 == 3 && nn == 6) {
    // prism: the two triangles are disjoint; each lateral quadrilateral joins
    // an edge of one to an edge of the other
    int t0 = -1, t1 = -1;
    for (int f = 0; f < 5; ++f)
      if (sz[f] == 3) (t0 < 0 ? t0 : t1) = f;
    unsigned A = 0, B = 0;
    for (int t = 0; t < 3; ++t) { A |= 1u << loc[t0][t]; B |= 1u << loc[t1][t]; }
    if (hexmap_popc(A) != 3 || hexmap_popc(B) != 3 || (A & B)) return CELLMAP_UNSUPPORTED;
    int k0 = 0;
    for (int k = 1; k < 6; ++k)
      if (node[k] < node[k0]) k0 = k;
    const unsigned bot = (A >> k0) & 1u ? A : B, top = bot == A ? B : A;
    L[0] = k0;
    int m = 1;
    for (int k = 0; k < 6; ++k)
      if (((bot >> k) & 1u) && k != k0) L[m++] = k;
    if (node[L[2]] < node[L[1]]) { const int t = L[1]; L[1] = L[2]; L[2] = t; }
    for (int i = 0; i < 3; ++i) {
      const unsigned up = adj[L[i]] & top;     // the lateral edge of node i
      if (hexmap_popc(up) != 1) return CELLMAP_UNSUPPORTED;
      for (int k = 0; k < 6; ++k)
        if ((up >> k) & 1u) L[3 + i] = k;
    }
    if (L[3] == L[4] || L[4] == L[5] || L[3] == L[5]) return CELLMAP_UNSUPPORTED;
    sh = topo::PRISM;
  } else if (nfc == 5 && n3 == 4 && n4 == 1 && nn == 5) {
    // pyramid: the quadrilateral is the base, the node off it the apex
    int fb = 0;
    while (sz[fb] != 4) ++fb;
    int apex = -1;
    for (int k = 0; k < 5; ++k)
      if (!((onf[k] >> fb) & 1u)) apex = k;
    if (apex < 0) return CELLMAP_UNSUPPORTED;
    int t0 = 0;
    for (int t = 1; t < 4; ++t)
      if (node[loc[fb][t]] < node[loc[fb][t0]]) t0 = t;
    const int nxt = loc[fb][(t0 + 1) & 3], prv = loc[fb][(t0 + 3) & 3];
    const int dir = node[nxt] < node[prv] ? 1 : 3;
    for (int i = 0; i < 4; ++i) L[i] = loc[fb][(t0 + dir * i) & 3];
    L[4] = apex;
    sh = topo::PYRAMID;
  } else {
    return CELLMAP_UNSUPPORTED;
  }
  // every face must be one of the shape's faces, as a node set, and every
  // face of the shape must be listed once
  int lof[8];
  for (int l = 0; l < topo::n_nodes(sh); ++l) lof[L[l]] = l;
  unsigned seen = 0;
  for (int f = 0; f < nfc; ++f) {
    unsigned set = 0;
    for (int t = 0; t < sz[f]; ++t) set |= 1u << lof[loc[f][t]];
    int match = -1;
    for (int lf = 0; lf < topo::n_faces(sh); ++lf) {
      unsigned ref = 0;
      for (int t = 0; t < topo::face_size(sh, lf); ++t) ref |= 1u << topo::face(sh, lf, t);
      if (ref == set && topo::face_size(sh, lf) == sz[f]) match = lf;
    }
    if (match < 0 || ((seen >> match) & 1u)) return CELLMAP_UNSUPPORTED;
    seen |= 1u << match;
    // consecutive entries of the listed face must be edges of the shape
    for (int t = 0; t < sz[f]; ++t) {
      const int a = lof[loc[f][t]], b = lof[loc[f][(t + 1) % sz[f]]];
      if (topo::pos_on_face(sh, match, a) < 0 || topo::pos_on_face(sh, match, b) < 0) return CELLMAP_UNSUPPORTED;
      const int pa = topo::pos_on_face(sh, match, a), pb = topo::pos_on_face(sh, match, b);
      const int n = sz[f];
      if ((pa + 1) % n != pb && (pb + 1) % n != pa) return CELLMAP_UNSUPPORTED;
    }
  }
  for (int l = 0; l < topo::n_nodes(sh); ++l) out[l] = node[L[l]];
  *shape = sh;
  return HEXMAP_OK;
}

}  // namespace vag
