// From the general polyhedral mesh descriptor of Sec. 3.1 (faces as cyclic
// node lists, cells as face lists, fracture faces as face ids) to the
// hexahedral numbering the kernels run on.
//
// A cell is a hexahedron when it has six faces of four nodes, eight distinct
// nodes each on three of the faces, every node with three edge neighbours,
// and faces that are the six faces of that cube graph.  Its canonical local
// numbering, independent of the order in which faces and their nodes are
// listed: node 0 is the smallest node id; 1, 2, 4 are its edge neighbours in
// increasing id; 3 is the other common neighbour of 1 and 2, 5 of 1 and 4, 6
// of 2 and 4; 7 is the last node.  Node l then sits at the lattice offset
// (l & 1, (l >> 1) & 1, (l >> 2) & 1) of the cell, which is the fast path's
// convention, and on a lattice whose node ids grow with x, then y, then z it
// is exactly the lattice numbering.  (The local matrices use |det| of every
// sub-tetrahedron, so a mirror-image numbering gives the same matrix.)
//
// Host and device code: the assembly converts device descriptors with a
// kernel, the server converts host descriptors on the host, and a CPU test
// compiles this header with g++.
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define VAG_HEXMAP_HD __host__ __device__
#else
#define VAG_HEXMAP_HD
#endif

namespace vag {

enum : int { HEXMAP_OK = 0, HEXMAP_BAD_INDEX = 1, HEXMAP_NOT_HEX = 2 };

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

// The four nodes of fracture face `fid`, in the face's cyclic order.
VAG_HEXMAP_HD inline int quad_of_face(const int32_t *fptr, const int32_t *fidx, int64_t fidx_len, int32_t n_faces,
                                      int32_t n_nodes, int32_t fid, int32_t out[4]) {
  if (fid < 0 || fid >= n_faces) return HEXMAP_BAD_INDEX;
  const int64_t p0 = fptr[fid], p1 = fptr[fid + 1];
  if (p0 < 0 || p1 > fidx_len || p1 < p0) return HEXMAP_BAD_INDEX;
  if (p1 - p0 != 4) return HEXMAP_NOT_HEX;
  for (int t = 0; t < 4; ++t) {
    const int32_t v = fidx[p0 + t];
    if (v < 0 || v >= n_nodes) return HEXMAP_BAD_INDEX;
    out[t] = v;
  }
  return HEXMAP_OK;
}

}  // namespace vag
