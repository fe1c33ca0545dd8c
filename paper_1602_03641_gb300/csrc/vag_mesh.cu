// The general polyhedral mesh descriptor of Sec. 3.1 (faces as cyclic node
// lists, cells as face lists, fracture faces as face ids) turned into the
// padded per-shape numbering on the device: one thread per cell recognises
// its shape and writes its canonical numbering (vag_cellmap.h), one thread
// per fracture face writes its three or four nodes.
#include <vector>

#include "vag_cellmap.h"
#include "vag_internal.cuh"

namespace vag {
namespace {

__global__ void k_cells_from_faces(int nc, const int32_t *__restrict__ fptr, const int32_t *__restrict__ fidx,
                                   int64_t fidx_len, const int32_t *__restrict__ cptr,
                                   const int32_t *__restrict__ cidx, int64_t cidx_len, int n_faces, int n_nodes,
                                   int32_t *__restrict__ cell_nodes, int8_t *__restrict__ cell_shape, int *err,
                                   unsigned *shapes) {
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= nc) return;
  int32_t out[8];
  int sh = 0;
  const int e = cell_from_faces(fptr, fidx, fidx_len, cptr, cidx, cidx_len, n_faces, n_nodes, K, out, &sh);
  if (e != HEXMAP_OK) {
    atomicOr(err, 1 << e);
    for (int l = 0; l < 8; ++l) out[l] = l < 4 ? 0 : -1;   // a valid placeholder; the call fails
    sh = topo::TET;
  }
  for (int l = 0; l < 8; ++l) cell_nodes[8 * (size_t)K + l] = out[l];
  cell_shape[K] = (int8_t)sh;
  atomicOr(shapes, 1u << sh);
}

__global__ void k_ffaces_of_faces(int nf, const int32_t *__restrict__ fptr, const int32_t *__restrict__ fidx,
                                  int64_t fidx_len, int n_faces, int n_nodes, const int32_t *__restrict__ ffid,
                                  int32_t *__restrict__ ff_nodes, int *err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nf) return;
  int32_t out[4];
  const int e = face_nodes_of(fptr, fidx, fidx_len, n_faces, n_nodes, ffid[i], out);
  if (e != HEXMAP_OK) {
    atomicOr(err, 1 << e);
    for (int t = 0; t < 4; ++t) out[t] = 0;
  }
  if (out[3] < 0) atomicOr(err, 1 << 8);   // a triangle
  for (int t = 0; t < 4; ++t) ff_nodes[4 * (size_t)i + t] = out[t];
}

// stream-ordered temporaries of the context's pool, freed on every path
struct Temps {
  Ctx *c;
  std::vector<void *> p;
  ~Temps() {
    for (void *q : p) ctx_free(c, q);
  }
  template <class T>
  T *get(size_t n) {
    T *q = static_cast<T *>(ctx_alloc(c, (n ? n : 1) * sizeof(T)));
    p.push_back(q);
    return q;
  }
};

}  // namespace

unsigned general_to_cells(Ctx *c, const vag_mesh &m, int mem, int32_t *cell_nodes, int32_t *ff_nodes,
                          int8_t *cell_shape, bool *tri_ff) {
  if (!m.face_node_ptr || !m.face_node_idx || !m.cell_face_ptr || !m.cell_face_idx || (m.n_ff && !m.ff_face_ids))
    fail(VAG_EINVAL, "general mesh descriptor: a face or cell array is NULL");
  if (m.n_faces <= 0) fail(VAG_EINVAL, "general mesh descriptor: n_faces must be positive");
  cudaStream_t st = c->stream;
  Temps tmp{c, {}};
  // the index arrays' lengths are the last offsets
  int32_t flen = 0, clen = 0;
  if (mem == VAG_MEM_HOST) {
    flen = m.face_node_ptr[m.n_faces];
    clen = m.cell_face_ptr[m.n_cells];
  } else {
    VAG_CUDA(cudaMemcpyAsync(&flen, m.face_node_ptr + m.n_faces, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    VAG_CUDA(cudaMemcpyAsync(&clen, m.cell_face_ptr + m.n_cells, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    VAG_CUDA(cudaStreamSynchronize(st));
  }
  if (flen < 0 || clen < 0) fail(VAG_EINVAL, "general mesh descriptor: negative offsets");
  const int32_t *fptr = m.face_node_ptr, *fidx = m.face_node_idx, *cptr = m.cell_face_ptr, *cidx = m.cell_face_idx,
                *ffid = m.ff_face_ids;
  if (mem == VAG_MEM_HOST) {   // device copies of the caller's host arrays
    auto up = [&](const int32_t *src, size_t n) {
      int32_t *d = tmp.get<int32_t>(n);
      if (n) VAG_CUDA(cudaMemcpyAsync(d, src, sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
      return (const int32_t *)d;
    };
    fptr = up(m.face_node_ptr, (size_t)m.n_faces + 1);
    fidx = up(m.face_node_idx, (size_t)flen);
    cptr = up(m.cell_face_ptr, (size_t)m.n_cells + 1);
    cidx = up(m.cell_face_idx, (size_t)clen);
    ffid = m.n_ff ? up(m.ff_face_ids, (size_t)m.n_ff) : nullptr;
  }
  int *err = tmp.get<int>(2);
  unsigned *shapes = reinterpret_cast<unsigned *>(err + 1);
  VAG_CUDA(cudaMemsetAsync(err, 0, 2 * sizeof(int), st));
  k_cells_from_faces<<<grid_for(m.n_cells, 128), 128, 0, st>>>(m.n_cells, fptr, fidx, flen, cptr, cidx, clen,
                                                                m.n_faces, m.n_nodes, cell_nodes, cell_shape, err,
                                                                shapes);
  note_launches(1);
  if (m.n_ff) {
    k_ffaces_of_faces<<<grid_for(m.n_ff, 128), 128, 0, st>>>(m.n_ff, fptr, fidx, flen, m.n_faces, m.n_nodes, ffid,
                                                              ff_nodes, err);
    note_launches(1);
  }
  VAG_CHECK_LAUNCH();
  int herr[2] = {0, 0};
  VAG_CUDA(cudaMemcpyAsync(herr, err, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  VAG_CUDA(cudaStreamSynchronize(st));
  if (herr[0] & (1 << HEXMAP_BAD_INDEX)) fail(VAG_EINVAL, "general mesh descriptor: an offset or id out of range");
  if (herr[0] & ((1 << HEXMAP_NOT_HEX) | (1 << CELLMAP_UNSUPPORTED)))
    fail(VAG_EMESH, "a cell is not a hexahedron, tetrahedron, prism or pyramid, or a fracture face has neither "
                    "three nor four distinct nodes");
  *tri_ff = (herr[0] & (1 << 8)) != 0;
  return (unsigned)herr[1];
}

}  // namespace vag
