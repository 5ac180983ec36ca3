// General (non-symmetric) storage of the iterates, the alternative to the
// symmetric storage of Section 5: every tile of both triangles is stored and
// every output tile of the square is computed, as the general-matrix
// implementation of the paper does (its symmetric counterpart stores only the
// upper triangle and is about twice as fast, Section 6).  The iterates are
// still symmetric matrices, so their tile pattern is symmetric and the
// truncation keeps or drops a tile together with its mirror (the selection is
// the one of the symmetric storage, made on the upper tiles).
//
// A general tile set is sorted by (I, J) over both triangles.  The product
// C = A B reads A by rows (CSR: the set itself) and B by columns (CSC: for
// column J the tiles (K, J), used untransposed).
#include "sp2_internal.h"

namespace sp2 {
namespace {

__device__ __forceinline__ int64_t lower_bound_col(const int32_t* __restrict__ col, int64_t lo, int64_t hi,
                                                   int32_t v) {
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (col[mid] < v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// bit J of row I for every stored tile (I, J) (one triangle or both)
__global__ void k_bits_general(const int32_t* __restrict__ brow, const int32_t* __restrict__ bcol, int64_t nnzb,
                               uint32_t* bits, int words) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nnzb) return;
  const int i = brow[t], j = bcol[t];
  atomicOr(&bits[(int64_t)i * words + (j >> 5)], 1u << (j & 31));
}

// CSC references of a general set with a symmetric pattern: tile t = (J, K)
// of row J stands for column J's entry K, i.e. the tile (K, J), found in row K
// and used untransposed (REF_T).  ref = that tile's slot (slot != nullptr) or
// its index.
__global__ void k_csc_refs(const int32_t* __restrict__ brow, const int32_t* __restrict__ bcol,
                           const int32_t* __restrict__ rowptr, const int32_t* __restrict__ slot, int64_t nnzb,
                           uint32_t* ref) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nnzb) return;
  const int J = brow[t], K = bcol[t];
  const int64_t u = lower_bound_col(bcol, rowptr[K], rowptr[K + 1], J);
  ref[t] = (uint32_t)(slot ? slot[u] : (int32_t)u) | REF_T;
}

// General set from the both-triangle view of a symmetric set: entry p of the
// view (row R, column col[p], stored tile ref[p], transposed when REF_T) becomes
// tile p = (R, col[p]) with its own values.  One CTA of 256 threads per row.
__global__ void __launch_bounds__(256)
    k_expand_general(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                     const uint32_t* __restrict__ ref, const double* __restrict__ src, int32_t* brow,
                     int32_t* bcol, double* dst) {
  const int R = blockIdx.x;
  for (int p = rowptr[R]; p < rowptr[R + 1]; ++p) {
    const uint32_t r = ref[p];
    const double* s = src + (int64_t)(r & ~REF_T) * TE;
    double* d = dst + (int64_t)p * TE;
    const bool tr = (r & REF_T) != 0;
    for (int e = threadIdx.x; e < TE; e += 256) {
      const int i = e >> 5, j = e & 31;
      d[e] = tr ? s[j * TB + i] : s[e];
    }
    if (threadIdx.x == 0) {
      brow[p] = R;
      bcol[p] = col[p];
    }
  }
}

__global__ void k_upper_flags(const int32_t* __restrict__ brow, const int32_t* __restrict__ bcol, int64_t nnzb,
                              int32_t* flag) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < nnzb) flag[t] = brow[t] <= bcol[t] ? 1 : 0;
}

// keep[t] of every tile of a general set from the keep flags of its upper
// tiles (keepU, indexed by the exclusive scan posU of the upper flags): a lower
// tile (I, J), I > J, takes the flag of its mirror (J, I).
__global__ void k_general_keep(const int32_t* __restrict__ brow, const int32_t* __restrict__ bcol,
                               const int32_t* __restrict__ rowptr, const int32_t* __restrict__ posU,
                               const int32_t* __restrict__ keepU, int64_t nnzb, int32_t* keep) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nnzb) return;
  const int I = brow[t], J = bcol[t];
  int64_t u = t;
  if (I > J) u = lower_bound_col(bcol, rowptr[J], rowptr[J + 1], I);
  keep[t] = keepU[posU[u]];
}

inline unsigned grid_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_bits_general(const TileSet& s, int nb, int words, uint32_t* bits, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(bits, 0, (size_t)nb * words * 4, st);
  if (e != cudaSuccess || s.nnzb == 0) return e;
  ++g_launches;
  k_bits_general<<<grid_for(s.nnzb, 256), 256, 0, st>>>(s.brow, s.bcol, s.nnzb, bits, words);
  return cudaGetLastError();
}

cudaError_t launch_csc_refs(const TileSet& s, const int32_t* slot, uint32_t* ref, cudaStream_t st) {
  if (s.nnzb == 0) return cudaSuccess;
  ++g_launches;
  k_csc_refs<<<grid_for(s.nnzb, 256), 256, 0, st>>>(s.brow, s.bcol, s.rowptr, slot, s.nnzb, ref);
  return cudaGetLastError();
}

cudaError_t launch_expand_general(const FullPattern& fp, int nb, const double* src, int32_t* brow, int32_t* bcol,
                                  double* dst, cudaStream_t st) {
  if (nb == 0) return cudaSuccess;
  ++g_launches;
  k_expand_general<<<(unsigned)nb, 256, 0, st>>>(fp.rowptr, fp.col, fp.ref, src, brow, bcol, dst);
  return cudaGetLastError();
}

cudaError_t launch_upper_flags(const TileSet& s, int32_t* flag, cudaStream_t st) {
  if (s.nnzb == 0) return cudaSuccess;
  ++g_launches;
  k_upper_flags<<<grid_for(s.nnzb, 256), 256, 0, st>>>(s.brow, s.bcol, s.nnzb, flag);
  return cudaGetLastError();
}

cudaError_t launch_general_keep(const TileSet& s, const int32_t* posU, const int32_t* keepU, int32_t* keep,
                                cudaStream_t st) {
  if (s.nnzb == 0) return cudaSuccess;
  ++g_launches;
  k_general_keep<<<grid_for(s.nnzb, 256), 256, 0, st>>>(s.brow, s.bcol, s.rowptr, posU, keepU, s.nnzb, keep);
  return cudaGetLastError();
}

}  // namespace sp2
