// Dense <-> tile conversion for sp2_create_dense and sp2_copy_D_dense.
//
// Section 1 states the problem for an N x N matrix F; the library works on
// 32 x 32 tiles of its upper block triangle (Section 5: symmetric storage,
// only the upper triangle is stored).  These kernels cut a dense row-major
// matrix into those tiles (leaving out the tiles that are exactly zero, keeping
// every diagonal tile) and assemble a dense matrix from the stored tiles of a
// symmetric tile set (each off-diagonal tile written twice, once transposed).
#include "sp2_internal.h"

namespace sp2 {
namespace {

constexpr int WARPS = 8;   // one warp per tile, 8 tiles per CTA

// flag[I * nb + J] = 1 iff J >= I and (I == J or tile (I, J) of F has a nonzero)
__global__ void __launch_bounds__(32 * WARPS)
    k_dense_tile_flags(const double* __restrict__ F, int64_t n, int64_t ld, int nb, int32_t* flag) {
  const int I = blockIdx.y;
  const int J = blockIdx.x * WARPS + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (J >= nb) return;
  int f = 0;
  if (J == I) {
    f = 1;
  } else if (J > I) {
    const int64_t c = (int64_t)J * TB + lane;
    bool nz = false;
    if (c < n) {
      for (int r = 0; r < TB; ++r) {
        const int64_t row = (int64_t)I * TB + r;
        if (row >= n) break;
        nz |= F[row * ld + c] != 0.0;
      }
    }
    f = __any_sync(0xffffffffu, nz) ? 1 : 0;
  }
  if (lane == 0) flag[(int64_t)I * nb + J] = f;
}

// Copies every flagged tile to position pos[I * nb + J] of the tile arrays
// (rows of a tile are coalesced 256-byte reads; rows and columns >= n are 0).
__global__ void __launch_bounds__(32 * WARPS)
    k_dense_tile_fill(const double* __restrict__ F, int64_t n, int64_t ld, int nb, const int32_t* __restrict__ flag,
                      const int32_t* __restrict__ pos, int32_t* brow, int32_t* bcol, double* pool) {
  const int I = blockIdx.y;
  const int J = blockIdx.x * WARPS + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (J >= nb || J < I) return;
  const int64_t e = (int64_t)I * nb + J;
  if (!flag[e]) return;
  const int64_t t = pos[e];
  if (lane == 0) {
    brow[t] = I;
    bcol[t] = J;
  }
  double* dst = pool + t * TE;
  const int64_t c = (int64_t)J * TB + lane;
  for (int r = 0; r < TB; ++r) {
    const int64_t row = (int64_t)I * TB + r;
    dst[r * TB + lane] = (row < n && c < n) ? F[row * ld + c] : 0.0;
  }
}

// out (n x n, leading dimension ld, zeroed by the caller) := the symmetric
// matrix whose upper tiles are given: tile (I, J) and, for I != J, its
// transpose at (J, I).  One warp per tile.
__global__ void __launch_bounds__(32 * WARPS)
    k_tiles_to_dense(const int32_t* __restrict__ brow, const int32_t* __restrict__ bcol,
                     const double* __restrict__ val, int64_t nnzb, int64_t n, int64_t ld, double* out) {
  const int64_t t = (int64_t)blockIdx.x * WARPS + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (t >= nnzb) return;
  const int I = brow[t], J = bcol[t];
  const double* src = val + t * TE;
  for (int r = 0; r < TB; ++r) {
    const int64_t row = (int64_t)I * TB + r, col = (int64_t)J * TB + lane;
    const double v = src[r * TB + lane];
    if (row < n && col < n) {
      out[row * ld + col] = v;
      if (I != J) out[col * ld + row] = v;
    }
  }
}

}  // namespace

cudaError_t launch_dense_tile_flags(const double* F, int64_t n, int64_t ld, int nb, int32_t* flag, cudaStream_t st) {
  const dim3 grid((unsigned)((nb + WARPS - 1) / WARPS), (unsigned)nb);
  ++g_launches;
  k_dense_tile_flags<<<grid, 32 * WARPS, 0, st>>>(F, n, ld, nb, flag);
  return cudaGetLastError();
}

cudaError_t launch_dense_tile_fill(const double* F, int64_t n, int64_t ld, int nb, const int32_t* flag,
                                   const int32_t* pos, int32_t* brow, int32_t* bcol, double* pool, cudaStream_t st) {
  const dim3 grid((unsigned)((nb + WARPS - 1) / WARPS), (unsigned)nb);
  ++g_launches;
  k_dense_tile_fill<<<grid, 32 * WARPS, 0, st>>>(F, n, ld, nb, flag, pos, brow, bcol, pool);
  return cudaGetLastError();
}

cudaError_t launch_tiles_to_dense(const int32_t* brow, const int32_t* bcol, const double* val, int64_t nnzb,
                                  int64_t n, int64_t ld, double* out, cudaStream_t st) {
  cudaError_t e = cudaMemset2DAsync(out, (size_t)ld * 8, 0, (size_t)n * 8, (size_t)n, st);
  if (e != cudaSuccess || nnzb == 0) return e;
  ++g_launches;
  k_tiles_to_dense<<<(unsigned)((nnzb + WARPS - 1) / WARPS), 32 * WARPS, 0, st>>>(brow, bcol, val, nnzb, n, ld, out);
  return cudaGetLastError();
}

}  // namespace sp2
