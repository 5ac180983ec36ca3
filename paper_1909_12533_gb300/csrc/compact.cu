// Compaction after truncation (integer, bit-exact): keep flags -> exclusive scan
// -> scatter of the tile index (row, column, value slot) -> row pointers.  Tile
// values are not moved: the kept tiles keep their slots in the value pool that
// the fused epilogue wrote, and the next step writes into the other pool.
#include "sp2_internal.h"

namespace sp2 {
namespace {

__global__ void k_scatter(const int32_t* __restrict__ keep, const int32_t* __restrict__ pos, int64_t n,
                          const int32_t* __restrict__ brow, const int32_t* __restrict__ bcol,
                          const int32_t* __restrict__ slot, int32_t* obrow, int32_t* obcol, int32_t* oslot) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n || !keep[t]) return;
  const int32_t p = pos[t];
  obrow[p] = brow[t];
  obcol[p] = bcol[t];
  oslot[p] = slot ? slot[t] : (int32_t)t;
}

// dst tile t = pool tile slot[t] (contiguous copy for the caller's view of D).
__global__ void k_gather(const int32_t* __restrict__ slot, const double* __restrict__ pool, double* dst) {
  const int64_t t = blockIdx.x;
  const double2* s = reinterpret_cast<const double2*>(pool + (int64_t)slot[t] * TE);
  double2* d = reinterpret_cast<double2*>(dst + t * TE);
  for (int q = threadIdx.x; q < TE / 2; q += blockDim.x) d[q] = s[q];
}

__global__ void k_copy2(const int32_t* __restrict__ a, const int32_t* __restrict__ b, int64_t n, int32_t* oa,
                        int32_t* ob) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  oa[t] = a[t];
  ob[t] = b[t];
}

inline unsigned grid_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_compact(const TileSet& in, const int32_t* keep, int nb, TileSet& out, int32_t* count_dev,
                           void* scan_tmp, int32_t* scan_buf, cudaStream_t st) {
  cudaError_t e = launch_scan_i32(keep, scan_buf, in.nnzb, count_dev, scan_tmp, st);
  if (e != cudaSuccess) return e;
  if (in.nnzb > 0)
    { ++g_launches; k_scatter<<<grid_for(in.nnzb, 256), 256, 0, st>>>(keep, scan_buf, in.nnzb, in.brow, in.bcol, in.slot, out.brow,
                                                       out.bcol, out.slot); }
  return cudaGetLastError();
}

cudaError_t launch_gather_tiles(const TileSet& s, const double* pool, double* dst, cudaStream_t st) {
  if (s.nnzb == 0) return cudaSuccess;
  { ++g_launches; k_gather<<<(unsigned)s.nnzb, 256, 0, st>>>(s.slot, pool, dst); }
  return cudaGetLastError();
}

cudaError_t launch_copy_index(const TileSet& s, int32_t* brow, int32_t* bcol, cudaStream_t st) {
  if (s.nnzb == 0) return cudaSuccess;
  { ++g_launches; k_copy2<<<grid_for(s.nnzb, 256), 256, 0, st>>>(s.brow, s.bcol, s.nnzb, brow, bcol); }
  return cudaGetLastError();
}

}  // namespace sp2
