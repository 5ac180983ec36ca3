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

__device__ __forceinline__ int64_t find_tile(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ bcol,
                                             int I, int J) {
  int64_t lo = rowptr[I], hi = rowptr[I + 1];
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (bcol[mid] < J) lo = mid + 1; else hi = mid;
  }
  return (lo < rowptr[I + 1] && bcol[lo] == J) ? lo : -1;
}

// dst tile t := scale * src tile (I, J) (0 when src has no such tile); with
// sym_diag the diagonal tiles are symmetrised, (W + W^T) / 2.
__global__ void __launch_bounds__(256) k_place(const int32_t* __restrict__ srowptr, const int32_t* __restrict__ sbcol,
                                               const int32_t* __restrict__ sslot, const double* __restrict__ spool,
                                               const int32_t* __restrict__ dbrow, const int32_t* __restrict__ dbcol,
                                               const int32_t* __restrict__ dslot, double* dpool, double scale,
                                               int sym_diag) {
  const int64_t t = blockIdx.x;
  const int I = dbrow[t], J = dbcol[t];
  const int64_t k = find_tile(srowptr, sbcol, I, J);
  double* d = dpool + (int64_t)(dslot ? dslot[t] : t) * TE;
  if (k < 0) {
    for (int q = threadIdx.x; q < TE; q += 256) d[q] = 0.0;
    return;
  }
  const double* s = spool + (int64_t)(sslot ? sslot[k] : k) * TE;
  for (int q = threadIdx.x; q < TE; q += 256) {
    double v = s[q];
    if (sym_diag && I == J) v = 0.5 * (v + s[(q & 31) * TB + (q >> 5)]);
    d[q] = scale * v;
  }
}

// Trace of the kept diagonal tiles of a tile set (the trace-correcting choice
// of Section 1 needs trace(X~) before the next product): rows I whose tile
// (I, I) is stored and kept (keep == nullptr: all kept) add the real part of
// the tile's diagonal.  One CTA, fixed summation order (deterministic).
constexpr int TRACE_T = 1024;
__global__ void __launch_bounds__(TRACE_T)
    k_trace_kept(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ bcol,
                 const int32_t* __restrict__ slot, const int32_t* __restrict__ keep,
                 const double* __restrict__ pool, int nb, int64_t n, double* out) {
  __shared__ double red[TRACE_T];
  double acc = 0.0;
  for (int I = threadIdx.x; I < nb; I += TRACE_T) {
    int lo = rowptr[I], hi = rowptr[I + 1];
    while (lo < hi) {   // first tile of row I with column >= I
      const int mid = (lo + hi) >> 1;
      if (bcol[mid] < I) lo = mid + 1;
      else hi = mid;
    }
    const int t = lo;
    if (t < rowptr[I + 1] && bcol[t] == I && (!keep || keep[t])) {
      const double* x = pool + (int64_t)(slot ? slot[t] : t) * TE;
      for (int r = 0; r < TB && (int64_t)I * TB + r < n; ++r) acc += x[r * (TB + 1)];
    }
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = TRACE_T / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

__global__ void k_iota(int32_t* p, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) p[i] = (int32_t)i;
}

inline unsigned grid_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_place(const TileSet& src, const double* spool, const TileSet& dst, double* dpool, double scale,
                         int sym_diag, cudaStream_t st) {
  if (dst.nnzb == 0) return cudaSuccess;
  { ++g_launches; k_place<<<(unsigned)dst.nnzb, 256, 0, st>>>(src.rowptr, src.bcol, src.slot, spool, dst.brow, dst.bcol, dst.slot, dpool, scale, sym_diag); }
  return cudaGetLastError();
}

cudaError_t launch_trace_kept(const TileSet& s, const int32_t* keep, const double* pool, int nb, int64_t n,
                              double* out, cudaStream_t st) {
  ++g_launches;
  k_trace_kept<<<1, TRACE_T, 0, st>>>(s.rowptr, s.bcol, s.slot, keep, pool, nb, n, out);
  return cudaGetLastError();
}

cudaError_t launch_iota(int32_t* p, int64_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  { ++g_launches; k_iota<<<grid_for(n, 256), 256, 0, st>>>(p, n); }
  return cudaGetLastError();
}

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
