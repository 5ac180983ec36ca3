// Algorithm 1 (Section 4, Step 1): Gershgorin bounds lambda_min <= lambda_1,
// lambda_max >= lambda_N of F, and X_0 = (lambda_max I - F) / (lambda_max - lambda_min)
// with the squared Frobenius norm of every tile (for the truncation of X_0).
#include "sp2_internal.h"

namespace sp2 {
namespace {

// One warp per tile row I, lane r = row inside the tile.  Row i's radius
// sum_{j != i} |F_ij| is accumulated sequentially over the row's tiles in
// ascending K, so the result does not depend on scheduling.  Each tile is
// read with coalesced loads and staged (in the orientation row I needs) in
// shared memory, rows padded to 33 doubles.
constexpr int GER_WARPS = 4;

__global__ void __launch_bounds__(32 * GER_WARPS) k_gershgorin(const int32_t* __restrict__ frowptr,
                                                               const int32_t* __restrict__ fcol,
                                                               const uint32_t* __restrict__ fref,
                                                               const double* __restrict__ pool, int nb, int64_t n,
                                                               double* rowlo, double* rowhi) {
  __shared__ double tile[GER_WARPS][TB][TB + 1];
  const int wid = threadIdx.x >> 5;
  const int I = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int r = threadIdx.x & 31;
  if (I >= nb) return;   // whole warps leave together
  const int64_t gi = (int64_t)I * TB + r;
  double (*ts)[TB + 1] = tile[wid];
  double d = 0.0, s = 0.0;
  for (int e = frowptr[I]; e < frowptr[I + 1]; ++e) {
    const int K = fcol[e];
    const uint32_t rf = fref[e];
    const double* T = pool + (int64_t)(rf & ~REF_T) * TE;
    const bool tr = (rf & REF_T) != 0;
    __syncwarp();
    for (int i = 0; i < TB; ++i) {
      const double v = T[i * TB + r];      // stored row i, column r
      if (tr) ts[r][i] = v;
      else ts[i][r] = v;
    }
    __syncwarp();
    for (int c = 0; c < TB; ++c) {
      const int64_t gk = (int64_t)K * TB + c;
      if (gk >= n) break;
      const double v = ts[r][c];
      if (gk == gi) d = v; else s += fabs(v);
    }
  }
  if (gi >= n) return;
  rowlo[gi] = d - s;
  rowhi[gi] = d + s;
}

__global__ void k_minmax(const double* __restrict__ lo, const double* __restrict__ hi, int64_t n, double* out2) {
  __shared__ double smin[32], smax[32];
  double mn = INFINITY, mx = -INFINITY;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    mn = fmin(mn, lo[i]);
    mx = fmax(mx, hi[i]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { smin[wid] = mn; smax[wid] = mx; }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    mn = lane < nw ? smin[lane] : INFINITY;
    mx = lane < nw ? smax[lane] : -INFINITY;
    for (int o = 16; o > 0; o >>= 1) {
      mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
      mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if (lane == 0) { out2[0] = mn; out2[1] = mx; }
  }
}

// One CTA (256 threads) per tile of F; X_0 takes F's tile pattern (every
// diagonal tile present).  Padding rows/columns (index >= n) are zero.
__global__ void __launch_bounds__(256) k_x0(const int32_t* __restrict__ brow, const int32_t* __restrict__ bcol,
                                            const int32_t* __restrict__ slot, const double* __restrict__ fpool,
                                            double* xpool, int64_t n, double lmax, double w, double* n2) {
  const int64_t t = blockIdx.x;
  const int I = brow[t], J = bcol[t];
  const double* src = fpool + (int64_t)slot[t] * TE;
  double* dst = xpool + (int64_t)slot[t] * TE;
  double acc = 0.0;
  for (int q = threadIdx.x; q < TE; q += blockDim.x) {
    const int r = q >> 5, c = q & 31;
    const int64_t gi = (int64_t)I * TB + r, gj = (int64_t)J * TB + c;
    double x = 0.0;
    if (gi < n && gj < n) x = ((gi == gj ? lmax : 0.0) - src[q]) / w;
    dst[q] = x;
    acc += x * x;
  }
  __shared__ double red[8];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
    n2[t] = s;
  }
}

}  // namespace

cudaError_t launch_gershgorin(const FullPattern& fp, const double* pool, int nb, int64_t n, double* rowlo,
                              double* rowhi, cudaStream_t st) {
  const int64_t thr = (int64_t)nb * 32;
  const int bs = 32 * GER_WARPS;
  ++g_launches;
  k_gershgorin<<<(unsigned)((thr + bs - 1) / bs), bs, 0, st>>>(fp.rowptr, fp.col, fp.ref, pool, nb, n, rowlo, rowhi);
  return cudaGetLastError();
}

cudaError_t launch_minmax(const double* lo, const double* hi, int64_t n, double* out2, cudaStream_t st) {
  { ++g_launches; k_minmax<<<1, 1024, 0, st>>>(lo, hi, n, out2); }
  return cudaGetLastError();
}

cudaError_t launch_x0(const TileSet& f, const double* fpool, double* xpool, int64_t n, double lmax, double w,
                      double* n2, cudaStream_t st) {
  if (f.nnzb == 0) return cudaSuccess;
  { ++g_launches; k_x0<<<(unsigned)f.nnzb, 256, 0, st>>>(f.brow, f.bcol, f.slot, fpool, xpool, n, lmax, w, n2); }
  return cudaGetLastError();
}

}  // namespace sp2
