// Truncation X~_i = X_i + E_i with ||E_i|| <= tau_i (Section 2, Eqs. (6)-(8)).
//
// Selection rule (the paper states only the bound, so this is a reading):
//  - Frobenius mode: sort the tiles by (||X_IJ||_F^2, I * nb + J) ascending and drop
//    the longest prefix whose weighted squared norms fit into tau^2; weight 2 for
//    off-diagonal tiles (their mirror is dropped too), 1 for diagonal tiles.
//  - Frob-Inf mode (Section 3, Eq. (13), square partition of `part` rows): every
//    super-block (R, C) gets the budget tau / max(m_R, m_C), m_R = number of
//    nonzero super-blocks in super-row R; the Frobenius rule runs inside each
//    super-block (weight 2 only for off-diagonal tiles of diagonal super-blocks).
//    Then every super-row sum of ||E_RC||_F is <= tau, so ||E||_2 <= ||E||_M <= tau.
//  - Sums are taken in integer units of budget * 2^-36 with each tile's share
//    rounded up, so they are exact, independent of summation order, and never
//    understate ||E||_F^2.
//
// GPU form: a segmented most-significant-digit radix select over the 96-bit key
// (63 bits of the squared norm's IEEE pattern -- non-negative doubles order like
// their bit patterns -- then the 32-bit linear tile index).  Twelve passes of
// 8 bits; each pass histograms the budget units of the remaining candidates and
// one thread per segment walks its 256 buckets.  No sort, no host round trip.
// A single segment of at most 2048 tiles runs the same passes in one CTA.
#include <cmath>
#include <vector>

#include "sp2_internal.h"

namespace sp2 {
namespace {

constexpr double Q_SCALE = 68719476736.0;          // 2^36
constexpr unsigned long long Q_BUDGET = 1ull << 36;
constexpr unsigned long long Q_CAP = 1ull << 37;
constexpr int MIXED_POWER_ITERS = 100;        // power steps of the mixed-norm bound

struct Work {
  unsigned long long* q;
  int32_t* seg;
  double* scale;
  unsigned long long* rem;
  unsigned long long* pref_hi;
  uint32_t* pref_lo;
  int32_t* state;
  int32_t* depth;
  unsigned long long* hist;
  int32_t* nz;
  int32_t* m;
  int64_t nseg;
  int32_t nsb;
};

inline size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

Work carve(void* base, int64_t nnzb, int64_t nseg, int nsb) {
  char* p = static_cast<char*>(base);
  Work w;
  w.q = reinterpret_cast<unsigned long long*>(p); p += align_up(nnzb * 8);
  w.seg = reinterpret_cast<int32_t*>(p); p += align_up(nnzb * 4);
  w.scale = reinterpret_cast<double*>(p); p += align_up(nseg * 8);
  w.rem = reinterpret_cast<unsigned long long*>(p); p += align_up(nseg * 8);
  w.pref_hi = reinterpret_cast<unsigned long long*>(p); p += align_up(nseg * 8);
  w.pref_lo = reinterpret_cast<uint32_t*>(p); p += align_up(nseg * 4);
  w.state = reinterpret_cast<int32_t*>(p); p += align_up(nseg * 4);
  w.depth = reinterpret_cast<int32_t*>(p); p += align_up(nseg * 4);
  w.hist = reinterpret_cast<unsigned long long*>(p); p += align_up(nseg * 256 * 8);
  w.nz = reinterpret_cast<int32_t*>(p); p += align_up((size_t)nsb * nsb * 4);
  w.m = reinterpret_cast<int32_t*>(p); p += align_up((size_t)nsb * 4);
  w.nseg = nseg;
  w.nsb = nsb;
  return w;
}

__global__ void k_nz(const int32_t* __restrict__ brow, const int32_t* __restrict__ bcol, int64_t nnzb, int pt,
                     int nsb, int32_t* nz) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nnzb) return;
  const int R = brow[t] / pt, C = bcol[t] / pt;
  nz[R * nsb + C] = 1;
  nz[C * nsb + R] = 1;
}

__global__ void k_m(const int32_t* __restrict__ nz, int nsb, int32_t* m) {
  const int R = blockIdx.x * blockDim.x + threadIdx.x;
  if (R >= nsb) return;
  int c = 0;
  for (int C = 0; C < nsb; ++C) c += nz[R * nsb + C];
  m[R] = c;
}

// mode 0: one segment, budget tau^2.  mode 1: segment R * nsb + C.
__global__ void k_seg_init(Work w, int mode, double tau) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= w.nseg) return;
  double budget;
  if (mode == 0) {
    budget = tau * tau;
  } else {
    const int R = (int)(s / w.nsb), C = (int)(s % w.nsb);
    const int mm = max(w.m[R], w.m[C]);
    const double beta = mm > 0 ? tau / (double)mm : 0.0;
    budget = beta * beta;
  }
  w.scale[s] = budget > 0.0 ? Q_SCALE / budget : 0.0;
  w.rem[s] = Q_BUDGET;
  w.pref_hi[s] = 0ull;
  w.pref_lo[s] = 0u;
  w.state[s] = 0;
  w.depth[s] = 0;
}

__global__ void k_q(const int32_t* __restrict__ brow, const int32_t* __restrict__ bcol,
                    const int32_t* __restrict__ slot, const double* __restrict__ n2, int64_t nnzb, int mode, int pt,
                    Work w) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nnzb) return;
  const int I = brow[t], J = bcol[t];
  int s = 0;
  double wt = (I == J) ? 1.0 : 2.0;
  if (mode == 1) {
    const int R = I / pt, C = J / pt;
    s = R * w.nsb + C;
    if (R != C) wt = 1.0;
  }
  w.seg[t] = s;
  const double v = n2[slot ? slot[t] : t];
  const double sc = w.scale[s];
  unsigned long long q;
  if (sc == 0.0) {
    q = (v == 0.0) ? 0ull : Q_CAP;
  } else {
    const double x = (wt * v) * sc;
    q = (x >= (double)Q_CAP) ? Q_CAP : (unsigned long long)ceil(x);
  }
  w.q[t] = q;
}

__device__ __forceinline__ bool is_candidate(unsigned long long hi, uint32_t lo, int p, unsigned long long ph,
                                             uint32_t pl) {
  if (p == 0) return true;
  if (p <= 8) return (hi >> (64 - 8 * p)) == ph;
  return hi == ph && (lo >> (32 - 8 * (p - 8))) == pl;
}

__device__ __forceinline__ int digit_of(unsigned long long hi, uint32_t lo, int p) {
  if (p < 8) return (int)((hi >> (56 - 8 * p)) & 0xFFull);
  return (int)((lo >> (24 - 8 * (p - 8))) & 0xFFu);
}

template <bool ONE_SEG>
__global__ void k_hist(const int32_t* __restrict__ brow, const int32_t* __restrict__ bcol,
                       const int32_t* __restrict__ slot, const double* __restrict__ n2, int64_t nnzb, int nb, int p,
                       Work w) {
  __shared__ unsigned long long sh[256];
  if (ONE_SEG) {
    for (int k = threadIdx.x; k < 256; k += blockDim.x) sh[k] = 0ull;
    __syncthreads();
  }
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < nnzb) {
    const int s = w.seg[t];
    if (w.state[s] == 0) {
      const unsigned long long hi = __double_as_longlong(n2[slot ? slot[t] : t]);
      const uint32_t lo = (uint32_t)brow[t] * (uint32_t)nb + (uint32_t)bcol[t];
      if (is_candidate(hi, lo, p, w.pref_hi[s], w.pref_lo[s])) {
        const int d = digit_of(hi, lo, p);
        if (ONE_SEG) atomicAdd(&sh[d], w.q[t]);
        else atomicAdd(&w.hist[(int64_t)s * 256 + d], w.q[t]);
      }
    }
  }
  if (ONE_SEG) {
    __syncthreads();
    for (int k = threadIdx.x; k < 256; k += blockDim.x)
      if (sh[k]) atomicAdd(&w.hist[k], sh[k]);
  }
}

__global__ void k_select(Work w, int p) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= w.nseg || w.state[s] != 0) return;
  unsigned long long rem = w.rem[s];
  const unsigned long long* h = w.hist + s * 256;
  int cut = -1;
  for (int d = 0; d < 256; ++d) {
    const unsigned long long v = h[d];
    if (v <= rem) rem -= v;
    else { cut = d; break; }
  }
  w.rem[s] = rem;
  if (cut < 0) {
    w.state[s] = 1;      // every candidate fits: drop all keys whose top 8p bits <= prefix
    w.depth[s] = p;
  } else if (p < 8) {
    w.pref_hi[s] = (w.pref_hi[s] << 8) | (unsigned long long)cut;
  } else {
    w.pref_lo[s] = (w.pref_lo[s] << 8) | (uint32_t)cut;
  }
}

__global__ void k_mark(const int32_t* __restrict__ brow, const int32_t* __restrict__ bcol,
                       const int32_t* __restrict__ slot, const double* __restrict__ n2, int64_t nnzb, int nb, Work w,
                       int32_t* keep) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nnzb) return;
  const int s = w.seg[t];
  const unsigned long long hi = __double_as_longlong(n2[slot ? slot[t] : t]);
  const uint32_t lo = (uint32_t)brow[t] * (uint32_t)nb + (uint32_t)bcol[t];
  const unsigned long long ph = w.pref_hi[s];
  const uint32_t pl = w.pref_lo[s];
  bool drop;
  if (w.state[s] == 1) {
    const int dep = w.depth[s];
    if (dep == 0) drop = true;
    else if (dep <= 8) drop = (hi >> (64 - 8 * dep)) <= ph;
    else {
      const uint32_t top = lo >> (32 - 8 * (dep - 8));
      drop = hi < ph || (hi == ph && top <= pl);
    }
  } else {
    drop = hi < ph || (hi == ph && lo < pl);
  }
  keep[t] = drop ? 0 : 1;
}

// One CTA for a single segment of at most SMALL_MAX tiles: the same twelve
// passes as k_hist + k_select + k_mark, keys held in shared memory, so a small
// truncation is one launch instead of about forty.  All sums are the same exact
// integers, so the keep flags equal the multi-launch path's.
constexpr int SMALL_MAX = 2048;
constexpr int SMALL_THREADS = 1024;

__global__ void __launch_bounds__(SMALL_THREADS)
    k_trunc_small(const int32_t* __restrict__ brow, const int32_t* __restrict__ bcol,
                  const int32_t* __restrict__ slot, const double* __restrict__ n2, int n, int nb, double budget,
                  int32_t* keep) {
  __shared__ unsigned long long s_hi[SMALL_MAX];
  __shared__ unsigned long long s_q[SMALL_MAX];
  __shared__ uint32_t s_lo[SMALL_MAX];
  __shared__ unsigned long long hist[256];
  __shared__ unsigned long long s_rem, s_ph;
  __shared__ uint32_t s_pl;
  __shared__ int s_state, s_depth;
  const double sc = budget > 0.0 ? Q_SCALE / budget : 0.0;
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const int I = brow[t], J = bcol[t];
    const double v = n2[slot ? slot[t] : t];
    const double wt = (I == J) ? 1.0 : 2.0;
    unsigned long long q;
    if (sc == 0.0) {
      q = (v == 0.0) ? 0ull : Q_CAP;
    } else {
      const double x = (wt * v) * sc;
      q = (x >= (double)Q_CAP) ? Q_CAP : (unsigned long long)ceil(x);
    }
    s_hi[t] = __double_as_longlong(v);
    s_lo[t] = (uint32_t)I * (uint32_t)nb + (uint32_t)J;
    s_q[t] = q;
  }
  if (threadIdx.x == 0) {
    s_rem = Q_BUDGET;
    s_ph = 0ull;
    s_pl = 0u;
    s_state = 0;
    s_depth = 0;
  }
  for (int p = 0; p < 12; ++p) {
    for (int k = threadIdx.x; k < 256; k += blockDim.x) hist[k] = 0ull;
    __syncthreads();
    if (s_state != 0) break;
    const unsigned long long ph = s_ph;
    const uint32_t pl = s_pl;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      const unsigned long long hi = s_hi[t];
      const uint32_t lo = s_lo[t];
      if (is_candidate(hi, lo, p, ph, pl)) atomicAdd(&hist[digit_of(hi, lo, p)], s_q[t]);
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      // bucket walk of k_select: lane l owns buckets 8l..8l+7, an inclusive
      // scan over the lanes finds the lane holding the cut
      const int lane = threadIdx.x;
      unsigned long long loc[8], sum = 0ull;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        loc[j] = hist[lane * 8 + j];
        sum += loc[j];
      }
      unsigned long long inc = sum;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const unsigned long long v = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += v;
      }
      const unsigned long long rem = s_rem;
      const unsigned bal = __ballot_sync(0xffffffffu, inc > rem);
      if (bal == 0u) {
        if (lane == 0) {
          s_state = 1;      // every candidate fits
          s_depth = p;
        }
      } else if (lane == __ffs(bal) - 1) {
        unsigned long long r = rem - (inc - sum);
        int cut = 8 * lane + 7;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (loc[j] <= r) {
            r -= loc[j];
          } else {
            cut = 8 * lane + j;
            break;
          }
        }
        s_rem = r;
        if (p < 8) s_ph = (ph << 8) | (unsigned long long)cut;
        else s_pl = (pl << 8) | (uint32_t)cut;
      }
    }
    __syncthreads();
  }
  __syncthreads();
  const unsigned long long ph = s_ph;
  const uint32_t pl = s_pl;
  const int state = s_state, dep = s_depth;
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const unsigned long long hi = s_hi[t];
    const uint32_t lo = s_lo[t];
    bool drop;
    if (state == 1) {
      if (dep == 0) drop = true;
      else if (dep <= 8) drop = (hi >> (64 - 8 * dep)) <= ph;
      else drop = hi < ph || (hi == ph && (lo >> (32 - 8 * (dep - 8))) <= pl);
    } else {
      drop = hi < ph || (hi == ph && lo < pl);
    }
    keep[t] = drop ? 0 : 1;
  }
}

// ||tile||_F^2 of contiguous tiles (fixed order: 4 strided partial sums per
// thread, then a fixed tree), one CTA of 256 threads per tile.
__global__ void __launch_bounds__(256) k_tile_norms(const double* __restrict__ val, double* n2) {
  const int64_t t = blockIdx.x;
  const double* x = val + t * TE;
  double a = 0.0;
  for (int q = threadIdx.x; q < TE; q += 256) a += x[q] * x[q];
  __shared__ double red[256];
  red[threadIdx.x] = a;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) n2[t] = red[0];
}

inline unsigned grid_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }


// ---------------------------------------------------------------- mixed norm
// Frobenius-spectral mixed norm of Section 3 on a partition of pt tiles:
// every tile gets its budget units q (weight 2 for an off-diagonal tile inside
// a diagonal block, units of tau^2 2^-36 rounded up, capped), the pattern of
// its squared norm (non-negative doubles order like their bit patterns) and
// its block index R * nsb + C.
__global__ void k_mixed_prep(const int32_t* __restrict__ brow, const int32_t* __restrict__ bcol,
                             const int32_t* __restrict__ slot, const double* __restrict__ n2, int64_t nnzb, int pt,
                             int nsb, double sc, unsigned long long* q, long long* bits, int32_t* blk) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nnzb) return;
  const int I = brow[t], J = bcol[t];
  const int R = I / pt, C = J / pt;
  const double wt = (R == C && I != J) ? 2.0 : 1.0;
  const double v = n2[slot ? slot[t] : t];
  const double x = (wt * v) * sc;
  q[t] = (x >= (double)Q_CAP) ? Q_CAP : (unsigned long long)ceil(x);
  bits[t] = __double_as_longlong(v);
  blk[t] = R * nsb + C;
}

// Block sums of the units of the tiles with bits <= theta (and the mirror block
// for R != C), exact integer atomics; cnt[0] counts the tiles with
// lo < bits <= hi (the bisection ends when none is left between its ends).
__global__ void k_mixed_probe(const unsigned long long* __restrict__ q, const long long* __restrict__ bits,
                              const int32_t* __restrict__ blk, int64_t nnzb, int nsb, long long theta, long long lo,
                              long long hi, unsigned long long* B2, unsigned long long* cnt) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  bool between = false;
  if (t < nnzb) {
    const long long b = bits[t];
    between = b > lo && b <= hi;
    if (b <= theta && q[t] != 0ull) {
      const int k = blk[t];
      const int R = k / nsb, C = k % nsb;
      atomicAdd(&B2[k], q[t]);
      if (R != C) atomicAdd(&B2[C * nsb + R], q[t]);
    }
  }
  const unsigned nb = __popc(__ballot_sync(0xffffffffu, between));
  if ((threadIdx.x & 31) == 0 && nb) atomicAdd(cnt, (unsigned long long)nb);
}

__global__ void k_mixed_keep(const long long* __restrict__ bits, int64_t nnzb, long long theta, int32_t* keep) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < nnzb) keep[t] = bits[t] <= theta ? 0 : 1;
}

}  // namespace

cudaError_t launch_tile_norms(const double* val, int64_t nnzb, double* n2, cudaStream_t st) {
  if (nnzb == 0) return cudaSuccess;
  { ++g_launches; k_tile_norms<<<(unsigned)nnzb, 256, 0, st>>>(val, n2); }
  return cudaGetLastError();
}

size_t trunc_work_bytes(int64_t nnzb, int nb, int64_t part_tiles) {
  const int nsb = (int)((nb + part_tiles - 1) / part_tiles);
  const int64_t nseg = (int64_t)nsb * nsb;
  return align_up(nnzb * 8) + align_up(nnzb * 4) + 5 * align_up(nseg * 8) + 3 * align_up(nseg * 4) +
         align_up(nseg * 256 * 8) + align_up((size_t)nsb * nsb * 4) + align_up((size_t)nsb * 4) + 1024;
}

// x: the tiles of X_i (slot indexes n2); n2[slot] = ||X_i tile||_F^2; keep[t] out.
cudaError_t launch_truncate(const TileSet& x, const double* n2, int nb, double tau, int mode, int64_t part_tiles,
                            void* work, int32_t* keep, cudaStream_t st) {
  const int64_t nnzb = x.nnzb;
  if (nnzb == 0) return cudaSuccess;
  const int nsb = (int)((nb + part_tiles - 1) / part_tiles);
  const int64_t nseg = mode == 1 ? (int64_t)nsb * nsb : 1;
  if (nseg == 1 && nnzb <= SMALL_MAX) {
    // one segment: mode 1 with a single super-block has m = 1, so its budget is tau^2 too
    { ++g_launches; k_trunc_small<<<1, SMALL_THREADS, 0, st>>>(x.brow, x.bcol, x.slot, n2, (int)nnzb, nb, tau * tau, keep); }
    return cudaGetLastError();
  }
  Work w = carve(work, nnzb, nseg, nsb);
  cudaError_t e;
  if (mode == 1) {
    e = cudaMemsetAsync(w.nz, 0, (size_t)nsb * nsb * 4, st);
    if (e != cudaSuccess) return e;
    { ++g_launches; k_nz<<<grid_for(nnzb, 256), 256, 0, st>>>(x.brow, x.bcol, nnzb, (int)part_tiles, nsb, w.nz); }
    { ++g_launches; k_m<<<grid_for(nsb, 128), 128, 0, st>>>(w.nz, nsb, w.m); }
  }
  { ++g_launches; k_seg_init<<<grid_for(nseg, 256), 256, 0, st>>>(w, mode, tau); }
  { ++g_launches; k_q<<<grid_for(nnzb, 256), 256, 0, st>>>(x.brow, x.bcol, x.slot, n2, nnzb, mode, (int)part_tiles, w); }
  for (int p = 0; p < 12; ++p) {
    e = cudaMemsetAsync(w.hist, 0, (size_t)nseg * 256 * 8, st);
    if (e != cudaSuccess) return e;
    if (nseg == 1) { ++g_launches; k_hist<true><<<grid_for(nnzb, 256), 256, 0, st>>>(x.brow, x.bcol, x.slot, n2, nnzb, nb, p, w); }
    else { ++g_launches; k_hist<false><<<grid_for(nnzb, 256), 256, 0, st>>>(x.brow, x.bcol, x.slot, n2, nnzb, nb, p, w); }
    { ++g_launches; k_select<<<grid_for(nseg, 128), 128, 0, st>>>(w, p); }
  }
  { ++g_launches; k_mark<<<grid_for(nnzb, 256), 256, 0, st>>>(x.brow, x.bcol, x.slot, n2, nnzb, nb, w, keep); }
  return cudaGetLastError();
}

}  // namespace sp2

namespace sp2 {

// Collatz-Wielandt upper bound of rho(M), M = sqrt(B2) (nsb x nsb, symmetric,
// non-negative): rows that are all zero are skipped; x starts at all ones and
// MIXED_POWER_ITERS times takes u = max_i (M x)_i / x_i, then x = (M x + u x)
// / max(M x + u x); the smallest u is returned.  Sequential row sums without
// fused multiply-adds.
double mixed_norm_bound_host(const unsigned long long* B2, int nsb) {
  std::vector<int> live;
  for (int i = 0; i < nsb; ++i) {
    bool nz = false;
    for (int j = 0; j < nsb && !nz; ++j) nz = B2[(size_t)i * nsb + j] != 0ull;
    if (nz) live.push_back(i);
  }
  const int m = (int)live.size();
  if (m == 0) return 0.0;
  std::vector<double> M((size_t)m * m), x(m, 1.0), y(m);
  for (int a = 0; a < m; ++a)
    for (int b = 0; b < m; ++b) M[(size_t)a * m + b] = std::sqrt((double)B2[(size_t)live[a] * nsb + live[b]]);
  double best = INFINITY;
  for (int it = 0; it < MIXED_POWER_ITERS; ++it) {
    for (int a = 0; a < m; ++a) {
      double acc = 0.0;
      for (int b = 0; b < m; ++b) {
        const double prod = M[(size_t)a * m + b] * x[b];
        acc = acc + prod;
      }
      y[a] = acc;
    }
    double u = 0.0;
    for (int a = 0; a < m; ++a) u = std::max(u, y[a] / x[a]);
    best = std::min(best, u);
    double mx = 0.0;
    for (int a = 0; a < m; ++a) {
      const double ux = u * x[a];
      y[a] = y[a] + ux;
      mx = std::max(mx, y[a]);
    }
    for (int a = 0; a < m; ++a) x[a] = y[a] / mx;
  }
  return best;
}

size_t mixed_work_bytes(int64_t nnzb, int nsb) {
  return align_up((size_t)nnzb * 8) * 2 + align_up((size_t)nnzb * 4) + align_up((size_t)nsb * nsb * 8) + 256;
}

// keep[t] for the mixed-norm selection (see the oracle's reading): bisection
// over the 63-bit patterns of the squared norms for the largest theta whose
// dropped set has a bound of at most tau (in units: 2^18); each probe is one
// kernel and a host round trip; the bisection stops early once no tile lies
// between its ends.  Synchronises the stream.
cudaError_t mixed_select(const TileSet& x, const double* n2, int nb, double tau, int64_t part_tiles, void* work,
                         int32_t* keep, cudaStream_t st) {
  const int64_t nnzb = x.nnzb;
  if (nnzb == 0) return cudaSuccess;
  const int pt = (int)part_tiles;
  const int nsb = (int)((nb + pt - 1) / pt);
  char* p = static_cast<char*>(work);
  unsigned long long* q = reinterpret_cast<unsigned long long*>(p); p += align_up((size_t)nnzb * 8);
  long long* bits = reinterpret_cast<long long*>(p); p += align_up((size_t)nnzb * 8);
  int32_t* blk = reinterpret_cast<int32_t*>(p); p += align_up((size_t)nnzb * 4);
  unsigned long long* B2 = reinterpret_cast<unsigned long long*>(p); p += align_up((size_t)nsb * nsb * 8);
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(p);
  const unsigned g = grid_for(nnzb, 256);
  const double sc = tau > 0.0 ? Q_SCALE / (tau * tau) : 0.0;
  ++g_launches;
  k_mixed_prep<<<g, 256, 0, st>>>(x.brow, x.bcol, x.slot, n2, nnzb, pt, nsb, sc, q, bits, blk);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // tau = 0 keeps lo = 0: only tiles that are exactly zero are dropped
  long long lo = 0, hi = 0x7FFFFFFFFFFFFFFFll;
  if (tau > 0.0) {
    std::vector<unsigned long long> h((size_t)nsb * nsb + 1);
    const double limit = 262144.0;   // tau in units of tau 2^-18
    while (hi - lo > 1) {
      const long long mid = lo + (hi - lo) / 2;
      if ((e = cudaMemsetAsync(B2, 0, (size_t)nsb * nsb * 8, st)) != cudaSuccess) return e;
      if ((e = cudaMemsetAsync(cnt, 0, 8, st)) != cudaSuccess) return e;
      ++g_launches;
      k_mixed_probe<<<g, 256, 0, st>>>(q, bits, blk, nnzb, nsb, mid, lo, hi, B2, cnt);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      if ((e = cudaMemcpyAsync(h.data(), B2, (size_t)nsb * nsb * 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return e;
      if ((e = cudaMemcpyAsync(h.data() + (size_t)nsb * nsb, cnt, 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return e;
      if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
      if (h[(size_t)nsb * nsb] == 0) break;   // no tile between lo and hi: the result is lo
      if (mixed_norm_bound_host(h.data(), nsb) <= limit) lo = mid;
      else hi = mid;
    }
  }
  ++g_launches;
  k_mixed_keep<<<g, 256, 0, st>>>(bits, nnzb, lo, keep);
  return cudaGetLastError();
}

}  // namespace sp2
