// Integer tile-pattern work (bit-exact): the symmetric bitmap of a tile set,
// both-triangle neighbour lists, the pattern of a product X~^2 (Section 5: the
// symmetric matrix is stored as its upper triangle only), prefix sums and
// input validation.
#include "sp2_internal.h"

namespace sp2 {

namespace {

__device__ __forceinline__ int warp_incl_scan(int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  return v;
}

__device__ __forceinline__ int warp_sum(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void k_bitmap(const int32_t* __restrict__ brow, const int32_t* __restrict__ bcol, int64_t nnzb,
                         uint32_t* bits, int words) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nnzb) return;
  const int i = brow[t], j = bcol[t];
  atomicOr(&bits[(int64_t)i * words + (j >> 5)], 1u << (j & 31));
  atomicOr(&bits[(int64_t)j * words + (i >> 5)], 1u << (i & 31));
}

__global__ void k_row_popc(const uint32_t* __restrict__ bits, int nb, int words, int32_t* counts) {
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= nb) return;
  int c = 0;
  for (int w = lane; w < words; w += 32) c += __popc(bits[(int64_t)row * words + w]);
  c = warp_sum(c);
  if (lane == 0) counts[row] = c;
}

// ---- three-phase exclusive scan of int32 (chunks of 4096) --------------------
constexpr int SCAN_T = 1024;
constexpr int SCAN_PER = 4;
constexpr int SCAN_CHUNK = SCAN_T * SCAN_PER;

__device__ int block_excl_scan(int v, int* total) {
  __shared__ int wsum[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (int)(blockDim.x >> 5);
  const int inc = warp_incl_scan(v);
  if (lane == 31) wsum[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    const int s = (lane < nw) ? wsum[lane] : 0;
    const int si = warp_incl_scan(s);
    wsum[lane] = si - s;
    if (lane == nw - 1) *total = si;
  }
  __syncthreads();
  const int r = inc - v + wsum[wid];
  __syncthreads();
  return r;
}

__global__ void k_scan_chunks(const int32_t* __restrict__ in, int64_t n, int32_t* chunk_sum) {
  const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK;
  int s = 0;
  for (int q = 0; q < SCAN_PER; ++q) {
    int64_t i = base + (int64_t)threadIdx.x * SCAN_PER + q;
    if (i < n) s += in[i];
  }
  __shared__ int tot;
  block_excl_scan(s, &tot);
  if (threadIdx.x == 0) chunk_sum[blockIdx.x] = tot;
}

__global__ void k_scan_partials(int32_t* chunk_sum, int64_t nchunks, int32_t* total_dev) {
  __shared__ int tot;
  int carry = 0;
  for (int64_t b0 = 0; b0 < nchunks; b0 += SCAN_T) {
    int64_t i = b0 + threadIdx.x;
    int v = (i < nchunks) ? chunk_sum[i] : 0;
    int ex = block_excl_scan(v, &tot);
    if (i < nchunks) chunk_sum[i] = ex + carry;
    carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0 && total_dev) *total_dev = carry;
}

__global__ void k_scan_apply(const int32_t* __restrict__ in, int64_t n, const int32_t* __restrict__ chunk_off,
                             int32_t* out) {
  const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK;
  int v[SCAN_PER];
  int s = 0;
  for (int q = 0; q < SCAN_PER; ++q) {
    int64_t i = base + (int64_t)threadIdx.x * SCAN_PER + q;
    v[q] = (i < n) ? in[i] : 0;
    s += v[q];
  }
  __shared__ int tot;
  int ex = block_excl_scan(s, &tot) + chunk_off[blockIdx.x];
  for (int q = 0; q < SCAN_PER; ++q) {
    int64_t i = base + (int64_t)threadIdx.x * SCAN_PER + q;
    if (i < n) out[i] = ex;
    ex += v[q];
  }
}

// n <= SCAN_CHUNK: the three passes above in one CTA.
__global__ void k_scan_one(const int32_t* __restrict__ in, int64_t n, int32_t* out, int32_t* total_dev) {
  int v[SCAN_PER];
  int s = 0;
  for (int q = 0; q < SCAN_PER; ++q) {
    const int64_t i = (int64_t)threadIdx.x * SCAN_PER + q;
    v[q] = (i < n) ? in[i] : 0;
    s += v[q];
  }
  __shared__ int tot;
  int ex = block_excl_scan(s, &tot);
  for (int q = 0; q < SCAN_PER; ++q) {
    const int64_t i = (int64_t)threadIdx.x * SCAN_PER + q;
    if (i < n) out[i] = ex;
    ex += v[q];
  }
  if (threadIdx.x == 0 && total_dev) *total_dev = tot;
}

__device__ __forceinline__ int64_t lower_bound_i32(const int32_t* a, int64_t lo, int64_t hi, int32_t key) {
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (a[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// One warp per row R: list the set bits of the row in ascending order and find
// the stored tile behind each one.
__global__ void k_fill_full(const uint32_t* __restrict__ bits, int nb, int words, const int32_t* __restrict__ frowptr,
                            const int32_t* __restrict__ up_rowptr, const int32_t* __restrict__ up_bcol,
                            const int32_t* __restrict__ up_slot, int32_t* col, uint32_t* ref) {
  const int R = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (R >= nb) return;
  int base = frowptr[R];
  for (int w0 = 0; w0 < words; w0 += 32) {
    const int w = w0 + lane;
    uint32_t m = (w < words) ? bits[(int64_t)R * words + w] : 0u;
    const int c = __popc(m);
    const int inc = warp_incl_scan(c);
    int off = base + inc - c;
    while (m) {
      const int b = __ffs(m) - 1;
      m &= m - 1;
      const int K = w * 32 + b;
      const int lo = K < R ? K : R, hi = K < R ? R : K;
      const int64_t p = lower_bound_i32(up_bcol, up_rowptr[lo], up_rowptr[lo + 1], hi);
      col[off] = K;
      ref[off] = (uint32_t)up_slot[p] | (K < R ? REF_T : 0u);
      ++off;
    }
    base += __shfl_sync(0xffffffffu, inc, 31);
  }
}

// Row I of the pattern of X_i = c0 I + c1 X~ + c2 X~^2 (Algorithm 2): OR over K
// in A's row I of B's bitmap row K (the product), OR A's own row I (the c1 X~
// term: a stored tile whose diagonal tiles were truncated away and that no K
// connects is still an output tile), restricted to J >= I, plus the diagonal.
__global__ void k_product_bits(const int32_t* __restrict__ arowptr, const int32_t* __restrict__ acol,
                               const uint32_t* __restrict__ abits, const uint32_t* __restrict__ bbits, int nb,
                               int words, int upper, uint32_t* out) {
  const int I = blockIdx.x;
  const int a0 = arowptr[I], a1 = arowptr[I + 1];
  for (int w = threadIdx.x; w < words; w += blockDim.x) {
    uint32_t acc = abits[(int64_t)I * words + w];
    for (int e = a0; e < a1; ++e) acc |= bbits[(int64_t)acol[e] * words + w];
    const int lo = w * 32;
    if (upper) {
      if (lo + 32 <= I) acc = 0;
      else if (lo < I) acc &= ~((1u << (I - lo)) - 1u);
    }
    if ((I >> 5) == w) acc |= 1u << (I & 31);
    out[(int64_t)I * words + w] = acc;
  }
}

__global__ void k_fill_upper(const uint32_t* __restrict__ bits, int nb, int words, const int32_t* __restrict__ rowptr,
                             int32_t* brow, int32_t* bcol, int32_t* slot) {
  const int R = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (R >= nb) return;
  int base = rowptr[R];
  for (int w0 = 0; w0 < words; w0 += 32) {
    const int w = w0 + lane;
    uint32_t m = (w < words) ? bits[(int64_t)R * words + w] : 0u;
    const int c = __popc(m);
    const int inc = warp_incl_scan(c);
    int off = base + inc - c;
    while (m) {
      const int b = __ffs(m) - 1;
      m &= m - 1;
      brow[off] = R;
      bcol[off] = w * 32 + b;
      if (slot) slot[off] = off;
      ++off;
    }
    base += __shfl_sync(0xffffffffu, inc, 31);
  }
}

__global__ void k_rowptr(const int32_t* __restrict__ brow, int64_t nnzb, int nb, int32_t* rowptr) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I > nb) return;
  rowptr[I] = (int32_t)lower_bound_i32(brow, 0, nnzb, I);
}

// flag bit 0: pattern error; bit 1: non-finite value.
__global__ void k_check_pattern(const int32_t* __restrict__ brow, const int32_t* __restrict__ bcol, int64_t nnzb,
                                int nb, int32_t* flag, int32_t* ndiag) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nnzb) return;
  const int i = brow[t], j = bcol[t];
  bool bad = i < 0 || j < i || j >= nb;
  if (t > 0) {
    const int pi = brow[t - 1], pj = bcol[t - 1];
    if (!(pi < i || (pi == i && pj < j))) bad = true;
  }
  if (bad) atomicOr(flag, 1);
  if (!bad && i == j) atomicAdd(ndiag, 1);
}

__global__ void k_check_finite(const double* __restrict__ val, int64_t count, int32_t* flag) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  bool bad = false;
  for (; i < count; i += stride) bad |= !isfinite(val[i]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 2);
}

inline unsigned grid_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

size_t scan_tmp_bytes(int64_t n) {
  const int64_t nch = (n + SCAN_CHUNK - 1) / SCAN_CHUNK;
  return (size_t)(nch + 1) * sizeof(int32_t);
}

cudaError_t launch_scan_i32(const int32_t* in, int32_t* out_excl, int64_t n, int32_t* total_dev, void* tmp,
                            cudaStream_t st) {
  if (n <= 0) {
    if (total_dev) return cudaMemsetAsync(total_dev, 0, sizeof(int32_t), st);
    return cudaSuccess;
  }
  const int64_t nch = (n + SCAN_CHUNK - 1) / SCAN_CHUNK;
  if (nch == 1) {
    { ++g_launches; k_scan_one<<<1, SCAN_T, 0, st>>>(in, n, out_excl, total_dev); }
    return cudaGetLastError();
  }
  int32_t* cs = static_cast<int32_t*>(tmp);
  { ++g_launches; k_scan_chunks<<<(unsigned)nch, SCAN_T, 0, st>>>(in, n, cs); }
  { ++g_launches; k_scan_partials<<<1, SCAN_T, 0, st>>>(cs, nch, total_dev); }
  { ++g_launches; k_scan_apply<<<(unsigned)nch, SCAN_T, 0, st>>>(in, n, cs, out_excl); }
  return cudaGetLastError();
}

cudaError_t launch_bitmap(const TileSet& s, int nb, FullPattern& fp, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(fp.bits, 0, (size_t)nb * fp.words * sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  if (s.nnzb > 0) { ++g_launches; k_bitmap<<<grid_for(s.nnzb, 256), 256, 0, st>>>(s.brow, s.bcol, s.nnzb, fp.bits, fp.words); }
  return cudaGetLastError();
}

cudaError_t launch_row_popc(const uint32_t* bits, int nb, int words, int32_t* counts, cudaStream_t st) {
  { ++g_launches; k_row_popc<<<grid_for((int64_t)nb * 32, 256), 256, 0, st>>>(bits, nb, words, counts); }
  return cudaGetLastError();
}

cudaError_t launch_fill_full(const TileSet& s, int nb, FullPattern& fp, cudaStream_t st) {
  { ++g_launches; k_fill_full<<<grid_for((int64_t)nb * 32, 256), 256, 0, st>>>(fp.bits, nb, fp.words, fp.rowptr, s.rowptr, s.bcol,
                                                                s.slot, fp.col, fp.ref); }
  return cudaGetLastError();
}

cudaError_t launch_product_bits(const FullPattern& a, const FullPattern& b, int nb, uint32_t* out_bits,
                                cudaStream_t st, bool upper) {
  const int t = a.words >= 128 ? 256 : (a.words >= 32 ? 128 : 32);
  { ++g_launches; k_product_bits<<<nb, t, 0, st>>>(a.rowptr, a.col, a.bits, b.bits, nb, a.words, upper ? 1 : 0, out_bits); }
  return cudaGetLastError();
}

cudaError_t launch_fill_upper_from_bits(const uint32_t* bits, int nb, int words, const int32_t* rowptr,
                                        int32_t* brow, int32_t* bcol, int32_t* slot, cudaStream_t st) {
  { ++g_launches; k_fill_upper<<<grid_for((int64_t)nb * 32, 256), 256, 0, st>>>(bits, nb, words, rowptr, brow, bcol, slot); }
  return cudaGetLastError();
}

cudaError_t launch_rowptr_from_brow(const int32_t* brow, int64_t nnzb, int nb, int32_t* rowptr, cudaStream_t st) {
  { ++g_launches; k_rowptr<<<grid_for(nb + 1, 256), 256, 0, st>>>(brow, nnzb, nb, rowptr); }
  return cudaGetLastError();
}

// flag[0]: error bits, flag[1]: number of diagonal tiles.
cudaError_t launch_check_pattern(const int32_t* brow, const int32_t* bcol, int64_t nnzb, int nb, const double* val,
                                 int64_t n, int32_t* flag, cudaStream_t st) {
  (void)n;
  cudaError_t e = cudaMemsetAsync(flag, 0, 2 * sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  if (nnzb > 0) {
    { ++g_launches; k_check_pattern<<<grid_for(nnzb, 256), 256, 0, st>>>(brow, bcol, nnzb, nb, flag, flag + 1); }
    const int64_t cnt = nnzb * TE;
    unsigned g = grid_for(cnt, 256);
    if (g > 152u * 32u) g = 152u * 32u;
    { ++g_launches; k_check_finite<<<g, 256, 0, st>>>(val, cnt, flag); }
  }
  return cudaGetLastError();
}

}  // namespace sp2
