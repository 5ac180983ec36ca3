// Tensor-core (tcgen05, sm_103a) symmetric block-sparse square with FP64-grade
// accuracy from FP16 slices, plus the fused epilogue of Algorithm 2.
//
// Slicing (a GB300-specific reading of "tile products in FP16 split precision"):
// every element x of X~ (|x| < 2 for an SP2 iterate, whose eigenvalues stay in
// about [0, 1]) is written on fixed absolute grids,
//     x ~= sum_{s=1..k} T_s * 2^-(11 s - 1),   T_s integers, |T_s| <= 2048,
// (11-bit slices; five slices use 10-bit ones, see slice_bits)
// so each slice T_s is exact in FP16.  The product of slices s and t has the
// unit 2^-(11 (s + t) - 2); all pairs with the same g = s + t share one FP32
// accumulator in tensor memory.  Their sums are integers: the g = 2 group
// (T_1 T_1) stays below 2^24 because rows of X~ have 2-norm <= ~1, so it is
// accumulated exactly; the smaller groups are exact in practice and their
// rounding error is scaled down by 2^-11 per group.  The epilogue combines the
// groups as an exact int64 fixed-point sum and converts once to FP64.  Pairs
// with s + t <= k + 1 are used (k = 4: 10 MMAs per K step, error ~2^-44 per
// element; k = 2 is the three-product hi+lo form).  Two places where the FP32
// sums would not stay exact are handled apart: the diagonal of S = X~^2, whose
// products of equal slices are all positive, is taken from FP64 squared row
// norms summed while the records are sliced; and long K loops (dense rows) are
// accumulated in segments whose exact sums the epilogue adds in int64.
//
// Operands are stored panel by panel: for a super-row R (tile rows 4R..4R+3)
// and a K tile present in any of its rows, one record holds slice s of the 4
// tiles as one contiguous 8 KB unit (the K-major layout the MMA reads, absent
// tiles zero), so one bulk copy moves a whole 128 x 32 operand slice.  The
// symmetric X~ needs one panel set for A and B alike.
//
// Most tiles of an SP2 iterate are small (density-matrix elements decay with
// distance): a tile with max |x| < 2^-11 has T_1 = 0, below 2^-22 also T_2 = 0.
// Each record notes its first slice that is not all zero.  For a K step the A
// record starts at slice fA, the B record at fB, and only the pairs s >= fA,
// t >= fB, s + t <= k + 1 are issued; only the slices they read are loaded.
// Pairs left out multiply zeros, so the result is the same bit for bit.
//
// Data path per CTA (one 128 x 128 output super-tile = 4 x 4 tiles of 32):
//   warp 0: producer -- for every K tile in the union of the super-rows'
//     patterns (32 at a time, found from the super-row bitmaps, their record
//     headers fetched one batch ahead), emits sub-steps of at most two A
//     slices x two B slices: each sub-step is one pipeline stage filled by up
//     to four 8 KB cp.async.bulk copies (completion tracked by an mbarrier
//     transaction count), described by a small stage record.
//   warp 1 lane 0: issues tcgen05.mma kind::f16 (M = 128, N = 128, K = 16) for
//     every slice pair of the record into the TMEM accumulator of its group,
//     then tcgen05.commit frees the stage.
//   all 8 warps: epilogue -- tcgen05.ld of the accumulators that were written,
//     exact fixed-point combination, X_new = c0 I + c1 X~ + c2 S in FP64,
//     per-tile ||X~ - S||^2, traces and ||X_new||^2, FP64 stores of the
//     output tiles present.
// Every wait is bounded; on timeout the kernel records an error flag, stops
// issuing work and still frees its tensor memory.
#include "sp2_internal.h"
#include <cuda_fp16.h>

namespace sp2 {
namespace {

constexpr int ST = 128;          // super-tile edge (4 tiles)

// Bits per slice: 11 (FP16 holds integers up to 2^11 exactly) for two to four
// slices; 10 for five, whose smaller digits keep the FP32 group sums of dense
// rows exact with room to spare (finest grid 2^-49, FP64 grade for |x| <= 1).
__host__ __device__ constexpr int slice_bits(int k) { return k == 5 ? 10 : 11; }
constexpr int SLICE_BYTES = 2048;  // one 32 x 32 FP16 slice

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// try_wait that lets the hardware suspend the thread for up to hint_ns (it
// resumes when the phase completes): for waiters off the critical path, so
// they do not take issue slots from the warps sharing their sub-partition.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, uint32_t parity, uint32_t hint_ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok != 0;
}

// Timeout sites of a launch, for the error message (err[1], bit 0 self-test
// probe, 8 copy warps, 9 copies still in flight at an error exit, 1 producer
// stage, 2 producer tile slot, 3 MMA data, 4 MMA TMEM or segment slot, 5 MMA
// drain, 6 epilogue tile, 7 epilogue segment).
__device__ __forceinline__ void note_timeout(int32_t* err, int where) {
  if (err) atomicOr(err + 1, 1 << where);
}

// Limit of every bounded wait of a launch (ns), set from the launch arguments.
__device__ __forceinline__ unsigned long long& wait_limit_ns() {
  __shared__ unsigned long long lim;
  return lim;
}

// Bounded wait with suspension between polls: false on timeout.
__device__ __forceinline__ bool mbar_wait_sleep(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = now_ns(), lim = wait_limit_ns();
  while (!mbar_try_wait_sleep(bar, parity, 20000u))
    if (now_ns() - t0 > lim) return false;
  return true;
}

// Bounded wait: false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = now_ns(), lim = wait_limit_ns();
  while (!mbar_try_wait(bar, parity))
    if (now_ns() - t0 > lim) return false;
  return true;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Exact int64 value of an FP32 that holds an integer (|x| < 2^31): split at
// 2^11 so both parts are below 2^22 and convert each with the FP32
// magic-number add (1.5 * 2^23), which stays on the FP32/ALU pipes.
__device__ __forceinline__ long long f32_int_to_ll(float x) {
  const float hi = truncf(x * 0x1p-11f);          // exact: power-of-two scale, integer part
  const float lo = fmaf(hi, -2048.0f, x);          // exact: |lo| < 2048
  const int ih = __float_as_int(hi + 12582912.0f) - 0x4B400000;
  const int il = __float_as_int(lo + 12582912.0f) - 0x4B400000;
  return (long long)ih * 2048 + il;
}

// The per-CTA fixed-point staging (two 128 KB slots per CTA, 38 MB in all) is
// written and read back by the same CTA within one tile: an L2 evict_last
// policy keeps it out of DRAM while the operand records stream past.
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

__device__ __forceinline__ longlong2 ld_staging(const longlong2* p, uint64_t pol) {
  long long a, b;
  asm volatile("ld.global.L2::cache_hint.v2.s64 {%0, %1}, [%2], %3;" : "=l"(a), "=l"(b) : "l"(p), "l"(pol));
  return make_longlong2(a, b);
}

__device__ __forceinline__ void st_staging(longlong2* p, longlong2 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v2.s64 [%0], {%1, %2}, %3;" ::"l"(p), "l"(v.x), "l"(v.y), "l"(pol)
               : "memory");
}

// x * 2^k, exact, by exponent arithmetic on the high word; x an integer-valued
// double (0 or |x| >= 1) and a normal result.
__device__ __forceinline__ double int_times_pow2(double x, int k) {
  const int hi = __double2hiint(x);
  return (hi & 0x7FFFFFFF) == 0 ? x : __hiloint2double(hi + (k << 20), __double2loint(x));
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// 2 z exactly (an exponent increment for normal z; the FP64 add otherwise).
__device__ __forceinline__ double twice(double z) {
  const int hi = __double2hiint(z);
  const int e = (hi >> 20) & 0x7FF;
  return (e != 0 && e < 0x7FE) ? __hiloint2double(hi + (1 << 20), __double2loint(z)) : z + z;
}

// Shared-memory matrix descriptor, no swizzle, K-major canonical layout:
// core matrices of 8 rows x 16 bytes (128 contiguous bytes), LBO = byte stride
// between core matrices along K, SBO = byte stride between 8-row groups.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // fixed 0b001 field of tcgen05 descriptors
  return d;                // base offset 0, relative LBO, no swizzle
}

// Instruction descriptor, kind::f16: FP16 A and B, FP32 D, both K-major, M = 128, N = 128.
constexpr uint32_t IDESC = (1u << 4) | (0u << 7) | (0u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ------------------------------------------------------------------ slicing
// One CTA per panel record e: the 4 tiles of the record (index words from
// k_panel_fill: compact tile index, bit 31 = use the stored tile transposed;
// all ones = absent), sliced and written as k units of 8 KB,
//   byte offset = s * 8192 + q * 2048 + g * 512 + c * 128 + r * 16 + j * 2
// for the element in row 8g + r, column 8c + j of tile q, slice s.  The header
// byte holds the first slice that is not all zero in any of the 4 tiles (k if
// none) in bits 0-2 and the tiles present in bits 4-7; units below that slice
// are all zero, are never read, and are not written.
//
// rsq (optional): rsq[128 e + 32 q + r] = sum_c x_rc^2 of row r of tile q in
// FP64, unscaled (0 for an absent tile).  Summed over the records of a
// super-row (k_row_sq_sum) they give the squared row norms of the matrix, the
// diagonal of its square.
template <int K>
__global__ void __launch_bounds__(256, 5) k_panel_slices(const uint4* __restrict__ index, const int32_t* __restrict__ slot,
                                                       const double* __restrict__ pool, __half* data,
                                                       uint8_t* head, int32_t* err, double* rsq, int lscale,
                                                       int report_range) {
  __shared__ __align__(16) __half sm[K * 4 * TE];
  __shared__ uint32_t wnz[8];
  __shared__ int first_s;
  const int64_t e = blockIdx.x;
  if (report_range && e == 0 && threadIdx.x == 0 && err) atomicOr(err, 4);
  const uint4 iw = index[e];
  const uint32_t wd[4] = {iw.x, iw.y, iw.z, iw.w};
  constexpr int W = slice_bits(K);
  constexpr int FIN = W * K - 1;                   // finest grid 2^-FIN
  constexpr int PER = TE / 256;                    // elements of a tile per thread
  // all loads first (16 per thread), then the integer work
  long long xb[4][PER];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const bool present = wd[q] != 0xFFFFFFFFu;
    const double* src = present ? pool + (int64_t)slot[wd[q] & ~REF_T] * TE : nullptr;
#pragma unroll
    for (int k = 0; k < PER; ++k) xb[q][k] = present ? __double_as_longlong(src[threadIdx.x + 256 * k]) : 0ll;
  }
  uint32_t nz = 0;                                 // bit s: slice s has a nonzero element
  uint32_t pres = 0;
  // Squared row sums (rsq): thread 32 w + l holds stored row w + 8 k, column
  // l.  Row w + 8 k of a tile used as stored is complete in warp w (a sum over
  // the lanes: lanes 8 k .. 8 k + 7 keep it in rs[q]); row l of a tile used
  // transposed is spread over the 8 warps (rs[q] = the sum over k here, over
  // the warps at the end).  Fixed order throughout (deterministic).
  static_assert(PER == 4, "four elements of a tile per thread");
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double rs[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    pres |= (wd[q] != 0xFFFFFFFFu ? 1u : 0u) << q;
    const bool tr = (wd[q] & REF_T) != 0;
    rs[q] = 0.0;
    if (rsq) {
      // FP64 is scarce on this part: squares and sums as fused multiply-adds
      double x[PER];
#pragma unroll
      for (int k = 0; k < PER; ++k) x[k] = __longlong_as_double(xb[q][k]);
      if (tr) {
        rs[q] = fma(x[3], x[3], fma(x[2], x[2], fma(x[1], x[1], x[0] * x[0])));
      } else {
        // reduce-scatter of the 4 rows over the lanes (the first step
        // exchanges the elements, the others the partial sums)
        const bool b16 = (lane & 16) != 0, b8 = (lane & 8) != 0;
        const double o0 = __shfl_xor_sync(0xffffffffu, b16 ? x[0] : x[2], 16);
        const double o1 = __shfl_xor_sync(0xffffffffu, b16 ? x[1] : x[3], 16);
        const double m0 = b16 ? x[2] : x[0], m1 = b16 ? x[3] : x[1];
        const double h0 = fma(m0, m0, o0 * o0), h1 = fma(m1, m1, o1 * o1);
        double t = (b8 ? h1 : h0) + __shfl_xor_sync(0xffffffffu, b8 ? h0 : h1, 8);
        t += __shfl_xor_sync(0xffffffffu, t, 4);
        t += __shfl_xor_sync(0xffffffffu, t, 2);
        t += __shfl_xor_sync(0xffffffffu, t, 1);
        rs[q] = t;
      }
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int i = threadIdx.x + 256 * k;
      // stored element (i / 32, i % 32) is element (r, c) of the panel's tile
      const int r = tr ? (i & 31) : (i >> 5), c = tr ? (i >> 5) : (i & 31);
      // v = x / scale * 2^FIN rounded to the nearest integer (ties to even),
      // from the bits of x = m 2^(ex - 1075): v = m >> sh on the integer pipes
      const long long x = xb[q][k];
      const int ex = (int)((x >> 52) & 0x7FF);
      long long v = 0;
      if (ex - lscale >= 1024) {           // |x / scale| >= 2, inf or NaN: flagged, clamped
        if (err) atomicOr(err, 4);
        v = (1ll << (FIN + 1)) - 1;
        if (x < 0) v = -v;
      } else if (ex != 0) {
        const unsigned long long m = ((unsigned long long)x & 0x000FFFFFFFFFFFFFull) | (1ull << 52);
        // sh >= 3 for every slice count used (FIN <= 49); a left shift, exact
        // (|v| < 2^(FIN + 1)), covers sh <= 0
        const int sh = 1075 + lscale - FIN - ex;
        unsigned long long qv = 0;
        if (sh <= 0) {
          qv = m << (-sh);
        } else if (sh < 64) {
          qv = m >> sh;
          const unsigned long long rem = m & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
          if (rem > half || (rem == half && (qv & 1ull))) ++qv;
        }
        v = x < 0 ? -(long long)qv : (long long)qv;
      }
      int T[K];
#pragma unroll
      for (int s = 0; s < K - 1; ++s) {
        const int sh = W * (K - 1 - s);
        const long long hi = (v + (1ll << (sh - 1))) >> sh;   // round to nearest (ties up)
        T[s] = (int)hi;
        v -= hi * (1ll << sh);
      }
      T[K - 1] = (int)v;
#pragma unroll
      for (int s = 0; s < K; ++s) {
        nz |= (T[s] != 0 ? 1u : 0u) << s;
        sm[(s * 4 + q) * TE + (r >> 3) * 256 + (c >> 3) * 64 + (r & 7) * 8 + (c & 7)] = __int2half_rn(T[s]);
      }
    }
  }
  nz = __reduce_or_sync(0xffffffffu, nz);
  if ((threadIdx.x & 31) == 0) wnz[threadIdx.x >> 5] = nz;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t m = 0;
    for (int w = 0; w < 8; ++w) m |= wnz[w];
    const int f = m ? __ffs(m) - 1 : K;
    first_s = f;
    head[e] = (uint8_t)(f | (pres << 4));
  }
  __syncthreads();
  // units below the first nonzero slice are all zero and never read: not written
  const uint4* s4 = reinterpret_cast<const uint4*>(sm);
  uint4* d4 = reinterpret_cast<uint4*>(data + e * (int64_t)(K * 4 * TE));
  for (int i = first_s * (4 * TE / 8) + threadIdx.x; i < K * 4 * TE / 8; i += blockDim.x) d4[i] = s4[i];
  if (!rsq) return;
  __syncthreads();                                 // sm is free: reused for the warp sums
  double* red = reinterpret_cast<double*>(sm);     // [8 warps][4 tiles][32 rows]
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if ((wd[q] & REF_T) != 0) {
      red[wid * 128 + q * 32 + lane] = rs[q];
    } else {
      red[wid * 128 + q * 32 + lane] = 0.0;
      __syncwarp();
      if ((lane & 7) == 0) red[wid * 128 + q * 32 + wid + 8 * (lane >> 3)] = rs[q];
    }
  }
  __syncthreads();
  if (threadIdx.x < 128) {
    double sum = 0.0;
#pragma unroll
    for (int u = 0; u < 8; ++u) sum += red[u * 128 + threadIdx.x];
    rsq[e * 128 + threadIdx.x] = sum;
  }
}

// dsq[128 P + j] = sum of rsq[128 e + j] over the panel records e of
// super-row P, in record order (the squared row norms; see k_panel_slices).
// One CTA of 128 threads per super-row.
__global__ void __launch_bounds__(128) k_row_sq_sum(const int32_t* __restrict__ spos, int words,
                                                    const double* __restrict__ rsq, int64_t n, double* dsq) {
  const int64_t P = blockIdx.x;
  const int j = threadIdx.x;
  const int64_t lo = spos[P * words], hi = spos[(P + 1) * words];
  double acc = 0.0;
  int64_t e = lo;
  for (; e + 4 <= hi; e += 4) {
    const double v0 = rsq[e * 128 + j], v1 = rsq[(e + 1) * 128 + j], v2 = rsq[(e + 2) * 128 + j],
                 v3 = rsq[(e + 3) * 128 + j];
    acc += v0;
    acc += v1;
    acc += v2;
    acc += v3;
  }
  for (; e < hi; ++e) acc += rsq[e * 128 + j];
  const int64_t gi = P * 128 + j;
  if (gi < n) dsq[gi] = acc;
}

// super-row bitmap: OR of the 4 tile rows
__global__ void k_super_bits(const uint32_t* __restrict__ bits, int nb, int words, int nsr, uint32_t* sb) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= (int64_t)nsr * words) return;
  const int R = (int)(i / words), w = (int)(i % words);
  uint32_t m = 0;
  for (int a = 0; a < 4; ++a) {
    const int row = 4 * R + a;
    if (row < nb) m |= bits[(int64_t)row * words + w];
  }
  sb[i] = m;
}

// Launch order of the super-tiles: blocks of RB super-rows x CB super-columns,
// row-major inside a block, blocks row-major.  CTAs that run at the same time
// then share A panels (same super-row) and B panels (same super-column), so the
// slices they stream are reused from L2 instead of each CTA pulling its own B
// panel from HBM.
constexpr int RB = 8, CB = 16;

__host__ __device__ inline int64_t blocked_size(int nsr) {
  const int64_t nbr = (nsr + RB - 1) / RB, nbc = (nsr + CB - 1) / CB;
  return nbr * nbc * RB * CB;
}

__device__ inline void blocked_decode(int64_t i, int nsr, int& R, int& C) {
  const int64_t nbc = (nsr + CB - 1) / CB;
  const int64_t b = i / (RB * CB), w = i % (RB * CB);
  R = (int)((b / nbc) * RB + w / CB);
  C = (int)((b % nbc) * CB + w % CB);
}

// flag of the i-th super-tile (R, C) in launch order: an output tile present
// (and R <= C unless the storage is general)
__global__ void k_super_flags(const uint32_t* __restrict__ obits, int nb, int words, int nsr, int general,
                              int32_t* flag) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= blocked_size(nsr)) return;
  int R, C;
  blocked_decode(i, nsr, R, C);
  int f = 0;
  if (R < nsr && C < nsr && (general || R <= C)) {
    for (int a = 0; a < 4 && !f; ++a) {
      const int row = 4 * R + a;
      if (row >= nb) break;
      const int col0 = 4 * C;
      const uint32_t m = obits[(int64_t)row * words + (col0 >> 5)] >> (col0 & 31);
      f = (m & 0xFu) != 0;
    }
  }
  flag[i] = f;
}

__global__ void k_super_fill(const int32_t* __restrict__ flag, const int32_t* __restrict__ pos, int64_t n, int nsr,
                             int32_t* list) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n || !flag[i]) return;
  int R, C;
  blocked_decode(i, nsr, R, C);
  list[pos[i]] = R * nsr + C;
}

// ------------------------------------------------------------------ main kernel
// One operand matrix of the product, as the kernel reads it: super-row
// bitmaps; the record of (super-row R, K tile) is number spos[R][word] +
// popcount of the lower bits of that word, with its header byte and k units
// of FP16 slices (see k_panel_slices).
struct TcOperand {
  const uint32_t* sbits;
  const int32_t* spos;
  const uint8_t* head;
  const __half* data;
};

struct TcArgs {
  TcOperand P, Q;           // S = sum_K P_IK Q_KJ  (+ Q_IK P_KJ when two_pass)
  int two_pass;
  const uint32_t* zbits;    // Z (the c1 term): pattern and FP64 values
  const int32_t* zrowptr;
  const uint32_t* zref;
  const int32_t* zslot;     // value slot of Z's tile index (nullptr: identity)
  const double* zpool;
  const uint32_t* obits;    // output pattern bitmap, upper tiles only
  const int32_t* orowptr;   // output tile row offsets
  const int32_t* list;      // active super-tiles, R * nsr + C
  const int32_t* count;     // number of active super-tiles (device)
  int32_t* work;            // work counter (zero at launch)
  double* opool;            // output tiles, slot = output index
  Partials part;
  double c0, c1, c2;
  double scale;             // product of the operands' slice scales
  int64_t n;
  int nb, words, nsr;
  int32_t* err;
  long long* scratch;       // per CTA, NSLOT slots: 128 x 128 fixed-point sums of a tile in its epilogue
  int seg_min;              // K loops of at least this many steps are cut into segments (0: never)
  int seg_ksteps;           // K steps per segment (8 or 16, divides the 32-step batch)
  unsigned long long wait_ns;   // limit of every bounded wait
  int selftest;             // 1: the producer first waits on a barrier nothing arrives at (timeout path test)
  int general;              // general storage: output tiles on both sides of the diagonal, weight 1 in e^2
  int split_supply;         // 1: the B units come through the copy warps (cp.async), the A units by bulk copy
  const double* dsq;        // S_ii = sum_k x_ik^2 in FP64 per global row (nullptr: from the tensor cores)
  int glo, ghi;             // slice-pair groups s + t of this launch (ghi - glo <= 3)
  int emode;                // 0: full epilogue; 1: write S (this launch's groups) into the output tiles only;
                            // 2: full epilogue on S + the S already in the output tiles
};

// A pipeline stage holds one sub-step: two A units and two B units, a unit
// being one slice of a 4-tile panel (128 rows x 32, 8 KB, 8-row groups 512 B
// apart).  A sub-step record (32 bits) tells the MMA issuer what it holds:
//   bits 3u..3u+2: slice of unit u (u = 0, 1: A units, u = 2, 3: B units),
//   bits 12-15: product mask, bit (2 i + j) for A unit i x B unit j,
//   bit 16: end of the super-tile, bit 17: no more super-tiles, bit 18: end of an
//   accumulation segment (no data).  A super-tile whose K loop has at least
//   seg_min K steps closes a segment after every 16 K steps: the epilogue adds
//   the segment's exact fixed-point sums into the scratch and frees the TMEM,
//   so no FP32 accumulator sums more than 16 K steps (512 products per
//   element) and the groups stay exact for dense operands.
constexpr int UNIT_BYTES = 4 * SLICE_BYTES;
constexpr int STAGE_BYTES = 4 * UNIT_BYTES;
constexpr int STAGES = 6;
constexpr uint32_t REC_END = 1u << 16;
constexpr int EPI_WARPS = 8;                       // epilogue warps 2..9
constexpr int COPY_WARPS = 2;                      // copy warps 10..11 (B units by 16-byte cp.async)
constexpr int TC_THREADS = 32 * (2 + EPI_WARPS + COPY_WARPS);   // + producer warp 0, MMA warp 1
constexpr uint32_t REC_LAST = 1u << 17;   // no more super-tiles (no data)
constexpr uint32_t REC_SEG = 1u << 18;    // end of an accumulation segment of the super-tile (no data)
constexpr uint32_t SEG_LAST = 1u << 31;   // segment record flag: last segment of its super-tile
constexpr int SEG_RING = 4;               // accumulation segments in flight between MMA and epilogue
constexpr int NSLOT = 3;                  // tiles in flight between the producer and the epilogue (2: 3% slower, 4: same)
constexpr int SEG_KSTEPS = 16;            // K steps per accumulation segment of a segmented tile (default)

// record header byte: first nonzero slice (bits 0-2), tiles present (bits 4-7)
constexpr uint32_t HEAD_NONE = 0x07u;   // header of a K index outside the step list

template <int K>
struct TcCfg {
  static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 + 128 * 16;
};

template <int K>
__global__ void __launch_bounds__(TC_THREADS, 1) k_square_tc(TcArgs a) {
  using Cfg = TcCfg<K>;
  constexpr unsigned FULLW = 0xffffffffu;
  // the group window and the epilogue mode vary only with five slices; fewer
  // slices take every group in one launch (compile-time constants)
  const int glo = K == 5 ? a.glo : 0, ghi = K == 5 ? a.ghi : K - 1, emode = K == 5 ? a.emode : 0;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* stage_base = smem_raw;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* acc_full = empty + STAGES;     // [SEG_RING] MMAs of a segment done (commit) + its record written
  uint64_t* tile_full = acc_full + SEG_RING;   // [NSLOT] tile slot written by the producer
  uint64_t* tile_empty = tile_full + NSLOT;    // [NSLOT] epilogue done with the tile slot (one arrive per warp)
  uint64_t* drain = tile_empty + NSLOT;    // MMAs issued before the exit are complete
  uint64_t* tmem_empty = drain + 1;        // [SEG_RING] every epilogue warp has read the segment's TMEM
  uint64_t* probe = tmem_empty + SEG_RING; // self-test: a barrier that nothing arrives at
  uint64_t* fill = probe + 1;              // [STAGES] stage record written: the copy warps may fill B
  const __half** srcb = reinterpret_cast<const __half**>(fill + STAGES);   // [STAGES] B record of the stage
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(srcb + STAGES);
  int32_t* tslot = reinterpret_cast<int32_t*>(tmem_slot + 2);      // [NSLOT] super-tile list index, -1: none
  int32_t* kcount = tslot + NSLOT;                                  // [NSLOT][16] triplets per output tile
  uint32_t* gmap = reinterpret_cast<uint32_t*>(kcount + 16 * NSLOT);   // [SEG_RING] groups written, block of each, last flag
  uint32_t* rec = gmap + SEG_RING;                                  // [STAGES] sub-step records
  int32_t* status = reinterpret_cast<int32_t*>(rec + STAGES);      // [0] a wait timed out
  uint4* ulist = reinterpret_cast<uint4*>(smem_raw + STAGES * STAGE_BYTES + 1024);   // [128] sub-steps of a batch

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      // the producer's arrival (with the bulk bytes), plus one per copy-warp thread
      mbar_init(&full[s], 1 + (a.split_supply ? 32 * COPY_WARPS : 0));
      mbar_init(&empty[s], 1);
      mbar_init(&fill[s], 1);
    }
    for (int b = 0; b < SEG_RING; ++b) {
      mbar_init(&acc_full[b], 2);
      mbar_init(&tmem_empty[b], EPI_WARPS);
    }
    for (int b = 0; b < NSLOT; ++b) {
      mbar_init(&tile_full[b], 1);
      mbar_init(&tile_empty[b], EPI_WARPS);
    }
    mbar_init(drain, 1);
    mbar_init(probe, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    status[0] = 0;
    wait_limit_ns() = a.wait_ns;
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int total = *a.count;

  // Persistent and warp-specialised: the producer (warp 0) takes super-tiles
  // from the work counter and streams their operand slices; the MMA issuer
  // (warp 1) accumulates each tile in TMEM blocks of 128 columns taken on
  // first use; the epilogue (warps 2-9) finishes tile i while tiles i + 1 and
  // i + 2 are being loaded and multiplied.  Tiles pass through NSLOT slots.
  if (warp == 0) {
    // ---------------- producer warp.  The record headers of 32 K steps are
    // fetched at a time (lane j: step j), one batch ahead of their use; the
    // lanes turn them into the batch's list of sub-steps in shared memory, and
    // lanes 0-3 issue the sub-steps, lane u copying unit u (A0, A1, B0, B1) and
    // lane 0 writing the stage record and arming its barrier.  Every lane keeps
    // its own copy of the stage counter; no warp votes per sub-step.
    int step = 0;
    int emitted = 0;   // stages whose copies were issued (lane 0's view)
    bool ok = true;
    // lanes 0-3: one sub-step (srcA / srcB: the K step's A and B panel records).
    // Lane 0 waits for the stage and the others take its result, so the four
    // lanes stay on the same stage phase.
    auto emit = [&](uint32_t rv, const __half* srcA, const __half* srcB) -> bool {
      const int s = step % STAGES;
      const uint32_t par = ((step / STAGES) & 1) ^ 1;
      ++step;
      int good = 1;
      if (lane == 0) good = mbar_wait(&empty[s], par) ? 1 : 0;
      good = __shfl_sync(0xFu, good, 0);
      if (!good) {
        if (lane == 0) {
          status[0] = 1;
          note_timeout(a.err, 1);
        }
        return false;
      }
      const uint32_t mask = (rv & (REC_END | REC_LAST | REC_SEG)) ? 0u : (rv >> 12) & 0xFu;
      // units A0, A1, B0, B1 read by a product of the mask; with the split
      // supply the B units go to the copy warps
      uint32_t use = ((mask & 0x3u) ? 1u : 0u) | ((mask & 0xCu) ? 2u : 0u) | ((mask & 0x5u) ? 4u : 0u) |
                     ((mask & 0xAu) ? 8u : 0u);
      if (a.split_supply) use &= 0x3u;
      if (lane == 0) {
        rec[s] = rv;
        srcb[s] = srcB;
        mbar_expect_tx(&full[s], (uint32_t)__popc(use) * UNIT_BYTES);
      }
      if ((use >> lane) & 1u)
        bulk_g2s(stage_base + s * STAGE_BYTES + lane * UNIT_BYTES,
                 (lane < 2 ? srcA : srcB) + (int64_t)((rv >> (3 * lane)) & 7u) * (UNIT_BYTES / 2), UNIT_BYTES,
                 &full[s]);
      if (a.split_supply && lane == 0) mbar_arrive(&fill[s]);   // release: record and B source visible
      emitted = step;
      return true;
    };
    // all lanes: a control sub-step (no data) through lanes 0-3
    auto emit_ctl = [&](uint32_t rv) -> bool {
      bool r = true;
      if (lane < 4) r = emit(rv, nullptr, nullptr);
      else ++step;
      return __shfl_sync(FULLW, r ? 1 : 0, 0) != 0;
    };
    // self-test of the timeout path: before any copy is issued, wait on a
    // barrier that nothing arrives at; the wait gives up after the wait limit,
    // the status is set, and the launch ends through the no-more-tiles path
    if (a.selftest) {
      int good = 1;
      if (lane == 0) good = mbar_wait(probe, 0) ? 1 : 0;
      good = __shfl_sync(FULLW, good, 0);
      if (!good && lane == 0) {
        status[0] = 1;
        note_timeout(a.err, 0);
      }
      __syncwarp();
    }
    for (int it = 0; ok; ++it) {
      const int b = it % NSLOT;
      // the slot's previous tile (it - NSLOT) has left the epilogue
      int good = 1;
      if (lane == 0) good = mbar_wait_sleep(&tile_empty[b], (((uint32_t)(it / NSLOT)) & 1u) ^ 1u) ? 1 : 0;
      good = __shfl_sync(FULLW, good, 0);
      if (!good) {
        if (lane == 0) { status[0] = 1; note_timeout(a.err, 2); }
        break;
      }
      int idx = 0;
      if (lane == 0) idx = atomicAdd(a.work, 1);
      idx = __shfl_sync(FULLW, idx, 0);
      if (idx >= total || *(volatile int32_t*)status != 0) {
        // no more tiles: tell the epilogue (slot) and the MMA issuer (record)
        if (lane == 0) {
          tslot[b] = -1;
          mbar_arrive(&tile_full[b]);
        }
        emit_ctl(REC_LAST);
        break;
      }
      const int stile = a.list[idx];
      const int R = stile / a.nsr, C = stile % a.nsr;
      // the epilogue learns the tile now (it drains segments while the tile is produced)
      if (lane == 0) {
        tslot[b] = idx;
        mbar_arrive(&tile_full[b]);
      }
      // K steps of the tile (both passes): long K loops are cut into segments
      int ktot = 0;
      if (a.seg_min > 0) {
        for (int pass = 0; pass < 1 + a.two_pass; ++pass) {
          const TcOperand& oa = pass == 0 ? a.P : a.Q;
          const TcOperand& ob = pass == 0 ? a.Q : a.P;
          for (int w = lane; w < a.words; w += 32)
            ktot += __popc(oa.sbits[(int64_t)R * a.words + w] & ob.sbits[(int64_t)C * a.words + w]);
        }
        ktot = __reduce_add_sync(FULLW, ktot);
      }
      const bool segmented = a.seg_min > 0 && ktot >= a.seg_min;
      int kdone = 0;
      int kc = 0;   // lane t < 16: K steps with A tile t / 4 and B tile t % 4 both present
      for (int pass = 0; pass < 1 + a.two_pass && ok; ++pass) {
        // pass 0: A = P (rows I), B = Q (rows J); pass 1: A = Q, B = P
        const TcOperand& opA = pass == 0 ? a.P : a.Q;
        const TcOperand& opB = pass == 0 ? a.Q : a.P;
        const int64_t offA = (int64_t)R * a.words, offB = (int64_t)C * a.words;
        for (int w0 = 0; w0 < a.words && ok; w0 += 32) {
          // lane L holds word w0 + L of both super-rows; the K steps are the set
          // bits of ma & mb, numbered through the inclusive prefix incl
          const int wl = w0 + lane;
          uint32_t ma = 0u, mb = 0u;
          int pa = 0, pb = 0;
          if (wl < a.words) {
            ma = opA.sbits[offA + wl];
            mb = opB.sbits[offB + wl];
            pa = opA.spos[offA + wl];
            pb = opB.spos[offB + wl];
          }
          const uint32_t mw = ma & mb;
          const int cnt = __popc(mw);
          int incl = cnt;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(FULLW, incl, o);
            if (lane >= o) incl += v;
          }
          const int total = __shfl_sync(FULLW, incl, 31);
          const int excl = incl - cnt;
          // records (A, B) of step j of this chunk and their header bytes
          auto fetch = [&](int j, int& ea, int& eb, uint32_t& ha, uint32_t& hb) {
            ea = eb = 0;
            ha = hb = HEAD_NONE;
            int L = 0;   // lanes whose prefix is <= j: the word lane of step j
#pragma unroll
            for (int h = 16; h > 0; h >>= 1)
              if (__shfl_sync(FULLW, incl, L + h - 1) <= j) L += h;
            const int Lc = min(L, 31);
            const uint32_t mL = __shfl_sync(FULLW, mw, Lc);
            const uint32_t maL = __shfl_sync(FULLW, ma, Lc);
            const uint32_t mbL = __shfl_sync(FULLW, mb, Lc);
            const int paL = __shfl_sync(FULLW, pa, Lc);
            const int pbL = __shfl_sync(FULLW, pb, Lc);
            const int exL = __shfl_sync(FULLW, excl, Lc);
            if (j < total) {
              uint32_t m = mL;
              for (int r = j - exL; r > 0; --r) m &= m - 1;
              const uint32_t below = (1u << (__ffs(m) - 1)) - 1u;
              ea = paL + __popc(maL & below);
              eb = pbL + __popc(mbL & below);
              ha = opA.head[ea];
              hb = opB.head[eb];
            }
          };
          int ea, eb;
          uint32_t ha, hb;
          fetch(lane, ea, eb, ha, hb);
          for (int jb = 0; jb < total && ok; jb += 32) {
            int ea_n, eb_n;
            uint32_t ha_n, hb_n;
            fetch(jb + 32 + lane, ea_n, eb_n, ha_n, hb_n);   // next batch, in flight during this one
            // triplet counts: K steps of this batch with A tile x and B tile y present
            const uint32_t pa4 = (ha >> 4) & 0xFu, pb4 = (hb >> 4) & 0xFu;
#pragma unroll
            for (int t = 0; t < 16; ++t) {
              const int c16 = __popc(__ballot_sync(FULLW, (pa4 >> (t >> 2)) & (pb4 >> (t & 3)) & 1u));
              if (lane == t) kc += c16;
            }
            // sub-steps of this lane's K step: pairs s >= fa, t >= fb with
            // glo <= s + t <= ghi (the launch's group window), two A and two B
            // slices each; the B pair starts where A slice a0 + 1 meets glo
            // (at most three sub-steps for every window used)
            const int fa = (int)(ha & 7u), fb = (int)(hb & 7u);
            uint32_t rv0 = 0u, rv1 = 0u, rv2 = 0u;
            int ns = 0;
            for (int a0 = fa; a0 <= K - 1 && a0 + fb <= ghi; a0 += 2) {
              for (int b0 = max(fb, glo - a0 - 1); b0 <= K - 1 && a0 + b0 <= ghi; b0 += 2) {
                uint32_t mask = 0;
                for (int i = 0; i < 2; ++i)
                  for (int jj = 0; jj < 2; ++jj) {
                    const int si = a0 + i, tj = b0 + jj;
                    if (si <= K - 1 && tj <= K - 1 && si + tj >= glo && si + tj <= ghi)
                      mask |= 1u << (2 * i + jj);
                  }
                if (!mask) continue;
                const uint32_t rv = (uint32_t)a0 | ((uint32_t)min(a0 + 1, K - 1) << 3) | ((uint32_t)b0 << 6) |
                                    ((uint32_t)min(b0 + 1, K - 1) << 9) | (mask << 12);
                if (ns == 0) rv0 = rv;
                else if (ns == 1) rv1 = rv;
                else rv2 = rv;
                ++ns;
              }
            }
            // a segmented tile also closes a segment before every seg_ksteps-th K
            // step inside the batch (the batch end closes one too)
            const int lead = (segmented && lane > 0 && (lane % a.seg_ksteps) == 0 && jb + lane < total) ? 1 : 0;
            int soff = ns + lead;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
              const int v = __shfl_up_sync(FULLW, soff, o);
              if (lane >= o) soff += v;
            }
            const int nsub = __shfl_sync(FULLW, soff, 31);
            soff -= ns;
            if (lead) ulist[soff - 1] = make_uint4(REC_SEG, 0u, 0u, 0u);
            if (ns > 0) ulist[soff] = make_uint4(rv0, (uint32_t)ea, (uint32_t)eb, 0u);
            if (ns > 1) ulist[soff + 1] = make_uint4(rv1, (uint32_t)ea, (uint32_t)eb, 0u);
            if (ns > 2) ulist[soff + 2] = make_uint4(rv2, (uint32_t)ea, (uint32_t)eb, 0u);
            __syncwarp();
            bool lok = true;
            if (lane < 4) {
              for (int u = 0; u < nsub; ++u) {
                const uint4 en = ulist[u];
                if (!emit(en.x, opA.data + (int64_t)en.y * (K * UNIT_BYTES / 2),
                          opB.data + (int64_t)en.z * (K * UNIT_BYTES / 2))) {
                  lok = false;
                  break;
                }
              }
            } else {
              step += nsub;
            }
            ok = __all_sync(FULLW, lok);
            __syncwarp();   // the list is rebuilt for the next batch
            kdone += min(32, total - jb);
            if (segmented && ok && kdone < ktot) ok = emit_ctl(REC_SEG);
            ea = ea_n;
            eb = eb_n;
            ha = ha_n;
            hb = hb_n;
          }
        }
      }
      // counts before the end record: the record's barrier, then the segment's,
      // order them before the epilogue's reads
      if (lane < 16) kcount[b * 16 + lane] = kc;
      __syncwarp();
      if (ok) ok = emit_ctl(REC_END);
    }
    // after a timeout anywhere in the CTA: wait (bounded) until the copies of
    // the last STAGES emitted stages have landed, so that no bulk copy into
    // this CTA's shared memory is in flight when the CTA exits
    if (lane == 0 && *(volatile int32_t*)status != 0) {
      for (int j = max(0, emitted - STAGES); j < emitted; ++j)
        if (!mbar_wait(&full[j % STAGES], (uint32_t)(j / STAGES) & 1u)) note_timeout(a.err, 9);
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer.  TMEM is four blocks of 128 columns; a group
    // accumulator of a segment (a whole super-tile, or 32 of its K steps) takes
    // a free block on its first product, and the blocks of a segment return to
    // the pool once every epilogue warp has read them (one arrival per warp on
    // the segment slot's tmem_empty barrier; segments are reclaimed in order).
    uint32_t free_mask = 0xFu;
    // blocks held by the segment in each ring slot (4 slots)
    uint32_t pend0 = 0u, pend1 = 0u, pend2 = 0u, pend3 = 0u;
    int released = 0;              // segments whose blocks are back in free_mask
    int seg = 0;                   // segments published
    unsigned long long nprod = 0;
    bool ok = true, done = false;
    // take back the blocks of the oldest segment that still holds some; false on timeout
    auto reclaim = [&]() -> bool {
      if (!mbar_wait(&tmem_empty[released & (SEG_RING - 1)], ((uint32_t)released >> 2) & 1u)) {
        note_timeout(a.err, 4);
        return false;
      }
      tc_fence_after();
      switch (released & (SEG_RING - 1)) {
        case 0: free_mask |= pend0; pend0 = 0u; break;
        case 1: free_mask |= pend1; pend1 = 0u; break;
        case 2: free_mask |= pend2; pend2 = 0u; break;
        default: free_mask |= pend3; pend3 = 0u; break;
      }
      ++released;
      return true;
    };
    // stage counter and phase kept incrementally; the shared-memory descriptor
    // of a unit is the stage's descriptor plus a constant (the start-address
    // field holds address / 16 in 14 bits; every address here is below 2^18)
    int s = 0;
    uint32_t par = 0;
    const uint64_t d0 = make_desc(smem_u32(stage_base), 128, 512);
    while (ok && !done) {
      uint32_t written = 0, gblk = 0, used = 0;
      uint32_t kind = 0;
      for (;;) {
        const int cs = s;
        const uint32_t cpar = par;
        if (++s == STAGES) { s = 0; par ^= 1u; }
        if (!mbar_wait(&full[cs], cpar)) { ok = false; note_timeout(a.err, 3); break; }
        tc_fence_after();
        // units written by cp.async (generic proxy) are read by the MMAs (async proxy)
        if (a.split_supply) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        const uint32_t rv = rec[cs];
        if (rv & (REC_END | REC_LAST | REC_SEG)) {
          mma_commit(&empty[cs]);
          kind = rv & (REC_END | REC_LAST | REC_SEG);
          break;
        }
        const uint64_t ds = d0 + (uint64_t)(cs * (STAGE_BYTES >> 4));
#pragma unroll
        for (int i = 0; i < 2; ++i) {
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            if (!((rv >> (12 + 2 * i + j)) & 1u)) continue;
            // group relative to the launch's window (at most four groups live)
            const int g = (int)((rv >> (3 * i)) & 7u) + (int)((rv >> (6 + 3 * j)) & 7u) - glo;
            if (!((written >> g) & 1u)) {
              while (free_mask == 0u && ok) ok = reclaim();
              if (!ok) break;
              const uint32_t blk = (uint32_t)(__ffs(free_mask) - 1);
              free_mask &= ~(1u << blk);
              used |= 1u << blk;
              gblk |= blk << (2 * g);
            }
            const uint32_t dcol = tmem + ((gblk >> (2 * g)) & 3u) * ST;
            const uint32_t acc = (written >> g) & 1u;
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
              const uint64_t ad = ds + (uint64_t)((i * UNIT_BYTES + kk * 256) >> 4);
              const uint64_t bd = ds + (uint64_t)(((2 + j) * UNIT_BYTES + kk * 256) >> 4);
              // the first MMA into a group accumulator of a segment overwrites it
              mma_f16(dcol, ad, bd, (kk > 0 || acc) ? 1u : 0u);
            }
            written |= 1u << g;
            ++nprod;
          }
          if (!ok) break;
        }
        mma_commit(&empty[cs]);
        if (!ok) break;
      }
      if (!ok) break;
      if (kind & REC_LAST) { done = true; break; }
      // publish the segment in ring slot seg % SEG_RING once the segment that used
      // the slot before has been read and its blocks reclaimed
      while (released < seg - (SEG_RING - 1) && ok) ok = reclaim();
      if (!ok) break;
      const int q = seg & (SEG_RING - 1);
      switch (q) {
        case 0: pend0 = used; break;
        case 1: pend1 = used; break;
        case 2: pend2 = used; break;
        default: pend3 = used; break;
      }
      gmap[q] = written | (gblk << 8) | ((kind & REC_END) ? SEG_LAST : 0u);
      mma_commit(&acc_full[q]);    // arrives once every MMA of the segment has completed
      mbar_arrive(&acc_full[q]);   // release: segment record visible to the epilogue
      ++seg;
    }
    if (!ok) status[0] = 1;
    // slice-pair products issued (each 2 MMAs of 128 x 128 x 16)
    if (a.err && nprod) atomicAdd(reinterpret_cast<unsigned long long*>(a.err + 2), nprod);
    mma_commit(drain);
    if (!mbar_wait(drain, 0)) { status[0] = 1; note_timeout(a.err, 5); }
  } else if (warp >= 2 + EPI_WARPS) {
    // ---------------- copy warps (split supply only).  Stage by stage, in the
    // producer's order: wait until the producer has written the stage record
    // (fill), copy the B units the record uses as 16-byte cp.async pieces (the
    // 64 threads take every 64th piece of an 8 KB unit), then arrive on the
    // stage's full barrier when this thread's copies have landed.  Control
    // records carry no data but are arrived at all the same.
    if (a.split_supply) {
      const int t = threadIdx.x - 32 * (2 + EPI_WARPS);   // 0 .. 63
      int ns = 0;
      uint32_t npar = 0;
      for (;;) {
        const int s = ns;
        const uint32_t par = npar;
        if (++ns == STAGES) { ns = 0; npar ^= 1u; }
        bool good = true;
        if (lane == 0) good = mbar_wait_sleep(&fill[s], par);
        good = __shfl_sync(FULLW, good ? 1 : 0, 0) != 0;
        if (!good) {
          if (lane == 0) {
            status[0] = 1;
            note_timeout(a.err, 8);
          }
          break;
        }
        const uint32_t rv = rec[s];
        if (!(rv & (REC_END | REC_LAST | REC_SEG))) {
          const uint32_t mask = (rv >> 12) & 0xFu;
          const __half* srcB = srcb[s];
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            if (!(mask & (j == 0 ? 0x5u : 0xAu))) continue;
            const char* src = reinterpret_cast<const char*>(srcB + (int64_t)((rv >> (6 + 3 * j)) & 7u) * (UNIT_BYTES / 2));
            const uint32_t dst = smem_u32(stage_base + s * STAGE_BYTES + (2 + j) * UNIT_BYTES);
#pragma unroll
            for (int c = t; c < UNIT_BYTES / 16; c += 32 * COPY_WARPS)
              asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + 16 * c), "l"(src + 16 * c)
                           : "memory");
          }
        }
        asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(&full[s])) : "memory");
        if (rv & REC_LAST) break;
      }
      asm volatile("cp.async.wait_all;" ::: "memory");
    }
  } else if (warp >= 2) {
    // ---------------- epilogue (warps 2-9, two per SM sub-partition: warp w
    // reads TMEM lanes 32 (w % 4)..+31 = tile row I0 + w % 4, lane = row inside
    // the tile; warps 2-5 take column tiles 0-1, warps 6-9 column tiles 2-3).
    // Phase 1 moves the exact fixed-point sums to the CTA's scratch and returns
    // the TMEM blocks, so the next tile's products run during phase 2, the FP64
    // arithmetic.
    const int quarter = warp & 3;
    const int bt0 = 2 * ((warp - 2) >> 2);
    const int r = lane;
    // unit of the finest group of the window: with W bits per slice, slice s
    // lies on the grid 2^-(W s + W - 1), so group g = s + t has the unit
    // 2^-(W g + 2 W - 2)
    constexpr int W = slice_bits(K);
    const double su = ldexp(1.0, -(W * ghi + 2 * W - 2)) * a.scale;   // S = fx * su, su a power of two
    const int lsu = ilogb(su);
    // X_new = c0 I + c1 X~ + c2 S.  Without acceleration (alpha = 1) the two
    // polynomials need fewer FP64 operations, with the same results:
    //   x^2 (c0 = c1 = 0, c2 = 1): S itself;  2x - x^2 (c0 = 0, c1 = 2, c2 = -1): 2 z - S.
    const int form = (a.c0 == 0.0 && a.c1 == 0.0 && a.c2 == 1.0) ? 1
                   : (a.c0 == 0.0 && a.c1 == 2.0 && a.c2 == -1.0) ? 2 : 0;
    // index of tile (row, col) in a pattern given by row bitmaps and row
    // offsets, -1 if absent; the lanes share the popcount of the row's words
    auto find = [&](const uint32_t* bits, const int32_t* rowptr, int row, int col) -> int {
      const uint32_t* rb = bits + (int64_t)row * a.words;
      const int wc = col >> 5;
      const uint32_t m = rb[wc];
      if (!((m >> (col & 31)) & 1u)) return -1;
      int cnt = 0;
      for (int w = lane; w < wc; w += 32) cnt += __popc(rb[w]);
      cnt = __reduce_add_sync(FULLW, cnt);
      return rowptr[row] + cnt + __popc(m & ((1u << (col & 31)) - 1u));
    };
    int seg = 0;   // segments consumed
    const uint64_t pol = policy_evict_last();
    for (int it = 0;; ++it) {
      const int b = it % NSLOT;
      const uint32_t par = ((uint32_t)(it / NSLOT)) & 1u;
      bool good = true;
      if (lane == 0) good = mbar_wait_sleep(&tile_full[b], par);
      good = __shfl_sync(FULLW, good ? 1 : 0, 0) != 0;
      if (!good) { if (lane == 0) { status[0] = 1; note_timeout(a.err, 6); } break; }
      __syncwarp();
      const int idx = tslot[b];
      if (idx < 0) break;
      const int stile = a.list[idx];
      const int R = stile / a.nsr, C = stile % a.nsr;
      const int I0 = 4 * R, J0 = 4 * C;
      const int Ia = I0 + quarter;           // tile row of this thread
      const int64_t gi = (int64_t)Ia * TB + r;
      long long* scr = a.scratch + ((int64_t)blockIdx.x * NSLOT + b) * (ST * ST) + (int64_t)(quarter * 32 + r) * ST;
      // output tile index of each column tile
      int oidx[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int Jb = J0 + bt0 + h;
        oidx[h] = (Ia < a.nb && Jb < a.nb && (a.general || Ia <= Jb)) ? find(a.obits, a.orowptr, Ia, Jb) : -1;
      }
      // Z_IJ of each output tile (X~_IJ in the forward step; absent -> null),
      // looked up and its row requested into L2 before the accumulators are
      // waited for, so that the chain of dependent loads overlaps the wait
      const double* Zt[2] = {nullptr, nullptr};
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (oidx[h] < 0 || emode == 1) continue;
        const int zp = find(a.zbits, a.zrowptr, Ia, J0 + bt0 + h);
        if (zp < 0) continue;
        const int64_t zi = (int64_t)(a.zref[zp] & ~REF_T);
        Zt[h] = a.zpool + (int64_t)(a.zslot ? a.zslot[zi] : zi) * TE;
        prefetch_l2(Zt[h] + r * TB);
        prefetch_l2(Zt[h] + r * TB + 16);
      }
      // phase 1, once per accumulation segment: TMEM -> the exact fixed-point
      // sums of this thread's row in the scratch (the first segment stores, the
      // others add), then the segment's TMEM blocks go back to the MMA issuer
      for (bool first = true;; first = false) {
        const int q = seg & (SEG_RING - 1);
        const uint32_t spar = ((uint32_t)seg >> 2) & 1u;
        if (lane == 0) good = mbar_wait_sleep(&acc_full[q], spar);
        good = __shfl_sync(FULLW, good ? 1 : 0, 0) != 0;
        if (!good) {
          if (lane == 0) note_timeout(a.err, 7);
          break;
        }
        __syncwarp();
        tc_fence_after();
        const uint32_t gm = gmap[q];
        const uint32_t written = gm & 0xFu;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int bt = bt0 + h;
          if (oidx[h] < 0) continue;      // warp-uniform
#pragma unroll
          for (int ch = 0; ch < 2; ++ch) {
            const int col0 = bt * 32 + ch * 16;
            long long fx[16];
            longlong2* sp = reinterpret_cast<longlong2*>(scr + col0);
            if (first) {
#pragma unroll
              for (int i = 0; i < 16; ++i) fx[i] = 0;
            } else {
#pragma unroll
              for (int i = 0; i < 8; ++i) {
                const longlong2 t2 = ld_staging(sp + i, pol);
                fx[2 * i] = t2.x;
                fx[2 * i + 1] = t2.y;
              }
            }
#pragma unroll
            for (int gg = 0; gg < 4; ++gg) {   // relative groups of the window
              if (gg <= ghi - glo && ((written >> gg) & 1u)) {   // warp-uniform: groups no product reached are zero
                float g[16];
                const uint32_t blk = (gm >> (8 + 2 * gg)) & 3u;
                tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + blk * ST + (uint32_t)col0, g);
#pragma unroll
                for (int i = 0; i < 16; ++i) fx[i] += f32_int_to_ll(g[i]) * (1ll << (W * (ghi - glo - gg)));
              }
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) st_staging(sp + i, make_longlong2(fx[2 * i], fx[2 * i + 1]), pol);
          }
        }
        // this warp's TMEM reads of the segment are complete
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tmem_empty[q]);
        ++seg;
        if (gm & SEG_LAST) break;
      }
      if (!good) { if (lane == 0) status[0] = 1; break; }
      // phase 2: X_new, per-tile ||X~ - S||^2, ||X_new||^2 and traces
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int bt = bt0 + h;
        const int Jb = J0 + bt;
        const int oi = oidx[h];
        if (oi < 0) continue;
        const double* Z = Zt[h];
        double trS = 0.0, trX = 0.0, n2 = 0.0, e2 = 0.0;
        double* O = a.opool + (int64_t)oi * TE;
        for (int ch = 0; ch < 2; ++ch) {     // 16 columns per chunk
          const int col0 = bt * 32 + ch * 16;
          double zv[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) zv[i] = 0.0;
          if (Z) {
            const double2* zp = reinterpret_cast<const double2*>(Z + r * TB + ch * 16);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const double2 t2 = zp[i];
              zv[2 * i] = t2.x;
              zv[2 * i + 1] = t2.y;
            }
          }
          long long fx[16];
          const longlong2* sp = reinterpret_cast<const longlong2*>(scr + col0);
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const longlong2 t2 = ld_staging(sp + i, pol);
            fx[2 * i] = t2.x;
            fx[2 * i + 1] = t2.y;
          }
          // emode 2: the finer groups' S, left in the output tile by the launch before
          double prev[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) prev[i] = 0.0;
          if (emode == 2) {
            const double2* pp = reinterpret_cast<const double2*>(O + r * TB + ch * 16);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const double2 t2 = pp[i];
              prev[2 * i] = t2.x;
              prev[2 * i + 1] = t2.y;
            }
          }
          double out[16];
          if (Z || form == 0) {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const int c = ch * 16 + i;
              const int64_t gj = (int64_t)Jb * TB + c;
              const bool inside = gi < a.n && gj < a.n;
              const double fxd = inside ? (double)fx[i] : 0.0;
              const double z = inside ? zv[i] : 0.0;
              const bool dg = inside && gi == gj;
              const double S0 = int_times_pow2(fxd, lsu);      // fx * su
              if (emode == 1) { out[i] = S0; continue; }     // finer groups only: S is stored
              // the diagonal of S = X~^2 is the squared row norm, taken in FP64
              // (its digit products are all positive and pass the exact range
              // of the FP32 group sums on dense rows)
              const double S = (dg && a.dsq) ? a.dsq[gi] : (emode == 2 ? S0 + prev[i] : S0);
              double xn;
              // c2 S = (c2 su) fx exactly (su is a power of two)
              if (form == 1) xn = S;
              else if (form == 2) xn = twice(z) - S;
              else xn = fma(a.c2, S, fma(a.c1, z, dg ? a.c0 : 0.0));
              out[i] = xn;
              const double df = z - S;
              e2 = fma(df, df, e2);
              n2 = fma(xn, xn, n2);
              if (dg) { trS += S; trX += z; }
            }
          } else {
            // no X~ tile here (z = 0) and X_new = S or 2 z - S = -S: every
            // (z - S)^2 equals xn^2, so one FMA per element gives both sums
            // (e2 is set from n2 below; the same values in the same order)
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const int c = ch * 16 + i;
              const int64_t gj = (int64_t)Jb * TB + c;
              const bool inside = gi < a.n && gj < a.n;
              const double fxd = inside ? (double)fx[i] : 0.0;
              const bool dg = inside && gi == gj;
              const double S0 = int_times_pow2(fxd, lsu);
              if (emode == 1) { out[i] = S0; continue; }
              const double S = (dg && a.dsq) ? a.dsq[gi] : (emode == 2 ? S0 + prev[i] : S0);
              const double xn = form == 1 ? S : 0.0 - S;
              out[i] = xn;
              n2 = fma(xn, xn, n2);
              if (dg) trS += S;
            }
          }
          double2* op = reinterpret_cast<double2*>(O + r * TB + ch * 16);
#pragma unroll
          for (int i = 0; i < 8; ++i) op[i] = make_double2(out[2 * i], out[2 * i + 1]);
        }
        if (emode == 1) continue;
        if (!Z && form != 0) e2 = n2;
        // warp reductions (the tile's 32 rows are this warp's 32 lanes)
        for (int o = 16; o > 0; o >>= 1) {
          e2 += __shfl_xor_sync(FULLW, e2, o);
          n2 += __shfl_xor_sync(FULLW, n2, o);
          trS += __shfl_xor_sync(FULLW, trS, o);
          trX += __shfl_xor_sync(FULLW, trX, o);
        }
        if (lane == 0) {
          const bool diag = Ia == Jb;
          a.part.e2[oi] = (diag || a.general ? 1.0 : 2.0) * e2;
          a.part.n2[oi] = n2;
          a.part.trS[oi] = diag ? trS : 0.0;
          a.part.trX[oi] = diag ? trX : 0.0;
          a.part.ktiles[oi] = kcount[b * 16 + quarter * 4 + bt];
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&tile_empty[b]);
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
  if (threadIdx.x == 0 && status[0] != 0 && a.err) atomicOr(a.err, 1);
}

inline unsigned grid_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

size_t panel_record_bytes(int k) { return (size_t)k * UNIT_BYTES; }

cudaError_t launch_panel_slices(const uint32_t* index, int64_t nrec, const int32_t* slot, const double* pool,
                                void* data, uint8_t* head, int k, int32_t* err, double* rsq, double scale,
                                bool report_range, cudaStream_t st) {
  if (nrec == 0) return cudaSuccess;
  const uint4* ix = reinterpret_cast<const uint4*>(index);
  __half* d = static_cast<__half*>(data);
  const int ls = ilogb(scale);   // scale is a power of two
  const int rr = report_range ? 1 : 0;
  const unsigned g = (unsigned)nrec;
  ++g_launches;
  if (k == 2) k_panel_slices<2><<<g, 256, 0, st>>>(ix, slot, pool, d, head, err, rsq, ls, rr);
  else if (k == 3) k_panel_slices<3><<<g, 256, 0, st>>>(ix, slot, pool, d, head, err, rsq, ls, rr);
  else if (k == 5) k_panel_slices<5><<<g, 256, 0, st>>>(ix, slot, pool, d, head, err, rsq, ls, rr);
  else k_panel_slices<4><<<g, 256, 0, st>>>(ix, slot, pool, d, head, err, rsq, ls, rr);
  return cudaGetLastError();
}

// number of set bits of each word
__global__ void k_popc_words(const uint32_t* __restrict__ bits, int64_t n, int32_t* cnt) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) cnt[i] = __popc(bits[i]);
}

// Record index words: one warp per tile row; every stored tile (row, K) of the
// both-triangle pattern writes its word (slot row % 4) of the record of
// (super-row row / 4, K): compact tile index, bit 31 when the stored tile is
// used transposed.  Words start all ones (absent).
__global__ void k_panel_fill(const int32_t* __restrict__ frowptr, const int32_t* __restrict__ fcol,
                             const uint32_t* __restrict__ fref, const uint32_t* __restrict__ sbits,
                             const int32_t* __restrict__ spos, int nb, int words, uint32_t* index) {
  const int row = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= nb) return;
  const int64_t o = (int64_t)(row >> 2) * words;
  for (int p = frowptr[row] + lane; p < frowptr[row + 1]; p += 32) {
    const int k = fcol[p];
    const int w = k >> 5;
    const int64_t e = spos[o + w] + __popc(sbits[o + w] & ((1u << (k & 31)) - 1u));
    index[e * 4 + (row & 3)] = fref[p];
  }
}

cudaError_t launch_row_sq_sum(const int32_t* spos, int nsr, int words, const double* rsq, int64_t n, double* dsq,
                              cudaStream_t st) {
  if (nsr == 0) return cudaSuccess;
  ++g_launches;
  k_row_sq_sum<<<(unsigned)nsr, 128, 0, st>>>(spos, words, rsq, n, dsq);
  return cudaGetLastError();
}

cudaError_t launch_popc_words(const uint32_t* bits, int64_t n, int32_t* cnt, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  ++g_launches;
  k_popc_words<<<grid_for(n, 256), 256, 0, st>>>(bits, n, cnt);
  return cudaGetLastError();
}

cudaError_t launch_panel_fill(const FullPattern& fp, int nb, const uint32_t* sbits, const int32_t* spos,
                              uint32_t* index, cudaStream_t st) {
  if (nb == 0) return cudaSuccess;
  ++g_launches;
  k_panel_fill<<<grid_for((int64_t)nb * 32, 256), 256, 0, st>>>(fp.rowptr, fp.col, fp.ref, sbits, spos, nb, fp.words,
                                                                 index);
  return cudaGetLastError();
}

// max |x| over the tiles of a set (for the power-of-two slice scale of G)
__global__ void k_absmax(const int32_t* __restrict__ slot, const double* __restrict__ pool, int64_t nnzb,
                         unsigned long long* out) {
  double m = 0.0;
  for (int64_t t = blockIdx.x; t < nnzb; t += gridDim.x) {
    const double* x = pool + (int64_t)slot[t] * TE;
    for (int q = threadIdx.x; q < TE; q += blockDim.x) m = fmax(m, fabs(x[q]));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

cudaError_t launch_absmax(const TileSet& x, const double* pool, unsigned long long* out, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess || x.nnzb == 0) return e;
  ++g_launches;
  k_absmax<<<(unsigned)std::min<int64_t>(x.nnzb, 152 * 8), 256, 0, st>>>(x.slot, pool, x.nnzb, out);
  return cudaGetLastError();
}

// upper-triangle bitmap of a tile set (bit J of row I for I <= J only)
__global__ void k_upper_bits(const int32_t* __restrict__ brow, const int32_t* __restrict__ bcol, int64_t nnzb,
                             uint32_t* bits, int words) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nnzb) return;
  const int i = brow[t], j = bcol[t];
  atomicOr(&bits[(int64_t)i * words + (j >> 5)], 1u << (j & 31));
}

cudaError_t launch_upper_bits(const TileSet& x, int nb, int words, uint32_t* bits, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(bits, 0, (size_t)nb * words * 4, st);
  if (e != cudaSuccess || x.nnzb == 0) return e;
  ++g_launches;
  k_upper_bits<<<grid_for(x.nnzb, 256), 256, 0, st>>>(x.brow, x.bcol, x.nnzb, bits, words);
  return cudaGetLastError();
}

cudaError_t launch_super_bits(const FullPattern& fp, int nb, int nsr, uint32_t* sb, cudaStream_t st) {
  ++g_launches;
  k_super_bits<<<grid_for((int64_t)nsr * fp.words, 256), 256, 0, st>>>(fp.bits, nb, fp.words, nsr, sb);
  return cudaGetLastError();
}

int64_t super_order_size(int nsr) { return blocked_size(nsr); }

cudaError_t launch_super_flags(const uint32_t* obits, int nb, int words, int nsr, int32_t* flag, cudaStream_t st,
                               bool general) {
  ++g_launches;
  k_super_flags<<<grid_for(blocked_size(nsr), 256), 256, 0, st>>>(obits, nb, words, nsr, general ? 1 : 0, flag);
  return cudaGetLastError();
}

cudaError_t launch_super_fill(const int32_t* flag, const int32_t* pos, int64_t n, int nsr, int32_t* list,
                              cudaStream_t st) {
  ++g_launches;
  k_super_fill<<<grid_for(n, 256), 256, 0, st>>>(flag, pos, n, nsr, list);
  return cudaGetLastError();
}

cudaError_t launch_square_tc(const TcLaunch& L, cudaStream_t st) {
  if (L.nsuper == 0) return cudaSuccess;
  TcArgs a;
  a.P = TcOperand{L.P.sbits, L.P.spos, L.P.head, static_cast<const __half*>(L.P.data)};
  a.Q = TcOperand{L.Q.sbits, L.Q.spos, L.Q.head, static_cast<const __half*>(L.Q.data)};
  a.two_pass = L.two_pass ? 1 : 0;
  a.zbits = L.Z->bits; a.zrowptr = L.Z->rowptr; a.zref = L.Z->ref; a.zslot = L.zslot; a.zpool = L.zpool;
  a.obits = L.obits; a.orowptr = L.orowptr; a.list = L.list; a.count = L.count; a.work = L.work;
  a.opool = L.opool;
  a.part = L.part; a.c0 = L.c0; a.c1 = L.c1; a.c2 = L.c2; a.scale = L.scale; a.n = L.n; a.nb = L.nb;
  a.words = L.words; a.nsr = L.nsr; a.err = L.err; a.scratch = static_cast<long long*>(L.scratch);
  a.seg_min = L.seg_min;
  a.seg_ksteps = L.seg_ksteps > 0 ? L.seg_ksteps : SEG_KSTEPS;
  a.wait_ns = L.wait_ns;
  a.selftest = L.selftest ? 1 : 0;
  a.general = L.general ? 1 : 0;
  a.split_supply = L.split_supply ? 1 : 0;
  a.dsq = L.dsq;
  a.glo = L.glo;
  a.ghi = L.ghi < 0 ? L.k - 1 : L.ghi;
  a.emode = L.emode;
  cudaError_t e = cudaSuccess;
  switch (L.k) {
    case 2:
      e = cudaFuncSetAttribute(k_square_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcCfg<2>::SMEM);
      if (e == cudaSuccess) { ++g_launches; k_square_tc<2><<<(unsigned)L.nsuper, TC_THREADS, TcCfg<2>::SMEM, st>>>(a); }
      break;
    case 3:
      e = cudaFuncSetAttribute(k_square_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcCfg<3>::SMEM);
      if (e == cudaSuccess) { ++g_launches; k_square_tc<3><<<(unsigned)L.nsuper, TC_THREADS, TcCfg<3>::SMEM, st>>>(a); }
      break;
    case 5:
      e = cudaFuncSetAttribute(k_square_tc<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcCfg<5>::SMEM);
      if (e == cudaSuccess) { ++g_launches; k_square_tc<5><<<(unsigned)L.nsuper, TC_THREADS, TcCfg<5>::SMEM, st>>>(a); }
      break;
    default:
      e = cudaFuncSetAttribute(k_square_tc<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcCfg<4>::SMEM);
      if (e == cudaSuccess) { ++g_launches; k_square_tc<4><<<(unsigned)L.nsuper, TC_THREADS, TcCfg<4>::SMEM, st>>>(a); }
      break;
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace sp2

namespace sp2 {
int tc_tile_slots() { return NSLOT; }
}  // namespace sp2
