// Tensor-core (tcgen05, sm_103a) symmetric block-sparse square with FP64-grade
// accuracy from FP16 slices, plus the fused epilogue of Algorithm 2.
//
// Slicing (a GB300-specific reading of "tile products in FP16 split precision"):
// every element x of X~ (|x| < 2 for an SP2 iterate, whose eigenvalues stay in
// about [0, 1]) is written on fixed absolute grids,
//     x ~= sum_{s=1..k} T_s * 2^-(11 s - 1),   T_s integers, |T_s| <= 2048,
// so each slice T_s is exact in FP16.  The product of slices s and t has the
// unit 2^-(11 (s + t) - 2); all pairs with the same g = s + t share one FP32
// accumulator in tensor memory.  Their sums are integers: the g = 2 group
// (T_1 T_1) stays below 2^24 because rows of X~ have 2-norm <= ~1, so it is
// accumulated exactly; the smaller groups are exact in practice and their
// rounding error is scaled down by 2^-11 per group.  The epilogue combines the
// groups as an exact int64 fixed-point sum and converts once to FP64.  Pairs
// with s + t <= k + 1 are used (k = 4: 10 MMAs per K step, error ~2^-44 per
// element; k = 2 is the three-product hi+lo form).
//
// Data path per CTA (one 128 x 128 output super-tile = 4 x 4 tiles of 32):
//   warp 0 lane 0: producer -- for every K tile in the union of the super-rows'
//     patterns, one cp.async.bulk (TMA engine) of the k slices of each of the
//     4 A tiles X~_{I+a,K} and 4 B tiles X~_{J+b,K} (8 KB each for k = 4) into a
//     pipeline stage, completion tracked by an mbarrier transaction count;
//     absent tiles come from a zero block.
//   warp 1 lane 0: issues tcgen05.mma kind::f16 (M = 128, N = 128, K = 16) for
//     every slice pair into the TMEM accumulator of its group, then
//     tcgen05.commit frees the stage.
//   all 8 warps: epilogue -- tcgen05.ld of the k accumulators, exact fixed-point
//     combination, X_new = c0 I + c1 X~ + c2 S in FP64, per-tile ||X~ - S||^2,
//     traces and ||X_new||^2, FP64 stores of the output tiles present.
// Every wait is bounded; on timeout the kernel records an error flag, stops
// issuing work and still frees its tensor memory.
#include "sp2_internal.h"
#include <cuda_fp16.h>

namespace sp2 {
namespace {

constexpr int ST = 128;          // super-tile edge (4 tiles)
constexpr int SLICE_BYTES = 2048;  // one 32 x 32 FP16 slice
constexpr unsigned long long WAIT_NS = 2000000000ull;   // bounded waits give up after ~2 s

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

// Bounded wait: false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = now_ns();
  while (!mbar_try_wait(bar, parity))
    if (now_ns() - t0 > WAIT_NS) return false;
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
// One CTA per stored tile t (values at pool slot slot[t]): write both
// orientations (the tile and its transpose) of the k slices, at index t, in
// the interleaved K-major layout
//   byte offset = g * (k * 512) + s * 512 + c * 128 + r * 16 + j * 2
// for the element in row 8g + r, column 8c + j of slice s.
template <int K>
__global__ void __launch_bounds__(256) k_make_slices(const int32_t* __restrict__ slot, const double* __restrict__ pool,
                                                      __half* slices, int32_t* err, double inv_scale) {
  // both orientations are assembled in shared memory, then written out with
  // coalesced 16-byte stores (2 * k * 2 KB per tile)
  __shared__ __align__(16) __half sm[2][K * TE];
  const int64_t t = blockIdx.x;
  const double* src = pool + (int64_t)slot[t] * TE;
  constexpr int FIN = 11 * K - 1;                  // finest grid 2^-FIN
  for (int q = threadIdx.x; q < TE; q += blockDim.x) {
    const int r = q >> 5, c = q & 31;
    double x = src[q] * inv_scale;
    if (!(fabs(x) < 2.0)) {
      if (err) atomicOr(err, 4);
      x = fmin(fmax(x, -1.999), 1.999);
    }
    long long v = __double2ll_rn(x * (double)(1ll << FIN));
    int T[K];
#pragma unroll
    for (int s = 0; s < K - 1; ++s) {
      const int sh = 11 * (K - 1 - s);
      const long long hi = (v + (1ll << (sh - 1))) >> sh;   // round to nearest (ties up)
      T[s] = (int)hi;
      v -= hi * (1ll << sh);
    }
    T[K - 1] = (int)v;
#pragma unroll
    for (int s = 0; s < K; ++s) {
      const __half h = __int2half_rn(T[s]);
      sm[0][(r >> 3) * (K * 256) + s * 256 + (c >> 3) * 64 + (r & 7) * 8 + (c & 7)] = h;
      sm[1][(c >> 3) * (K * 256) + s * 256 + (r >> 3) * 64 + (c & 7) * 8 + (r & 7)] = h;
    }
  }
  __syncthreads();
  const uint4* s4 = reinterpret_cast<const uint4*>(&sm[0][0]);
  uint4* d4 = reinterpret_cast<uint4*>(slices + t * 2 * (int64_t)K * TE);
  for (int i = threadIdx.x; i < 2 * K * TE / 8; i += blockDim.x) d4[i] = s4[i];
}

__global__ void k_zero_half(__half* p, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) p[i] = __float2half(0.0f);
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

// flag of the i-th super-tile (R, C) in launch order: R <= C and an output tile present
__global__ void k_super_flags(const uint32_t* __restrict__ obits, int nb, int words, int nsr, int32_t* flag) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= blocked_size(nsr)) return;
  int R, C;
  blocked_decode(i, nsr, R, C);
  int f = 0;
  if (R < nsr && C < nsr && R <= C) {
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
// One operand matrix of the product: both-triangle pattern, super-row bitmap
// and FP16 slices (indexed by value slot).
struct TcOperand {
  const uint32_t* bits;
  const int32_t* frowptr;
  const uint32_t* fref;
  const uint32_t* sbits;
  const __half* slices;
};

struct TcArgs {
  TcOperand P, Q;           // S = sum_K P_IK Q_KJ  (+ Q_IK P_KJ when two_pass)
  int two_pass;
  const uint32_t* zbits;    // Z (the c1 term): pattern and FP64 values
  const int32_t* zrowptr;
  const uint32_t* zref;
  const int32_t* zslot;     // value slot of Z's tile index (nullptr: identity)
  const double* zpool;
  const __half* zero;       // K * 1024 zeros
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
};

template <int K>
struct TcCfg {
  static constexpr int TILE_BLOCK = K * SLICE_BYTES;          // k slices of one tile
  static constexpr int STAGE_BYTES = 8 * TILE_BLOCK;          // 4 A + 4 B tiles
  static constexpr int STAGES = (K >= 4) ? 3 : (K == 3 ? 4 : 6);
  static constexpr int SMEM = STAGES * STAGE_BYTES + 1024;
  // unit of the finest group, 2^-(11 (k + 1) - 2)
  static constexpr double UNIT = 1.0 / (double)(1ull << (11 * (K + 1) - 2));
};

template <int K>
__global__ void __launch_bounds__(256, 1) k_square_tc(TcArgs a) {
  using Cfg = TcCfg<K>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* stage_base = smem_raw;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + Cfg::STAGES * Cfg::STAGE_BYTES);
  uint64_t* empty = full + Cfg::STAGES;
  uint64_t* accb = empty + Cfg::STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accb + 1);
  int32_t* kcount = reinterpret_cast<int32_t*>(tmem_slot + 2);   // [16] triplets per tile
  int32_t* status = kcount + 16;                                   // [0] timeout, [1] steps, [2] tile index

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < Cfg::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accb, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    status[0] = 0;
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

  // Persistent: every CTA takes super-tiles from the work counter until none are
  // left.  Pipeline stages and barrier phases continue across tiles (step_base),
  // TMEM is allocated once; the accumulator barrier flips once per tile.
  int step_base = 0;        // steps issued by this CTA before the current tile
  uint64_t zero_slots = 0;  // producer: 8 bits per stage, slots that hold zeros
  bool alive = true;
  for (uint32_t tile_iter = 0; alive; ++tile_iter) {
    if (threadIdx.x == 0) status[2] = atomicAdd(a.work, 1);
    if (threadIdx.x < 16) kcount[threadIdx.x] = 0;
    __syncthreads();
    const int idx = status[2];
    if (idx >= total || status[0] != 0) break;
    const int st = a.list[idx];
    const int R = st / a.nsr, C = st % a.nsr;
    const int I0 = 4 * R, J0 = 4 * C;

    if (warp == 0) {
      // ---------------- producer warp: lane q < 8 owns operand tile q (A rows
      // I0..I0+3, then B rows J0..J0+3); the 8 tile lookups and bulk copies of a
      // K step run in parallel, lane 0 arms the stage barrier first.
      const int q = lane;
      const int row = (q < 4) ? I0 + q : J0 + (q - 4);
      const bool own = q < 8 && row < a.nb;
      int step = step_base;
      bool ok = true;
      for (int pass = 0; pass < 1 + a.two_pass && ok; ++pass) {
        // pass 0: A = P (rows I), B = Q (rows J); pass 1: A = Q, B = P
        const TcOperand& opA = pass == 0 ? a.P : a.Q;
        const TcOperand& opB = pass == 0 ? a.Q : a.P;
        const TcOperand& mine = (q < 4) ? opA : opB;
        const uint32_t* sA = opA.sbits + (int64_t)R * a.words;
        const uint32_t* sB = opB.sbits + (int64_t)C * a.words;
        int base = own ? mine.frowptr[row] : 0;
        for (int w = 0; w < a.words && ok; ++w) {
          uint32_t m = sA[w] & sB[w];
          const uint32_t rb = own ? mine.bits[(int64_t)row * a.words + w] : 0u;
          while (m) {
            const int b = __ffs(m) - 1;
            m &= m - 1;
            const int s = step % Cfg::STAGES;
            const uint32_t par = ((step / Cfg::STAGES) & 1) ^ 1;
            // the tile lookup does not depend on the stage: issue it before waiting
            const bool present = (rb >> b) & 1u;
            const void* src = nullptr;
            if (present) {
              const uint32_t rf = mine.fref[base + __popc(rb & ((1u << b) - 1u))];
              src = mine.slices + ((int64_t)(rf & ~REF_T) * 2 + ((rf & REF_T) ? 1 : 0)) * (int64_t)K * TE;
            }
            const uint32_t pres = __ballot_sync(0xffffffffu, q < 8 && present) & 0xFFu;
            int good = 1;
            if (lane == 0) good = mbar_wait(&empty[s], par) ? 1 : 0;
            good = __shfl_sync(0xffffffffu, good, 0);
            if (!good) { ok = false; if (lane == 0) status[0] = 1; break; }
            unsigned char* dst = stage_base + s * Cfg::STAGE_BYTES;
            // zero-fill absent slots that do not hold zeros yet (whole warp, 16-byte stores)
            uint32_t fill = ~pres & ~(uint32_t)(zero_slots >> (8 * s)) & 0xFFu;
            if (fill) {
              while (fill) {
                const int slot = __ffs(fill) - 1;
                fill &= fill - 1;
                uint4* z4 = reinterpret_cast<uint4*>(dst + slot * Cfg::TILE_BLOCK);
                for (int i = lane; i < Cfg::TILE_BLOCK / 16; i += 32) z4[i] = make_uint4(0u, 0u, 0u, 0u);
              }
              asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
              __syncwarp();
            }
            zero_slots = (zero_slots & ~(0xFFull << (8 * s))) | ((uint64_t)(~pres & 0xFFu) << (8 * s));
            if (lane == 0) mbar_expect_tx(&full[s], (uint32_t)__popc(pres) * Cfg::TILE_BLOCK);
            __syncwarp();
            if (q < 8 && present) bulk_g2s(dst + q * Cfg::TILE_BLOCK, src, Cfg::TILE_BLOCK, &full[s]);
            if (lane == 0) {
              const int amask = pres & 0xF, bmask = (pres >> 4) & 0xF;
              for (int x = 0; x < 4; ++x)
                for (int y = 0; y < 4; ++y)
                  if (((amask >> x) & 1) && ((bmask >> y) & 1)) kcount[x * 4 + y] += 1;
            }
            ++step;
          }
          base += __popc(rb);
        }
      }
      if (lane == 0) status[1] = step - step_base;
    } else if (warp == 1 && lane == 0) {
      // ---------------- MMA issuer
      int nsteps = 0;
      for (int w = 0; w < a.words; ++w)
        nsteps += __popc(a.P.sbits[(int64_t)R * a.words + w] & a.Q.sbits[(int64_t)C * a.words + w]);
      if (a.two_pass)
        for (int w = 0; w < a.words; ++w)
          nsteps += __popc(a.Q.sbits[(int64_t)R * a.words + w] & a.P.sbits[(int64_t)C * a.words + w]);
      bool ok = true;
      for (int ls = 0; ls < nsteps; ++ls) {
        const int step = step_base + ls;
        const int s = step % Cfg::STAGES;
        const uint32_t par = (step / Cfg::STAGES) & 1;
        if (!mbar_wait(&full[s], par)) { ok = false; status[0] = 1; break; }
        tc_fence_after();
        const uint32_t sA = smem_u32(stage_base + s * Cfg::STAGE_BYTES);
        const uint32_t sB = sA + 4 * Cfg::TILE_BLOCK;
#pragma unroll
        for (int ps = 0; ps < K; ++ps) {
#pragma unroll
          for (int pt = 0; pt < K; ++pt) {
            if (ps + pt > K - 1) continue;          // s + t <= k + 1 (1-based)
            const uint32_t dcol = tmem + (uint32_t)((ps + pt) * ST);
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
              const uint64_t ad = make_desc(sA + ps * 512 + kk * 256, 128, K * 512);
              const uint64_t bd = make_desc(sB + pt * 512 + kk * 256, 128, K * 512);
              // the first MMA into each group accumulator of a tile (its first
              // step, first K half, ps = 0) overwrites it; all others accumulate
              mma_f16(dcol, ad, bd, (ls > 0 || kk > 0 || ps > 0) ? 1u : 0u);
            }
          }
        }
        mma_commit(&empty[s]);
      }
      if (!ok) status[0] = 1;
      mma_commit(accb);   // arrives once every MMA issued above has completed
    }
    __syncwarp();
    __syncthreads();

    // ---------------- epilogue (all 8 warps)
    const int nsteps = status[1];
    step_base += nsteps;
    // block-uniform outcome of the bounded wait (a late completion must not split the CTA)
    const bool acc_ok = !__syncthreads_or(!mbar_wait(accb, tile_iter & 1u) || status[0] != 0);
    if (!acc_ok) alive = false;
    tc_fence_after();
    const int quarter = warp & 3;          // TMEM lanes 32*quarter .. +31
    const int half = warp >> 2;            // columns 64*half .. +63
    const int Ia = I0 + quarter;           // tile row of this thread
    const int r = lane;                    // row inside the tile
    const int64_t gi = (int64_t)Ia * TB + r;
    for (int hb = 0; hb < 2 && alive; ++hb) {   // two tiles per half: b = 2*half + hb
      const int b = 2 * half + hb;
      const int Jb = J0 + b;
      const bool valid = Ia < a.nb && Jb < a.nb && Ia <= Jb;
      // output tile index (if present in the output pattern)
      int oidx = -1;
      if (valid) {
        const uint32_t* ob = a.obits + (int64_t)Ia * a.words;
        const uint32_t mo = ob[Jb >> 5];
        if ((mo >> (Jb & 31)) & 1u) {
          int pos = a.orowptr[Ia];
          for (int w = 0; w < (Jb >> 5); ++w) pos += __popc(ob[w]);
          oidx = pos + __popc(mo & ((1u << (Jb & 31)) - 1u));
        }
      }
      // Z_IJ (X~_IJ in the forward step; absent -> 0)
      const double* Zt = nullptr;
      if (oidx >= 0) {
        const uint32_t* bz = a.zbits + (int64_t)Ia * a.words;
        const uint32_t mz = bz[Jb >> 5];
        if ((mz >> (Jb & 31)) & 1u) {
          int pos = a.zrowptr[Ia];
          for (int w = 0; w < (Jb >> 5); ++w) pos += __popc(bz[w]);
          pos += __popc(mz & ((1u << (Jb & 31)) - 1u));
          const int64_t zi = (int64_t)(a.zref[pos] & ~REF_T);
          Zt = a.zpool + (int64_t)(a.zslot ? a.zslot[zi] : zi) * TE;
        }
      }
      double e2 = 0.0, trS = 0.0, trX = 0.0, n2 = 0.0;
      // S = fx * UNIT * scale with fx the exact fixed-point sum of the groups; the
      // unit is folded into the coefficients: xn = c0 [diag] + c1 z + (c2 su) fx
      const double su = Cfg::UNIT * a.scale;
      const double c2u = a.c2 * su;
      for (int ch = 0; ch < 2; ++ch) {     // 16 columns per chunk
        const int col0 = b * 32 + ch * 16;
        double zv[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) zv[i] = 0.0;
        if (oidx >= 0 && Zt) {
          const double2* zp = reinterpret_cast<const double2*>(Zt + r * TB + ch * 16);
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const double2 t2 = zp[i];
            zv[2 * i] = t2.x;
            zv[2 * i + 1] = t2.y;
          }
        }
        float g[K][16];
        if (nsteps > 0) {
#pragma unroll
          for (int gg = 0; gg < K; ++gg)
            tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(gg * ST + col0), g[gg]);
        } else {
#pragma unroll
          for (int gg = 0; gg < K; ++gg)
#pragma unroll
            for (int i = 0; i < 16; ++i) g[gg][i] = 0.0f;
        }
        if (oidx < 0) continue;
        double* O = a.opool + (int64_t)oidx * TE;
        double out[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int c = ch * 16 + i;
          const int64_t gj = (int64_t)Jb * TB + c;
          const bool inside = gi < a.n && gj < a.n;
          long long fx = 0;
#pragma unroll
          for (int gg = 0; gg < K; ++gg) fx += f32_int_to_ll(g[gg][i]) * (1ll << (11 * (K - 1 - gg)));
          const double fxd = inside ? (double)fx : 0.0;
          const double z = inside ? zv[i] : 0.0;
          const bool dg = inside && gi == gj;
          const double xn = inside ? fma(c2u, fxd, fma(a.c1, z, dg ? a.c0 : 0.0)) : 0.0;
          out[i] = xn;
          const double d = fma(fxd, -su, z);
          e2 = fma(d, d, e2);
          n2 = fma(xn, xn, n2);
          if (dg) { trS += fxd * su; trX += z; }
        }
        double2* op = reinterpret_cast<double2*>(O + r * TB + ch * 16);
#pragma unroll
        for (int i = 0; i < 8; ++i) op[i] = make_double2(out[2 * i], out[2 * i + 1]);
      }
      // warp reductions (the tile's 32 rows are this warp's 32 lanes)
      for (int o = 16; o > 0; o >>= 1) {
        e2 += __shfl_xor_sync(0xffffffffu, e2, o);
        n2 += __shfl_xor_sync(0xffffffffu, n2, o);
        trS += __shfl_xor_sync(0xffffffffu, trS, o);
        trX += __shfl_xor_sync(0xffffffffu, trX, o);
      }
      if (lane == 0 && oidx >= 0) {
        const bool diag = Ia == Jb;
        a.part.e2[oidx] = (diag ? 1.0 : 2.0) * e2;
        a.part.n2[oidx] = n2;
        a.part.trS[oidx] = diag ? trS : 0.0;
        a.part.trX[oidx] = diag ? trX : 0.0;
        a.part.ktiles[oidx] = kcount[quarter * 4 + b];
      }
    }
    if (threadIdx.x == 0 && a.err) {
      if (!acc_ok) atomicOr(a.err, 1);
      // K steps issued (hardware MMA work = steps * pairs * 2 MMAs of 128x128x16)
      atomicAdd(reinterpret_cast<unsigned long long*>(a.err + 2), (unsigned long long)nsteps);
    }
    // TMEM reads of this tile are complete before the next tile's MMAs start
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
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

size_t slice_block_bytes(int k) { return (size_t)k * SLICE_BYTES; }

cudaError_t launch_make_slices(const TileSet& x, const double* pool, void* slices, int k, int32_t* err,
                               double scale, cudaStream_t st) {
  if (x.nnzb == 0) return cudaSuccess;
  __half* s = static_cast<__half*>(slices);
  const double inv = 1.0 / scale;   // scale is a power of two: exact
  if (k == 2) { ++g_launches; k_make_slices<2><<<(unsigned)x.nnzb, 256, 0, st>>>(x.slot, pool, s, err, inv); }
  else if (k == 3) { ++g_launches; k_make_slices<3><<<(unsigned)x.nnzb, 256, 0, st>>>(x.slot, pool, s, err, inv); }
  else { ++g_launches; k_make_slices<4><<<(unsigned)x.nnzb, 256, 0, st>>>(x.slot, pool, s, err, inv); }
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

cudaError_t launch_zero_half(void* p, int64_t n, cudaStream_t st) {
  ++g_launches;
  k_zero_half<<<grid_for(n, 256), 256, 0, st>>>(static_cast<__half*>(p), n);
  return cudaGetLastError();
}

cudaError_t launch_super_bits(const FullPattern& fp, int nb, int nsr, uint32_t* sb, cudaStream_t st) {
  ++g_launches;
  k_super_bits<<<grid_for((int64_t)nsr * fp.words, 256), 256, 0, st>>>(fp.bits, nb, fp.words, nsr, sb);
  return cudaGetLastError();
}

int64_t super_order_size(int nsr) { return blocked_size(nsr); }

cudaError_t launch_super_flags(const uint32_t* obits, int nb, int words, int nsr, int32_t* flag, cudaStream_t st) {
  ++g_launches;
  k_super_flags<<<grid_for(blocked_size(nsr), 256), 256, 0, st>>>(obits, nb, words, nsr, flag);
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
  a.P = TcOperand{L.P->bits, L.P->rowptr, L.P->ref, L.Psbits, static_cast<const __half*>(L.Pslices)};
  a.Q = TcOperand{L.Q->bits, L.Q->rowptr, L.Q->ref, L.Qsbits, static_cast<const __half*>(L.Qslices)};
  a.two_pass = L.two_pass ? 1 : 0;
  a.zbits = L.Z->bits; a.zrowptr = L.Z->rowptr; a.zref = L.Z->ref; a.zslot = L.zslot; a.zpool = L.zpool;
  a.zero = static_cast<const __half*>(L.zero);
  a.obits = L.obits; a.orowptr = L.orowptr; a.list = L.list; a.count = L.count; a.work = L.work;
  a.opool = L.opool;
  a.part = L.part; a.c0 = L.c0; a.c1 = L.c1; a.c2 = L.c2; a.scale = L.scale; a.n = L.n; a.nb = L.nb;
  a.words = L.P->words; a.nsr = L.nsr; a.err = L.err;
  cudaError_t e = cudaSuccess;
  switch (L.k) {
    case 2:
      e = cudaFuncSetAttribute(k_square_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcCfg<2>::SMEM);
      if (e == cudaSuccess) { ++g_launches; k_square_tc<2><<<(unsigned)L.nsuper, 256, TcCfg<2>::SMEM, st>>>(a); }
      break;
    case 3:
      e = cudaFuncSetAttribute(k_square_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcCfg<3>::SMEM);
      if (e == cudaSuccess) { ++g_launches; k_square_tc<3><<<(unsigned)L.nsuper, 256, TcCfg<3>::SMEM, st>>>(a); }
      break;
    default:
      e = cudaFuncSetAttribute(k_square_tc<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcCfg<4>::SMEM);
      if (e == cudaSuccess) { ++g_launches; k_square_tc<4><<<(unsigned)L.nsuper, 256, TcCfg<4>::SMEM, st>>>(a); }
      break;
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace sp2
