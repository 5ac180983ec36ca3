// FP64 symmetric block-sparse square with the fused epilogue of Algorithm 2.
//
// For every output tile (I, J), I <= J, of the product pattern:
//   S_IJ = sum_{K in R(I) & R(J)} X~_IK X~_KJ            (X~_KJ = X~_JK^T, symmetry)
//   X_new = c0 I + c1 X~_IJ + c2 S_IJ                     (Algorithm 2: p=1 gives
//           c0=(1-a)^2, c1=2a(1-a), c2=a^2; p=0 gives c0=0, c1=2a, c2=-a^2)
// and per tile the partial sums of ||X~ - S||_F^2 (weight 2 off the diagonal:
// the mirrored tile is not stored), trace(S), trace(X~) on diagonal tiles and
// ||X_new tile||_F^2 for the truncation.  e_{i-1} = ||X~_{i-1} - X~_{i-1}^2||_F and
// t_{i-1} = trace(X~_{i-1} - X~_{i-1}^2) (Algorithm 2) come out of the same pass.
//
// Sym-sum mode (used by the adjoint): S_IJ = sum_K A_IK B_KJ + B_IK A_KJ.
//
// GB300's FP64 rate is the bound here (about 1.2 TFLOP/s for DFMA, the same
// for the FP64 MMA instruction), so the kernel is written for a busy FP64 pipe:
// one CTA of 256 threads per output tile, 4 outputs per thread, both operand
// tiles staged in shared memory (transposed on the fly when the stored tile is
// the mirror), several CTAs per SM hide the load latency.
#include "sp2_internal.h"

namespace sp2 {
namespace {

struct PatDev {
  const uint32_t* bits;
  const int32_t* rowptr;
  const uint32_t* ref;
};

struct SqDev {
  PatDev A, B, Z;
  const double* apool;
  const double* bpool;
  const double* zpool;
  const int32_t* obrow;
  const int32_t* obcol;
  const int32_t* oslot;
  double* opool;
  double c0, c1, c2;
  int64_t n;
  int words;
  int general;   // both triangles stored: no mirror weight
  Partials part;
};

__device__ __forceinline__ void load_tile(double (*S)[TB + 1], const double* __restrict__ src, bool trans) {
#pragma unroll
  for (int q = 0; q < TE / 256; ++q) {
    const int idx = threadIdx.x + 256 * q;
    const int r = idx >> 5, c = idx & 31;
    const double v = src[idx];
    if (trans) S[c][r] = v; else S[r][c] = v;
  }
}

// acc += sum_K P_IK Q_KJ over K in R_P(I) & R_Q(J); Q_KJ = (Q_JK)^T.
__device__ __forceinline__ int accumulate(const PatDev& P, const double* __restrict__ ppool, const PatDev& Q,
                                          const double* __restrict__ qpool, int I, int J, int words,
                                          double (*As)[TB + 1], double (*Bs)[TB + 1], double acc[2][2]) {
  const uint32_t* bi = P.bits + (int64_t)I * words;
  const uint32_t* bj = Q.bits + (int64_t)J * words;
  int baseI = P.rowptr[I], baseJ = Q.rowptr[J];
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  int nk = 0;
  for (int w = 0; w < words; ++w) {
    const uint32_t mi = bi[w], mj = bj[w];
    uint32_t m = mi & mj;
    while (m) {
      const int b = __ffs(m) - 1;
      m &= m - 1;
      const uint32_t below = (1u << b) - 1u;
      const uint32_t ra = P.ref[baseI + __popc(mi & below)];
      const uint32_t rb = Q.ref[baseJ + __popc(mj & below)];
      // P_IK: stored tile, transposed when it is the mirror.
      load_tile(As, ppool + (int64_t)(ra & ~REF_T) * TE, (ra & REF_T) != 0);
      // Q_KJ = (Q_JK)^T: Q_JK is the stored tile (or its mirror), so transpose
      // exactly when Q_JK is not itself the mirror.
      load_tile(Bs, qpool + (int64_t)(rb & ~REF_T) * TE, (rb & REF_T) == 0);
      __syncthreads();
#pragma unroll 8
      for (int k = 0; k < TB; ++k) {
        const double a0 = As[ty][k], a1 = As[ty + 16][k];
        const double b0 = Bs[k][tx], b1 = Bs[k][tx + 16];
        acc[0][0] = fma(a0, b0, acc[0][0]);
        acc[0][1] = fma(a0, b1, acc[0][1]);
        acc[1][0] = fma(a1, b0, acc[1][0]);
        acc[1][1] = fma(a1, b1, acc[1][1]);
      }
      __syncthreads();
      ++nk;
    }
    baseI += __popc(mi);
    baseJ += __popc(mj);
  }
  return nk;
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < 8; ++k) s += red[k];
  return s;
}

template <bool SYM>
__global__ void __launch_bounds__(256) k_square_f64(SqDev a) {
  __shared__ double As[TB][TB + 1];
  __shared__ double Bs[TB][TB + 1];
  __shared__ double red[8];
  const int64_t t = blockIdx.x;
  const int I = a.obrow[t], J = a.obcol[t];
  double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  int nk = accumulate(a.A, a.apool, a.B, a.bpool, I, J, a.words, As, Bs, acc);
  if (SYM) nk += accumulate(a.B, a.bpool, a.A, a.apool, I, J, a.words, As, Bs, acc);

  // Z_IJ (X~_IJ in the forward step): present iff bit J of Z's row I is set.
  const uint32_t* bz = a.Z.bits + (int64_t)I * a.words;
  const int wj = J >> 5;
  const uint32_t mz = bz[wj];
  const bool hasZ = (mz >> (J & 31)) & 1u;
  const double* Zt = nullptr;
  if (hasZ) {
    int pos = a.Z.rowptr[I];
    for (int w = 0; w < wj; ++w) pos += __popc(bz[w]);
    pos += __popc(mz & ((1u << (J & 31)) - 1u));
    Zt = a.zpool + (int64_t)(a.Z.ref[pos] & ~REF_T) * TE;  // I <= J: never a mirror
  }
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  double* O = a.opool + (int64_t)a.oslot[t] * TE;
  double e2 = 0.0, trS = 0.0, trX = 0.0, n2 = 0.0;
#pragma unroll
  for (int u = 0; u < 2; ++u) {
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int r = ty + 16 * u, c = tx + 16 * v;
      const int64_t gi = (int64_t)I * TB + r, gj = (int64_t)J * TB + c;
      const bool inside = gi < a.n && gj < a.n;
      const double s = inside ? acc[u][v] : 0.0;
      const double z = (inside && hasZ) ? Zt[r * TB + c] : 0.0;
      const bool dg = inside && gi == gj;
      const double xn = inside ? ((dg ? a.c0 : 0.0) + a.c1 * z) + a.c2 * s : 0.0;
      O[r * TB + c] = xn;
      const double d = z - s;
      e2 += d * d;
      n2 += xn * xn;
      if (dg) { trS += s; trX += z; }
    }
  }
  const double w = (I == J || a.general) ? 1.0 : 2.0;
  e2 = block_sum(e2, red);
  if (threadIdx.x == 0) a.part.e2[t] = w * e2;
  n2 = block_sum(n2, red);
  if (threadIdx.x == 0) a.part.n2[t] = n2;
  if (I == J) {
    trS = block_sum(trS, red);
    if (threadIdx.x == 0) a.part.trS[t] = trS;
    trX = block_sum(trX, red);
    if (threadIdx.x == 0) a.part.trX[t] = trX;
  } else if (threadIdx.x == 0) {
    a.part.trS[t] = 0.0;
    a.part.trX[t] = 0.0;
  }
  if (threadIdx.x == 0) a.part.ktiles[t] = nk;
}

// Fixed-order two-level reduction of the per-tile partials.  Block g sums the
// contiguous range [g c, (g+1) c), c = ceil(nt / RED_BLOCKS): thread k takes
// entries k, k + 256, ... of the range in order, then a fixed tree; one block
// then sums the RED_BLOCKS results with the same tree.  The result depends on
// nt only, not on scheduling.
constexpr int RED_BLOCKS = 256;

struct RedPart {
  double e2, trS, trX;
  long long k;
};

__device__ void block_tree(double a, double b, double c, long long k, RedPart* out) {
  __shared__ double s0[256], s1[256], s2[256];
  __shared__ long long s3[256];
  s0[threadIdx.x] = a; s1[threadIdx.x] = b; s2[threadIdx.x] = c; s3[threadIdx.x] = k;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      s0[threadIdx.x] += s0[threadIdx.x + h];
      s1[threadIdx.x] += s1[threadIdx.x + h];
      s2[threadIdx.x] += s2[threadIdx.x + h];
      s3[threadIdx.x] += s3[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = RedPart{s0[0], s1[0], s2[0], s3[0]};
}

__global__ void __launch_bounds__(256) k_reduce_part(Partials p, int64_t nt, RedPart* part) {
  const int64_t c = (nt + RED_BLOCKS - 1) / RED_BLOCKS;
  const int64_t lo = (int64_t)blockIdx.x * c, hi = min(nt, lo + c);
  double a = 0.0, b = 0.0, d = 0.0;
  long long k = 0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += 256) {
    a += p.e2[i];
    b += p.trS[i];
    d += p.trX[i];
    k += p.ktiles[i];
  }
  block_tree(a, b, d, k, &part[blockIdx.x]);
}

__global__ void __launch_bounds__(256) k_reduce_step(const RedPart* __restrict__ part, StepScalars* out) {
  const RedPart q = part[threadIdx.x];   // RED_BLOCKS == blockDim.x
  __shared__ RedPart r;
  block_tree(q.e2, q.trS, q.trX, q.k, &r);
  __syncthreads();
  if (threadIdx.x == 0) {
    out->e2 = r.e2;
    out->trS = r.trS;
    out->trX = r.trX;
    out->triplets = r.k;
  }
}

PatDev dev(const FullPattern* f) { return PatDev{f->bits, f->rowptr, f->ref}; }

}  // namespace

cudaError_t launch_square_f64(const SquareArgs& a, cudaStream_t st) {
  if (a.out->nnzb == 0) return cudaSuccess;
  SqDev d;
  d.A = dev(a.A); d.B = dev(a.B); d.Z = dev(a.Z);
  d.apool = a.apool; d.bpool = a.bpool; d.zpool = a.zpool;
  d.obrow = a.out->brow; d.obcol = a.out->bcol; d.oslot = a.out->slot; d.opool = a.outpool;
  d.c0 = a.c0; d.c1 = a.c1; d.c2 = a.c2;
  d.n = a.n; d.words = a.A->words;
  d.general = a.general ? 1 : 0;
  d.part = a.part;
  if (a.sym_sum) { ++g_launches; k_square_f64<true><<<(unsigned)a.out->nnzb, 256, 0, st>>>(d); }
  else { ++g_launches; k_square_f64<false><<<(unsigned)a.out->nnzb, 256, 0, st>>>(d); }
  return cudaGetLastError();
}

size_t reduce_work_bytes() { return RED_BLOCKS * sizeof(RedPart); }

cudaError_t launch_reduce_step(const Partials& p, int64_t ntiles, StepScalars* out, void* work, cudaStream_t st) {
  RedPart* part = static_cast<RedPart*>(work);
  g_launches += 2;
  k_reduce_part<<<RED_BLOCKS, 256, 0, st>>>(p, ntiles, part);
  k_reduce_step<<<1, RED_BLOCKS, 0, st>>>(part, out);
  return cudaGetLastError();
}

}  // namespace sp2
