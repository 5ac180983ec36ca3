// Measurement program (not part of libsp2): back-to-back tcgen05.mma kind::f16
// (M = 128, N = 64, 128 or 256, K = 16), operands in shared memory (no-swizzle
// K-major, the layout type of the square's slice units), one CTA per SM, no other
// traffic.  Gives the cycles per MMA that the tensor-core square is compared
// with.  The final wait is bounded (2 s) and reported through the error word.
// Build and run: nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o mma_rate mma_rate.cu && ./mma_rate
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
template <int N>
__global__ void __launch_bounds__(128, 1) k_rate(int nmma, long long* cycles, int* err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tslot;
  const int warp = threadIdx.x >> 5;
  // zero operands: A 128 x 16 (4 KB) x 2 buffers, B N x 16 x 2 buffers
  for (int i = threadIdx.x; i < (2 * 4096 + 2 * N * 32) / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(sm)[i] = make_uint4(0, 0, 0, 0);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(&tslot)) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tslot;
  if (threadIdx.x == 0) {
    const uint32_t idesc = (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((128u >> 4) << 24);
    const uint32_t a0 = smem_u32(sm), b0 = a0 + 2 * 4096;
    const long long t0 = clock64();
    for (int i = 0; i < nmma; ++i) {
      const uint64_t ad = make_desc(a0 + (i & 1) * 4096, 128, 256);
      const uint64_t bd = make_desc(b0 + (i & 1) * (N * 32), 128, 256);
      asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                   "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                   "l"(ad), "l"(bd), "r"(idesc), "r"(i > 0 ? 1 : 0) : "memory");
    }
    const long long t1 = clock64();
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(&bar)) : "memory");
    uint32_t ok = 0;
    unsigned long long g0, g1;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(g0));
    g1 = g0;
    while (!ok && g1 - g0 < 2000000000ull) {
      asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                   : "=r"(ok) : "r"(smem_u32(&bar)) : "memory");
      asm volatile("mov.u64 %0, %globaltimer;" : "=l"(g1));
    }
    if (!ok) atomicOr(err, 1);
    const long long t2 = clock64();
    cycles[blockIdx.x * 2] = t1 - t0;
    cycles[blockIdx.x * 2 + 1] = t2 - t0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
  }
}
template <int N>
void run(int sms) {
  const int nmma = 8192;
  long long* d; int* e; cudaMalloc(&d, sms * 16); cudaMalloc(&e, 4); cudaMemset(e, 0, 4);
  const int smem = 2 * 4096 + 2 * N * 32;
  cudaFuncSetAttribute(k_rate<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  k_rate<N><<<sms, 128, smem>>>(nmma, d, e);
  cudaEvent_t a, b; cudaEventCreate(&a); cudaEventCreate(&b);
  cudaEventRecord(a);
  k_rate<N><<<sms, 128, smem>>>(nmma, d, e);
  cudaEventRecord(b);
  cudaError_t rc = cudaDeviceSynchronize();
  float ms = 0; cudaEventElapsedTime(&ms, a, b);
  long long h[2]; cudaMemcpy(h, d, 16, cudaMemcpyDeviceToHost);
  int he; cudaMemcpy(&he, e, 4, cudaMemcpyDeviceToHost);
  const double flop = 2.0 * 128 * N * 16 * (double)nmma * sms;
  printf("N=%d rc=%d err=%d: %.3f ms, %.1f TFLOP/s; CTA0 issue %lld cyc, total %lld cyc -> %.1f cyc/MMA\n", N, (int)rc, he, ms,
         flop / ms / 1e9, h[0], h[1], (double)h[1] / nmma);
  cudaFree(d); cudaFree(e);
}
int main() {
  int sms = 0; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  run<128>(sms);
  run<256>(sms);
  run<64>(sms);
  return 0;
}
