// sp2_truncate_noalloc: the truncation selection of sp2_truncate for callers
// that cannot allocate device memory themselves -- code running inside a CUDA
// graph that is being captured, inside another library's allocation-free
// callback, or under an allocator that forbids cudaMalloc after start-up.
// Its scratch (tile norms and the radix-select work area) is one file-scope
// device array of fixed size; no call here allocates or frees memory.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "sp2_internal.h"

namespace sp2 {
namespace {

constexpr int64_t NOALLOC_MAX_TILES = 1 << 18;     // 262,144 tiles (2 GiB of FP64 tile values)
constexpr int64_t NOALLOC_MAX_SEGMENTS = 1024;      // Frob-Inf: at most 32 x 32 super-blocks
constexpr size_t NOALLOC_SCRATCH_BYTES = 8u << 20;  // 8 MiB, checked against the need below

// Every GPU that loads this library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void* g_scratch_ptr[MAX_DEVICES] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the host-side name of the array is not a device address).  The
// address stays valid for the life of the device's primary context; a
// cudaDeviceReset of that device invalidates it (see include/sp2.h).
int scratch_for_current_device(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
    cudaGetLastError();
    return SP2_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return SP2_ERR_CUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return SP2_OK;
}

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace
}  // namespace sp2

using namespace sp2;

extern "C" int sp2_truncate_noalloc(const int32_t* brow, const int32_t* bcol, const double* val, int64_t n,
                                    int64_t nnzb, double tau, int32_t mode, int64_t frobinf_part, int32_t* keep,
                                    void* cuda_stream) {
  if (n <= 0 || nnzb < 0 || !(tau >= 0.0) || !std::isfinite(tau)) return SP2_ERR_INVALID_ARG;
  if (nnzb > 0 && (!brow || !bcol || !val || !keep)) return SP2_ERR_INVALID_ARG;
  if (mode != SP2_TRUNC_FROBENIUS && mode != SP2_TRUNC_FROBINF) return SP2_ERR_INVALID_ARG;
  if (mode == SP2_TRUNC_FROBINF && (frobinf_part < TB || frobinf_part % TB)) return SP2_ERR_INVALID_ARG;
  const int64_t nb64 = (n + TB - 1) / TB;
  if (nb64 > 65535) return SP2_ERR_INVALID_ARG;
  // Frobenius mode is one segment (the super-block size only matters for Frob-Inf)
  const int64_t part_tiles = mode == SP2_TRUNC_FROBINF ? frobinf_part / TB : std::max<int64_t>(nb64, 1);
  const int64_t nsb = (nb64 + part_tiles - 1) / part_tiles;
  const int64_t nseg = mode == SP2_TRUNC_FROBINF ? nsb * nsb : 1;
  if (nnzb > NOALLOC_MAX_TILES || nseg > NOALLOC_MAX_SEGMENTS) return SP2_ERR_TOO_LARGE;
  if (nnzb == 0) return SP2_OK;
  // scratch layout: tile norms, then the radix-select work area, sized by the
  // same function that sizes it for sp2_truncate
  const size_t n2_bytes = align256((size_t)nnzb * 8);
  const size_t need = n2_bytes + trunc_work_bytes(nnzb, (int)nb64, part_tiles);
  if (need > NOALLOC_SCRATCH_BYTES) return SP2_ERR_TOO_LARGE;
  void* base = nullptr;
  const int rc = scratch_for_current_device(&base);
  if (rc != SP2_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  double* n2 = static_cast<double*>(base);
  void* work = static_cast<unsigned char*>(base) + n2_bytes;
  TileSet ts;
  ts.nnzb = nnzb;
  ts.brow = const_cast<int32_t*>(brow);
  ts.bcol = const_cast<int32_t*>(bcol);
  ts.slot = nullptr;
  if (launch_tile_norms(val, nnzb, n2, st) != cudaSuccess ||
      launch_truncate(ts, n2, (int)nb64, tau, mode, part_tiles, work, keep, st) != cudaSuccess) {
    cudaGetLastError();
    return SP2_ERR_CUDA;
  }
  return SP2_OK;
}
