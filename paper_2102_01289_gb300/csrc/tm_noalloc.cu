// tm_noalloc.cu -- integral images without any allocation.
//
// tm_integral_image needs scratch device memory (one job descriptor and the
// tile sums of the integral images) and obtains it with cudaMallocAsync. Some
// callers cannot allocate at all: code running under a real-time or frame-
// deadline contract that forbids allocator calls after start-up, code that
// runs inside another framework's memory-pool or allocation callbacks (where
// re-entering the CUDA allocator is not allowed), and processes that have
// reserved all device memory up front. tm_integral_image_noalloc serves them
// with a file-scope static device array instead; every GPU that loads this
// library holds the array until the process exits.
#include <cstring>
#include <mutex>

#include "tm.h"
#include "tm_kernels.cuh"

using namespace tmk;

namespace {

constexpr size_t kScratchBytes = (size_t)8 << 20;  // 8 MiB

// Shared by every call on a device: [job descriptor | integral-image scratch].
static __device__ __align__(256) unsigned char g_integral_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void *g_scratch_addr[kMaxDevices];  // device address of the array, per device

size_t round256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

extern "C" tm_status tm_integral_image_noalloc(const int32_t *q, int32_t width, int32_t height,
                                               int64_t *s1, int64_t *s2, void *stream) {
  if (!q || !s1 || !s2 || s1 == s2) return TM_EINVAL;
  if (width < 1 || height < 1 || (long long)width * height > (1LL << 31) - 1) return TM_EINVAL;
  const size_t job_bytes = round256(sizeof(Job));
  int nseg = 1, seg_rows = 1;
  integral_layout(width, height, (kScratchBytes - job_bytes) / 8, nseg, seg_rows);
  const size_t need = job_bytes + 8 * integral_scratch_elems(width, height, nseg);
  if (need > kScratchBytes) return TM_EINVAL;  // larger than the static scratch
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return TM_ECUDA;
  }
  void *base = nullptr;
  {
    // First call on this device (with it current): the host cannot use the
    // array's name as a device address, so look the address up once.
    std::lock_guard<std::mutex> g(g_setup_mu);
    if (!g_scratch_addr[dev]) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_integral_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return TM_ECUDA;
      }
      g_scratch_addr[dev] = p;
    }
    base = g_scratch_addr[dev];
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Job J;
  memset(&J, 0, sizeof J);
  J.in.W = width;
  J.in.H = height;
  J.q = const_cast<int32_t *>(q);
  J.s1 = reinterpret_cast<long long *>(s1);
  J.s2 = reinterpret_cast<long long *>(s2);
  J.nseg = nseg;
  J.seg_rows = seg_rows;
  J.segtot = reinterpret_cast<long long *>(static_cast<char *>(base) + job_bytes);
  // The scratch is fully rewritten before it is read, so nothing
  // left in the array by an earlier call needs clearing. The descriptor comes
  // from pageable memory: the copy has consumed it when this call returns.
  if (cudaMemcpyAsync(base, &J, sizeof(Job), cudaMemcpyHostToDevice, st) != cudaSuccess) {
    cudaGetLastError();
    return TM_ECUDA;
  }
  launch_integral_jobs(static_cast<const Job *>(base), 1, integral_tile_blocks(width, nseg), integral_col_blocks(width),
                       st);
  if (cudaGetLastError() != cudaSuccess) return TM_ECUDA;
  return TM_OK;
}
