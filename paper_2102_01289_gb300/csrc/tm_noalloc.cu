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
#include "tm.h"
#include "tm_host.h"
#include "tm_kernels.cuh"

using namespace tmk;

namespace {

constexpr size_t kScratchBytes = (size_t)8 << 20;  // 8 MiB

// Shared by every call on a device: [job descriptor | integral-image scratch].
static __device__ __align__(256) unsigned char g_integral_scratch[kScratchBytes];

size_t round256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

extern "C" tm_status tm_integral_image_noalloc(const int32_t *q, int32_t width, int32_t height,
                                               int64_t *s1, int64_t *s2, void *stream) {
  if (!q || !s1 || !s2 || s1 == s2)
    return fail_noctx(TM_EINVAL, "tm_integral_image_noalloc: null or aliased plane pointer");
  if (width < 1 || height < 1 || (long long)width * height > (1LL << 31) - 1)
    return fail_noctx(TM_EINVAL, "tm_integral_image_noalloc: width and height must be >= 1, below 2^31 pixels");
  const size_t job_bytes = round256(sizeof(Job));
  int nseg = 1, seg_rows = 1;
  integral_layout(width, height, (kScratchBytes - job_bytes) / 8, nseg, seg_rows);
  const size_t need = job_bytes + 8 * integral_scratch_elems(width, height, nseg);
  if (need > kScratchBytes)
    return fail_noctx(TM_EINVAL, "tm_integral_image_noalloc: the image needs more than the 8 MiB static scratch "
                                 "(use tm_integral_image)");
  // In host code the array's name is not a device address: look the address
  // up with the caller's device current. The lookup allocates nothing; doing
  // it on every call keeps it right for whichever device (or context after a
  // device reset) is current.
  void *base = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&base, g_integral_scratch);
  if (e != cudaSuccess || !base) {
    cudaGetLastError();
    return fail_noctx(TM_ECUDA, "tm_integral_image_noalloc: cudaGetSymbolAddress of the static scratch failed");
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Job J{};
  J.in.W = width;
  J.in.H = height;
  J.q = const_cast<int32_t *>(q);
  J.s1 = reinterpret_cast<long long *>(s1);
  J.s2 = reinterpret_cast<long long *>(s2);
  J.nseg = nseg;
  J.seg_rows = seg_rows;
  J.segtot = reinterpret_cast<long long *>(static_cast<char *>(base) + job_bytes);
  // The descriptor travels as a kernel parameter of the copy kernel (nothing
  // is read from host memory after this call returns); the scratch after it is
  // fully rewritten before it is read, so nothing an earlier call left there
  // needs clearing.
  put_jobs(&J, 1, static_cast<Job *>(base), st);
  launch_integral_jobs(static_cast<const Job *>(base), 1, integral_tile_blocks(width, nseg), integral_col_blocks(width),
                       st);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail_noctx(TM_ECUDA, "tm_integral_image_noalloc: kernel launch failed");
  return TM_OK;
}
