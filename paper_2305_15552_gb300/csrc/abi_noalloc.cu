// C ABI: a Gram product that allocates no device memory.
//
// eig_gram takes its per-CTA partial sums from a stream-ordered allocation.  Some callers cannot
// allocate while they run: a framework that has reserved the whole device memory for its own
// pool (so cudaMalloc/cudaMallocAsync would fail or fight its allocator), or code on a
// latency-critical path that must not enter the driver's allocator at all.  For them
// eig_gram_noalloc computes the same product with its scratch in a file-scope __device__ array
// of fixed size that every device loading this library holds until the process exits.
#include <mutex>

#include "common.cuh"
#include "dense.cuh"

namespace eig {
namespace {

// 4 MiB of partials: up to 512 CTA partials of a 32 x 32 Gram.
constexpr int kNoAllocParts = 512;
constexpr int kNoAllocMaxBlock = 32;
constexpr size_t kNoAllocScratchDoubles = (size_t)kNoAllocParts * kNoAllocMaxBlock * kNoAllocMaxBlock;
__device__ __align__(256) double g_gram_scratch[kNoAllocScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array for the current device (looked up once per device).
eig_status scratch_address(void** out) {
  int dev = 0;
  EIG_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return EIG_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    EIG_CUDA_TRY(cudaGetSymbolAddress(&p, g_gram_scratch));
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return EIG_OK;
}

}  // namespace
}  // namespace eig

using namespace eig;

extern "C" {

eig_status eig_gram_noalloc_parts(const void* A, const void* B, int64_t n, int nb, eig_dtype vec_type, double* G,
                                  int max_parts, void* stream) {
  static_assert((size_t)kNoAllocParts * kNoAllocMaxBlock * kNoAllocMaxBlock <= kNoAllocScratchDoubles,
                "the scratch array holds every partial of the largest block");
  if (!A || !B || !G || n < 1 || nb < 1 || nb > kNoAllocMaxBlock) return EIG_EINVAL;
  if (vec_type != EIG_F32 && vec_type != EIG_F64) return EIG_EINVAL;
  if (max_parts < 1 || max_parts > kNoAllocParts) return EIG_EINVAL;
  void* scratch = nullptr;
  EIG_TRY(scratch_address(&scratch));
  BlockList bl;
  bl.n = 2;
  bl.p[0] = A;
  bl.p[1] = B;
  const int pa = 0, pb = 1;
  // every CTA overwrites all of its partials, so the array needs no clearing between calls
  return gram_multi(bl, &pa, &pb, 1, nb, n, vec_type, G, scratch, as_stream(stream), max_parts);
}

eig_status eig_gram_noalloc(const void* A, const void* B, int64_t n, int nb, eig_dtype vec_type, double* G,
                            void* stream) {
  return eig_gram_noalloc_parts(A, B, n, nb, vec_type, G, kNoAllocParts, stream);
}

}  // extern "C"
