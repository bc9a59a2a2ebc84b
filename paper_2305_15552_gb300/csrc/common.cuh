// Shared helpers of the GB300 eigensolver library: status plumbing, error-checked CUDA calls,
// device memory ownership, and small warp-level primitives.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/eig.h"

namespace eig {

// Thread-local message of the last failing CUDA call.
void set_cuda_error(cudaError_t e, const char* what, const char* file, int line);

#define EIG_CUDA_TRY(call)                                                   \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      ::eig::set_cuda_error(e_, #call, __FILE__, __LINE__);                  \
      return e_ == cudaErrorMemoryAllocation ? EIG_ENOMEM : EIG_ECUDA;       \
    }                                                                        \
  } while (0)

// Raises a kernel's dynamic shared-memory limit to at least `bytes` and never lowers it.  The
// attribute is per function and process-wide, so host threads that launch the same kernel
// with different sizes (the instances of a batch) must not undercut each other's launches.
cudaError_t ensure_dyn_smem(const void* kern, size_t bytes);
template <typename K>
inline cudaError_t ensure_dyn_smem(K* kern, size_t bytes) {
  return ensure_dyn_smem(reinterpret_cast<const void*>(kern), bytes);
}

// Count of kernel launches made by this library (every launch site checks through here).
void count_launch();

#define EIG_LAUNCH_CHECK(what)                                               \
  do {                                                                       \
    ::eig::count_launch();                                                   \
    cudaError_t e_ = cudaGetLastError();                                     \
    if (e_ != cudaSuccess) {                                                 \
      ::eig::set_cuda_error(e_, what, __FILE__, __LINE__);                   \
      return EIG_ECUDA;                                                      \
    }                                                                        \
  } while (0)

#define EIG_TRY(call)                                                        \
  do {                                                                       \
    eig_status s_ = (call);                                                  \
    if (s_ != EIG_OK) return s_;                                             \
  } while (0)

__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

inline size_t dtype_size(eig_dtype t) { return t == EIG_F64 ? 8 : (t == EIG_F32 ? 4 : 2); }

// Device buffer owned by the library (cudaMalloc / cudaFree).
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  // Ensures at least `b` bytes; contents are not preserved when it grows.
  eig_status reserve(size_t b) {
    if (b <= bytes && p) return EIG_OK;
    release();
    if (b == 0) return EIG_OK;
    cudaError_t e = cudaMalloc(&p, b);
    if (e != cudaSuccess) {
      set_cuda_error(e, "cudaMalloc", __FILE__, __LINE__);
      p = nullptr;
      return EIG_ENOMEM;
    }
    bytes = b;
    return EIG_OK;
  }
  template <typename T> T* as() const { return reinterpret_cast<T*>(p); }
};

// SM count of the device current at the first call (thread-safe initialisation: concurrent
// solves of a batch call this from several host threads).
inline int num_sms() {
  static const int sms = []() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
  }();
  return sms;
}

// ---------------------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ float bf16_to_f32(uint16_t b) {
  return __uint_as_float(static_cast<uint32_t>(b) << 16);
}

template <typename V> struct ValLoad;
template <> struct ValLoad<float> {
  typedef float storage;
  __device__ __forceinline__ static float get(const float* p, int64_t i) { return __ldg(p + i); }
};
template <> struct ValLoad<double> {
  typedef double storage;
  __device__ __forceinline__ static double get(const double* p, int64_t i) { return __ldg(p + i); }
};
template <> struct ValLoad<uint16_t> {
  typedef uint16_t storage;
  __device__ __forceinline__ static float get(const uint16_t* p, int64_t i) {
    return bf16_to_f32(__ldg(p + i));
  }
};

// Value from a shared-memory (or any generic) pointer, widened to the arithmetic type.
template <typename V> struct ValSmem;
template <> struct ValSmem<float> {
  __device__ __forceinline__ static float get(const float* p, int i) { return p[i]; }
};
template <> struct ValSmem<double> {
  __device__ __forceinline__ static double get(const double* p, int i) { return p[i]; }
};
template <> struct ValSmem<uint16_t> {
  __device__ __forceinline__ static float get(const uint16_t* p, int i) { return bf16_to_f32(p[i]); }
};

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace eig
