// Short per-lane vectors (<= 16 bytes) so that shared/global accesses are 128-bit wide.
#pragma once
#include <cuda_runtime.h>

namespace eig {

template <typename T, int N> struct Vec {
  T v[N];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = T(0);
  }
};

template <typename T, int N> struct VecIO;

template <typename T> struct VecIO<T, 1> {
  __device__ __forceinline__ static Vec<T, 1> ld(const T* p) { Vec<T, 1> r; r.v[0] = *p; return r; }
  __device__ __forceinline__ static void st(T* p, const Vec<T, 1>& a) { *p = a.v[0]; }
};
template <> struct VecIO<float, 2> {
  __device__ __forceinline__ static Vec<float, 2> ld(const float* p) {
    float2 t = *reinterpret_cast<const float2*>(p); Vec<float, 2> r; r.v[0] = t.x; r.v[1] = t.y; return r;
  }
  __device__ __forceinline__ static void st(float* p, const Vec<float, 2>& a) {
    *reinterpret_cast<float2*>(p) = make_float2(a.v[0], a.v[1]);
  }
};
template <> struct VecIO<float, 4> {
  __device__ __forceinline__ static Vec<float, 4> ld(const float* p) {
    float4 t = *reinterpret_cast<const float4*>(p);
    Vec<float, 4> r; r.v[0] = t.x; r.v[1] = t.y; r.v[2] = t.z; r.v[3] = t.w; return r;
  }
  __device__ __forceinline__ static void st(float* p, const Vec<float, 4>& a) {
    *reinterpret_cast<float4*>(p) = make_float4(a.v[0], a.v[1], a.v[2], a.v[3]);
  }
};
template <> struct VecIO<double, 2> {
  __device__ __forceinline__ static Vec<double, 2> ld(const double* p) {
    double2 t = *reinterpret_cast<const double2*>(p); Vec<double, 2> r; r.v[0] = t.x; r.v[1] = t.y; return r;
  }
  __device__ __forceinline__ static void st(double* p, const Vec<double, 2>& a) {
    *reinterpret_cast<double2*>(p) = make_double2(a.v[0], a.v[1]);
  }
};

// Elements per lane so that one lane moves at most 16 bytes of a row of nb elements.
template <typename T, int NB> struct LaneShape {
  static constexpr int EPL = (NB * (int)sizeof(T) >= 16) ? (16 / (int)sizeof(T)) : NB;
  static constexpr int L = NB / EPL;   // lanes per matrix entry (per X row)
  static constexpr int E = 32 / L;     // entries processed per warp step
};

}  // namespace eig
