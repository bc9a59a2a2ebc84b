// C ABI: step-level entry points (Gram, CholQR2, projected eigenproblems, RMM-DIIS small solves).
#include <vector>

#include "common.cuh"
#include "dense.cuh"
#include "rmm.cuh"
#include "small.cuh"

namespace eig {

// Stream-ordered scratch for one ABI call.
struct AsyncScratch {
  void* p = nullptr;
  cudaStream_t st;
  explicit AsyncScratch(cudaStream_t s) : st(s) {}
  eig_status get(size_t bytes) {
    cudaError_t e = cudaMallocAsync(&p, bytes, st);
    if (e != cudaSuccess) { set_cuda_error(e, "cudaMallocAsync", __FILE__, __LINE__); p = nullptr; return EIG_ENOMEM; }
    return EIG_OK;
  }
  ~AsyncScratch() { if (p) cudaFreeAsync(p, st); }
};

__global__ void k_small_matmul(const double* __restrict__ A, const double* __restrict__ B, int k,
                               double* __restrict__ C) {
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int i = e / k, j = e % k;
    double s = 0.0;
    for (int l = 0; l < k; ++l) s += A[i * k + l] * B[l * k + j];
    C[e] = s;
  }
}

// CholQR2 of X (in place); X2 (optional, same shape) receives the same right factors, so that
// X2 <- X2 R^{-1} (used for H Q = (H Y) R^{-1}).
eig_status cholqr2_impl2(void* X, void* X2, int64_t n, int k, eig_dtype vt, double* R, cudaStream_t st) {
  AsyncScratch sc(st);
  const size_t gb = gram_scratch_bytes(1, k);
  EIG_TRY(sc.get(gb + 4 * (size_t)k * k * 8 + small_chol_inv_work_bytes(k) + 256 * 4));
  unsigned char* base = (unsigned char*)sc.p;
  double* part = (double*)base;
  double* G = (double*)(base + gb);
  double* R1 = G + k * k;
  double* Ri = R1 + k * k;
  double* R2 = Ri + k * k;
  double* work = R2 + k * k;
  int* info = (int*)((unsigned char*)work + small_chol_inv_work_bytes(k));
  int hinfo = 0;
  for (int pass = 0; pass < 2; ++pass) {
    BlockList bl;
    bl.n = 1;
    bl.p[0] = X;
    const int pa = 0, pb = 0;
    EIG_TRY(gram_multi(bl, &pa, &pb, 1, k, n, vt, G, part, st));
    EIG_TRY(small_chol_inv(G, k, 1e-14, pass == 0 ? R1 : R2, Ri, nullptr, work, info, st));
    EIG_CUDA_TRY(cudaMemcpyAsync(&hinfo, info, 4, cudaMemcpyDeviceToHost, st));
    EIG_CUDA_TRY(cudaStreamSynchronize(st));
    if (hinfo != SMALL_OK) return EIG_EBREAKDOWN;
    // X <- X R^{-1}: block_apply cannot work in place; stage through a copy
    void* tmp = nullptr;
    EIG_CUDA_TRY(cudaMallocAsync(&tmp, (size_t)n * k * dtype_size(vt), st));
    for (int which = 0; which < (X2 ? 2 : 1); ++which) {
      void* Xw = which ? X2 : X;
      EIG_CUDA_TRY(cudaMemcpyAsync(tmp, Xw, (size_t)n * k * dtype_size(vt), cudaMemcpyDeviceToDevice, st));
      BlockList in;
      in.n = 1;
      in.p[0] = tmp;
      eig_status s = block_apply(in, k, Ri, k, Xw, 0.0, n, vt, st);
      if (s != EIG_OK) { cudaFreeAsync(tmp, st); return s; }
    }
    cudaFreeAsync(tmp, st);
  }
  k_small_matmul<<<1, 256, 0, st>>>(R2, R1, k, R);
  EIG_LAUNCH_CHECK("k_small_matmul");
  EIG_CUDA_TRY(cudaStreamSynchronize(st));
  return EIG_OK;
}

}  // namespace eig

using namespace eig;

extern "C" {

eig_status eig_gram(const void* A, const void* B, int64_t n, int nb, eig_dtype vec_type, double* G, void* stream) {
  if (!A || !B || !G || n < 1 || nb < 1 || nb > 64) return EIG_EINVAL;
  if (vec_type != EIG_F32 && vec_type != EIG_F64) return EIG_EINVAL;
  cudaStream_t st = as_stream(stream);
  AsyncScratch sc(st);
  EIG_TRY(sc.get(gram_scratch_bytes(1, nb)));
  BlockList bl;
  bl.n = 2;
  bl.p[0] = A;
  bl.p[1] = B;
  const int pa = 0, pb = 1;
  return gram_multi(bl, &pa, &pb, 1, nb, n, vec_type, G, sc.p, st);
}

eig_status eig_cholqr2(void* X, int64_t n, int k, eig_dtype vec_type, double* R, void* stream) {
  if (!X || !R || n < 1 || k < 1 || k > 64 || n < k) return EIG_EINVAL;
  if (vec_type != EIG_F32 && vec_type != EIG_F64) return EIG_EINVAL;
  return cholqr2_impl2(X, nullptr, n, k, vec_type, R, as_stream(stream));
}

eig_status eig_small_syev(const double* A, int k, int m, double* w, double* Z, void* stream) {
  if (!A || !w || !Z || k < 1 || m < 1 || m > k || k > kSmallMax || m > 256) return EIG_EINVAL;
  cudaStream_t st = as_stream(stream);
  AsyncScratch sc(st);
  EIG_TRY(sc.get(small_syev_work_bytes(k, m) + 256));
  return small_syev(A, k, m, w, Z, sc.p, nullptr, st);
}

eig_status eig_small_rr(const double* A, const double* G, int k, int nb, double piv_tol, double* theta, double* C,
                        int* info_host, void* stream) {
  if (!A || !G || !theta || !C || k < 1 || nb < 1 || nb > k || k > 4 * kSmallMax) return EIG_EINVAL;
  cudaStream_t st = as_stream(stream);
  AsyncScratch sc(st);
  EIG_TRY(sc.get(small_rr_work_bytes(k, nb) + 256));
  int* dinfo = (int*)((unsigned char*)sc.p + small_rr_work_bytes(k, nb));
  EIG_TRY(small_rr(A, G, k, nb, piv_tol, theta, C, nullptr, sc.p, dinfo, st));
  int hinfo = 0;
  EIG_CUDA_TRY(cudaMemcpyAsync(&hinfo, dinfo, 4, cudaMemcpyDeviceToHost, st));
  EIG_CUDA_TRY(cudaStreamSynchronize(st));
  if (info_host) *info_host = hinfo;
  return EIG_OK;
}

eig_status eig_rmm_rr2(const double* dots, const int* active, int m, double* theta, double* g, void* stream) {
  if (!dots || !active || !theta || !g || m < 1 || m > 32) return EIG_EINVAL;
  return rmm_rr2(dots, active, m, theta, g, as_stream(stream));
}

eig_status eig_rmm_diis(const double* B, const int* slots, int s, const int* active, int m, double* alpha,
                        void* stream) {
  if (!B || !slots || !active || !alpha || m < 1 || m > 32 || s < 1 || s > kRmmSMax) return EIG_EINVAL;
  Window w;
  w.s = s;
  for (int i = 0; i < s; ++i) {
    if (slots[i] < 0 || slots[i] >= kRmmSMax) return EIG_EINVAL;
    w.slot[i] = slots[i];
  }
  return rmm_diis(B, w, active, m, alpha, as_stream(stream));
}

}  // extern "C"
