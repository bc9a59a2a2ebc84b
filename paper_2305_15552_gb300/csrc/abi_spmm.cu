// C ABI: library-level calls and the SpMM plan entry points.
#include "common.cuh"
#include "spmm.cuh"

#include <atomic>
#include <mutex>
#include <unordered_map>

namespace eig {
cudaError_t ensure_dyn_smem(const void* kern, size_t bytes) {
  static std::mutex mu;
  static std::unordered_map<const void*, size_t> limit;
  std::lock_guard<std::mutex> lock(mu);
  size_t& cur = limit[kern];
  if (bytes <= cur) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}
static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
static thread_local char g_cuda_msg[512] = {0};
void set_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  snprintf(g_cuda_msg, sizeof(g_cuda_msg), "%s: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
}
}  // namespace eig

extern "C" {

const char* eig_strerror(eig_status s) {
  switch (s) {
    case EIG_OK: return "EIG_OK";
    case EIG_EINVAL: return "EIG_EINVAL: invalid argument";
    case EIG_ENOMEM: return "EIG_ENOMEM: device allocation failed";
    case EIG_ECUDA: return "EIG_ECUDA: CUDA error";
    case EIG_ENOT_CONVERGED: return "EIG_ENOT_CONVERGED: maxiter reached";
    case EIG_EBREAKDOWN: return "EIG_EBREAKDOWN: numerically rank-deficient basis";
    case EIG_ETIMEOUT: return "EIG_ETIMEOUT: bounded device wait gave up";
    case EIG_EDUPLICATE: return "EIG_EDUPLICATE: duplicate eigenpairs";
    case EIG_EUNSUPPORTED: return "EIG_EUNSUPPORTED: not supported by this build";
  }
  return "unknown eig_status";
}

const char* eig_last_cuda_error(void) { return eig::g_cuda_msg; }

const char* eig_version(void) { return "0.1.0 sm_103a"; }

int64_t eig_launch_count(void) { return eig::g_launches.load(std::memory_order_relaxed); }

eig_status eig_spmm_plan_create(const eig_csr_upper* H, int row_block, int col_block, int copy, void* stream,
                                void** plan) {
  return eig_spmm_plan_create_ex(H, row_block, col_block, EIG_LAYOUT_AUTO, copy, stream, plan);
}

eig_status eig_spmm_plan_create_ex(const eig_csr_upper* H, int row_block, int col_block, int layout, int copy,
                                   void* stream, void** plan) {
  if (!plan) return EIG_EINVAL;
  *plan = nullptr;
  if (layout < EIG_LAYOUT_AUTO || layout > EIG_LAYOUT_CSR) return EIG_EINVAL;
  eig::SpmmPlan* P = new (std::nothrow) eig::SpmmPlan();
  if (!P) return EIG_ENOMEM;
  eig_status s = eig::spmm_plan_build(P, H, row_block, col_block, layout, copy, eig::as_stream(stream));
  if (s != EIG_OK) {
    cudaStreamSynchronize(eig::as_stream(stream));
    delete P;
    return s;
  }
  *plan = P;
  return EIG_OK;
}

void eig_spmm_plan_destroy(void* plan) {
  if (!plan) return;
  cudaDeviceSynchronize();
  delete static_cast<eig::SpmmPlan*>(plan);
}

eig_status eig_spmm_plan_info(const void* plan, eig_spmm_info* info) {
  if (!plan || !info) return EIG_EINVAL;
  const eig::SpmmPlan* P = static_cast<const eig::SpmmPlan*>(plan);
  info->n = P->n;
  info->nnz = P->nnz;
  info->row_block = P->R;
  info->col_block = P->C;
  info->n_row_blocks = P->nRB;
  info->n_col_blocks = P->nCB;
  info->n_tiles = P->n_tiles;
  info->n_slots = P->n_slots;
  info->scratch_bytes_per_col = P->n_slots * (int64_t)P->C;
  info->val_type = P->val_type;
  info->layout = P->layout;
  const int64_t vb = (int64_t)eig::dtype_size(P->val_type);
  if (P->layout == EIG_LAYOUT_MIRRORED) {
    info->layout_entries = P->m_nblk * 256;
    info->device_bytes = P->m_nblk * 256 * (2 + vb) + P->m_npan * 256;
  } else if (P->layout == EIG_LAYOUT_HALF) {
    info->layout_entries = P->tiled_entries;
    info->device_bytes = P->tiled_entries * (1 + vb) + P->tiled_rp * 2;
  } else {
    info->layout_entries = P->nnz;
    info->device_bytes = P->nnz * (4 + vb) + (P->n + 1) * 8;
  }
  return EIG_OK;
}

eig_status eig_spmm(void* plan, const void* X, void* Y, int nb, eig_dtype vec_type, void* stream) {
  if (!plan || !X || !Y) return EIG_EINVAL;
  return eig::spmm_run(static_cast<eig::SpmmPlan*>(plan), X, Y, nb, vec_type, eig::as_stream(stream));
}

eig_status eig_spmm_cheb(void* plan, const void* X, void* Y, int nb, eig_dtype vec_type, const void* Qp,
                         const int* active, double alpha, double c, int first, void* stream) {
  if (!plan || !X || !Y || !active) return EIG_EINVAL;
  return eig::spmm_run_cheb(static_cast<eig::SpmmPlan*>(plan), X, Y, nb, vec_type, Qp, active, alpha, c, first,
                            eig::as_stream(stream));
}

}  // extern "C"
