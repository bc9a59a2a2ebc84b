// Symmetric half-stored SpMM plan (internal interface shared by the C ABI and the solvers).
#pragma once
#include "common.cuh"

namespace eig {

struct SpmmPlan {
  int64_t n = 0, nnz = 0;
  int R = 256, C = 128;                 // row block / column block sizes
  int64_t nRB = 0, nCB = 0;
  eig_dtype val_type = EIG_F32;
  // matrix (owned when copied)
  const int64_t* rowptr = nullptr;
  const int32_t* col = nullptr;
  const void* val = nullptr;
  DevBuf own_rowptr, own_col, own_val;
  // tile lists: tiles of row block I are tile_col[tile_ptr[I] .. tile_ptr[I+1]), ascending J
  int64_t n_tiles = 0, n_slots = 0;
  DevBuf tile_ptr;     // int64[nRB+1]
  DevBuf tile_col;     // int32[n_tiles]
  DevBuf tile_slot;    // int32[n_tiles]: scratch slot of a non-local tile, -1 for local
  // transpose schedule: slots landing in column block J, ascending source row block
  DevBuf sched_ptr;    // int64[n_sched+1]
  DevBuf sched_cb;     // int32[n_sched]: column blocks that receive at least one slot
  DevBuf sched_slot;   // int32[n_slots]
  int64_t n_sched = 0;
  DevBuf diag;         // float64[n]: H_ii (used by the Jacobi preconditioner)
  DevBuf scratch;      // transposed partial products, n_slots * C * nb * sizeof(T)
  double algorithmic_bytes(int nb, size_t vec_bytes) const;
};

eig_status spmm_plan_build(SpmmPlan* P, const eig_csr_upper* H, int R, int C, int copy, cudaStream_t st);
eig_status spmm_run(SpmmPlan* P, const void* X, void* Y, int nb, eig_dtype vt, cudaStream_t st);
// Scratch bytes spmm_run needs for (nb, vec type); caller-provided scratch variant below.
size_t spmm_scratch_bytes(const SpmmPlan* P, int nb, eig_dtype vt);
eig_status spmm_run_with_scratch(SpmmPlan* P, const void* X, void* Y, int nb, eig_dtype vt, void* scratch,
                                 cudaStream_t st);

}  // namespace eig
