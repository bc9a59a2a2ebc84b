// Solver handle and per-solve context (internal).
#pragma once
#include <cmath>
#include <functional>
#include <vector>

#include "common.cuh"
#include "spmm.cuh"

namespace eig {

struct PinnedBuf {
  void* p = nullptr;
  size_t bytes = 0;
  ~PinnedBuf() { if (p) cudaFreeHost(p); }
  eig_status reserve(size_t b) {
    if (b <= bytes && p) return EIG_OK;
    if (p) cudaFreeHost(p);
    p = nullptr;
    bytes = 0;
    cudaError_t e = cudaMallocHost(&p, b);
    if (e != cudaSuccess) { set_cuda_error(e, "cudaMallocHost", __FILE__, __LINE__); p = nullptr; return EIG_ENOMEM; }
    bytes = b;
    return EIG_OK;
  }
  template <typename T> T* as() const { return reinterpret_cast<T*>(p); }
};

struct Handle {
  SpmmPlan plan;
  int64_t n = 0;
  int n_ev = 0, nb = 0;
  bool have = false;
  std::vector<double> theta, relres;
  DevBuf Xres;                 // FP64 n x n_ev (row-major)
  // workspaces kept across solves
  DevBuf blk[8];               // n x nb blocks (front methods)
  DevBuf big;                  // histories / Krylov bases
  DevBuf small;                // projected problems, partials
  DevBuf tmp64a, tmp64b;       // n x nb FP64 temporaries
  PinnedBuf host;
  // learned preconditioner: (|H| 1)_i (computed on first use) and sample workspaces
  DevBuf lp_rowabs;
  bool lp_rowabs_ok = false;
  DevBuf lp_buf[3], lp_small;
};

struct ProductBatcher;

// Per-solve context
struct Ctx {
  Handle* h;
  cudaStream_t st;
  eig_opts o;
  eig_stats* s;
  // lock-step batches: every product goes through the batcher, which launches the products of
  // all running instances together (batch.cu); req_ev orders this stream's work before it
  ProductBatcher* batch = nullptr;
  cudaEvent_t req_ev = nullptr;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> spmm_ev;
  std::vector<int> spmm_shape;   // product shape of each timed call (index of eig_stats' by-shape arrays)
  void count_spmm(int nb, eig_dtype vt, int64_t spmv_cols);
  eig_status spmm(const void* X, void* Y, int nb, eig_dtype vt, int64_t spmv_cols);
  // one SpMV: column col of a block with row stride ld (decoupled RMM-DIIS, Sec. 4.3)
  eig_status spmv_col(const void* X, void* Y, int ld, int col, eig_dtype vt);
  // H r for the RMM-DIIS block: one SpMM, or (decoupled, once opts.rmm_decouple wanted vectors
  // have converged) one SpMV per active column
  eig_status rmm_product(const void* X, void* Y, int mp, eig_dtype vt, const std::vector<int>& act, int nev);
  // spmm with a fused Chebyshev step (spmm_run_cheb); EIG_EUNSUPPORTED leaves Y untouched
  eig_status spmm_cheb(const void* X, void* Y, int nb, eig_dtype vt, int64_t spmv_cols, const void* Qp,
                       const int* active, double alpha, double cshift, int first);
  // one convergence-history row (opts.trace), count <= n_ev values of theta and relres
  void trace(int phase, int it, const double* th, const double* rel, int count) {
    if (!o.trace || s->trace_rows >= o.trace_cap) return;
    const int ne = h->n_ev;
    double* row = o.trace + (size_t)s->trace_rows * (2 + 2 * ne);
    row[0] = phase;
    row[1] = it;
    for (int j = 0; j < ne; ++j) {
      row[2 + j] = j < count ? th[j] : NAN;
      row[2 + ne + j] = j < count ? rel[j] : NAN;
    }
    s->trace_rows++;
  }
  eig_status sync() {
    EIG_CUDA_TRY(cudaStreamSynchronize(st));
    return EIG_OK;
  }
  ~Ctx();
};

// The batcher's side of a product (batch.cu): posts job, waits for the round's launch, and
// orders c.st after it.  EIG_EUNSUPPORTED for a Chebyshev step the plan cannot fuse (nothing
// posted).
eig_status batch_product(ProductBatcher* b, Ctx& c, const SpmmJob& job, int nb, eig_dtype vt, bool cheb);
// Solve with an optional batcher (eig_solve: none).
eig_status solve_handle(void* handle, eig_method method, const eig_opts* opts, eig_stats* stats,
                        ProductBatcher* batch);

// Stop rule of a front method: called after every iteration with the ascending Ritz values and
// relative residuals of the leading `count` (>= n_ev) pairs; returns a switch reason (> 0) to stop.
typedef std::function<int(int it, const double* theta, const double* relres, int count)> StopFn;

eig_status run_lobpcg(Ctx& c, const double* X0, int x0_cols, int maxiter, const StopFn& stop, int* iters,
                      int* reason, bool* converged, double* X64_out, std::vector<double>* theta_out);
eig_status run_rmmdiis(Ctx& c, const double* X0, int maxiter, int* iters, bool* converged,
                       std::vector<double>* theta_out);
eig_status run_lanczos(Ctx& c, const double* X0, int x0_cols, int* iters, bool* converged,
                       std::vector<double>* theta_out);
eig_status run_block_lanczos(Ctx& c, const double* X0, int x0_cols, int maxiter, const StopFn& stop, int* iters,
                             int* reason, bool* converged, std::vector<double>* theta_out);
eig_status run_chebfsi(Ctx& c, const double* X0, int x0_cols, int* iters, bool* converged,
                       std::vector<double>* theta_out);

// helpers shared by the drivers (solver.cu)
eig_status fill_random(double* X, int64_t count, uint64_t seed, cudaStream_t st);
eig_status pad_columns(const double* src, int ks, double* dst, int kd, int64_t n, cudaStream_t st);
// dst (n x kd) columns j < min(ks, kd) <- src (n x ks); other columns untouched
eig_status overlay_columns(const double* src, int ks, double* dst, int kd, int64_t n, cudaStream_t st);
eig_status find_duplicates(Ctx& c, const double* X, int m, int ld, const std::vector<double>& theta,
                           bool* duplicate);
eig_status certify(Ctx& c, const double* X, const std::vector<double>& theta, std::vector<double>* relres,
                   bool* duplicate);
// (|H| 1)_i of the handle's matrix into h->lp_rowabs (once per handle).
eig_status lp_ensure_rowabs(Handle* h, cudaStream_t st);
inline int next_pow2(int v) { int p = 1; while (p < v) p <<= 1; return p; }

}  // namespace eig
