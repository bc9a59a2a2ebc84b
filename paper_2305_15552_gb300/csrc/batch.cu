// Many independent instances: concurrent solves of a batch of handles, and an autotuner of the
// SpMM plan shape.
//
// The paper's point about eigenpair-level concurrency (Secs. 1, 4.3) is that small independent
// pieces of work only fill a wide machine when they run side by side.  A batch of uneven
// matrices is the extreme case: one instance of 2e4 rows leaves most of the 152 SMs idle, and a
// solve synchronises with the host once per iteration.  eig_solve_batch therefore runs the
// instances from a pool of host threads, each with its own non-blocking stream, so that the
// kernels and host round trips of different instances overlap.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "solver.cuh"
#include "spmm.cuh"

namespace eig {
namespace {

template <typename T>
__global__ void k_tune_fill(T* X, int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    // deterministic values in [-1, 1)
    uint32_t h = (uint32_t)(i * 2654435761u) ^ 0x9E3779B9u;
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    X[i] = (T)((double)(h & 0xFFFFFF) / 8388608.0 - 1.0);
  }
}

bool is_hard_error(eig_status s) {
  return s != EIG_OK && s != EIG_ENOT_CONVERGED && s != EIG_EDUPLICATE;
}

}  // namespace

// Lock-step products of a batch: every running instance's next SpMM (or fused Chebyshev step)
// is posted here, and once all running instances have posted, the last poster launches the
// round -- one launch per shape over the posted products' concatenated row blocks (the
// (instance, row block) work list) on the batcher's stream, after every poster's stream has
// reached its post (events), with every poster's stream ordered after the launch.  An
// instance that finished (converged or stopped) no longer counts, so the work list of each
// round holds exactly the running instances: the per-instance convergence mask.
struct ProductBatcher {
  struct Req {
    SpmmJob job;
    int nb;
    eig_dtype vt;
    bool cheb;
    cudaEvent_t ready;
    eig_status rc;
  };
  std::mutex mu;
  std::condition_variable cv;
  int running = 0;
  uint64_t round = 0;
  std::vector<Req> reqs;
  std::vector<eig_status> results;    // of the last launched round, by post order
  cudaStream_t ls = nullptr;
  cudaEvent_t done = nullptr;
  int64_t launches = 0, products = 0; // batched launches issued, products they carried

  // all posted; called with mu held
  void launch_round() {
    results.assign(reqs.size(), EIG_OK);
    for (auto& r : reqs) cudaStreamWaitEvent(ls, r.ready, 0);
    std::map<std::tuple<int, int, int>, std::vector<int>> groups;
    for (int i = 0; i < (int)reqs.size(); ++i)
      groups[std::make_tuple(reqs[i].nb, (int)reqs[i].vt, reqs[i].cheb ? 1 : 0)].push_back(i);
    for (auto& g : groups) {
      const int nb = std::get<0>(g.first);
      const eig_dtype vt = (eig_dtype)std::get<1>(g.first);
      const bool cheb = std::get<2>(g.first) != 0;
      std::vector<SpmmJob> jobs;
      for (int i : g.second) jobs.push_back(reqs[i].job);
      eig_status s = spmm_run_batch(jobs.data(), (int)jobs.size(), nb, vt, cheb, ls);
      if (s == EIG_OK) {
        ++launches;
        products += (int64_t)jobs.size();
      } else if (s == EIG_EUNSUPPORTED) {
        // shapes without a batched kernel: the products one by one, same stream, same order
        s = EIG_OK;
        for (int i : g.second) {
          const SpmmJob& j = reqs[i].job;
          eig_status t = cheb ? spmm_run_cheb(j.P, j.X, j.Y, nb, vt, j.Qp, j.active, j.alpha, j.c, j.first, ls)
                              : spmm_run(j.P, j.X, j.Y, nb, vt, ls);
          results[i] = t;
        }
      }
      if (s != EIG_OK)
        for (int i : g.second) results[i] = s;
    }
    cudaEventRecord(done, ls);
    reqs.clear();
    ++round;
    cv.notify_all();
  }
};

eig_status batch_product(ProductBatcher* b, Ctx& c, const SpmmJob& job, int nb, eig_dtype vt, bool cheb) {
  if (!c.req_ev) EIG_CUDA_TRY(cudaEventCreateWithFlags(&c.req_ev, cudaEventDisableTiming));
  EIG_CUDA_TRY(cudaEventRecord(c.req_ev, c.st));
  std::unique_lock<std::mutex> lock(b->mu);
  const size_t mine = b->reqs.size();
  b->reqs.push_back({job, nb, vt, cheb, c.req_ev, EIG_OK});
  const uint64_t r = b->round;
  if ((int)b->reqs.size() >= b->running) {
    b->launch_round();
  } else if (!b->cv.wait_for(lock, std::chrono::seconds(120), [&] { return b->round != r; })) {
    // an instance that neither posts nor leaves for two minutes (host work of that length)
    // does not hold the others: the round goes out with the products posted so far
    if (b->round == r) b->launch_round();
  }
  const eig_status rc = b->results[mine];
  // ordered on this stream before any later round records `done` again: that round needs this
  // instance's next post, which comes after this wait
  cudaStreamWaitEvent(c.st, b->done, 0);
  return rc;
}
}  // namespace eig

using namespace eig;

extern "C" {

eig_status eig_create_batch(const eig_csr_upper* Hs, int count, int n_ev, int block, int layout, void** handles) {
  if (count < 0 || (count > 0 && (!Hs || !handles))) return EIG_EINVAL;
  for (int i = 0; i < count; ++i) handles[i] = nullptr;
  for (int i = 0; i < count; ++i) {
    const eig_status s = eig_create_ex(&Hs[i], n_ev, block, layout, &handles[i]);
    if (s != EIG_OK) {
      for (int j = 0; j < i; ++j) {
        eig_destroy(handles[j]);
        handles[j] = nullptr;
      }
      return s;
    }
  }
  return EIG_OK;
}

eig_status eig_solve_batch_ex(void* const* handles, int count, eig_method method, const eig_opts* opts,
                              int per_instance_opts, int threads, int flags, eig_status* status, eig_stats* stats) {
  if (count < 0 || (count > 0 && !handles)) return EIG_EINVAL;
  if (per_instance_opts && !opts) return EIG_EINVAL;
  if (flags & ~EIG_BATCH_LOCKSTEP) return EIG_EINVAL;
  for (int i = 0; i < count; ++i)
    if (!handles[i]) return EIG_EINVAL;
  if (count == 0) return EIG_OK;
  int dev = 0;
  EIG_CUDA_TRY(cudaGetDevice(&dev));
  const int nt = std::max(1, std::min(count, threads > 0 ? threads : 16));
  const bool lockstep = (flags & EIG_BATCH_LOCKSTEP) != 0;
  ProductBatcher pb;
  if (lockstep) {
    EIG_CUDA_TRY(cudaStreamCreateWithFlags(&pb.ls, cudaStreamNonBlocking));
    EIG_CUDA_TRY(cudaEventCreateWithFlags(&pb.done, cudaEventDisableTiming));
    pb.running = nt;   // every worker's first instance; a worker leaves when the list is exhausted
  }
  auto leave = [&]() {
    std::lock_guard<std::mutex> lock(pb.mu);
    --pb.running;
    if (!pb.reqs.empty() && (int)pb.reqs.size() >= pb.running) pb.launch_round();
  };
  std::vector<eig_status> st(count, EIG_OK);
  std::vector<eig_stats> ss(count);
  std::atomic<int> next(0);
  std::atomic<int> setup_error(0);
  auto worker = [&]() {
    cudaStream_t s = nullptr;
    if (cudaSetDevice(dev) != cudaSuccess || cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      setup_error = 1;
      if (lockstep) leave();
      return;
    }
    for (int i = next++; i < count; i = next++) {
      eig_opts o;
      if (!opts) eig_default_opts(&o);
      else o = per_instance_opts ? opts[i] : opts[0];
      if (!o.stream) o.stream = s;
      st[i] = solve_handle(handles[i], method, &o, &ss[i], lockstep ? &pb : nullptr);
    }
    if (lockstep) leave();
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  };
  std::vector<std::thread> pool;
  pool.reserve(nt);
  for (int t = 0; t < nt; ++t) pool.emplace_back(worker);
  for (auto& th : pool) th.join();
  if (lockstep) {
    cudaStreamSynchronize(pb.ls);
    cudaEventDestroy(pb.done);
    cudaStreamDestroy(pb.ls);
  }
  if (setup_error) return EIG_ECUDA;
  eig_status first = EIG_OK;
  for (int i = 0; i < count; ++i) {
    if (status) status[i] = st[i];
    if (stats) {
      stats[i] = ss[i];
      if (lockstep) {
        stats[i].batch_launches = pb.launches;
        stats[i].batch_products = pb.products;
      }
    }
    if (first == EIG_OK && is_hard_error(st[i])) first = st[i];
  }
  return first;
}

eig_status eig_solve_batch(void* const* handles, int count, eig_method method, const eig_opts* opts,
                           int per_instance_opts, int threads, eig_status* status, eig_stats* stats) {
  return eig_solve_batch_ex(handles, count, method, opts, per_instance_opts, threads, 0, status, stats);
}

eig_status eig_autotune_spmm(const eig_csr_upper* H, int nb, eig_dtype vec_type, int reps, eig_tune_result* best,
                             eig_tune_result* all, int* n_all, void* stream) {
  if (!H || !best || nb < 1 || nb > 32 || (nb & (nb - 1)) || reps < 1) return EIG_EINVAL;
  if (vec_type != EIG_F32 && vec_type != EIG_F64) return EIG_EINVAL;
  cudaStream_t st = as_stream(stream);
  const int64_t n = H->n, nnz = H->nnz;
  if (n < 1 || nnz < 0) return EIG_EINVAL;
  const size_t vb = H->val_type == EIG_F64 ? 8 : (H->val_type == EIG_F32 ? 4 : 2);
  // one device copy of H shared by every candidate plan
  DevBuf rp, cl, vl;
  eig_csr_upper Hd = *H;
  if (!H->on_device) {
    EIG_TRY(rp.reserve((size_t)(n + 1) * 8));
    EIG_TRY(cl.reserve(std::max<int64_t>(nnz, 1) * 4));
    EIG_TRY(vl.reserve(std::max<int64_t>(nnz, 1) * vb));
    EIG_CUDA_TRY(cudaMemcpyAsync(rp.p, H->rowptr, (size_t)(n + 1) * 8, cudaMemcpyHostToDevice, st));
    if (nnz) {
      EIG_CUDA_TRY(cudaMemcpyAsync(cl.p, H->col, (size_t)nnz * 4, cudaMemcpyHostToDevice, st));
      EIG_CUDA_TRY(cudaMemcpyAsync(vl.p, H->val, (size_t)nnz * vb, cudaMemcpyHostToDevice, st));
    }
    Hd.rowptr = rp.as<int64_t>();
    Hd.col = cl.as<int32_t>();
    Hd.val = vl.p;
    Hd.on_device = 1;
  }
  const size_t es = vec_type == EIG_F64 ? 8 : 4;
  DevBuf X, Y;
  EIG_TRY(X.reserve((size_t)n * nb * es));
  EIG_TRY(Y.reserve((size_t)n * nb * es));
  const int fg = num_sms() * 4;
  if (vec_type == EIG_F64) k_tune_fill<double><<<fg, 256, 0, st>>>(X.as<double>(), n * nb);
  else k_tune_fill<float><<<fg, 256, 0, st>>>(X.as<float>(), n * nb);
  EIG_LAUNCH_CHECK("k_tune_fill");
  static const int cand[][3] = {{EIG_LAYOUT_MIRRORED, 256, 64}, {EIG_LAYOUT_HALF, 256, 64},
                                {EIG_LAYOUT_HALF, 128, 64},     {EIG_LAYOUT_HALF, 512, 128},
                                {EIG_LAYOUT_CSR, 256, 64},      {EIG_LAYOUT_CSR, 128, 32},
                                {EIG_LAYOUT_CSR, 512, 64}};
  const int ncand = (int)(sizeof(cand) / sizeof(cand[0]));
  cudaEvent_t e0, e1;
  EIG_CUDA_TRY(cudaEventCreate(&e0));
  EIG_CUDA_TRY(cudaEventCreate(&e1));
  int nres = 0;
  best->ms = -1.0;
  eig_status rc = EIG_OK;
  for (int q = 0; q < ncand && rc == EIG_OK; ++q) {
    SpmmPlan* P = new (std::nothrow) SpmmPlan();
    if (!P) { rc = EIG_ENOMEM; break; }
    eig_status s = spmm_plan_build(P, &Hd, cand[q][1], cand[q][2], cand[q][0], 0, st);
    // a layout the matrix or the memory does not allow is skipped
    if (s == EIG_OK && P->layout != cand[q][0]) s = EIG_EUNSUPPORTED;
    double ms = -1.0;
    if (s == EIG_OK) {
      for (int w = 0; w < 2 && s == EIG_OK; ++w) s = spmm_run(P, X.p, Y.p, nb, vec_type, st);
      if (s == EIG_OK) {
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps && s == EIG_OK; ++r) s = spmm_run(P, X.p, Y.p, nb, vec_type, st);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) s = EIG_ECUDA;
        float f = 0.f;
        cudaEventElapsedTime(&f, e0, e1);
        ms = f / reps;
      }
    }
    cudaStreamSynchronize(st);
    delete P;
    if (s == EIG_ECUDA) rc = s;
    if (s != EIG_OK) continue;
    eig_tune_result r{cand[q][0], cand[q][1], cand[q][2], ms};
    if (all) all[nres] = r;
    ++nres;
    if (best->ms < 0.0 || ms < best->ms) *best = r;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (n_all) *n_all = nres;
  if (rc != EIG_OK) return rc;
  return nres ? EIG_OK : EIG_EUNSUPPORTED;
}

eig_status eig_autotune_cheb(void* handle, const int* degrees, int count, const eig_opts* base, int* best_degree,
                             double* ms, int* converged) {
  if (!handle || !degrees || count < 1 || !best_degree) return EIG_EINVAL;
  for (int i = 0; i < count; ++i)
    if (degrees[i] < 1) return EIG_EINVAL;
  *best_degree = 0;
  double best = -1.0;
  auto opts_for = [&](int degree) {
    eig_opts o;
    if (base) o = *base;
    else eig_default_opts(&o);
    o.cheb_degree = degree;
    o.timing = 1;
    return o;
  };
  // one untimed solve first: lazy module loading, kernel attributes and workspace growth are
  // then paid before any candidate is timed
  {
    eig_opts o = opts_for(degrees[0]);
    eig_stats st;
    const eig_status s = eig_solve(handle, EIG_CHEBFILTER, &o, &st);
    if (is_hard_error(s) && s != EIG_EBREAKDOWN) return s;
  }
  constexpr int kReps = 3;   // the median of three timed solves per degree
  for (int i = 0; i < count; ++i) {
    eig_opts o = opts_for(degrees[i]);
    double t[kReps];
    eig_status s = EIG_OK;
    int r = 0;
    for (; r < kReps; ++r) {
      eig_stats st;
      s = eig_solve(handle, EIG_CHEBFILTER, &o, &st);
      if (s != EIG_OK) break;   // not converged, duplicate pairs or breakdown: not a candidate
      t[r] = st.time_ms_total;
    }
    if (is_hard_error(s) && s != EIG_EBREAKDOWN) return s;   // a CUDA / allocation / argument error
    const bool ok = (r == kReps);
    double med = 0.0;
    if (ok) {
      std::sort(t, t + kReps);
      med = t[kReps / 2];
    }
    if (ms) ms[i] = med;
    if (converged) converged[i] = ok ? 1 : 0;
    if (ok && (best < 0.0 || med < best)) {
      best = med;
      *best_degree = degrees[i];
    }
  }
  return *best_degree ? EIG_OK : EIG_ENOT_CONVERGED;
}

}  // extern "C"
