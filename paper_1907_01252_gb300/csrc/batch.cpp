// Batches of independent FSI problems on one GPU: host-side scheduler.
//
// The paper runs one problem at a time and parallelises its time slices. A
// batch of independent problems (different meshes, materials and slice counts)
// has no coupling at all, so the GPU-native layout is concurrency: worker host
// threads, each with its own non-blocking CUDA stream and its own context,
// pull problems from one queue ordered by estimated cost (longest first) and
// run the Parareal iteration of Sec. 3 on each. Kernels of different workers
// overlap on the GPU; the single-slice coarse sweeps, which alone leave most
// SMs idle, overlap with other problems' batched fine sweeps.
//
// This file uses the public C ABI only (fsi_setup, parareal_iterate,
// fsi_destroy); results are bit-identical to running each problem alone.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <mutex>
#include <numeric>
#include <string>
#include <system_error>
#include <thread>
#include <vector>

#include "../../include/fsi.h"
#include "fsi_internal.h"

namespace {

int batch_fail(int code, const std::string& msg) { return fsi_record_error(code, msg); }

// Work estimate of one instance in dof-steps: fine steps of every slice still
// iterated (Parareal iteration i re-solves slices i-1 .. N-1), plus the
// single-slice coarse steps weighted by kCoarseWeight. A single-slice coarse
// step on one GPU costs about as much as eight batched fine steps of one slice
// (measured on the 128 x 32 workload: 0.11 s vs 14 ms), because one slice
// cannot fill the GPU.
constexpr double kCoarseWeight = 8.0;

double instance_cost(const fsi_instance& I, int n_dofs) {
  const int N = std::max(I.params.n_slices, 1);
  const int K = std::min(std::max(I.max_iter, 0), N);
  double fine = 0.0, coarse = (double)N * I.params.m_coarse;   // predictor sweep
  for (int i = 1; i <= K; ++i) {
    fine += (double)(N - i + 1) * I.params.m_fine;
    coarse += (double)(N - i) * I.params.m_coarse;
  }
  return (double)n_dofs * (fine + kCoarseWeight * coarse);
}

double now_s() {
  using clk = std::chrono::steady_clock;
  return std::chrono::duration<double>(clk::now().time_since_epoch()).count();
}

}  // namespace

extern "C" {

int fsi_batch_plan(const fsi_instance* inst, int n, int workers, int* order, int* worker, double* cost,
                   double* makespan) {
  if (n < 0 || workers < 1 || (n > 0 && (!inst || !order || !worker || !cost)))
    return batch_fail(FSI_EINVAL, "bad batch plan arguments");
  for (int i = 0; i < n; ++i) {
    int nodes = 0, dofs = 0, nnzb = 0;
    const int rc = fsi_mesh_size(&inst[i].mesh, &nodes, &dofs, &nnzb);
    if (rc != FSI_OK) return batch_fail(rc, "instance " + std::to_string(i) + ": " + fsi_last_error());
    cost[i] = instance_cost(inst[i], dofs);
  }
  // longest first (ties by index), each to the least loaded worker (ties by index)
  std::iota(order, order + n, 0);
  std::stable_sort(order, order + n, [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<double> load(workers, 0.0);
  for (int k = 0; k < n; ++k) {
    const int w = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    worker[order[k]] = w;
    load[w] += cost[order[k]];
  }
  if (makespan) *makespan = n > 0 ? *std::max_element(load.begin(), load.end()) : 0.0;
  return FSI_OK;
}

int fsi_batch_parareal(fsi_instance* inst, int n, int workers, void* stream) {
  if (n < 0 || workers < 1 || (n > 0 && !inst)) return batch_fail(FSI_EINVAL, "bad batch arguments");
  if (n == 0) return FSI_OK;
  for (int i = 0; i < n; ++i)
    if (!inst[i].U || inst[i].params.n_slices < 1 || inst[i].max_iter < 0)
      return batch_fail(FSI_EINVAL, "instance " + std::to_string(i) + ": null state or bad slice/iteration count");
  std::vector<int> order(n), planned(n);
  std::vector<double> cost(n);
  int rc = fsi_batch_plan(inst, n, workers, order.data(), planned.data(), cost.data(), nullptr);
  if (rc != FSI_OK) return rc;
  const int W = std::min(workers, n);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return batch_fail(FSI_ECUDA, "cudaGetDevice failed");
  cudaStream_t caller = (cudaStream_t)stream;
  cudaEvent_t start;
  if (cudaEventCreateWithFlags(&start, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventRecord(start, caller) != cudaSuccess)
    return batch_fail(FSI_ECUDA, "cannot order the batch after the caller's stream");

  std::atomic<int> next{0};
  std::mutex mu;                 // guards deferred, first_rc, first_msg
  std::vector<int> deferred;     // instances whose set-up ran out of device memory
  int first_rc = FSI_OK;
  std::string first_msg;
  auto run_one = [&](int idx, int w, cudaStream_t s, bool may_defer) {
    fsi_instance& I = inst[idx];
    const double t0 = now_s();
    fsi_params p = I.params;
    p.max_batch = p.n_slices;
    fsi_ctx* c = nullptr;
    int r = fsi_setup(&I.mesh, &p, &c);
    if (r == FSI_ENOMEM && may_defer) {
      std::lock_guard<std::mutex> lk(mu);
      deferred.push_back(idx);
      return;
    }
    std::string msg;
    if (r == FSI_OK) {
      fsi_parareal_stats st{};
      st.history = I.stats.history;
      st.history_len = I.stats.history_len;
      r = parareal_iterate(c, I.U, I.max_iter, I.tol, &st, s);
      if (r != FSI_OK) msg = fsi_last_error();
      I.stats = st;
      cudaStreamSynchronize(s);
    } else {
      msg = fsi_last_error();
    }
    fsi_destroy(c);
    I.status = r;
    I.worker = w;
    I.seconds = now_s() - t0;
    if (r != FSI_OK) {
      std::lock_guard<std::mutex> lk(mu);
      if (first_rc == FSI_OK) {
        first_rc = r;
        first_msg = "instance " + std::to_string(idx) + ": " + msg;
      }
    }
  };

  std::vector<cudaStream_t> streams(W, nullptr);
  std::vector<std::thread> threads;
  threads.reserve(W);
  auto worker_main = [&](int w) {
    cudaSetDevice(dev);
    if (cudaStreamCreateWithFlags(&streams[w], cudaStreamNonBlocking) != cudaSuccess) {
      std::lock_guard<std::mutex> lk(mu);
      if (first_rc == FSI_OK) first_rc = FSI_ECUDA, first_msg = "worker stream creation failed";
      streams[w] = nullptr;
    } else {
      cudaStreamWaitEvent(streams[w], start, 0);
    }
    for (;;) {
      const int k = next.fetch_add(1);
      if (k >= n) break;
      if (!streams[w]) {   // no stream: leave the instance to the serial pass below
        std::lock_guard<std::mutex> lk(mu);
        deferred.push_back(order[k]);
        continue;
      }
      run_one(order[k], w, streams[w], true);
    }
  };
  for (int w = 0; w < W; ++w) {
    try {
      threads.emplace_back(worker_main, w);
    } catch (const std::system_error&) {   // fewer workers than asked for
      break;
    }
  }
  for (auto& t : threads) t.join();
  // problems no worker took (no thread could be started) join the serial pass
  for (int k = next.load(); k < n; ++k) deferred.push_back(order[k]);
  // instances that did not fit next to the others run one at a time
  std::sort(deferred.begin(), deferred.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  cudaStream_t s0 = nullptr;
  if (!deferred.empty() && cudaStreamCreateWithFlags(&s0, cudaStreamNonBlocking) == cudaSuccess) {
    cudaStreamWaitEvent(s0, start, 0);
    for (int idx : deferred) run_one(idx, 0, s0, false);
  } else {
    for (int idx : deferred) {
      inst[idx].status = FSI_ECUDA;
      if (first_rc == FSI_OK) first_rc = FSI_ECUDA, first_msg = "no stream for deferred instances";
    }
  }
  // the caller's stream continues after every worker's work
  for (cudaStream_t s : streams)
    if (s) {
      cudaEvent_t done;
      if (cudaEventCreateWithFlags(&done, cudaEventDisableTiming) == cudaSuccess) {
        cudaEventRecord(done, s);
        cudaStreamWaitEvent(caller, done, 0);
        cudaEventDestroy(done);
      }
      cudaStreamDestroy(s);
    }
  if (s0) cudaStreamDestroy(s0);
  cudaEventDestroy(start);
  if (first_rc != FSI_OK) return batch_fail(first_rc, first_msg);
  return FSI_OK;
}

int fsi_batch_autotune(fsi_instance* inst, int n, const int* candidates, int n_candidates, double* seconds,
                       int* best, void* stream) {
  if (!candidates || n_candidates < 1 || !seconds || !best) return batch_fail(FSI_EINVAL, "bad autotune arguments");
  for (int c = 0; c < n_candidates; ++c)
    if (candidates[c] < 1) return batch_fail(FSI_EINVAL, "worker counts must be >= 1");
  cudaStream_t s = (cudaStream_t)stream;
  // one untimed run takes the one-time costs (module load, graph capture)
  int rc = fsi_batch_parareal(inst, n, candidates[0], stream);
  if (rc != FSI_OK) return rc;
  *best = candidates[0];
  double best_t = 0.0;
  for (int c = 0; c < n_candidates; ++c) {
    if (cudaStreamSynchronize(s) != cudaSuccess) return batch_fail(FSI_ECUDA, "stream synchronisation failed");
    const double t0 = now_s();
    rc = fsi_batch_parareal(inst, n, candidates[c], stream);
    if (rc != FSI_OK) return rc;
    if (cudaStreamSynchronize(s) != cudaSuccess) return batch_fail(FSI_ECUDA, "stream synchronisation failed");
    seconds[c] = now_s() - t0;
    if (c == 0 || seconds[c] < best_t) {
      best_t = seconds[c];
      *best = candidates[c];
    }
  }
  return FSI_OK;
}

}  // extern "C"
