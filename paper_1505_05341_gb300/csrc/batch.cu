// Batched runner: many catalogues (uneven sizes, mixed mesh sizes) in one CUDA
// graph launch.  The paper's motivation is measuring hundreds of mock catalogues
// (Sec. 1); this is a throughput arrangement of the same per-catalogue steps.
//
// Catalogues are spread over B concurrent stream branches by longest-processing-
// time-first on an estimate of their cost; every (branch, configuration class)
// owns one plan, reused by that branch's catalogues in sequence.  The whole batch
// -- assignment, transforms, shell sums and the copy of each result row -- is
// captured once into a graph and replayed by every ys_batch_run with the same
// catalogue pointers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "ys_internal.h"

namespace ys {
ys_status autotune(Plan& p, const ys_catalog& gal, const ys_catalog& ran, int reps, ys_tuning* out,
                   std::string& why);
}

struct ys_batch_s {
  int n = 0, branches = 1;
  std::vector<ys_config> cfgs;
  std::vector<int> cls;                   // configuration class per catalogue
  std::vector<int> branch;                // stream branch per catalogue
  std::vector<std::vector<ys_plan*>> plans;  // [branch][class]
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;        // fork + one join per branch
  cudaGraphExec_t exec = nullptr;
  std::vector<ys_catalog> captured_gal, captured_ran;
  double* captured_out = nullptr;
  int64_t stride = 0;
};

namespace {

bool same_class(const ys_config& a, const ys_config& b) {
  return a.n_mesh == b.n_mesh && a.box_len == b.box_len && a.box_min[0] == b.box_min[0] &&
         a.box_min[1] == b.box_min[1] && a.box_min[2] == b.box_min[2] && a.observer[0] == b.observer[0] &&
         a.observer[1] == b.observer[1] && a.observer[2] == b.observer[2] && a.assign == b.assign &&
         a.interlace == b.interlace && a.compensate == b.compensate && a.ell_max == b.ell_max &&
         a.k_min == b.k_min && a.dk == b.dk && a.n_bins == b.n_bins && a.alpha == b.alpha;
}

bool same_catalog(const ys_catalog& a, const ys_catalog& b) {
  return a.x == b.x && a.y == b.y && a.z == b.z && a.w == b.w && a.nbar == b.nbar && a.n == b.n;
}

void destroy_batch(ys_batch* b) {
  if (!b) return;
  for (auto& row : b->plans)
    for (ys_plan* p : row)
      if (p) ys_plan_destroy(p);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (cudaStream_t s : b->streams)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->events)
    if (e) cudaEventDestroy(e);
  delete b;
}

ys_status capture(ys_batch* b, const ys_catalog* gal, const ys_catalog* ran, double* d_out) {
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  cudaStream_t s0 = b->streams[0];
  cudaError_t e = cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal);
  if (e) return YS_ERR_CUDA;
  cudaError_t e2 = cudaEventRecord(b->events[0], s0);
  for (int br = 1; br < b->branches && !e2; ++br) e2 = cudaStreamWaitEvent(b->streams[br], b->events[0], 0);
  for (int i = 0; i < b->n && !e2; ++i) {
    ys::Plan& p = b->plans[b->branch[i]][b->cls[i]]->p;
    e2 = ys::launch_assign(p, gal[i], ran[i]);
    if (!e2) e2 = ys::launch_measure(p);
    if (!e2)
      e2 = cudaMemcpyAsync(d_out + (size_t)i * b->stride, p.d_result, sizeof(double) * p.row_len,
                           cudaMemcpyDeviceToDevice, p.stream);
  }
  for (int br = 1; br < b->branches && !e2; ++br) {
    e2 = cudaEventRecord(b->events[br], b->streams[br]);
    if (!e2) e2 = cudaStreamWaitEvent(s0, b->events[br], 0);
  }
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(s0, &graph);
  if (!e && !e2) e = cudaGraphInstantiate(&b->exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e || e2) {
    ys::g_last_cuda_error = cudaGetErrorString(e2 ? e2 : e);
    cudaGetLastError();
    b->exec = nullptr;
    return YS_ERR_CUDA;
  }
  b->captured_gal.assign(gal, gal + b->n);
  b->captured_ran.assign(ran, ran + b->n);
  b->captured_out = d_out;
  return YS_OK;
}

}  // namespace

extern "C" {

ys_status ys_batch_create(const ys_config* cfgs, int32_t n, int32_t branches, ys_batch** out) {
  if (!cfgs || !out || n <= 0 || branches <= 0 || branches > 32) return YS_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < n; ++i)
    if (cfgs[i].max_particles <= 0) return YS_ERR_ARG;  // capacity must be known before capture
  ys_batch* b = new (std::nothrow) ys_batch;
  if (!b) return YS_ERR_OOM;
  b->n = n;
  b->branches = std::min<int>(branches, n);
  b->cfgs.assign(cfgs, cfgs + n);
  // configuration classes
  std::vector<int> reps;  // first catalogue of each class
  b->cls.resize(n);
  for (int i = 0; i < n; ++i) {
    int c = -1;
    for (size_t k = 0; k < reps.size(); ++k)
      if (same_class(cfgs[reps[k]], cfgs[i])) c = (int)k;
    if (c < 0) {
      c = (int)reps.size();
      reps.push_back(i);
    }
    b->cls[i] = c;
  }
  // longest-processing-time-first over the branches (cost ~ N^3 log N + particles)
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  auto cost = [&](int i) {
    const double N = cfgs[i].n_mesh;
    return N * N * N * std::log2(N) * (cfgs[i].interlace ? 2.0 : 1.0) + 40.0 * (double)cfgs[i].max_particles;
  };
  std::sort(order.begin(), order.end(), [&](int a, int c) { return cost(a) > cost(c); });
  std::vector<double> load(b->branches, 0.0);
  b->branch.resize(n);
  for (int i : order) {
    const int br = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    b->branch[i] = br;
    load[br] += cost(i);
  }
  b->streams.assign(b->branches, nullptr);
  b->events.assign(b->branches, nullptr);
  for (int br = 0; br < b->branches; ++br) {
    if (cudaStreamCreateWithFlags(&b->streams[br], cudaStreamNonBlocking) ||
        cudaEventCreateWithFlags(&b->events[br], cudaEventDisableTiming)) {
      destroy_batch(b);
      return YS_ERR_CUDA;
    }
  }
  // one plan per (branch, class) that has catalogues, sized for its largest one
  b->plans.assign(b->branches, std::vector<ys_plan*>(reps.size(), nullptr));
  int row_max = 0;
  for (int br = 0; br < b->branches; ++br)
    for (size_t c = 0; c < reps.size(); ++c) {
      int64_t cap = 0;
      for (int i = 0; i < n; ++i)
        if (b->branch[i] == br && b->cls[i] == (int)c) cap = std::max<int64_t>(cap, cfgs[i].max_particles);
      if (cap == 0) continue;
      ys_config cc = cfgs[reps[c]];
      cc.max_particles = cap;
      cc.stream = b->streams[br];
      ys_status st = ys_plan_create(&cc, &b->plans[br][c]);
      if (st != YS_OK) {
        destroy_batch(b);
        return st;
      }
      row_max = std::max(row_max, b->plans[br][c]->p.row_len);
    }
  b->stride = row_max;
  *out = b;
  return YS_OK;
}

int64_t ys_batch_result_stride(const ys_batch* batch) { return batch ? batch->stride : 0; }

ys_status ys_batch_autotune(ys_batch* b, const ys_catalog* gal, const ys_catalog* ran, int32_t reps) {
  if (!b || !gal || !ran) return YS_ERR_ARG;
  for (int br = 0; br < b->branches; ++br)
    for (size_t c = 0; c < b->plans[br].size(); ++c) {
      ys_plan* pl = b->plans[br][c];
      if (!pl) continue;
      // tune on the largest catalogue of this plan
      int pick = -1;
      for (int i = 0; i < b->n; ++i)
        if (b->branch[i] == br && b->cls[i] == (int)c &&
            (pick < 0 || gal[i].n + ran[i].n > gal[pick].n + ran[pick].n))
          pick = i;
      std::string why;
      ys_status st = ys::autotune(pl->p, gal[pick], ran[pick], reps, nullptr, why);
      if (st != YS_OK) {
        ys::g_last_cuda_error = why;
        return st;
      }
    }
  for (cudaStream_t s : b->streams) cudaStreamSynchronize(s);
  if (b->exec) {  // launch shapes changed
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  return YS_OK;
}

ys_status ys_batch_run(ys_batch* b, const ys_catalog* gal, const ys_catalog* ran, double* d_results, void* stream) {
  if (!b || !gal || !ran || !d_results) return YS_ERR_ARG;
  for (int i = 0; i < b->n; ++i) {
    if (gal[i].n < 0 || ran[i].n < 0 || gal[i].n + ran[i].n > b->cfgs[i].max_particles) return YS_ERR_ARG;
    if ((gal[i].n > 0 && (!gal[i].x || !gal[i].y || !gal[i].z)) || (ran[i].n > 0 && (!ran[i].x || !ran[i].y || !ran[i].z)))
      return YS_ERR_ARG;
  }
  bool same = b->exec && b->captured_out == d_results;
  for (int i = 0; same && i < b->n; ++i)
    same = same_catalog(b->captured_gal[i], gal[i]) && same_catalog(b->captured_ran[i], ran[i]);
  if (!same) {
    ys_status st = capture(b, gal, ran, d_results);
    if (st != YS_OK) return st;
    for (auto& row : b->plans)
      for (ys_plan* p : row)
        if (p) p->p.assigned = true;
  }
  cudaError_t e = cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream));
  if (e) {
    ys::g_last_cuda_error = cudaGetErrorString(e);
    return YS_ERR_CUDA;
  }
  return YS_OK;
}

ys_status ys_batch_destroy(ys_batch* b) {
  if (!b) return YS_OK;
  for (cudaStream_t s : b->streams)
    if (s) cudaStreamSynchronize(s);
  destroy_batch(b);
  return YS_OK;
}

ys_status ys_plan_autotune(ys_plan* plan, const ys_catalog* gal, const ys_catalog* ran, int32_t reps,
                           ys_tuning* out) {
  if (!plan || !gal || !ran || gal->n < 0 || ran->n < 0) return YS_ERR_ARG;
  std::string why;
  ys_status st = ys::autotune(plan->p, *gal, *ran, reps, out, why);
  if (st != YS_OK) ys::g_last_cuda_error = why;
  return st;
}

}  // extern "C"
