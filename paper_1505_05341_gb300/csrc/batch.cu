// Batched runner: many catalogues (uneven sizes, mixed mesh sizes) in one CUDA
// graph launch.  The paper's motivation is measuring hundreds of mock catalogues
// (Sec. 1); this is a throughput arrangement of the same per-catalogue steps.
//
// Catalogues with the same configuration form a class.  A class owns one to four
// sets of up to YZ_MAX_LANES plans ("lanes", each with its own meshes, ring and transforms)
// and is measured in waves: every lane of a set assigns one catalogue, then one
// persistent y,z launch walks the items of all the wave's catalogues through one
// ticket queue, one x-stage launch covers all their pencil blocks, and one finalize
// launch writes each result row straight into the caller's array.  Consecutive waves
// go round the sets, each on its own stream, so that one wave's assignment overlaps
// another's transforms; classes run on further streams.
// The whole batch is captured once into a graph and replayed by every ys_batch_run
// with the same catalogue pointers.
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
  int n = 0, lanes = 1;
  std::vector<ys_config> cfgs;
  std::vector<int> cls;                        // configuration class per catalogue
  std::vector<std::vector<int>> members;       // catalogues of each class, in order
  std::vector<std::vector<std::vector<ys_plan*>>> plans;  // [class][set][lane]
  std::vector<std::vector<int>> set_stream;    // stream index of each class's sets
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;             // fork + one join per stream
  cudaGraphExec_t exec = nullptr;
  std::vector<ys_catalog> captured_gal, captured_ran;
  double* captured_out = nullptr;
  int64_t stride = 0;
};

namespace {

constexpr int kMaxStreams = 8;

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
  for (auto& sets : b->plans)
    for (auto& row : sets)
      for (ys_plan* p : row)
        if (p) ys_plan_destroy(p);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (cudaStream_t s : b->streams)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->events)
    if (e) cudaEventDestroy(e);
  delete b;
}

// Launch shapes tuned on lane 0, given to the class's other lanes.
void copy_tuning(ys::Plan& dst, const ys::Plan& src) {
  ys::set_tiles(dst, src.geom.tdim[0], src.geom.tdim[1], src.geom.tdim[2]);
  dst.direct_assign = src.direct_assign;
  ys::set_yz_grid(dst, src.yz_grid, src.ring_lead_pct);
  ys::set_x_pencils(dst, src.x_pencils);
  if (dst.measure_exec) {
    cudaGraphExecDestroy(dst.measure_exec);
    dst.measure_exec = nullptr;
  }
}

ys_status capture(ys_batch* b, const ys_catalog* gal, const ys_catalog* ran, double* d_out) {
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  cudaStream_t s0 = b->streams[0];
  const int ns = (int)b->streams.size();
  cudaError_t e = cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal);
  if (e) return YS_ERR_CUDA;
  cudaError_t e2 = cudaEventRecord(b->events[0], s0);
  for (int s = 1; s < ns && !e2; ++s) e2 = cudaStreamWaitEvent(b->streams[s], b->events[0], 0);
  for (size_t c = 0; c < b->members.size() && !e2; ++c) {
    const std::vector<int>& mem = b->members[c];
    const int nsets = (int)b->plans[c].size();
    const int W = (int)b->plans[c][0].size();
    int wave = 0;
    for (size_t w0 = 0; w0 < mem.size() && !e2; w0 += W, ++wave) {
      const int w = (int)std::min<size_t>(W, mem.size() - w0);
      const std::vector<ys_plan*>& set = b->plans[c][wave % nsets];
      ys::Plan* lanes[ys::YZ_MAX_LANES];
      double* rows[ys::YZ_MAX_LANES];
      for (int l = 0; l < w && !e2; ++l) {
        const int i = mem[w0 + l];
        lanes[l] = &set[l]->p;
        rows[l] = d_out + (size_t)i * b->stride;
        e2 = ys::launch_assign(*lanes[l], gal[i], ran[i]);
      }
      if (!e2) e2 = ys::launch_measure_lanes(lanes, w, rows);
    }
  }
  for (int s = 1; s < ns && !e2; ++s) {
    e2 = cudaEventRecord(b->events[s], b->streams[s]);
    if (!e2) e2 = cudaStreamWaitEvent(s0, b->events[s], 0);
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

ys_status ys_batch_create(const ys_config* cfgs, int32_t n, int32_t lanes, ys_batch** out) {
  if (!cfgs || !out || n <= 0 || lanes <= 0 || lanes > 32) return YS_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < n; ++i)
    if (cfgs[i].max_particles <= 0) return YS_ERR_ARG;  // capacity must be known before capture
  ys_batch* b = new (std::nothrow) ys_batch;
  if (!b) return YS_ERR_OOM;
  b->n = n;
  b->lanes = std::min<int>(lanes, ys::YZ_MAX_LANES);
  b->cfgs.assign(cfgs, cfgs + n);
  // configuration classes, each with its catalogues in input order
  std::vector<int> reps;  // first catalogue of each class
  b->cls.resize(n);
  for (int i = 0; i < n; ++i) {
    int c = -1;
    for (size_t k = 0; k < reps.size(); ++k)
      if (same_class(cfgs[reps[k]], cfgs[i])) c = (int)k;
    if (c < 0) {
      c = (int)reps.size();
      reps.push_back(i);
      b->members.emplace_back();
    }
    b->cls[i] = c;
    b->members[c].push_back(i);
  }
  const int nclass = (int)reps.size();
  // lane sets per class (each on its own stream): as many as its waves, the streams
  // shared out among the classes and at most 4
  const int W = b->lanes;
  std::vector<int> nsets(nclass);
  int want = 0;
  for (int c = 0; c < nclass; ++c) {
    const int waves = ((int)b->members[c].size() + W - 1) / W;
    nsets[c] = std::max(1, std::min({waves, kMaxStreams / std::max(1, nclass), 4}));
    want += nsets[c];
  }
  const int ns = std::min(want, kMaxStreams);
  b->streams.assign(ns, nullptr);
  b->events.assign(ns, nullptr);
  for (int s = 0; s < ns; ++s) {
    if (cudaStreamCreateWithFlags(&b->streams[s], cudaStreamNonBlocking) ||
        cudaEventCreateWithFlags(&b->events[s], cudaEventDisableTiming)) {
      destroy_batch(b);
      return YS_ERR_CUDA;
    }
  }
  // each set of each class on a stream (round robin) with min(lanes, its catalogues)
  // plans, each sized for the class's largest catalogue
  b->set_stream.assign(nclass, {});
  b->plans.assign(nclass, {});
  int row_max = 0, next_stream = 0;
  for (int c = 0; c < nclass; ++c) {
    int64_t cap = 0;
    for (int i : b->members[c]) cap = std::max<int64_t>(cap, cfgs[i].max_particles);
    const int Wc = std::min<int>(W, (int)b->members[c].size());
    b->plans[c].assign(nsets[c], {});
    for (int k = 0; k < nsets[c]; ++k) {
      const int sidx = next_stream++ % ns;
      b->set_stream[c].push_back(sidx);
      ys_config cc = cfgs[reps[c]];
      cc.max_particles = cap;
      cc.stream = b->streams[sidx];
      for (int l = 0; l < Wc; ++l) {
        ys_plan* pl = nullptr;
        ys_status st = ys_plan_create(&cc, &pl);
        if (st != YS_OK) {
          destroy_batch(b);
          return st;
        }
        b->plans[c][k].push_back(pl);
        row_max = std::max(row_max, pl->p.row_len);
      }
    }
  }
  b->stride = row_max;
  *out = b;
  return YS_OK;
}

int64_t ys_batch_result_stride(const ys_batch* batch) { return batch ? batch->stride : 0; }

ys_status ys_batch_autotune(ys_batch* b, const ys_catalog* gal, const ys_catalog* ran, int32_t reps) {
  if (!b || !gal || !ran) return YS_ERR_ARG;
  for (size_t c = 0; c < b->plans.size(); ++c) {
    // tune lane 0 on the class's largest catalogue; the other lanes take its shapes
    int pick = -1;
    for (int i : b->members[c])
      if (pick < 0 || gal[i].n + ran[i].n > gal[pick].n + ran[pick].n) pick = i;
    std::string why;
    ys::Plan& p0 = b->plans[c][0][0]->p;
    ys_status st = ys::autotune(p0, gal[pick], ran[pick], reps, nullptr, why);
    if (st != YS_OK) {
      ys::g_last_cuda_error = why;
      return st;
    }
    for (auto& set : b->plans[c])
      for (ys_plan* pl : set)
        if (&pl->p != &p0) copy_tuning(pl->p, p0);
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
    for (auto& sets : b->plans)
      for (auto& row : sets)
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
