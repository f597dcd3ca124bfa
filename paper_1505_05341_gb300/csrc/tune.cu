// Autotuner: picks, by timing on the caller's catalogue, the scatter tile shape (or
// the direct assignment), the grid and ring lead of the persistent y,z kernel and
// the x stage's FFT tile for one plan.  Not part of the method
// (the paper runs on CPUs); it only chooses among configurations that compute the
// same result.
#include <cuda_runtime.h>

#include <cfloat>
#include <string>

#include "ys_internal.h"

namespace ys {
namespace {

// Mean device time (ms) of fn() over reps launches on the plan's stream, after one
// untimed call.
template <class F>
cudaError_t time_ms(Plan& p, int reps, F fn, float* out) {
  cudaError_t e = fn();
  if (e) return e;
  cudaEvent_t a, b;
  if ((e = cudaEventCreate(&a))) return e;
  if ((e = cudaEventCreate(&b))) {
    cudaEventDestroy(a);
    return e;
  }
  e = cudaEventRecord(a, p.stream);
  for (int r = 0; r < reps && !e; ++r) e = fn();
  if (!e) e = cudaEventRecord(b, p.stream);
  if (!e) e = cudaEventSynchronize(b);
  float ms = 0.f;
  if (!e) e = cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *out = ms / reps;
  return e;
}

}  // namespace

ys_status autotune(Plan& p, const ys_catalog& gal, const ys_catalog& ran, int reps, ys_tuning* out,
                   std::string& why) {
  ys_status st = ensure_particles(p, gal.n + ran.n);
  if (st != YS_OK) return st;
  reps = reps < 1 ? 1 : reps;
  // 1. scatter tile shape
  int best_tile = -1;
  float best_assign = FLT_MAX;
  for (int c = 0; c < (int)(sizeof(kTileCandidates) / sizeof(kTileCandidates[0])); ++c) {
    const auto& t = kTileCandidates[c];
    const size_t smem = sizeof(float) * p.m * (size_t)std::min(t[0], p.n) * std::min(t[1], p.n) * std::min(t[2], p.n);
    if (smem > 200u * 1024u) continue;
    set_tiles(p, t[0], t[1], t[2]);
    float ms = 0.f;
    cudaError_t e = time_ms(p, reps, [&] { return launch_assign(p, gal, ran); }, &ms);
    if (e) {
      why = cudaGetErrorString(e);
      return YS_ERR_CUDA;
    }
    if (ms < best_assign) {
      best_assign = ms;
      best_tile = c;
    }
  }
  const auto& bt = kTileCandidates[best_tile < 0 ? 0 : best_tile];
  set_tiles(p, bt[0], bt[1], bt[2]);
  // 1b. direct assignment into an L2-resident mesh, where the mesh set is small enough
  p.direct_assign = false;
  if (p.direct_ok) {
    p.direct_assign = true;
    float ms = 0.f;
    cudaError_t e1 = time_ms(p, reps, [&] { return launch_assign(p, gal, ran); }, &ms);
    if (e1) {
      why = cudaGetErrorString(e1);
      return YS_ERR_CUDA;
    }
    if (ms < best_assign) best_assign = ms;
    else p.direct_assign = false;
  }
  cudaError_t e = launch_assign(p, gal, ran);
  if (e) {
    why = cudaGetErrorString(e);
    return YS_ERR_CUDA;
  }
  p.assigned = true;
  // 2. grid of the persistent y,z kernel (the whole measurement is timed)
  const int grids[3] = {p.yz_grid_max, (p.yz_grid_max * 3) / 4, p.yz_grid_max / 2};
  int best_grid = p.yz_grid_max;
  float best_measure = FLT_MAX;
  for (int g : grids) {
    if (g < 1) continue;
    set_yz_grid(p, g);
    float ms = 0.f;
    e = time_ms(p, reps, [&] { return launch_measure(p); }, &ms);
    if (e) {
      why = cudaGetErrorString(e);
      return YS_ERR_CUDA;
    }
    if (ms < best_measure) {
      best_measure = ms;
      best_grid = g;
    }
  }
  set_yz_grid(p, best_grid);
  // 3. lead of the y,z ring at that grid
  int best_pct = p.ring_lead_pct;
  for (int pct : {70, 140, kRingLeadPctMax}) {
    set_yz_grid(p, best_grid, pct);
    float ms = 0.f;
    e = time_ms(p, reps, [&] { return launch_measure(p); }, &ms);
    if (e) {
      why = cudaGetErrorString(e);
      return YS_ERR_CUDA;
    }
    if (ms < best_measure) {
      best_measure = ms;
      best_pct = pct;
    }
  }
  set_yz_grid(p, best_grid, best_pct);
  // 4. the x stage's FFT tile (pencils per CTA): the default and its alternative; a
  // tile the device cannot run (shared memory) is skipped
  int best_px = p.x_pencils;
  for (int px : {k3_pencils(p.n), k3_pencils_alt(p.n)}) {
    if (px == best_px) continue;
    if (set_x_pencils(p, px) != YS_OK) continue;
    float ms = 0.f;
    e = time_ms(p, reps, [&] { return launch_measure(p); }, &ms);
    if (e) {
      cudaGetLastError();
      continue;
    }
    if (ms < best_measure) {
      best_measure = ms;
      best_px = px;
    }
  }
  if (set_x_pencils(p, best_px) != YS_OK) {
    why = "could not restore the x-stage tile";
    return YS_ERR_CUDA;
  }
  // the captured measurement graph holds the old launch shapes
  if (p.measure_exec) {
    cudaGraphExecDestroy(p.measure_exec);
    p.measure_exec = nullptr;
  }
  for (int c = 0; c < YS_NUM_KERNEL_CLASSES; ++c) {
    p.launches[c] = 0;
    p.ms[c] = 0.0;
  }
  if (out) {
    for (int a = 0; a < 3; ++a) out->tile[a] = p.direct_assign ? 0 : p.geom.tdim[a];
    out->yz_grid = p.yz_grid;
    out->ring_lead = p.ring_lead;
    out->assign_ms = best_assign;
    out->measure_ms = best_measure;
    out->x_pencils = p.x_pencils;
  }
  return YS_OK;
}

}  // namespace ys
