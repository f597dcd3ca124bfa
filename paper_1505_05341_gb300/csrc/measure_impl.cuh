// Host-side launch sequence of the spectral steps for one mesh size N (one
// translation unit per N instantiates it, so the sizes compile in parallel).
#pragma once
#include <algorithm>

#include "spectra.cuh"

namespace ys {

cudaError_t launch_finalize(Plan* const* lanes, int W, double* const* rows);

// CTAs of the persistent y,z kernel that fit on the device at once.
template <int N, int ELL>
int yz_grid(cudaError_t* err) {
  using Y = YZ<N, ELL>;
  int dev = 0, sms = 0, per = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (!e) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (!e) e = cudaFuncSetAttribute(k_yz<N, ELL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Y::smem);
  if (!e) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_yz<N, ELL>, Y::THREADS, Y::smem);
  if (err) *err = e;
  return e ? 0 : std::max(1, per) * sms;
}

// l_max = 6 needs the 29 basis lines of a column item in shared memory: N <= 512.
template <int N>
constexpr bool ell6_supported() { return N <= 512; }

template <int N>
int yz_grid_n(int ell, cudaError_t* err) {
  switch (ell) {
    case 0: return yz_grid<N, 0>(err);
    case 2: return yz_grid<N, 2>(err);
    case 6:
      if constexpr (ell6_supported<N>()) return yz_grid<N, 6>(err);
      if (err) *err = cudaErrorInvalidValue;
      return 0;
    default: return yz_grid<N, 4>(err);
  }
}

// The launches below take the lanes (plans of one configuration, each with its own
// catalogue already assigned) measured together; a single plan is one lane.  Work is
// queued on lane 0's stream.
template <int N, int ELL>
cudaError_t run_yz(Plan* const* lanes, int W) {
  using Y = YZ<N, ELL>;
  Plan& p0 = *lanes[0];
  cudaError_t err;
  YZMulti pm{};
  int items = 0;
  for (int l = 0; l < W; ++l) {
    Plan& p = *lanes[l];
    if ((err = cudaMemsetAsync(p.d_sync, 0, sizeof(int) * (2 * p.m * N + 2), p0.stream))) return err;
    YZParams& prm = pm.lane[l];
    prm.mesh = p.d_mesh;
    prm.rel = p.d_rel;
    prm.tw = p.d_tw;
    prm.ring = p.d_z;
    prm.gout = p.d_g;
    prm.col_off = p.d_col_off;
    prm.done_z = p.d_sync;
    prm.done_y = p.d_sync + p.m * N;
    prm.ticket = p.d_sync + 2 * p.m * N;
    prm.err = p.d_sync + 2 * p.m * N + 1;
    prm.nzc = p.nzc;
    prm.np = p.np_pad;
    prm.m = p.m;
    prm.S = p.ring_slots;
    prm.D = p.ring_lead;
    prm.spin_limit = p.yz_wait_ns;  // 1 s unless a test shortened it; then the kernel reports a timeout
    prm.skip_plane = p.fault_skip_plane;
    items += (p.m * N + p.ring_lead) * (N / Y::R + p.nzc);
    pm.end[l] = items;
  }
  pm.nlanes = W;
  pm.ticket = p0.d_sync + 2 * p0.m * N;
  if ((err = cudaFuncSetAttribute(k_yz<N, ELL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Y::smem)))
    return err;
  LaunchScope ls(p0, 4);
  k_yz<N, ELL><<<p0.yz_grid, Y::THREADS, Y::smem, p0.stream>>>(pm);
  return cudaGetLastError();
}

template <int N, int ELL, int M, int PX>
cudaError_t run_x_p(Plan* const* lanes, int W) {
  using XC = XCombine<N, ELL, M, PX>;
  Plan& p = *lanes[0];
  const int nbins = p.cfg.n_bins;
  cudaError_t err;
  int dev0 = 0, smem_max = 0;
  if ((err = cudaGetDevice(&dev0))) return err;
  if ((err = cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev0))) return err;
  // Float-bin copies: several per warp (lanes spread over them) while that costs no
  // resident CTA, else one per warp while it fits, else one shared copy (many shells).
  auto occupancy = [&](int nwb, int* per) -> cudaError_t {
    const size_t sm = XC::smem(nbins, nwb);
    if (sm > (size_t)smem_max) {
      *per = 0;
      return cudaSuccess;
    }
    cudaError_t e = cudaFuncSetAttribute(k_x_combine<N, ELL, M, PX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (!e) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per, k_x_combine<N, ELL, M, PX>, XC::THREADS, sm);
    return e;
  };
  int nwb = 1, per = 0, per_warp = 0;
  if ((err = occupancy(XC::NW, &per_warp))) return err;
  if (per_warp > 0) {
    nwb = XC::NW;
    per = per_warp;
    for (int c : {8, 4, 2}) {
      int pc = 0;
      if ((err = occupancy(XC::NW * c, &pc))) return err;
      if (pc >= per_warp) {
        nwb = XC::NW * c;
        break;
      }
    }
  } else if ((err = occupancy(1, &per))) {
    return err;
  }
  const size_t smem = XC::smem(nbins, nwb);
  if (smem > (size_t)smem_max) return cudaErrorInvalidConfiguration;
  if ((err = cudaFuncSetAttribute(k_x_combine<N, ELL, M, PX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
    return err;
  int dev = 0, sms = 0;
  if ((err = cudaGetDevice(&dev))) return err;
  if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))) return err;
  XMulti pm{};
  for (int l = 0; l < W; ++l) {
    pm.map[l] = lanes[l]->gmap;
    pm.acc[l] = lanes[l]->d_acc;
    pm.err[l] = lanes[l]->d_sync + 2 * lanes[l]->m * N + 1;
  }
  pm.nlanes = W;
  // the resident CTAs are shared among the lanes
  const int npb = p.np_pad / XC::P;
  const int resident = std::max(1, per) * sms;
  const int grid = std::max(1, std::min(npb, (resident + W - 1) / W));
  LaunchScope ls(p, 6);
  k_x_combine<N, ELL, M, PX><<<dim3(grid, W), XC::THREADS, smem, p.stream>>>(pm, p.np_pad, p.d_pencil, p.d_tw, p.d_invw,
                                                                         p.d_phase, p.d_lut, p.n2_hi, nbins, nwb);
  return cudaGetLastError();
}

// The x stage with the plan's current pencils per CTA.
template <int N, int ELL, int M>
cudaError_t run_x(Plan* const* lanes, int W) {
  if (lanes[0]->x_pencils == k3_pencils_alt(N)) return run_x_p<N, ELL, M, k3_pencils_alt(N)>(lanes, W);
  return run_x_p<N, ELL, M, k3_pencils(N)>(lanes, W);
}

// Dynamic shared memory of the x stage for mesh size N (independent of interlacing),
// with nwb copies of the float shell bins.
template <int N>
size_t x_smem_n(int nbins, int nwb, int ell) {
  return ell == 6 ? XCombine<N, 6, 2>::smem(nbins, nwb) : XCombine<N, 4, 2>::smem(nbins, nwb);
}

template <int N, int ELL>
cudaError_t run_ell(Plan* const* lanes, int W) {
  cudaError_t err;
  if (lanes[0]->np > 0) {
    if ((err = run_yz<N, ELL>(lanes, W))) return err;
    if ((err = (lanes[0]->m == 2 ? run_x<N, ELL, 2>(lanes, W) : run_x<N, ELL, 1>(lanes, W)))) return err;
  }
  return cudaSuccess;
}

// Measurement of W lanes of one configuration; lane l's result row goes to rows[l].
template <int N>
cudaError_t run_measure_n(Plan* const* lanes, int W, double* const* rows) {
  cudaError_t err;
  Plan& p0 = *lanes[0];
  for (int l = 0; l < W; ++l)
    if ((err = cudaMemsetAsync(lanes[l]->d_acc, 0, sizeof(double) * 4 * p0.cfg.n_bins, p0.stream))) return err;
  switch (p0.ell) {
    case 0: err = run_ell<N, 0>(lanes, W); break;
    case 2: err = run_ell<N, 2>(lanes, W); break;
    case 4: err = run_ell<N, 4>(lanes, W); break;
    case 6:
      if constexpr (ell6_supported<N>()) {
        err = run_ell<N, 6>(lanes, W);
        break;
      }
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
  if (err) return err;
  return launch_finalize(lanes, W, rows);
}

}  // namespace ys
