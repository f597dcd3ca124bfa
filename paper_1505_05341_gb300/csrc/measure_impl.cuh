// Host-side launch sequence of the spectral steps for one mesh size N (one
// translation unit per N instantiates it, so the sizes compile in parallel).
#pragma once
#include <algorithm>

#include "spectra.cuh"

namespace ys {

cudaError_t launch_finalize(Plan& p);

template <int N, int ELL>
cudaError_t run_yz(Plan& p) {
  using T = GroupTable<ELL>;
  cudaStream_t st = p.stream;
  cudaError_t err;
  const size_t smem_rows = sizeof(float2) * N + sizeof(float2) * KZ_ROWS * (N + 1) + sizeof(float) * KZ_ROWS * N;
  const int kc = std::max(1, std::min(p.nzc, (int)(98304 / (T::NB * (N + 1) * sizeof(float2)))));
  const size_t smem_cols = sizeof(float2) * N + sizeof(float2) * T::NB * kc * (N + 1);
  if ((err = cudaFuncSetAttribute(k_yz_rows<N, ELL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_rows)))
    return err;
  if ((err = cudaFuncSetAttribute(k_yz_cols<N, ELL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cols)))
    return err;
  const size_t n3 = (size_t)N * N * N;
  for (int mj = 0; mj < p.m; ++mj) {
    const float* rel = p.d_rel + (size_t)mj * 3 * N;
    for (int ix0 = 0; ix0 < N; ix0 += p.batch) {
      const int nb = std::min(p.batch, N - ix0);
      {
        LaunchScope ls(p, 4);
        k_yz_rows<N, ELL><<<dim3(N / KZ_ROWS, nb), KZ_THREADS, smem_rows, st>>>(
          p.d_mesh + mj * n3, ix0, rel, rel + N, rel + 2 * N, p.d_tw, p.d_z, p.nzc, p.batch);
        if ((err = cudaGetLastError())) return err;
      }
      LaunchScope ls(p, 5);
      k_yz_cols<N, ELL><<<dim3((p.nzc + kc - 1) / kc, nb), KY_THREADS, smem_cols, st>>>(
          p.d_z, ix0, p.nzc, p.batch, kc, p.d_col_off, p.d_tw, p.d_g, mj, p.np);
      if ((err = cudaGetLastError())) return err;
    }
  }
  return cudaSuccess;
}

template <int N, int ELL, int M>
cudaError_t run_x(Plan& p) {
  using XC = XCombine<N, ELL, M>;
  const int nbins = p.cfg.n_bins;
  const size_t smem = x_combine_smem<N, ELL, M>(nbins);
  cudaError_t err;
  if ((err = cudaFuncSetAttribute(k_x_combine<N, ELL, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
    return err;
  const int npb = (p.np + XC::P - 1) / XC::P;
  const int grid = std::max(1, std::min(npb, 152 * 4));
  LaunchScope ls(p, 6);
  k_x_combine<N, ELL, M><<<grid, XC::THREADS, smem, p.stream>>>(p.d_g, p.np, p.d_pencil, p.d_tw, p.d_invw,
                                                                 p.d_phase, p.d_lut, p.n2_hi, p.d_acc, nbins);
  return cudaGetLastError();
}

template <int N, int ELL>
cudaError_t run_ell(Plan& p) {
  cudaError_t err;
  if (p.np > 0) {
    if ((err = run_yz<N, ELL>(p))) return err;
    if ((err = (p.m == 2 ? run_x<N, ELL, 2>(p) : run_x<N, ELL, 1>(p)))) return err;
  }
  return cudaSuccess;
}

template <int N>
cudaError_t run_measure_n(Plan& p) {
  cudaError_t err;
  if ((err = cudaMemsetAsync(p.d_acc, 0, sizeof(double) * 3 * p.cfg.n_bins, p.stream))) return err;
  switch (p.ell) {
    case 0: err = run_ell<N, 0>(p); break;
    case 2: err = run_ell<N, 2>(p); break;
    case 4: err = run_ell<N, 4>(p); break;
    default: return cudaErrorInvalidValue;
  }
  if (err) return err;
  return launch_finalize(p);
}

}  // namespace ys
