// Power-spectrum wedges from the multipoles (Sec. 5, Eqs. 16-17): the moments of the
// estimator with top hats 0 <= mu <= 1/2 (P_perp) and 1/2 < mu <= 1 (P_para) in
// place of the Legendre weight, approximated by the first three even multipoles,
//   P_perp = P_0 - 3/8 P_2 + 15/128 P_4,   P_para = P_0 + 3/8 P_2 - 15/128 P_4.
// An epilogue on result rows in the layout of ys_measure_multipoles_async.
#include <cuda_runtime.h>

#include "ys_internal.h"

namespace ys {
namespace {

__global__ void k_wedges(const double* __restrict__ rows, int n_cat, int64_t stride, int n_bins,
                         double* __restrict__ out) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n_cat * n_bins) return;
  const int c = (int)(idx / n_bins), b = (int)(idx % n_bins);
  const double* row = rows + (size_t)c * stride;
  const double p0 = row[2 * n_bins + b], p2 = row[3 * n_bins + b], p4 = row[4 * n_bins + b];
  double* o = out + (size_t)c * 2 * n_bins;
  o[b] = p0 - 0.375 * p2 + 0.1171875 * p4;
  o[n_bins + b] = p0 + 0.375 * p2 - 0.1171875 * p4;
}

}  // namespace
}  // namespace ys

extern "C" ys_status ys_wedges(const double* d_rows, int32_t n_cat, int64_t stride, int32_t n_bins, double* d_out,
                               void* stream) {
  if (!d_rows || !d_out || n_cat <= 0 || n_bins <= 0 || stride < 5 * (int64_t)n_bins + 5) return YS_ERR_ARG;
  const int64_t total = (int64_t)n_cat * n_bins;
  ys::k_wedges<<<(unsigned)((total + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(d_rows, n_cat, stride,
                                                                                              n_bins, d_out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    ys::g_last_cuda_error = cudaGetErrorString(e);
    return YS_ERR_CUDA;
  }
  return YS_OK;
}
