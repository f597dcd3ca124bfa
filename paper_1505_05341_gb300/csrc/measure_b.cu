// Spectral kernels instantiated for mesh sizes: 128 192
#include "measure_impl.cuh"
namespace ys {
template cudaError_t run_measure_n<128>(Plan* const*, int, double* const*);
template int yz_grid_n<128>(int, cudaError_t*);
template size_t x_smem_n<128>(int, int, int);
template cudaError_t run_measure_n<192>(Plan* const*, int, double* const*);
template int yz_grid_n<192>(int, cudaError_t*);
template size_t x_smem_n<192>(int, int, int);
}  // namespace ys
