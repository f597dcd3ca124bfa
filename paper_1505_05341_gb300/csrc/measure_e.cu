// Spectral kernels instantiated for mesh sizes: 768 1024
#include "measure_impl.cuh"
namespace ys {
template cudaError_t run_measure_n<768>(Plan* const*, int, double* const*);
template int yz_grid_n<768>(int, cudaError_t*);
template size_t x_smem_n<768>(int, int, int);
template cudaError_t run_measure_n<1024>(Plan* const*, int, double* const*);
template int yz_grid_n<1024>(int, cudaError_t*);
template size_t x_smem_n<1024>(int, int, int);
}  // namespace ys
