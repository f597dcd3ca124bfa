// Spectral kernels instantiated for mesh sizes: 256 384
#include "measure_impl.cuh"
namespace ys {
template cudaError_t run_measure_n<256>(Plan* const*, int, double* const*);
template int yz_grid_n<256>(int, cudaError_t*);
template size_t x_smem_n<256>(int, int, int);
template cudaError_t run_measure_n<384>(Plan* const*, int, double* const*);
template int yz_grid_n<384>(int, cudaError_t*);
template size_t x_smem_n<384>(int, int, int);
}  // namespace ys
