// Spectral kernels instantiated for mesh sizes: 512
#include "measure_impl.cuh"
namespace ys {
template cudaError_t run_measure_n<512>(Plan* const*, int, double* const*);
template int yz_grid_n<512>(int, cudaError_t*);
template size_t x_smem_n<512>(int, int, int);
}  // namespace ys
