// Spectral kernels instantiated for mesh sizes: 16 32 64 96
#include "measure_impl.cuh"
namespace ys {
template cudaError_t run_measure_n<16>(Plan* const*, int, double* const*);
template int yz_grid_n<16>(int, cudaError_t*);
template size_t x_smem_n<16>(int, int, int);
template cudaError_t run_measure_n<32>(Plan* const*, int, double* const*);
template int yz_grid_n<32>(int, cudaError_t*);
template size_t x_smem_n<32>(int, int, int);
template cudaError_t run_measure_n<64>(Plan* const*, int, double* const*);
template int yz_grid_n<64>(int, cudaError_t*);
template size_t x_smem_n<64>(int, int, int);
template cudaError_t run_measure_n<96>(Plan* const*, int, double* const*);
template int yz_grid_n<96>(int, cudaError_t*);
template size_t x_smem_n<96>(int, int, int);
}  // namespace ys
