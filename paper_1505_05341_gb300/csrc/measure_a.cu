// Spectral kernels instantiated for mesh sizes: 16 32 64 96
#include "measure_impl.cuh"
namespace ys {
template cudaError_t run_measure_n<16>(Plan&);
template cudaError_t run_measure_n<32>(Plan&);
template cudaError_t run_measure_n<64>(Plan&);
template cudaError_t run_measure_n<96>(Plan&);
}  // namespace ys
