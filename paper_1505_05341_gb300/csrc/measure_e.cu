// Spectral kernels instantiated for mesh sizes: 768 1024
#include "measure_impl.cuh"
namespace ys {
template cudaError_t run_measure_n<768>(Plan&);
template cudaError_t run_measure_n<1024>(Plan&);
}  // namespace ys
