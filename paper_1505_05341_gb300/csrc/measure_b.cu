// Spectral kernels instantiated for mesh sizes: 128 192
#include "measure_impl.cuh"
namespace ys {
template cudaError_t run_measure_n<128>(Plan&);
template cudaError_t run_measure_n<192>(Plan&);
}  // namespace ys
