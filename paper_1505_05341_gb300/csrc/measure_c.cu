// Spectral kernels instantiated for mesh sizes: 256 384
#include "measure_impl.cuh"
namespace ys {
template cudaError_t run_measure_n<256>(Plan&);
template cudaError_t run_measure_n<384>(Plan&);
}  // namespace ys
