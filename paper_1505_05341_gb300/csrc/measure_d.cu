// Spectral kernels instantiated for mesh sizes: 512
#include "measure_impl.cuh"
namespace ys {
template cudaError_t run_measure_n<512>(Plan&);
}  // namespace ys
