// Red-black smoother kernels of FP32 levels with isotropic moduli (lambda, mu), compiled
// apart so that the smoother's units build in parallel.
#include "elas_sweep_impl.cuh"

namespace elas {

extern template void launch_tiled<2, 16>(const Lv<float>&, const float*, float*, const float*, int, const NullInfo&, const double*,
                                  cudaStream_t);
extern template void launch_tiled<2, 8>(const Lv<float>&, const float*, float*, const float*, int, const NullInfo&, const double*,
                                  cudaStream_t);
template void sweep_int_variant<float, 2, false, kMlDefault>(int, size_t, const Lv<float>&, const float*, float*, const float*, int,
                                                const NullInfo&, const double*, cudaStream_t);

}  // namespace elas
