// Shared-memory tiled smoother kernels (FP32 levels, blocked FP32 moduli).
#include "elas_sweep_impl.cuh"

namespace elas {

template void launch_tiled<21, 16>(const Lv<float>&, const float*, float*, const float*, int, const NullInfo&, const double*,
                                  cudaStream_t);
template void launch_tiled<21, 8>(const Lv<float>&, const float*, float*, const float*, int, const NullInfo&, const double*,
                                  cudaStream_t);
template void launch_tiled<2, 16>(const Lv<float>&, const float*, float*, const float*, int, const NullInfo&, const double*,
                                  cudaStream_t);
template void launch_tiled<2, 8>(const Lv<float>&, const float*, float*, const float*, int, const NullInfo&, const double*,
                                  cudaStream_t);

}  // namespace elas
