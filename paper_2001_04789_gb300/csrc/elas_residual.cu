// Residual launcher, FP32 levels.
#include "elas_residual_impl.cuh"

namespace elas {

template void launch_residual<float, float>(const Lv<float>&, const float*, const float*, const NullInfo*,
                                            const double*, float*, double*, int*, cudaStream_t);

}  // namespace elas
