// Residual launcher, FP64 levels (the refinement's residual writes FP64 or FP32).
#include "elas_residual_impl.cuh"

namespace elas {

template void launch_residual<double, double>(const Lv<double>&, const double*, const double*, const NullInfo*,
                                              const double*, double*, double*, int*, cudaStream_t);
template void launch_residual<double, float>(const Lv<double>&, const double*, const double*, const NullInfo*,
                                             const double*, float*, double*, int*, cudaStream_t);

}  // namespace elas
