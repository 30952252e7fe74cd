// Red-black smoother launchers and autotuner, FP32 levels.
#include "elas_sweep_impl.cuh"

namespace elas {

template int tune_sweep<float>(const Lv<float>&, const float*, float*, const float*, cudaStream_t, float*);
template void launch_half_sweep<float>(const Lv<float>&, const float*, float*, const float*, int, const NullInfo*,
                                       const double*, cudaStream_t);

}  // namespace elas
