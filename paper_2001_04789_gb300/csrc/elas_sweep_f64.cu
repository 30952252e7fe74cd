// Red-black smoother launchers and autotuner, FP64 levels.
#include "elas_sweep_impl.cuh"

namespace elas {

template int tune_sweep<double>(const Lv<double>&, const double*, double*, const double*, cudaStream_t, float*);
template void launch_half_sweep<double>(const Lv<double>&, const double*, double*, const double*, int, const NullInfo*,
                                       const double*, cudaStream_t);

}  // namespace elas
