// Red-black smoother kernels of FP32 levels that read FP16 moduli records.
#include "elas_sweep_impl.cuh"

namespace elas {

template void sweep_int_variant<float, 2, false, kMlHalf>(int, size_t, const Lv<float>&, const float*, float*, const float*, int,
                                                const NullInfo&, const double*, cudaStream_t);
template void sweep_int_variant<float, 21, false, kMlHalf>(int, size_t, const Lv<float>&, const float*, float*, const float*, int,
                                                const NullInfo&, const double*, cudaStream_t);

}  // namespace elas
