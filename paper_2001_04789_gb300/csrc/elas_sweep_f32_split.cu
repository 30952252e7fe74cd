// Red-black smoother kernels of FP32 levels whose general moduli are stored colour-split
// with the modulus divergence (centre records only), compiled apart so that the
// smoother's units build in parallel.
#include "elas_sweep_impl.cuh"

namespace elas {

template void sweep_int_variant<float, 21, true, kMlSplit>(int, size_t, const Lv<float>&, const float*, float*, const float*, int,
                                                const NullInfo&, const double*, cudaStream_t);

}  // namespace elas
