// Red-black smoother launchers and autotuner, FP32 levels.  The kernel instances compile
// in the companion units: FP16-moduli shapes (elas_sweep_f32_h.cu), isotropic moduli
// (elas_sweep_f32_iso.cu), colour-split moduli (elas_sweep_f32_split.cu) and the
// shared-memory tiled kernel (elas_sweep_f32_tiled.cu).
#include "elas_sweep_impl.cuh"

namespace elas {

extern template void sweep_int_variant<float, 2, false, kMlDefault>(int, size_t, const Lv<float>&, const float*, float*, const float*, int,
                                                const NullInfo&, const double*, cudaStream_t);
extern template void sweep_int_variant<float, 2, false, kMlHalf>(int, size_t, const Lv<float>&, const float*, float*, const float*, int,
                                                const NullInfo&, const double*, cudaStream_t);
extern template void sweep_int_variant<float, 21, false, kMlHalf>(int, size_t, const Lv<float>&, const float*, float*, const float*, int,
                                                const NullInfo&, const double*, cudaStream_t);
extern template void sweep_int_variant<float, 21, true, kMlSplit>(int, size_t, const Lv<float>&, const float*, float*, const float*, int,
                                                const NullInfo&, const double*, cudaStream_t);
extern template void launch_tiled<21, 16>(const Lv<float>&, const float*, float*, const float*, int, const NullInfo&, const double*,
                                  cudaStream_t);
extern template void launch_tiled<21, 8>(const Lv<float>&, const float*, float*, const float*, int, const NullInfo&, const double*,
                                  cudaStream_t);
extern template void launch_tiled<2, 16>(const Lv<float>&, const float*, float*, const float*, int, const NullInfo&, const double*,
                                  cudaStream_t);
extern template void launch_tiled<2, 8>(const Lv<float>&, const float*, float*, const float*, int, const NullInfo&, const double*,
                                  cudaStream_t);

template int tune_sweep<float>(const Lv<float>&, const float*, float*, const float*, cudaStream_t, float*);
template void launch_half_sweep<float>(const Lv<float>&, const float*, float*, const float*, int, const NullInfo*,
                                       const double*, cudaStream_t);

}  // namespace elas
