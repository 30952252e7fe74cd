// Launcher of the residual kernel (one launch covers edges, faces and interior).
#include "elas_kernels.cuh"

namespace elas {

template <typename T, typename TR>
void launch_residual(const Lv<T>& L, const T* u, const T* f, const NullInfo* nf, const double* lam, TR* r,
                     double* partials, int* nblocks, cudaStream_t s) {
    NullInfo nfv{};
    if (nf) nfv = *nf;
    const BndSegs sg = bnd_segs(L, kBlock);
    const int nb = sg.f2 + blocks_for(interior_count(L));
    if (nblocks) *nblocks = nb;
    if (!nb) return;
    count_launch();
    if (partials) {
        if (L.K == 2) k_residual<T, TR, 2, true, false><<<nb, kBlock, 0, s>>>(L, u, f, nfv, lam, r, partials, sg);
        else if (L.divc) k_residual<T, TR, 21, true, true><<<nb, kBlock, 0, s>>>(L, u, f, nfv, lam, r, partials, sg);
        else k_residual<T, TR, 21, true, false><<<nb, kBlock, 0, s>>>(L, u, f, nfv, lam, r, partials, sg);
    } else {
        if (L.K == 2) k_residual<T, TR, 2, false, false><<<nb, kBlock, 0, s>>>(L, u, f, nfv, lam, r, nullptr, sg);
        else if (L.divc) k_residual<T, TR, 21, false, true><<<nb, kBlock, 0, s>>>(L, u, f, nfv, lam, r, nullptr, sg);
        else k_residual<T, TR, 21, false, false><<<nb, kBlock, 0, s>>>(L, u, f, nfv, lam, r, nullptr, sg);
    }
}

template void launch_residual<double, double>(const Lv<double>&, const double*, const double*, const NullInfo*,
                                              const double*, double*, double*, int*, cudaStream_t);
template void launch_residual<double, float>(const Lv<double>&, const double*, const double*, const NullInfo*,
                                             const double*, float*, double*, int*, cudaStream_t);
template void launch_residual<float, float>(const Lv<float>&, const float*, const float*, const NullInfo*,
                                            const double*, float*, double*, int*, cudaStream_t);

}  // namespace elas
