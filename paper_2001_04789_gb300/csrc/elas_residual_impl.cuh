// Launcher of the residual kernel (one launch covers edges, faces and interior),
// instantiated per precision in elas_residual.cu (FP32) and elas_residual_f64.cu.
#pragma once
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
    // FP64 levels of general moduli carry the precomputed divergence; FP32 levels read
    // their moduli as FP32 blocks or FP16 records
    if constexpr (sizeof(T) == 8) {
        if (L.K == 21 && L.divc) {
            if (partials) k_residual<T, TR, 21, true, true, kMlDefault><<<nb, kBlock, 0, s>>>(L, u, f, nfv, lam, r, partials, sg);
            else k_residual<T, TR, 21, false, true, kMlDefault><<<nb, kBlock, 0, s>>>(L, u, f, nfv, lam, r, nullptr, sg);
            return;
        }
    }
    if constexpr (sizeof(T) == 4) {
        if (L.K == 21 && L.mlay == kModSplit) {
            // colour-split records with the divergence
            if (partials) k_residual<T, TR, 21, true, true, kMlSplit><<<nb, kBlock, 0, s>>>(L, u, f, nfv, lam, r, partials, sg);
            else k_residual<T, TR, 21, false, true, kMlSplit><<<nb, kBlock, 0, s>>>(L, u, f, nfv, lam, r, nullptr, sg);
            return;
        }
    }
    if (L.modh) {
        if (partials) {
            if (L.K == 2) k_residual<T, TR, 2, true, false, kMlHalf><<<nb, kBlock, 0, s>>>(L, u, f, nfv, lam, r, partials, sg);
            else k_residual<T, TR, 21, true, false, kMlHalf><<<nb, kBlock, 0, s>>>(L, u, f, nfv, lam, r, partials, sg);
        } else {
            if (L.K == 2) k_residual<T, TR, 2, false, false, kMlHalf><<<nb, kBlock, 0, s>>>(L, u, f, nfv, lam, r, nullptr, sg);
            else k_residual<T, TR, 21, false, false, kMlHalf><<<nb, kBlock, 0, s>>>(L, u, f, nfv, lam, r, nullptr, sg);
        }
    } else {
        if (partials) {
            if (L.K == 2) k_residual<T, TR, 2, true, false, kMlDefault><<<nb, kBlock, 0, s>>>(L, u, f, nfv, lam, r, partials, sg);
            else k_residual<T, TR, 21, true, false, kMlDefault><<<nb, kBlock, 0, s>>>(L, u, f, nfv, lam, r, partials, sg);
        } else {
            if (L.K == 2) k_residual<T, TR, 2, false, false, kMlDefault><<<nb, kBlock, 0, s>>>(L, u, f, nfv, lam, r, nullptr, sg);
            else k_residual<T, TR, 21, false, false, kMlDefault><<<nb, kBlock, 0, s>>>(L, u, f, nfv, lam, r, nullptr, sg);
        }
    }
}

}  // namespace elas
