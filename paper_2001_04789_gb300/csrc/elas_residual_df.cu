// Double-float refinement residual of a mixed solve (kernels in elas_kernels.cuh) and
// the splits that keep its double-float inputs in step with the FP64 fields.
#include <algorithm>

#include "elas_kernels.cuh"

namespace elas {
namespace {

__global__ void k_split_df(const double* __restrict__ a, dfloat* __restrict__ out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = df_split(a[i]);
}

__global__ void k_add_correction_df(Lv<double> L, double* __restrict__ u, const float* __restrict__ e,
                                    dfloat* __restrict__ u2) {
    if (L.active && *L.active == 0) return;
    add_correction_df_body<float>(L, u, e, u2, blockIdx.x * blockDim.x + threadIdx.x);
}

}  // namespace

int residual_df_block_count(const Lv<dfloat>& L) { return residual_df_blocks<kDfNodesPerThread>(L); }

void launch_residual_df(const Lv<dfloat>& L, const dfloat* u, const dfloat* f, const NullInfo* nf, const double* lam,
                        float* r, double* partials, int* nblocks, cudaStream_t s) {
    NullInfo nfv{};
    if (nf) nfv = *nf;
    const int nb = residual_df_block_count(L);
    if (nblocks) *nblocks = nb;
    if (!nb) return;
    count_launch();
    constexpr int P = kDfNodesPerThread;
    if (L.K == 21 && L.divc) k_residual_df<21, true, true, P><<<nb, kBlock, 0, s>>>(L, u, f, nfv, lam, r, partials);
    else if (L.K == 21) k_residual_df<21, true, false, P><<<nb, kBlock, 0, s>>>(L, u, f, nfv, lam, r, partials);
    else k_residual_df<2, true, false, P><<<nb, kBlock, 0, s>>>(L, u, f, nfv, lam, r, partials);
}

void launch_split_df(const double* a, dfloat* out, size_t n, cudaStream_t s) {
    if (!n) return;
    count_launch();
    const size_t want = (n + kBlock - 1) / kBlock;
    const int nb = (int)std::min<size_t>(want, (size_t)152 * 16);
    k_split_df<<<nb, kBlock, 0, s>>>(a, out, n);
}

void launch_add_correction_df(const Lv<double>& L, double* u, const float* e, dfloat* u2, cudaStream_t s) {
    count_launch();
    k_add_correction_df<<<blocks_for(L.N), kBlock, 0, s>>>(L, u, e, u2);
}

}  // namespace elas
