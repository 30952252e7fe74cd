// Batched engine: one launch per phase of a multigrid cycle covers every member of a
// batch of grids.  A phase's tasks (one per member taking part) and its block map (the
// task and the block within it, for every block of the launch) live in device memory;
// each block loads its task into shared memory and runs the same per-node code as the
// single-grid kernels on that member's level, with the member's own block partition, so
// each member's result is identical to its lone solve.
// Converged members (their active flag cleared on the device) skip their blocks.
#include "elas_kernels.cuh"

namespace elas {
namespace {

constexpr int kBatchBlock = 256;

__device__ __forceinline__ bool inactive(const int* a) { return a && *a == 0; }

// The block's task, copied into shared memory by the whole block (so that the level's
// fields are read at shared-memory latency), and the block's index within its task,
// both from the phase's block map (one (task, local block) pair per block).
template <typename Task>
__device__ __forceinline__ int load_task(const Task* __restrict__ tasks, const int2* __restrict__ bmap, Task& dst) {
    const int2 m = bmap[blockIdx.x];
    const int* src = reinterpret_cast<const int*>(tasks + m.x);
    int* d = reinterpret_cast<int*>(&dst);
    for (int k = threadIdx.x; k < (int)(sizeof(Task) / sizeof(int)); k += blockDim.x) d[k] = src[k];
    __syncthreads();
    return m.y;
}

template <int KIND, bool HM, int ML>
__global__ void __launch_bounds__(kBatchBlock, 3)
    k_batch_sweep(const SweepTask<float>* __restrict__ tasks, const int2* __restrict__ bmap, int colour) {
    __shared__ __align__(16) SweepTask<float> t;
    const int b = load_task(tasks, bmap, t), tid = threadIdx.x;
    const Lv<float>& L = t.L;
    if (inactive(L.active)) return;
    const BndSegs sg = bnd_segs(L, kBatchBlock);
    if (b < sg.f2) {
        if (b < sg.e) sweep_bnd_body<float, KIND>(L, t.u, t.uo, t.f, colour, t.nf, t.lam, (b * kBatchBlock + tid) >> 5, tid & 31);
        else if (b < sg.f0) sweep_face_body<float, KIND, 0>(L, t.u, t.uo, t.f, colour, t.nf, t.lam, (b - sg.e) * kBatchBlock + tid);
        else if (b < sg.f1) sweep_face_body<float, KIND, 1>(L, t.u, t.uo, t.f, colour, t.nf, t.lam, (b - sg.f0) * kBatchBlock + tid);
        else sweep_face_body<float, KIND, 2>(L, t.u, t.uo, t.f, colour, t.nf, t.lam, (b - sg.f1) * kBatchBlock + tid);
        return;
    }
    sweep_pair_body<float, KIND, HM, ML>(L, t.u, t.uo, t.f, colour, t.nf, t.lam, (b - sg.f2) * kBatchBlock + tid);
}

template <typename T, typename TR, int KIND, bool NORM, bool HM, int ML>
__global__ void __launch_bounds__(kBatchBlock, sizeof(T) == 4 ? 4 : 2)
    k_batch_resid(const ResidTask<T, TR>* __restrict__ tasks, const int2* __restrict__ bmap) {
    __shared__ __align__(16) ResidTask<T, TR> t;
    const int b = load_task(tasks, bmap, t), tid = threadIdx.x;
    const Lv<T>& L = t.L;
    if (inactive(L.active)) return;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const BndSegs sg = bnd_segs(L, kBlock);
    if (b < sg.e) residual_bnd_body<T, TR, KIND, NORM>(L, t.u, t.f, t.nf, t.lam, t.r, (b * kBlock + tid) >> 5, tid & 31, acc);
    else if (b < sg.f0) residual_face_body<T, TR, KIND, 0, NORM>(L, t.u, t.f, t.nf, t.lam, t.r, (b - sg.e) * kBlock + tid, acc);
    else if (b < sg.f1) residual_face_body<T, TR, KIND, 1, NORM>(L, t.u, t.f, t.nf, t.lam, t.r, (b - sg.f0) * kBlock + tid, acc);
    else if (b < sg.f2) residual_face_body<T, TR, KIND, 2, NORM>(L, t.u, t.f, t.nf, t.lam, t.r, (b - sg.f1) * kBlock + tid, acc);
    else residual_int_body<T, TR, KIND, NORM, HM, ML>(L, t.u, t.f, t.nf, t.lam, t.r, (b - sg.f2) * kBlock + tid, acc);
    if (NORM) block_reduce_norms_at(acc, t.nf.m > 0 ? 7 : 1, t.partials, b);
}

__global__ void k_batch_restrict(const RestrictTask<float>* __restrict__ tasks, const int2* __restrict__ bmap) {
    __shared__ __align__(16) RestrictTask<float> t;
    const int b = load_task(tasks, bmap, t);
    if (inactive(t.Lf.active)) return;
    restrict_body<float>(t.Lf, t.Lc, t.r, t.fc, t.nf, t.dlam, b * kBlock + threadIdx.x);
}

__global__ void k_batch_prolong(const ProlongTask<float>* __restrict__ tasks, const int2* __restrict__ bmap) {
    __shared__ __align__(16) ProlongTask<float> t;
    const int b = load_task(tasks, bmap, t);
    if (inactive(t.Lf.active)) return;
    prolong_body<float>(t.Lf, t.Lc, t.ec, t.u, b * kBlock + threadIdx.x);
}

__global__ void k_batch_zero(const ZeroTask<float>* __restrict__ tasks, const int2* __restrict__ bmap) {
    const int2 m = bmap[blockIdx.x];
    const ZeroTask<float>& t = tasks[m.x];
    if (inactive(t.active)) return;
    const size_t k = (size_t)m.y * kBlock + threadIdx.x;
    if (k < t.n) t.a[k] = 0.f;
}

__global__ void k_batch_gather(const BottomTask<float>* __restrict__ tasks, const int2* __restrict__ bmap) {
    const int2 m = bmap[blockIdx.x];
    const BottomTask<float>& t = tasks[m.x];
    if (inactive(t.L.active)) return;
    const int k = m.y * kBlock + threadIdx.x;
    if (k < t.ntot) t.work[k] = k < t.nfree ? (double)t.f[t.dofs[k]] : 0.0;
}

__global__ void k_batch_matvec(const BottomTask<float>* __restrict__ tasks, const int2* __restrict__ bmap) {
    const int2 m = bmap[blockIdx.x];
    const BottomTask<float>& t = tasks[m.x];
    if (inactive(t.L.active)) return;
    bottom_matvec_body<float>(t.dofs, t.nfree, t.ntot, t.Ainv, t.work, t.u, m.y);
}

__global__ void k_batch_finalize(const FinalizeTask* __restrict__ tasks, int n) {
    const FinalizeTask& t = tasks[blockIdx.x];
    if (inactive(t.bf.active)) return;
    finalize_body(t.partials, t.nblocks, t.nf, t.Ginv, t.G, t.lam, t.dlam, t.alam, t.adlam, t.out, 1, t.bf);
}

__global__ void k_batch_corr(const CorrTask* __restrict__ tasks, const int2* __restrict__ bmap) {
    __shared__ __align__(16) CorrTask t;
    const int b = load_task(tasks, bmap, t);
    if (inactive(t.L.active)) return;
    if (t.u2) add_correction_df_body<float>(t.L, t.u, t.e, t.u2, b * kBlock + threadIdx.x);
    else add_correction_body<float>(t.L, t.u, t.e, b * kBlock + threadIdx.x);
}

template <int KIND, bool HM>
__global__ void __launch_bounds__(kBlock, 2)
    k_batch_resid_df(const ResidTask<dfloat, float>* __restrict__ tasks, const int2* __restrict__ bmap) {
    __shared__ __align__(16) ResidTask<dfloat, float> t;
    const int b = load_task(tasks, bmap, t);
    if (inactive(t.L.active)) return;
    residual_df_block<KIND, true, HM, kDfNodesPerThread>(t.L, t.u, t.f, t.nf, t.lam, t.r, t.partials, b);
}

template <int KIND, bool HM, int ML>
void sweep_launch(const BatchPhase& ph, cudaStream_t s) {
    k_batch_sweep<KIND, HM, ML><<<ph.blocks, kBatchBlock, 0, s>>>((const SweepTask<float>*)ph.tasks, ph.bmap, ph.colour);
}

template <typename T, typename TR, bool NORM>
void resid_launch(const BatchPhase& ph, cudaStream_t s) {
    const auto* t = (const ResidTask<T, TR>*)ph.tasks;
    if (sizeof(T) == 8) {
        if (ph.K == 21) k_batch_resid<T, TR, 21, NORM, true, kMlDefault><<<ph.blocks, kBlock, 0, s>>>(t, ph.bmap);
        else k_batch_resid<T, TR, 2, NORM, false, kMlDefault><<<ph.blocks, kBlock, 0, s>>>(t, ph.bmap);
    } else if (ph.ml == kMlSplit) {
        k_batch_resid<T, TR, 21, NORM, true, kMlSplit><<<ph.blocks, kBlock, 0, s>>>(t, ph.bmap);
    } else if (ph.K == 21) {
        k_batch_resid<T, TR, 21, NORM, false, kMlDefault><<<ph.blocks, kBlock, 0, s>>>(t, ph.bmap);
    } else {
        k_batch_resid<T, TR, 2, NORM, false, kMlDefault><<<ph.blocks, kBlock, 0, s>>>(t, ph.bmap);
    }
}

}  // namespace

int batch_task_blocks(int kind, const void* task) {
    auto nb = [](size_t n, int bs) { return (int)((n + bs - 1) / bs); };
    switch (kind) {
        case kPhaseSweep: {
            const auto& t = *(const SweepTask<float>*)task;
            return bnd_segs(t.L, kBatchBlock).f2 + nb(interior_pairs(t.L), kBatchBlock);
        }
        case kPhaseResid32: {
            const auto& t = *(const ResidTask<float, float>*)task;
            return bnd_segs(t.L, kBlock).f2 + nb(interior_count(t.L), kBlock);
        }
        case kPhaseResid64: {
            const auto& t = *(const ResidTask<double, float>*)task;
            return bnd_segs(t.L, kBlock).f2 + nb(interior_count(t.L), kBlock);
        }
        case kPhaseResidDf: return residual_df_blocks<kDfNodesPerThread>(((const ResidTask<dfloat, float>*)task)->L);
        case kPhaseRestrict: return nb(((const RestrictTask<float>*)task)->Lc.N, kBlock);
        case kPhaseProlong: return nb(((const ProlongTask<float>*)task)->Lf.N, kBlock);
        case kPhaseZero: return nb(((const ZeroTask<float>*)task)->n, kBlock);
        case kPhaseGather: return nb(((const BottomTask<float>*)task)->ntot, kBlock);
        case kPhaseMatvec: return ((const BottomTask<float>*)task)->nfree;
        case kPhaseFinalize: return 1;
        case kPhaseCorr: return nb(((const CorrTask*)task)->L.N, kBlock);
    }
    return 0;
}

void batch_phase_launch(const BatchPhase& ph, cudaStream_t s) {
    if (ph.n <= 0 || ph.blocks <= 0) return;
    count_launch();
    switch (ph.kind) {
        case kPhaseSweep:
            if (ph.ml == kMlSplit) sweep_launch<21, true, kMlSplit>(ph, s);
            else if (ph.K == 21) sweep_launch<21, false, kMlDefault>(ph, s);
            else sweep_launch<2, false, kMlDefault>(ph, s);
            break;
        case kPhaseResid32: resid_launch<float, float, false>(ph, s); break;
        case kPhaseResid64: resid_launch<double, float, true>(ph, s); break;
        case kPhaseResidDf: {
            const auto* t = (const ResidTask<dfloat, float>*)ph.tasks;
            if (ph.K == 21) k_batch_resid_df<21, true><<<ph.blocks, kBlock, 0, s>>>(t, ph.bmap);
            else k_batch_resid_df<2, false><<<ph.blocks, kBlock, 0, s>>>(t, ph.bmap);
            break;
        }
        case kPhaseRestrict: k_batch_restrict<<<ph.blocks, kBlock, 0, s>>>((const RestrictTask<float>*)ph.tasks, ph.bmap); break;
        case kPhaseProlong: k_batch_prolong<<<ph.blocks, kBlock, 0, s>>>((const ProlongTask<float>*)ph.tasks, ph.bmap); break;
        case kPhaseZero: k_batch_zero<<<ph.blocks, kBlock, 0, s>>>((const ZeroTask<float>*)ph.tasks, ph.bmap); break;
        case kPhaseGather: k_batch_gather<<<ph.blocks, kBlock, 0, s>>>((const BottomTask<float>*)ph.tasks, ph.bmap); break;
        case kPhaseMatvec: k_batch_matvec<<<ph.blocks, kBlock, 0, s>>>((const BottomTask<float>*)ph.tasks, ph.bmap); break;
        case kPhaseFinalize: k_batch_finalize<<<ph.n, kSumThreads, 0, s>>>((const FinalizeTask*)ph.tasks, ph.n); break;
        case kPhaseCorr: k_batch_corr<<<ph.blocks, kBlock, 0, s>>>((const CorrTask*)ph.tasks, ph.bmap); break;
    }
}

}  // namespace elas
