// Launch shapes of the red-black smoother, their autotuner and the half-sweep launcher.
// Instantiated per precision (elas_sweep_f32.cu, elas_sweep_f64.cu); the FP32 isotropic
// instances compile in elas_sweep_f32_iso.cu.
#pragma once
#include <array>

#include "elas_kernels.cuh"

namespace elas {

// ---- launch variants of the interior smoother and their tuning table -----------------
// (threads per block, minimum resident blocks per SM) pairs; the second number
// bounds the registers per thread and so trades registers for resident warps.
// Variants 5 and 6 are the shared-memory tiled kernel (32 x 16 and 32 x 8 tiles, FP32
// levels with blocked FP32 moduli only); 7 and 8 the z-marching tiled kernel of
// colour-split levels (32 x 16 and 32 x 8 tiles, displacement staged); their pair holds
// (threads, resident blocks per SM).
static const int kSweepVariants[kNumSweepVariants][2] = {{256, 1}, {256, 2}, {256, 3}, {256, 4}, {128, 8},
                                                         {256, 1}, {128, 2}, {256, 1}, {128, 3}};
constexpr int kFirstTiledVariant = 5;
constexpr int kFirstSplitTiledVariant = 7;

// Tuning key: level dimensions, moduli kind, precision and the moduli source (1: FP64
// levels with the precomputed divergence, 2: FP32 colour-split records, 0: otherwise).
template <typename T>
static std::array<int, 6> tune_key(const Lv<T>& L) {
    return {L.n[0], L.n[1], L.n[2], L.K, (int)sizeof(T), L.divc ? 1 : (L.mlay == kModSplit ? 2 : 0)};
}

template <typename T>
static int sweep_variant_for(const Lv<T>& L) {
    return tune_lookup(tune_key(L), kDefaultSweepVariant);
}

template <typename T>
static void set_sweep_variant(const Lv<T>& L, int v) {
    tune_store(tune_key(L), v);
}

static int sm_count() {
    static int n = [] {
        int dev = 0, c = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
        return c > 0 ? c : 1;
    }();
    return n;
}

// z planes per block of the tiled smoother: the chunking with the fewest plane steps
// per SM, counting whole waves of resident blocks and two prologue planes per block.
static int tiled_zlen(int columns, int nzi, int per_sm) {
    const long slots = (long)sm_count() * per_sm;
    int best = nzi;
    long best_cost = -1;
    for (int zc = 1; zc <= nzi; ++zc) {
        const int zl = (nzi + zc - 1) / zc;
        if ((nzi + zl - 1) / zl != zc) continue;
        const long blocks = (long)columns * zc;
        const long cost = ((blocks + slots - 1) / slots) * (zl + 2);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = zl;
        }
    }
    return best;
}

template <int KIND, int TY>
void launch_tiled(const Lv<float>& L, const float* u_in, float* u_out, const float* f, int colour,
                         const NullInfo& nfv, const double* lam, cudaStream_t s) {
    using S = TiledShape<KIND, TY>;
    static const bool attr = [] {
        cudaFuncSetAttribute(k_half_sweep_tiled<KIND, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)S::SMEM);
        return true;
    }();
    (void)attr;
    int cnt[3];
    for (int d = 0; d < 3; ++d) cnt[d] = L.per[d] ? L.n[d] : L.n[d] - 2;
    const int gx = (cnt[0] + kTileX - 1) / kTileX, gy = (cnt[1] + TY - 1) / TY;
    const int zl = tiled_zlen(gx * gy, cnt[2], TY <= 8 ? 2 : 1);
    const dim3 grid(gx, gy, (cnt[2] + zl - 1) / zl);
    k_half_sweep_tiled<KIND, TY><<<grid, 16 * TY, S::SMEM, s>>>(L, u_in, u_out, f, colour, nfv, lam, zl);
}

template <int TY, int MINB>
void launch_tiled_split(const Lv<float>& L, const float* u_in, float* u_out, const float* f, int colour,
                        const NullInfo& nfv, const double* lam, cudaStream_t s) {
    using S = SplitTile<TY>;
    int cnt[3];
    for (int d = 0; d < 3; ++d) cnt[d] = L.per[d] ? L.n[d] : L.n[d] - 2;
    const int gx = (cnt[0] + kTileX - 1) / kTileX, gy = (cnt[1] + TY - 1) / TY;
    const int zl = cnt[2] > 0 ? tiled_zlen(gx * gy, cnt[2], MINB) : 1;
    const int gz = cnt[2] > 0 ? (cnt[2] + zl - 1) / zl : 0;
    const BndSegs sg = bnd_segs(L, S::NT);
    const int nb = sg.f2 + gx * gy * gz;
    if (!nb) return;
    static const bool attr = [] {
        cudaFuncSetAttribute(k_half_sweep_tiled_split<TY, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)S::SMEM);
        return true;
    }();
    (void)attr;
    count_launch();
    k_half_sweep_tiled_split<TY, MINB><<<nb, S::NT, S::SMEM, s>>>(L, u_in, u_out, f, colour, nfv, lam, sg, gx, gy, zl);
}

// The tiled kernel reads the blocked FP32 moduli copy directly: not for FP64 levels or
// FP16 moduli.
template <typename T>
static bool variant_ok(const Lv<T>& L, int v) {
    if (sizeof(T) == 4 && L.modh) return v == 1 || v == 2;   // FP16 records: two shapes
    if (sizeof(T) == 4 && L.mlay == kModSplit) return v < kFirstTiledVariant || v >= kFirstSplitTiledVariant;
    if (v >= kFirstSplitTiledVariant) return false;
    if (v < kFirstTiledVariant) return true;
    return sizeof(T) == 4 && L.mlay == kModBlocked && !L.divc;
}

// Edge, corner and face nodes of a half-sweep as launches of their own (with the tiled
// interior kernel, whose grid is three-dimensional).
template <typename T>
static void launch_boundary_sweep(const Lv<T>& L, const T* u_in, T* u_out, const T* f, int colour,
                                  const NullInfo& nfv, const double* lam, cudaStream_t s) {
    launch_faces_sweep<T, 0>(L, u_in, u_out, f, colour, nfv, lam, s);
    launch_faces_sweep<T, 1>(L, u_in, u_out, f, colour, nfv, lam, s);
    launch_faces_sweep<T, 2>(L, u_in, u_out, f, colour, nfv, lam, s);
    if (L.nbnd) {
        count_launch();
        if (L.K == 2) k_half_sweep_bnd<T, 2><<<blocks_for((size_t)L.nbnd * 32), kBlock, 0, s>>>(L, u_in, u_out, f, colour, nfv, lam);
        else k_half_sweep_bnd<T, 21><<<blocks_for((size_t)L.nbnd * 32), kBlock, 0, s>>>(L, u_in, u_out, f, colour, nfv, lam);
    }
}

// One half-sweep with interior shape v: the untiled shapes take every node in one
// launch; the tiled ones launch the boundary nodes separately.
template <typename T, int KIND, bool HM, int MH>
void sweep_int_variant(int v, size_t np, const Lv<T>& L, const T* u_in, T* u_out, const T* f, int colour,
                       const NullInfo& nfv, const double* lam, cudaStream_t s) {
    if constexpr (sizeof(T) == 4 && !HM && MH == kMlDefault) {
        if (v >= kFirstTiledVariant && variant_ok(L, v) && colour < 2) {   // tiled: red-black only
            if (np) {
                count_launch();
                if (v == kFirstTiledVariant) launch_tiled<KIND, 16>(L, u_in, u_out, f, colour, nfv, lam, s);
                else launch_tiled<KIND, 8>(L, u_in, u_out, f, colour, nfv, lam, s);
            }
            launch_boundary_sweep(L, u_in, u_out, f, colour, nfv, lam, s);
            return;
        }
    }
    if constexpr (sizeof(T) == 4 && MH == kMlSplit) {
        if (v >= kFirstSplitTiledVariant && variant_ok(L, v) && colour < 2) {   // red-black only
            if (v == kFirstSplitTiledVariant) launch_tiled_split<16, 1>(L, u_in, u_out, f, colour, nfv, lam, s);
            else launch_tiled_split<8, 3>(L, u_in, u_out, f, colour, nfv, lam, s);
            return;
        }
    }
    if (v >= kFirstTiledVariant || !variant_ok(L, v)) v = kDefaultSweepVariant;
    if constexpr (MH == kMlHalf) {
        // FP16 records: shapes (256,2) and (256,3) only
        const int bs = 256;
        const BndSegs sg = bnd_segs(L, bs);
        const int nb = sg.f2 + (int)((np + bs - 1) / bs);
        if (!nb) return;
        count_launch();
        if (v == 1) k_half_sweep_int<T, KIND, HM, kMlHalf, 256, 2><<<nb, 256, 0, s>>>(L, u_in, u_out, f, colour, nfv, lam, sg);
        else k_half_sweep_int<T, KIND, HM, kMlHalf, 256, 3><<<nb, 256, 0, s>>>(L, u_in, u_out, f, colour, nfv, lam, sg);
    } else {
        const int bs = kSweepVariants[v][0];
        const BndSegs sg = bnd_segs(L, bs);
        const int nb = sg.f2 + (int)((np + bs - 1) / bs);
        if (!nb) return;
        count_launch();
        switch (v) {
            case 0: k_half_sweep_int<T, KIND, HM, MH, 256, 1><<<nb, 256, 0, s>>>(L, u_in, u_out, f, colour, nfv, lam, sg); break;
            case 1: k_half_sweep_int<T, KIND, HM, MH, 256, 2><<<nb, 256, 0, s>>>(L, u_in, u_out, f, colour, nfv, lam, sg); break;
            case 2: k_half_sweep_int<T, KIND, HM, MH, 256, 3><<<nb, 256, 0, s>>>(L, u_in, u_out, f, colour, nfv, lam, sg); break;
            case 3: k_half_sweep_int<T, KIND, HM, MH, 256, 4><<<nb, 256, 0, s>>>(L, u_in, u_out, f, colour, nfv, lam, sg); break;
            default: k_half_sweep_int<T, KIND, HM, MH, 128, 8><<<nb, 128, 0, s>>>(L, u_in, u_out, f, colour, nfv, lam, sg); break;
        }
    }
}

// Moduli kind -> kernel instance.
template <typename T>
static void dispatch_sweep(int v, size_t np, const Lv<T>& L, const T* u_in, T* u_out, const T* f, int colour,
                           const NullInfo& nfv, const double* lam, cudaStream_t s) {
    if constexpr (sizeof(T) == 8) {
        // FP64 levels of general moduli always carry the divergence
        if (L.K == 2) sweep_int_variant<T, 2, false, kMlDefault>(v, np, L, u_in, u_out, f, colour, nfv, lam, s);
        else sweep_int_variant<T, 21, true, kMlDefault>(v, np, L, u_in, u_out, f, colour, nfv, lam, s);
    } else if (L.modh) {
        if (L.K == 2) sweep_int_variant<T, 2, false, kMlHalf>(v, np, L, u_in, u_out, f, colour, nfv, lam, s);
        else sweep_int_variant<T, 21, false, kMlHalf>(v, np, L, u_in, u_out, f, colour, nfv, lam, s);
    } else if (L.K == 21 && L.mlay == kModSplit) {
        // colour-split records with the divergence: centre moduli only
        sweep_int_variant<T, 21, true, kMlSplit>(v, np, L, u_in, u_out, f, colour, nfv, lam, s);
    } else {
        if (L.K == 2) sweep_int_variant<T, 2, false, kMlDefault>(v, np, L, u_in, u_out, f, colour, nfv, lam, s);
        else sweep_int_variant<T, 21, false, kMlDefault>(v, np, L, u_in, u_out, f, colour, nfv, lam, s);
    }
}

// Time every variant of the interior half-sweep on one level (buffers as given) and
// keep the fastest in the tuning table.  Returns the chosen variant.
template <typename T>
int tune_sweep(const Lv<T>& L, const T* u_in, T* u_out, const T* f, cudaStream_t s, float* ms_out) {
    const size_t np = interior_pairs(L);
    if (!np) return kDefaultSweepVariant;
    NullInfo nfv{};
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    int best = kDefaultSweepVariant;
    float best_ms = 1e30f;
    for (int v = 0; v < kNumSweepVariants; ++v) {
        if (!variant_ok(L, v)) {
            if (ms_out) ms_out[v] = -1.f;
            continue;
        }
        auto run = [&]() {
            dispatch_sweep<T>(v, np, L, u_in, u_out, f, 0, nfv, nullptr, s);
        };
        run();
        cudaEventRecord(a, s);
        const int reps = 5;
        for (int r = 0; r < reps; ++r) run();
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        ms /= reps;
        if (ms_out) ms_out[v] = ms;
        if (cudaGetLastError() == cudaSuccess && ms < best_ms) {
            best_ms = ms;
            best = v;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    set_sweep_variant(L, best);
    return best;
}


template <typename T>
void launch_half_sweep(const Lv<T>& L, const T* u_in, T* u_out, const T* f, int colour, const NullInfo* nf,
                       const double* lam, cudaStream_t s) {
    NullInfo nfv{};
    if (nf) nfv = *nf;
    const size_t np = interior_pairs(L);
    const int v = sweep_variant_for(L);
    dispatch_sweep<T>(v, np, L, u_in, u_out, f, colour, nfv, lam, s);
}

}  // namespace elas
