// Host-side interface between the C ABI layer and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include <array>

#include "elas_device.cuh"

namespace elas {

constexpr int kBlock = 256;
constexpr int kMaxPartials = 4096;   // reduction blocks per launch (grid-stride beyond)
constexpr int kPartialStride = 8;    // doubles per block partial: sumsq + 6 W^T r + pad

// Boundary data of the finest level used by the right-hand side.
struct BoundaryData {
    double uniform[6][3];
    const double* face[6];          // per-node data of face f (3 x N), or null
};

struct RhsInputs {
    const double* eps0;             // 6 x N or null
    const double* body;             // 3 x N or null
    double mean_strain[6];
    int has_mean_strain;
};

// Number of kernel launches issued by this library since load (all contexts).
unsigned long long launch_count();
void count_launch(int n = 1);

// Interior smoother launch variants (block size, minimum blocks per SM) and the
// autotuner that picks one per level shape and precision.
constexpr int kNumSweepVariants = 9;
constexpr int kDefaultSweepVariant = 0;
template <typename T>
int tune_sweep(const Lv<T>& L, const T* u_in, T* u_out, const T* f, cudaStream_t s, float* ms_out);
int tune_lookup(const std::array<int, 6>& key, int fallback);   // key: nx ny nz K bytes layout
void tune_store(const std::array<int, 6>& key, int variant);
int tune_table_dump(char* buf, int cap);
int tune_table_load(const char* text);
unsigned long long tune_version();   // changes whenever the table does (captured launches depend on it)

// Launchers (all enqueue on `s`).
void launch_rhs(const Lv<double>& L, const RhsInputs& in, const BoundaryData& bd, double* f, cudaStream_t s);
void launch_dirichlet(const Lv<double>& L, const BoundaryData& bd, double* u, int keep_free, cudaStream_t s);

template <typename T>
void launch_apply(const Lv<T>& L, const T* u, T* out, cudaStream_t s);

// r = f - load - A u (load optional: the equilibrating load as 6 numbers t, w, applied
// as t + w x d); writes r as TR; per-block partials of sum r^2 and of the six
// rigid-motion moments of r when partials != null.
template <typename T, typename TR>
void launch_residual(const Lv<T>& L, const T* u, const T* f, const NullInfo* nf, const double* lam,
                     TR* r, double* partials, int* nblocks, cudaStream_t s);

// The same residual of an FP64 level in double-float arithmetic from double-float copies
// of u, f, the moduli (with the divergence) and the stored rows (L: the level with those
// planes), written as FP32; partials (required) as launch_residual's.  Interior threads take
// kDfNodesPerThread nodes each.
constexpr int kDfNodesPerThread = 8;
void launch_residual_df(const Lv<dfloat>& L, const dfloat* u, const dfloat* f, const NullInfo* nf, const double* lam,
                        float* r, double* partials, int* nblocks, cudaStream_t s);
int residual_df_block_count(const Lv<dfloat>& L);
// out[i] = a[i] split into hi + lo (n elements)
void launch_split_df(const double* a, dfloat* out, size_t n, cudaStream_t s);
// u += e on the non-Dirichlet rows (as launch_add_correction) and u2 := split(u) everywhere
void launch_add_correction_df(const Lv<double>& L, double* u, const float* e, dfloat* u2, cudaStream_t s);

// One colour of the red-black block smoother, u_in -> u_out (all nodes written).
template <typename T>
void launch_half_sweep(const Lv<T>& L, const T* u_in, T* u_out, const T* f, int colour,
                       const NullInfo* nf, const double* lam, cudaStream_t s);

// fc = R (r - dlam.W) (dlam optional)
template <typename T>
void launch_restrict(const Lv<T>& Lf, const Lv<T>& Lc, const T* r, T* fc, const NullInfo* nf,
                     const double* dlam, cudaStream_t s);

template <typename T>
void launch_prolong_add(const Lv<T>& Lf, const Lv<T>& Lc, const T* ec, T* u, cudaStream_t s);

template <typename T>
void launch_restrict_moduli(const Lv<T>& Lf, const Lv<T>& Lc, const T* mf, T* mc, cudaStream_t s);

// FP64 moduli planes (K x N) -> the FP32 blocked copy or the FP16 node records of an FP32
// level (entries to allocate: moduli_copy_entries).
size_t moduli_copy_entries(int N, int K, bool half);
// Coefficients of the level's edge and corner rows (L.nbnd x kEdgeCoef) into out.
template <typename T>
void launch_edge_coef(const Lv<T>& L, T* out, cudaStream_t s);
void launch_moduli_copy(const double* in, float* out, int N, int K, cudaStream_t s);
// Colour-split FP32 records (moduli + divergence, kModSplit) of a general-moduli level with
// odd nx and ny: whether a level takes them, their element count, and the copy from the
// FP64 moduli and divergence planes.
bool split_layout_applies(const int n[3], int K);
size_t split_entries(int N);
void launch_moduli_split(const double* mod, const double* divc, float* out, int N, cudaStream_t s);
void launch_moduli_copy(const double* in, __half* out, int N, int K, cudaStream_t s);
// M_iV = sum_j d_j C_(ij)V (18 planes) of a general-moduli FP64 level (setup)
void launch_divc(const Lv<double>& L, double* M, cudaStream_t s);
void launch_add_correction(const Lv<double>& L, double* u, const float* e, cudaStream_t s);
void launch_add_correction64(const Lv<double>& L, double* u, const double* e, cudaStream_t s);

// Coarsest level: dense matrix over the listed free DOFs (plus m bordering rows and
// columns of the free rigid modes), its inverse, and the solve.
void launch_bottom_assemble(const Lv<double>& L, const int* dofs, int nfree, const NullInfo& nf,
                            double* A, cudaStream_t s);
void launch_invert(double* A, double* Ainv, int n, double* fcol, int* singular_flag, cudaStream_t s);  // fcol: n doubles of scratch
template <typename T>
void launch_bottom_solve(const Lv<T>& L, const int* dofs, int nfree, int ntot, const double* Ainv,
                         const T* f, T* u, double* work, cudaStream_t s);

// Deterministic final reduction of residual partials; when nf.m > 0 also the
// equilibrating-load update dlam = G^-1 W^T r, lam += dlam (if update_lam),
// and the norm of r - dlam.W.  out[0] = sum r^2 (corrected).
// Per-member convergence control of a batched solve (all null = not batched).
struct BatchFlags {
    int* active;        // 1 while the member still iterates
    int* count;         // residual evaluations so far
    double* hist;       // relative residual history
    int hist_len;
    double r0, tol;
    int max_cycles;
};
void launch_finalize(const double* partials, int nblocks, const NullInfo& nf, const double* Ginv,
                     const double* G, double* lam, double* dlam, double* alam, double* adlam, double* out,
                     int update_lam, cudaStream_t s, BatchFlags bflags = BatchFlags{});

// Block partials of the six raw rigid-motion moments of u (sum u, sum d x u over the
// non-Dirichlet rows); with gram = q + 1, column q of W^T W (setup).
void launch_null_dots(const Lv<double>& L, const NullInfo& nf, const double* u, double* partials,
                      int* nblocks, int gram, cudaStream_t s);
void launch_sum_partials(const double* partials, int nblocks, int width, double* out, cudaStream_t s);
// u -= sum_q coef[q] W_q with coef = Ginv (W^T u), from the six raw moments of u
// (sum u, sum d x u; launch_null_dots + launch_sum_partials with width 6): the motion
// (t, w) = basis coef is formed on the device in `motion` (6 doubles), then
// u -= t + w x d on the non-Dirichlet rows.
void launch_remove_null(const Lv<double>& L, const NullInfo& nf, const double* Ginv, const double* moment,
                        double* motion, double* u, cudaStream_t s);

// Stress sigma = C : (grad u + mean - eps0) of an FP64 level, 6 x N (11 22 33 23 31 12);
// eps0 optional (6 x N), mean the mean strain of a periodic cell (zero otherwise).
struct MeanStrain {
    double e[6];
};
void launch_stress(const Lv<double>& L, const double* u, const double* eps0, const MeanStrain& mean, double* out,
                   cudaStream_t s);

// ---- batched engine: one launch per phase over a work list of members ------------------
// Each phase (a half-sweep of one level, a residual, a restriction, ...) of a batch of
// grids is one launch.  Its tasks (one per member taking part) sit in device memory with
// their block offsets; a block finds its task by binary search over the offsets and runs
// the same per-node code as the single-grid kernels on that member's level, so every
// member computes exactly what it computes alone.
enum : int {
    kPhaseSweep = 0,      // SweepTask<float>: half-sweep (colour in the phase)
    kPhaseResid32 = 1,    // ResidTask<float, float>: FP32 residual, no norm
    kPhaseResid64 = 2,    // ResidTask<double, float>: FP64 residual written as FP32, with partials
    kPhaseRestrict = 3,   // RestrictTask<float>
    kPhaseProlong = 4,    // ProlongTask<float>
    kPhaseZero = 5,       // ZeroTask<float>
    kPhaseGather = 6,     // BottomTask<float>: right-hand side of the bottom solve
    kPhaseMatvec = 7,     // BottomTask<float>: dense inverse times it
    kPhaseFinalize = 8,   // FinalizeTask
    kPhaseCorr = 9,       // CorrTask: FP64 u += FP32 e
    kPhaseResidDf = 10,   // ResidTask<dfloat, float>: double-float residual written as FP32, with partials
};
template <typename T>
struct SweepTask {
    Lv<T> L;
    const T* u;
    T* uo;
    const T* f;
    NullInfo nf;
    const double* lam;
};
template <typename T, typename TR>
struct ResidTask {
    Lv<T> L;
    const T* u;
    const T* f;
    NullInfo nf;
    const double* lam;
    TR* r;
    double* partials;
};
template <typename T>
struct RestrictTask {
    Lv<T> Lf, Lc;
    const T* r;
    T* fc;
    NullInfo nf;
    const double* dlam;
};
template <typename T>
struct ProlongTask {
    Lv<T> Lf, Lc;
    const T* ec;
    T* u;
};
template <typename T>
struct ZeroTask {
    T* a;
    size_t n;
    const int* active;
};
template <typename T>
struct BottomTask {
    Lv<T> L;
    const int* dofs;
    int nfree, ntot;
    const double* Ainv;
    const T* f;
    T* u;
    double* work;
};
struct FinalizeTask {
    const double* partials;
    int nblocks;
    NullInfo nf;
    const double *Ginv, *G;
    double *lam, *dlam, *alam, *adlam, *out;
    BatchFlags bf;
};
struct CorrTask {
    Lv<double> L;
    double* u;
    const float* e;
    dfloat* u2;   // non-null: also refresh the double-float copy of u
};
// A phase ready to launch: kind, member count, tasks and the block map in device memory
// (for every block of the launch: its task and its block index within that task), total
// blocks, the half-sweep colour and the moduli variant of the sweep and residual kernels
// (moduli kind 2 or 21 and layout kMl*).
struct BatchPhase {
    int kind = 0, n = 0, blocks = 0, colour = 0, K = 2, ml = 0;
    const void* tasks = nullptr;
    const int2* bmap = nullptr;
};
// Blocks one task of a phase takes (the member's own block partition).
int batch_task_blocks(int kind, const void* task);
void batch_phase_launch(const BatchPhase& ph, cudaStream_t s);

// ALU peak microbenchmark: one launch of independent FMA chains on every SM (precision 0 =
// FP64, 1 = FP32); returns the FLOPs of the launch and its device time in *ms.  out: a
// device buffer of 256 elements (never written in practice).
double measure_fma_flops(int precision, int iters, float* ms, void* out, cudaStream_t s);

// ---- block-structured AMR transfers ------------------------------------------------
// Placement of one AMR level's grid in its level's global node index space.
struct AmrBox {
    int grid_lo[3];
    int valid_lo[3];
    int valid_hi[3];
    int ghost[6];
    int count[3];      // global node count of the level per direction
};

// mode 0: ghost nodes := I(coarse); mode 1: valid non-Dirichlet nodes += I(coarse)
template <typename T>
void launch_amr_interp(const Lv<T>& Lf, const AmrBox& bf, const Lv<T>& Lc, const AmrBox& bc, const T* cfield,
                       T* ffield, int mode, cudaStream_t s);
// covered coarse nodes := coincident fine values
void launch_amr_inject(const Lv<double>& Lf, const AmrBox& bf, const Lv<double>& Lc, const AmrBox& bc,
                       const double* ffield, double* cfield, cudaStream_t s);
// covered coarse nodes := renormalised restriction of a K-plane fine field over the fine
// box's valid nodes; on coarse Dirichlet rows: zero (zero_dirichlet 1), kept (2), or the
// restricted value (0)
template <typename T>
void launch_amr_restrict(const Lv<T>& Lf, const AmrBox& bf, const Lv<T>& Lc, const AmrBox& bc, const T* ffield,
                         T* cfield, int K, int zero_dirichlet, cudaStream_t s);
// partials of sum res^2 over valid nodes not covered by the next level (cov may be null)
int launch_amr_norm(const Lv<double>& L, const AmrBox& b, const AmrBox* cov, const double* res, double* partials,
                    cudaStream_t s);
// u += cor on every node that is not a ghost
template <typename TU, typename TC>
void launch_amr_add(const Lv<TU>& L, const AmrBox& b, TU* u, const TC* cor, cudaStream_t s);
// a := (TO) b over n elements
template <typename TO, typename TI>
void launch_cast(TO* a, const TI* b, size_t n, cudaStream_t s);

}  // namespace elas
