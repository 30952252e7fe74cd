// C ABI of the solver: contexts, grids and their multigrid hierarchy, setup,
// FP64 and mixed-precision solves, single-operation entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <deque>
#include <functional>
#include <mutex>
#include <map>
#include <vector>

#include "../../include/elas.h"
#include "elas_internal.h"

using namespace elas;

struct elas_ctx_s {
    int device = 0;
    size_t budget = 0;
    size_t in_use = 0;
    elas_allocator alloc{};
    bool has_alloc = false;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    double* host_status = nullptr;   // pinned readback buffer
    // profiling: event pairs recorded around finest-level launches
    bool profile = false;
    std::vector<cudaEvent_t> pool;
    size_t pool_used = 0;
    std::vector<std::pair<int, size_t>> pending;   // (class, index of start event)
    double prof_ms[ELAS_PROF_CLASSES] = {0, 0, 0, 0};
    long long prof_count[ELAS_PROF_CLASSES] = {0, 0, 0, 0};
    std::vector<cudaStream_t> branch;        // streams of the batched graph's branches
    std::vector<cudaEvent_t> branch_ev;
    struct BatchPlan* plan = nullptr;         // the batched engine's last plan and graph
    std::vector<elas_server_s*> servers;      // live servers (their requests hold grids)
};

// Whether a live server of the context holds a waiting or active request on grid g (as
// its grid or as a level of its AMR layout) or on AMR layout a; such objects must not be
// destroyed until the request retires.
bool server_holds(elas_ctx c, elas_grid g, elas_amr a);

namespace {

// Start / stop an event-bracketed launch of a profiled class (no-op when profiling is off).
size_t prof_begin(elas_ctx c, int cls) {
    if (!c->profile) return (size_t)-1;
    while (c->pool.size() < c->pool_used + 2) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        c->pool.push_back(e);
    }
    const size_t i = c->pool_used;
    c->pool_used += 2;
    cudaEventRecord(c->pool[i], c->stream);
    c->pending.push_back({cls, i});
    return i;
}

void prof_end(elas_ctx c, size_t i) {
    if (i == (size_t)-1) return;
    cudaEventRecord(c->pool[i + 1], c->stream);
}

// Fold pending event pairs into the totals (after a stream synchronisation).
void prof_collect(elas_ctx c) {
    if (!c->profile) return;
    for (auto& pr : c->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->pool[pr.second], c->pool[pr.second + 1]) == cudaSuccess) {
            c->prof_ms[pr.first] += ms;
            c->prof_count[pr.first] += 1;
        }
    }
    c->pending.clear();
    c->pool_used = 0;
}

struct Level {
    int n[3];
    int N;
    Lv<double> L64;
    Lv<float> L32;
    double *mod64 = nullptr, *u = nullptr, *ua = nullptr, *f = nullptr, *r = nullptr, *divc = nullptr;
    float *mod32 = nullptr, *u32 = nullptr, *ua32 = nullptr, *f32 = nullptr, *r32 = nullptr;
    __half* mod16 = nullptr;   // FP16 moduli of the FP32 V-cycle (half_moduli grids)
    bool split = false;        // mod32 holds colour-split records with the divergence
    int* bnd = nullptr;   // boundary-plane nodes of this level
    int nbnd = 0;
    double* bcoef64 = nullptr;   // edge and corner row coefficients (kEdgeCoef per node)
    // the FP32 copy's list and coefficients (general moduli on small levels list every
    // face node there, see face_list_mask)
    int* bnd32 = nullptr;
    int nbnd32 = 0;
    float* bcoef32 = nullptr;
    NullInfo nf{};
    // double-float copies read by the refinement residual of a mixed solve (finest level of
    // a mixed grid): moduli (K planes, then the 18 divergence planes), u, f, stored rows
    dfloat *m2 = nullptr, *u2 = nullptr, *f2 = nullptr, *bc2 = nullptr;
};

}  // namespace

struct elas_grid_s {
    elas_ctx ctx = nullptr;
    elas_grid_desc desc{};
    std::vector<Level> lv;
    int K = 2;
    // finest-level inputs
    double* eps0 = nullptr;
    double* body = nullptr;
    double mean[6] = {0, 0, 0, 0, 0, 0};
    int has_mean = 0;
    int bc_type[6][3];
    double bc_val[6][3];
    double* face[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    std::map<double**, double*> kept;   // buffers of cleared inputs, reused when set again
    // bottom
    int* dofs = nullptr;
    int nfree = 0, ntot = 0;
    double *Ainv = nullptr, *Awork = nullptr, *bwork = nullptr;
    int* flag = nullptr;
    // equilibrating load
    double *G = nullptr, *Ginv = nullptr, *lam = nullptr, *dlam = nullptr, *status = nullptr, *partials = nullptr;
    double *alam = nullptr, *adlam = nullptr;   // loads as rigid motions (t, w)
    double r0 = 0.0;
    double r0inf = 0.0;   // ||r_0||_inf
    bool moduli_set = false;
    bool dirty = true;         // moduli or boundary types changed: rebuild everything
    bool rhs_dirty = true;     // only loads / boundary data changed: rebuild the right-hand side
    bool gram_valid = false;   // W^T W of the finest level (depends on boundary types, not moduli)
    unsigned long long gen = 0;   // full set-ups so far (a cached batch plan checks it)
    unsigned long long df_gen = ~0ull;   // set-up whose moduli the double-float copies hold
    // smoother and cycle of the solve in progress (from its options)
    int smoother = ELAS_SMOOTH_RB;
    int cycle = ELAS_CYCLE_V;
    double omega = 2.0 / 3.0;
    std::vector<std::pair<void*, size_t>> allocs;
    int amr_refs = 0;   // live AMR layouts that hold the grid as a level
    // captured multigrid cycles (see run_cycle), keyed by precision, level, start and cycle
    // type, valid for the set-up, launch-shape table, options and stream they were
    // captured with
    struct CycleGraph {
        cudaGraphExec_t exec = nullptr;   // null: capture failed, launch directly
        int launches = 0;
    };
    std::map<int, CycleGraph> cyc;
    unsigned long long cyc_gen = ~0ull, cyc_tune = ~0ull;
    int cyc_nu1 = -1, cyc_nu2 = -1, cyc_smoother = -1;
    double cyc_omega = -1.0;
    const void* cyc_nf = nullptr;
    const void* cyc_dlam = nullptr;
    cudaStream_t cyc_stream = nullptr;
};

namespace {

int set_err(elas_ctx c, int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

// Calls that launch on a grid or change it are refused while a server request holds the
// grid: an admitted request keeps its per-grid state (activity flags, iterate, loads) in
// the grid between server steps, and a waiting one is solved from the grid as it will be.
int refuse_if_served(elas_grid g) {
    return server_holds(g->ctx, g, nullptr)
               ? set_err(g->ctx, ELAS_ERR_STATE, "grid has a waiting or active server request")
               : ELAS_OK;
}

#define CUDA_TRY(ctx, call)                                                                      \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return set_err(ctx, ELAS_ERR_DEVICE, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define CHECK_LAUNCH(ctx) CUDA_TRY(ctx, cudaGetLastError())

void* ctx_alloc(elas_ctx c, size_t bytes) {
    if (bytes == 0) bytes = 256;
    bytes = (bytes + 255) & ~size_t(255);
    if (c->budget && c->in_use + bytes > c->budget) return nullptr;
    void* p = nullptr;
    if (c->has_alloc) {
        p = c->alloc.alloc(bytes, c->alloc.user, (void*)c->stream);
    } else {
        if (cudaMallocAsync(&p, bytes, c->stream) != cudaSuccess) p = nullptr;
    }
    if (p) c->in_use += bytes;
    return p;
}

void ctx_free(elas_ctx c, void* p, size_t bytes) {
    if (!p) return;
    if (bytes == 0) bytes = 256;
    bytes = (bytes + 255) & ~size_t(255);
    if (c->has_alloc) c->alloc.free(p, bytes, c->alloc.user, (void*)c->stream);
    else cudaFreeAsync(p, c->stream);
    c->in_use -= bytes;
}

template <typename P>
int galloc(elas_grid g, P** out, size_t count) {
    const size_t bytes = count * sizeof(P);
    if (g->ctx->budget && g->ctx->in_use + ((bytes + 255) & ~size_t(255)) > g->ctx->budget)
        return set_err(g->ctx, ELAS_ERR_OUT_OF_BUDGET, "HBM budget of the context exceeded");
    void* p = ctx_alloc(g->ctx, bytes);
    if (!p) return set_err(g->ctx, ELAS_ERR_ALLOC, "device allocation failed");
    g->allocs.push_back({p, bytes});
    *out = (P*)p;
    return ELAS_OK;
}

template <typename T>
void fill_lv(Lv<T>& L, const int n[3], const int per[3], const double h[3], int K, const int bct[6][3]) {
    for (int d = 0; d < 3; ++d) {
        L.n[d] = n[d];
        L.per[d] = per[d];
        L.h[d] = (T)h[d];
        L.inv2h[d] = (T)(1.0 / (2.0 * h[d]));
        L.invh[d] = (T)(1.0 / h[d]);
        L.invh2[d] = (T)(1.0 / (h[d] * h[d]));
    }
    L.inv4hh[0] = (T)(1.0 / (4.0 * h[1] * h[2]));
    L.inv4hh[1] = (T)(1.0 / (4.0 * h[0] * h[2]));
    L.inv4hh[2] = (T)(1.0 / (4.0 * h[0] * h[1]));
    L.N = n[0] * n[1] * n[2];
    L.K = K;
    for (int f = 0; f < 6; ++f)
        for (int c = 0; c < 3; ++c) L.bc[f][c] = (signed char)(per[f / 2] ? 0 : bct[f][c]);
    L.mod = nullptr;
    L.bnodes = nullptr;
    L.nbnd = 0;
    L.divc = nullptr;
    L.active = nullptr;
    L.modh = nullptr;
    L.mlay = kModPlanes;
    L.bcoef = nullptr;
    L.msplit1 = 0;
    L.omega = (T)1;
    L.xface_list = 0;
}

// The level seen by the double-float residual: the FP64 view's geometry, boundary types
// and flags with double-float constants and the double-float planes.
Lv<dfloat> df_view(const Level& v) {
    const Lv<double>& S = v.L64;
    Lv<dfloat> L{};
    for (int d = 0; d < 3; ++d) {
        L.n[d] = S.n[d];
        L.per[d] = S.per[d];
        L.h[d] = dfloat(S.h[d]);
        L.inv2h[d] = dfloat(S.inv2h[d]);
        L.invh[d] = dfloat(S.invh[d]);
        L.invh2[d] = dfloat(S.invh2[d]);
        L.inv4hh[d] = dfloat(S.inv4hh[d]);
    }
    L.N = S.N;
    L.K = S.K;
    L.mlay = kModPlanes;
    for (int f = 0; f < 6; ++f)
        for (int c = 0; c < 3; ++c) L.bc[f][c] = S.bc[f][c];
    L.mod = v.m2;
    L.bnodes = S.bnodes;
    L.nbnd = S.nbnd;
    L.divc = (S.K == 21 && v.divc && v.m2) ? v.m2 + (size_t)21 * v.N : nullptr;
    L.active = S.active;
    L.modh = nullptr;
    L.bcoef = v.bc2;
    L.msplit1 = 0;
    L.omega = dfloat(S.omega);
    L.xface_list = S.xface_list;
    return L;
}

// Face directions (bit A) whose face nodes take their rows from stored coefficients (a
// warp per node) rather than from the face kernels; FP32 copies only.  Levels of 2^20
// nodes and more list the x faces, whose stencil neighbours lie nx apart (rows evaluated
// from the fields read one sector per value; 257^3 half-sweep 0.53 -> 0.48 ms).  Levels of
// general moduli with up to 300000 nodes (65^3 and coarser) list every face: there the
// face kernels' rows (tens of dependent moduli and displacement loads, long code) dominate
// the launches; measured V-cycles of a 65^3 hierarchy 0.87 -> 0.44 ms.  Not so with
// isotropic moduli (two moduli per node make the face rows cheap), nor on 129^3 (the
// coefficients add to a bandwidth-bound launch: 1.37 -> 1.60 ms).  FP64 levels store the
// edge and corner rows only: a stored row there costs 243 FMAs on the narrow FP64 pipe per
// application (33^3 FP64 solves 133 -> 91 per second with every face listed) and 243
// evaluations of the generic row in FP64 at every set-up (the x faces of 257^3: tens of
// milliseconds per new moduli field).
constexpr size_t kAllFacesListMaxNodes = 300000;
constexpr size_t kXFaceListMinNodes = size_t(1) << 20;
int face_list_mask(const int n[3], const int per[3], bool fp32, bool general) {
    if (!fp32) return 0;
    const size_t N = (size_t)n[0] * n[1] * n[2];
    int m = 0;
    if (general && N <= kAllFacesListMaxNodes) m = 7;
    else if (N >= kXFaceListMinNodes) m = 1;
    for (int d = 0; d < 3; ++d)
        if (per[d]) m &= ~(1 << d);
    return m;
}

bool coarsenable(const int n[3], const int per[3]) {
    int mx = 0;
    for (int d = 0; d < 3; ++d) {
        if (per[d]) {
            if (n[d] % 2 != 0 || n[d] / 2 < 4) return false;
        } else {
            if ((n[d] - 1) % 2 != 0 || (n[d] - 1) / 2 + 1 < 3) return false;
        }
        mx = n[d] > mx ? n[d] : mx;
    }
    return mx > 5;
}

std::vector<std::array<int, 3>> level_dims(const elas_grid_desc& d) {
    std::vector<std::array<int, 3>> out;
    std::array<int, 3> n = {d.n[0], d.n[1], d.n[2]};
    out.push_back(n);
    while (d.max_levels != 1 && coarsenable(n.data(), d.periodic)) {
        for (int k = 0; k < 3; ++k) n[k] = d.periodic[k] ? n[k] / 2 : (n[k] - 1) / 2 + 1;
        out.push_back(n);
    }
    return out;
}

// ---- host: free rigid modes --------------------------------------------------------
// Symmetric 6x6 eigen-decomposition by cyclic Jacobi rotations.
void jacobi6(double A[6][6], double V[6][6], double ev[6]) {
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) V[i][j] = i == j ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < 6; ++i)
            for (int j = i + 1; j < 6; ++j) off += A[i][j] * A[i][j];
        if (off < 1e-300) break;
        for (int p = 0; p < 6; ++p)
            for (int q = p + 1; q < 6; ++q) {
                if (std::fabs(A[p][q]) < 1e-300) continue;
                const double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < 6; ++k) {
                    const double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - s * akq;
                    A[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < 6; ++k) {
                    const double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - s * aqk;
                    A[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 6; ++k) {
                    const double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - s * vkq;
                    V[k][q] = s * vkp + c * vkq;
                }
            }
    }
    for (int i = 0; i < 6; ++i) ev[i] = A[i][i];
}

int host_row_type(const int bct[6][3], const int per[3], const int n[3], const int c[3], int comp) {
    bool any = false, dir = false, neu = false;
    for (int d = 0; d < 3; ++d) {
        if (per[d]) continue;
        int f = -1;
        if (c[d] == 0) f = 2 * d;
        else if (c[d] == n[d] - 1) f = 2 * d + 1;
        if (f < 0) continue;
        any = true;
        dir |= bct[f][comp] == ELAS_BC_DIRICHLET;
        neu |= bct[f][comp] == ELAS_BC_NEUMANN;
    }
    if (!any) return ROW_INTERIOR;
    return dir ? ROW_DIRICHLET : (neu ? ROW_NEUMANN : ROW_TRACTION);
}

NullInfo null_space(const elas_grid_desc& d, const int n[3], const double h[3], const int bct[6][3]) {
    NullInfo nf{};
    for (int k = 0; k < 3; ++k) {
        nf.lo[k] = d.lo[k];
        nf.h[k] = h[k];
        nf.ctr[k] = d.lo[k] + 0.5 * h[k] * (n[k] - 1);
        nf.off[k] = nf.lo[k] - nf.ctr[k];
        nf.off32[k] = (float)nf.off[k];
        nf.h32[k] = (float)h[k];
    }
    bool allowed[6] = {true, true, true, true, true, true};
    for (int a = 0; a < 3; ++a) {
        const int b = (a + 1) % 3, c = (a + 2) % 3;
        if (d.periodic[b] || d.periodic[c]) allowed[3 + a] = false;
    }
    double M[6][6] = {};
    // rigid-mode values at every Dirichlet row
    int c[3];
    for (c[2] = 0; c[2] < n[2]; ++c[2])
        for (c[1] = 0; c[1] < n[1]; ++c[1])
            for (c[0] = 0; c[0] < n[0]; ++c[0]) {
                bool bnd = false;
                for (int k = 0; k < 3; ++k)
                    if (!d.periodic[k] && (c[k] == 0 || c[k] == n[k] - 1)) bnd = true;
                if (!bnd) {  // skip the interior of the box quickly
                    if (!d.periodic[0] && c[0] == 0 && n[0] > 2) { c[0] = n[0] - 2; }
                    continue;
                }
                for (int comp = 0; comp < 3; ++comp) {
                    if (host_row_type(bct, d.periodic, n, c, comp) != ROW_DIRICHLET) continue;
                    double x[3];
                    for (int k = 0; k < 3; ++k) x[k] = d.lo[k] + h[k] * c[k] - nf.ctr[k];
                    double R[6];
                    for (int m = 0; m < 3; ++m) R[m] = (m == comp) ? 1.0 : 0.0;
                    for (int a = 0; a < 3; ++a) {
                        const int b = (a + 1) % 3, e = (a + 2) % 3;
                        R[3 + a] = (comp == b) ? -x[e] : (comp == e ? x[b] : 0.0);
                    }
                    for (int i = 0; i < 6; ++i)
                        for (int j = 0; j < 6; ++j) M[i][j] += R[i] * R[j];
                }
            }
    // restrict to allowed modes: disallowed ones get a large diagonal so they are not null
    double scale = 1.0;
    for (int i = 0; i < 6; ++i) scale = std::fmax(scale, M[i][i]);
    for (int i = 0; i < 6; ++i)
        if (!allowed[i]) {
            for (int j = 0; j < 6; ++j) M[i][j] = M[j][i] = 0.0;
            M[i][i] = scale;
        }
    double V[6][6], ev[6];
    jacobi6(M, V, ev);
    nf.m = 0;
    for (int k = 0; k < 6; ++k) {
        if (ev[k] <= 1e-12 * scale) {
            for (int i = 0; i < 6; ++i) nf.basis[i][nf.m] = V[i][k];
            ++nf.m;
        }
    }
    return nf;
}

// small dense inverse on the host (m <= 6)
bool invert_small(const double* A, double* X, int m) {
    double a[6][12];
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < 2 * m; ++j) a[i][j] = j < m ? A[i * m + j] : (j - m == i ? 1.0 : 0.0);
    for (int c = 0; c < m; ++c) {
        int p = c;
        for (int r = c + 1; r < m; ++r)
            if (std::fabs(a[r][c]) > std::fabs(a[p][c])) p = r;
        if (a[p][c] == 0.0) return false;
        for (int j = 0; j < 2 * m; ++j) std::swap(a[c][j], a[p][j]);
        const double iv = 1.0 / a[c][c];
        for (int j = 0; j < 2 * m; ++j) a[c][j] *= iv;
        for (int r = 0; r < m; ++r)
            if (r != c) {
                const double fct = a[r][c];
                for (int j = 0; j < 2 * m; ++j) a[r][j] -= fct * a[c][j];
            }
    }
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) X[i * m + j] = a[i][m + j];
    return true;
}

BoundaryData boundary_data(elas_grid g) {
    BoundaryData bd;
    for (int f = 0; f < 6; ++f) {
        for (int c = 0; c < 3; ++c) bd.uniform[f][c] = g->bc_val[f][c];
        bd.face[f] = g->face[f];
    }
    return bd;
}

int read_status(elas_grid g, double* out, int count) {
    elas_ctx c = g->ctx;
    CUDA_TRY(c, cudaMemcpyAsync(c->host_status, g->status, sizeof(double) * count, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    for (int i = 0; i < count; ++i) out[i] = c->host_status[i];
    return ELAS_OK;
}

// Right-hand side of the finest level and ||r_0|| (loads and boundary data only).
int setup_rhs(elas_grid g) {
    elas_ctx c = g->ctx;
    cudaStream_t s = c->stream;
    Level& L0 = g->lv[0];
    // right-hand side
    RhsInputs in{};
    in.eps0 = g->eps0;
    in.body = g->body;
    for (int k = 0; k < 6; ++k) in.mean_strain[k] = g->mean[k];
    in.has_mean_strain = g->has_mean;
    launch_rhs(g->lv[0].L64, in, boundary_data(g), g->lv[0].f, s);
    CHECK_LAUNCH(c);
    // ||r_0||: residual of the Dirichlet-only field
    {
        launch_dirichlet(L0.L64, boundary_data(g), L0.ua, 0, s);
        CHECK_LAUNCH(c);
        int nb = 0;
        launch_residual<double, double>(L0.L64, L0.ua, L0.f, nullptr, nullptr, L0.r, g->partials, &nb, s);
        CHECK_LAUNCH(c);
        NullInfo none{};
        launch_finalize(g->partials, nb, none, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, g->status, 0, s);
        CHECK_LAUNCH(c);
        double st[2];
        int rc = read_status(g, st, 2);
        if (rc) return rc;
        g->r0 = std::sqrt(st[0]);
        g->r0inf = st[1];
    }
    g->rhs_dirty = false;
    return ELAS_OK;
}

// ---- setup: coarse moduli, FP32 copies, RHS, equilibrating-load data, bottom ----------
int setup(elas_grid g) {
    if (!g->dirty && !g->rhs_dirty) return ELAS_OK;
    elas_ctx c = g->ctx;
    cudaStream_t s = c->stream;
    if (!g->moduli_set) return set_err(c, ELAS_ERR_STATE, "moduli not set");
    const int nl = (int)g->lv.size();
    if (!g->dirty) return setup_rhs(g);
    for (int l = 1; l < nl; ++l) {
        launch_restrict_moduli<double>(g->lv[l - 1].L64, g->lv[l].L64, g->lv[l - 1].mod64, g->lv[l].mod64, s);
        CHECK_LAUNCH(c);
    }
    for (int l = 0; l < nl; ++l) {
        if (g->lv[l].divc) {
            Lv<double> Lm = g->lv[l].L64;
            Lm.divc = nullptr;
            launch_divc(Lm, g->lv[l].divc, s);
            CHECK_LAUNCH(c);
        }
    }
    if (g->desc.mixed) {
        for (int l = 0; l < nl; ++l) {
            Level& v = g->lv[l];
            if (v.mod16) launch_moduli_copy(v.mod64, v.mod16, v.N, g->K, s);
            else if (v.split) launch_moduli_split(v.mod64, v.divc, v.mod32, v.N, s);
            else launch_moduli_copy(v.mod64, v.mod32, v.N, g->K, s);
            CHECK_LAUNCH(c);
        }
    }
    // coefficients of the edge and corner rows (they depend on moduli and boundary types)
    for (int l = 0; l < nl; ++l) {
        Level& v = g->lv[l];
        if (v.nbnd) launch_edge_coef<double>(v.L64, v.bcoef64, s);
        if (v.nbnd32 && v.bcoef32) launch_edge_coef<float>(v.L32, v.bcoef32, s);
        CHECK_LAUNCH(c);
    }
    // equilibrating load of the finest level: G = W^T W, Ginv
    Level& L0 = g->lv[0];
    const int m = L0.nf.m;
    if (m > 0 && !g->gram_valid) {
        std::vector<double> Gh(m * m), Gi(m * m);
        for (int q = 0; q < m; ++q) {
            int nb = 0;
            launch_null_dots(L0.L64, L0.nf, nullptr, g->partials, &nb, q + 1, s);
            CHECK_LAUNCH(c);
            launch_sum_partials(g->partials, nb, m, g->status, s);
            CHECK_LAUNCH(c);
            double row[8];
            int rc = read_status(g, row, m);
            if (rc) return rc;
            for (int k = 0; k < m; ++k) Gh[q * m + k] = row[k];
        }
        if (!invert_small(Gh.data(), Gi.data(), m)) return set_err(c, ELAS_ERR_STATE, "singular rigid-mode Gram matrix");
        CUDA_TRY(c, cudaMemcpyAsync(g->G, Gh.data(), sizeof(double) * m * m, cudaMemcpyHostToDevice, s));
        CUDA_TRY(c, cudaMemcpyAsync(g->Ginv, Gi.data(), sizeof(double) * m * m, cudaMemcpyHostToDevice, s));
        CUDA_TRY(c, cudaStreamSynchronize(s));
        g->gram_valid = true;
    }
    // bottom: dense inverse of the coarsest operator (bordered when singular)
    if (g->ntot > 0) {
        Level& B = g->lv[nl - 1];
        launch_bottom_assemble(B.L64, g->dofs, g->nfree, B.nf, g->Awork, s);
        CHECK_LAUNCH(c);
        CUDA_TRY(c, cudaMemsetAsync(g->flag, 0, sizeof(int), s));
        launch_invert(g->Awork, g->Ainv, g->ntot, g->bwork, g->flag, s);
        CHECK_LAUNCH(c);
        int flag = 0;
        CUDA_TRY(c, cudaMemcpyAsync(&flag, g->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(c, cudaStreamSynchronize(s));
        if (flag) return set_err(c, ELAS_ERR_STATE, "coarsest operator is singular");
    }
    {
        int rc = setup_rhs(g);
        if (rc) return rc;
    }
    g->dirty = false;
    g->rhs_dirty = false;
    ++g->gen;
    return ELAS_OK;
}

// ---- cycles ------------------------------------------------------------------------
template <typename T>
struct Fields {
    static T* u(Level& v);
    static T* ua(Level& v);
    static T* f(Level& v);
    static T* r(Level& v);
    static const Lv<T>& L(Level& v);
};
template <>
struct Fields<double> {
    static double* u(Level& v) { return v.u; }
    static double* ua(Level& v) { return v.ua; }
    static double* f(Level& v) { return v.f; }
    static double* r(Level& v) { return v.r; }
    static const Lv<double>& L(Level& v) { return v.L64; }
};
template <>
struct Fields<float> {
    static float* u(Level& v) { return v.u32; }
    static float* ua(Level& v) { return v.ua32; }
    static float* f(Level& v) { return v.f32; }
    static float* r(Level& v) { return v.r32; }
    static const Lv<float>& L(Level& v) { return v.L32; }
};

// `sweeps` sweeps of a smoother on level l, in place on u (ping-pong through ua): red-black
// (two passes a sweep), eight colours (eight passes) or damped Jacobi (one pass).
template <typename T>
void smooth_with(elas_grid g, int l, int sweeps, int kind, double omega, T* u, T* ua, const T* f, const NullInfo* nf,
                 const double* lam) {
    Level& v = g->lv[l];
    elas_ctx c = g->ctx;
    cudaStream_t s = c->stream;
    const int cls = sizeof(T) == 8 ? ELAS_PROF_SWEEP64_L0 : ELAS_PROF_SWEEP32_L0;
    Lv<T> L = Fields<T>::L(v);
    L.omega = (T)omega;
    int passes = 0, first = 0;
    if (kind == ELAS_SMOOTH_GS8) passes = 8, first = 2;
    else if (kind == ELAS_SMOOTH_JACOBI) passes = 1, first = kJacobiColour;
    else passes = 2, first = 0;
    const int total = sweeps * passes;
    for (int k = 0; k < total; ++k) {
        const int colour = kind == ELAS_SMOOTH_JACOBI ? kJacobiColour : first + k % passes;
        const size_t e = l == 0 ? prof_begin(c, cls) : (size_t)-1;
        if (k % 2 == 0) launch_half_sweep<T>(L, u, ua, f, colour, nf, lam, s);
        else launch_half_sweep<T>(L, ua, u, f, colour, nf, lam, s);
        prof_end(c, e);
    }
    if (total % 2) cudaMemcpyAsync(u, ua, sizeof(T) * 3 * (size_t)v.N, cudaMemcpyDeviceToDevice, s);
}

template <typename T>
void smooth(elas_grid g, int l, int sweeps, const NullInfo* nf, const double* lam) {
    Level& v = g->lv[l];
    smooth_with<T>(g, l, sweeps, g->smoother, g->omega, Fields<T>::u(v), Fields<T>::ua(v), Fields<T>::f(v), nf, lam);
}

// Correction cycle on level l >= 1 (or l = 0 of the FP32 cycle): u_l from zero (or from
// its current value).  cycle: ELAS_CYCLE_V, or ELAS_CYCLE_F, whose coarse-grid correction
// is an F-cycle on the next level followed by a V-cycle from its result (Section 3.1).
// From the finest level the cycles of the coarser levels run as captured graphs
// (run_cycle); below it they recurse directly (inside such a capture).
template <typename T>
void run_cycle(elas_grid g, int l, int nu1, int nu2, const NullInfo* nf, const double* dlam, bool zero_init,
               int cycle);

template <typename T>
void vcycle(elas_grid g, int l, int nu1, int nu2, const NullInfo* nf0, const double* dlam0, bool zero_init = true,
            int cycle = ELAS_CYCLE_V) {
    Level& v = g->lv[l];
    cudaStream_t s = g->ctx->stream;
    const int nl = (int)g->lv.size();
    if (l == nl - 1) {
        launch_bottom_solve<T>(Fields<T>::L(v), g->dofs, g->nfree, g->ntot, g->Ainv, Fields<T>::f(v), Fields<T>::u(v),
                               g->bwork, s);
        return;
    }
    const NullInfo* nf = (l == 0) ? nf0 : nullptr;
    const double* lam = (l == 0) ? dlam0 : nullptr;
    if (zero_init) cudaMemsetAsync(Fields<T>::u(v), 0, sizeof(T) * 3 * (size_t)v.N, s);
    smooth<T>(g, l, nu1, nf, lam);
    const size_t e = l == 0 ? prof_begin(g->ctx, sizeof(T) == 8 ? ELAS_PROF_RESID64_L0 : ELAS_PROF_RESID32_L0)
                            : (size_t)-1;
    launch_residual<T, T>(Fields<T>::L(v), Fields<T>::u(v), Fields<T>::f(v), nf, lam, Fields<T>::r(v), nullptr,
                          nullptr, s);
    prof_end(g->ctx, e);
    Level& w = g->lv[l + 1];
    launch_restrict<T>(Fields<T>::L(v), Fields<T>::L(w), Fields<T>::r(v), Fields<T>::f(w), nullptr, nullptr, s);
    auto descend = l == 0 ? run_cycle<T> : vcycle<T>;
    if (cycle == ELAS_CYCLE_F) {
        descend(g, l + 1, nu1, nu2, nullptr, nullptr, true, ELAS_CYCLE_F);
        descend(g, l + 1, nu1, nu2, nullptr, nullptr, false, ELAS_CYCLE_V);
    } else {
        descend(g, l + 1, nu1, nu2, nullptr, nullptr, true, ELAS_CYCLE_V);
    }
    launch_prolong_add<T>(Fields<T>::L(v), Fields<T>::L(w), Fields<T>::u(w), Fields<T>::u(v), s);
    smooth<T>(g, l, nu2, nf, lam);
}

void cycle_graphs_free(elas_grid g) {
    for (auto& kv : g->cyc)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    g->cyc.clear();
}

// One multigrid cycle from level l (vcycle's arguments), launched from a CUDA graph of
// its whole launch sequence.  A cycle below the finest level is several dozen launches
// of small kernels, so launching them one by one costs more host time than the GPU
// spends on them; the graph of each (precision, level, start, cycle type) is captured
// on first use and replayed until the set-up, the launch-shape table, the smoothing
// options or the stream change.  Levels below the finest hold no profiled launches.
// With a batch's activity flags set, within another capture, or where the stream cannot
// be captured, the cycle is launched directly.  Replays compute exactly what the direct
// launches compute.
template <typename T>
void run_cycle(elas_grid g, int l, int nu1, int nu2, const NullInfo* nf, const double* dlam, bool zero_init,
               int cycle) {
    elas_ctx c = g->ctx;
    cudaStream_t s = c->stream;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        cs = cudaStreamCaptureStatusActive;
    }
    if (l == 0 || cs != cudaStreamCaptureStatusNone || g->lv[l].L32.active || g->lv[l].L64.active) {
        vcycle<T>(g, l, nu1, nu2, nf, dlam, zero_init, cycle);
        return;
    }
    const unsigned long long tv = tune_version();
    if (g->cyc_gen != g->gen || g->cyc_tune != tv || g->cyc_nu1 != nu1 || g->cyc_nu2 != nu2 ||
        g->cyc_smoother != g->smoother || g->cyc_omega != g->omega || g->cyc_stream != s ||
        g->cyc_nf != (const void*)nf || g->cyc_dlam != (const void*)dlam) {
        cycle_graphs_free(g);
        g->cyc_gen = g->gen;
        g->cyc_tune = tv;
        g->cyc_nu1 = nu1;
        g->cyc_nu2 = nu2;
        g->cyc_smoother = g->smoother;
        g->cyc_omega = g->omega;
        g->cyc_stream = s;
        g->cyc_nf = nf;
        g->cyc_dlam = dlam;
    }
    const int key = (sizeof(T) == 8 ? 1 << 16 : 0) | (l << 8) | (zero_init ? 2 : 0) | (cycle == ELAS_CYCLE_F ? 1 : 0);
    auto it = g->cyc.find(key);
    if (it == g->cyc.end()) {
        elas_grid_s::CycleGraph cg;
        const unsigned long long l0 = launch_count();
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            vcycle<T>(g, l, nu1, nu2, nf, dlam, zero_init, cycle);
            const cudaError_t e = cudaStreamEndCapture(s, &graph);
            if (e == cudaSuccess && graph && cudaGraphInstantiate(&cg.exec, graph, 0) != cudaSuccess) cg.exec = nullptr;
        }
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();   // a refused capture leaves no error behind: launch directly
        cg.launches = (int)(launch_count() - l0);
        count_launch(-cg.launches);   // captured, not launched: counted per replay
        it = g->cyc.emplace(key, cg).first;
    }
    if (it->second.exec && cudaGraphLaunch(it->second.exec, s) == cudaSuccess) {
        count_launch(it->second.launches);
        return;
    }
    cudaGetLastError();
    vcycle<T>(g, l, nu1, nu2, nf, dlam, zero_init, cycle);
}

// The refinement residual of a mixed solve: double-float (from the grid's double-float
// copies, kept in step with u by outer_begin and outer_correct) or FP64, both written as
// FP32 into the FP32 level's right-hand side with FP64 block partials of the norms.
// The copies are made on the first solve that takes the double-float residual (grids of
// AMR layouts never do) and refreshed after each full set-up.
constexpr double kDfMinTol = 1e-11;   // AUTO: below this tolerance the FP64 residual
bool outer_df(elas_grid g, const elas_solve_opts* o) {
    if (!g->desc.mixed || g->lv.size() < 2 || o->outer_residual == ELAS_OUTER_FP64) return false;
    if (o->outer_residual == ELAS_OUTER_DF) return true;
    return o->fixed_cycles > 0 || o->rel_tol >= kDfMinTol;
}

// Allocate (once) and fill (after a set-up) the double-float copies of the finest level's
// moduli, divergence and stored rows; u and f are split at the start of each solve.  Each
// copy is allocated on its own, so a call after a refused allocation completes the set.
int df_prepare(elas_grid g) {
    Level& v = g->lv[0];
    const size_t N = (size_t)v.N;
    int rc = ELAS_OK;
    if (!v.m2 || !v.u2 || !v.f2 || (v.nbnd && !v.bc2)) {
        g->df_gen = ~0ull;
        if (!v.m2) rc = galloc(g, &v.m2, (size_t)(g->K == 21 ? 39 : 2) * N);
        if (!rc && !v.u2) rc = galloc(g, &v.u2, 3 * N);
        if (!rc && !v.f2) rc = galloc(g, &v.f2, 3 * N);
        if (!rc && v.nbnd && !v.bc2) rc = galloc(g, &v.bc2, (size_t)v.nbnd * kEdgeCoef);
        if (rc) return rc;
    }
    if (g->df_gen != g->gen) {
        elas_ctx c = g->ctx;
        cudaStream_t s = c->stream;
        launch_split_df(v.mod64, v.m2, (size_t)g->K * N, s);
        if (v.divc) launch_split_df(v.divc, v.m2 + 21 * N, 18 * N, s);
        if (v.bc2) launch_split_df(v.bcoef64, v.bc2, (size_t)v.nbnd * kEdgeCoef, s);
        CHECK_LAUNCH(c);
        g->df_gen = g->gen;
    }
    return ELAS_OK;
}

void outer_begin(elas_grid g, bool df, cudaStream_t s) {
    if (!df) return;
    Level& L0 = g->lv[0];
    launch_split_df(L0.u, L0.u2, 3 * (size_t)L0.N, s);
    launch_split_df(L0.f, L0.f2, 3 * (size_t)L0.N, s);
}

void outer_residual(elas_grid g, bool df, const NullInfo* nf0, const double* load, int* nb, cudaStream_t s) {
    Level& L0 = g->lv[0];
    if (df) launch_residual_df(df_view(L0), L0.u2, L0.f2, nf0, load, L0.f32, g->partials, nb, s);
    else launch_residual<double, float>(L0.L64, L0.u, L0.f, nf0, load, L0.f32, g->partials, nb, s);
}

void outer_correct(elas_grid g, bool df, cudaStream_t s) {
    Level& L0 = g->lv[0];
    if (df) launch_add_correction_df(L0.L64, L0.u, L0.u32, L0.u2, s);
    else launch_add_correction(L0.L64, L0.u, L0.u32, s);
}

// Every member of a batch takes the same residual arithmetic.
bool batch_df(elas_grid* grids, int n, const elas_solve_opts* o) {
    for (int i = 0; i < n; ++i)
        if (!outer_df(grids[i], o)) return false;
    return n > 0;
}

int remove_rigid(elas_grid g) {
    Level& L0 = g->lv[0];
    if (L0.nf.m == 0) return ELAS_OK;
    elas_ctx c = g->ctx;
    int nb = 0;
    launch_null_dots(L0.L64, L0.nf, L0.u, g->partials, &nb, 0, c->stream);
    CHECK_LAUNCH(c);
    launch_sum_partials(g->partials, nb, 6, g->status + 8, c->stream);
    CHECK_LAUNCH(c);
    launch_remove_null(L0.L64, L0.nf, g->Ginv, g->status + 8, g->status + 16, L0.u, c->stream);
    CHECK_LAUNCH(c);
    return ELAS_OK;
}

int level_alloc(elas_grid g, Level& v, bool mixed) {
    int rc;
    const size_t N = (size_t)v.N;
    if ((rc = galloc(g, &v.mod64, (size_t)g->K * N))) return rc;
    if (g->K == 21 && (rc = galloc(g, &v.divc, 18 * N))) return rc;
    if ((rc = galloc(g, &v.u, 3 * N))) return rc;
    if ((rc = galloc(g, &v.ua, 3 * N))) return rc;
    if ((rc = galloc(g, &v.f, 3 * N))) return rc;
    if ((rc = galloc(g, &v.r, 3 * N))) return rc;
    if (mixed) {
        v.split = !g->desc.half_moduli && split_layout_applies(v.n, g->K);
        if (g->desc.half_moduli) {
            if ((rc = galloc(g, &v.mod16, moduli_copy_entries(v.N, g->K, true)))) return rc;
        } else if (v.split) {
            if ((rc = galloc(g, &v.mod32, split_entries(v.N)))) return rc;
        } else if ((rc = galloc(g, &v.mod32, moduli_copy_entries(v.N, g->K, false)))) {
            return rc;
        }
        if ((rc = galloc(g, &v.u32, 3 * N))) return rc;
        if ((rc = galloc(g, &v.ua32, 3 * N))) return rc;
        if ((rc = galloc(g, &v.f32, 3 * N))) return rc;
        if ((rc = galloc(g, &v.r32, 3 * N))) return rc;
    }
    v.L64.mod = v.mod64;
    v.L32.mod = v.mod32;
    v.L32.mlay = v.mod16 ? kModRecords : (v.split ? kModSplit : (v.mod32 ? kModBlocked : kModPlanes));
    v.L32.msplit1 = v.split ? split_half_entries((v.N + 1) / 2) : 0;
    // lists of the nodes whose rows are stored as coefficients (the FP64 level's and the
    // FP32 copy's): the nodes on two or three boundary planes, and the face nodes of the
    // directions in face_list_mask; the other face nodes are enumerated arithmetically by
    // the face kernels
    const int* per = g->desc.periodic;
    const int m64 = face_list_mask(v.n, per, false, g->K == 21), m32 = face_list_mask(v.n, per, true, g->K == 21);
    auto make_list = [&](int fmask) {
        std::vector<int> b;
        for (int z = 0; z < v.n[2]; ++z)
            for (int y = 0; y < v.n[1]; ++y)
                for (int x = 0; x < v.n[0]; ++x) {
                    const int fx = !per[0] && (x == 0 || x == v.n[0] - 1);
                    const int fy = !per[1] && (y == 0 || y == v.n[1] - 1);
                    const int fz = !per[2] && (z == 0 || z == v.n[2] - 1);
                    const int on = fx + fy + fz;
                    const int dirs = fx | (fy << 1) | (fz << 2);
                    if (on >= 2 || (on == 1 && (dirs & fmask))) b.push_back(x + v.n[0] * (y + v.n[1] * z));
                }
        return b;
    };
    elas_ctx c = g->ctx;
    const std::vector<int> b64 = make_list(m64);
    v.L64.xface_list = m64;
    v.nbnd = (int)b64.size();
    if (v.nbnd) {
        if ((rc = galloc(g, &v.bnd, b64.size()))) return rc;
        if ((rc = galloc(g, &v.bcoef64, b64.size() * kEdgeCoef))) return rc;
        CUDA_TRY(c, cudaMemcpyAsync(v.bnd, b64.data(), sizeof(int) * b64.size(), cudaMemcpyHostToDevice, c->stream));
    }
    v.L32.xface_list = m32;
    if (mixed) {
        const std::vector<int> b32 = m32 == m64 ? b64 : make_list(m32);
        v.nbnd32 = (int)b32.size();
        if (v.nbnd32) {
            if (m32 == m64) {
                v.bnd32 = v.bnd;
            } else {
                if ((rc = galloc(g, &v.bnd32, b32.size()))) return rc;
                CUDA_TRY(c, cudaMemcpyAsync(v.bnd32, b32.data(), sizeof(int) * b32.size(), cudaMemcpyHostToDevice,
                                            c->stream));
            }
            if ((rc = galloc(g, &v.bcoef32, b32.size() * kEdgeCoef))) return rc;
        }
    }
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return ELAS_OK;
}

void refresh_lv(elas_grid g) {
    const int nl = (int)g->lv.size();
    for (int l = 0; l < nl; ++l) {
        Level& v = g->lv[l];
        double h[3];
        for (int d = 0; d < 3; ++d) {
            const double span = g->desc.hi[d] - g->desc.lo[d];
            const double h0 = g->desc.periodic[d] ? span / g->desc.n[d] : span / (g->desc.n[d] - 1);
            h[d] = h0 * (double)(1 << l);
        }
        fill_lv(v.L64, v.n, g->desc.periodic, h, g->K, g->bc_type);
        fill_lv(v.L32, v.n, g->desc.periodic, h, g->K, g->bc_type);
        v.L64.mod = v.mod64;
        v.L32.mod = v.mod32;
        v.L64.bnodes = v.bnd;
        v.L32.bnodes = v.bnd32;
        v.L64.bcoef = v.bcoef64;
        v.L32.bcoef = v.bcoef32;
        v.L64.nbnd = v.nbnd;
        v.L32.nbnd = v.nbnd32;
        v.L64.xface_list = face_list_mask(v.n, g->desc.periodic, false, g->K == 21);
        v.L32.xface_list = face_list_mask(v.n, g->desc.periodic, true, g->K == 21);
        v.L64.divc = v.divc;
        v.L32.modh = v.mod16;
        v.L32.mlay = v.mod16 ? kModRecords : (v.split ? kModSplit : (v.mod32 ? kModBlocked : kModPlanes));
        v.L32.msplit1 = v.split ? split_half_entries((v.N + 1) / 2) : 0;
        v.nf = null_space(g->desc, v.n, h, g->bc_type);
    }
}

int rebuild_bottom_dofs(elas_grid g) {
    Level& B = g->lv.back();
    std::vector<int> dofs;
    int c[3];
    for (int comp = 0; comp < 3; ++comp)
        for (c[2] = 0; c[2] < B.n[2]; ++c[2])
            for (c[1] = 0; c[1] < B.n[1]; ++c[1])
                for (c[0] = 0; c[0] < B.n[0]; ++c[0])
                    if (host_row_type(g->bc_type, g->desc.periodic, B.n, c, comp) != ROW_DIRICHLET)
                        dofs.push_back(comp * B.N + c[0] + B.n[0] * (c[1] + B.n[1] * c[2]));
    int nfree = (int)dofs.size();
    int ntot = nfree + B.nf.m;
    elas_ctx ctx = g->ctx;
    if (g->desc.max_levels == 1) {
        nfree = ntot = 0;   // smoothed only, no bottom solve
        g->nfree = g->ntot = 0;
        return ELAS_OK;
    }
    if (ntot > 6000)
        return set_err(ctx, ELAS_ERR_INVALID_ARG,
                       "node counts do not coarsen to a small bottom level (use n = 2^k m + 1 with small m)");
    if (ntot != g->ntot || !g->dofs) {
        // (re)allocate: sizes change only with the boundary types
        int rc;
        if ((rc = galloc(g, &g->dofs, (size_t)3 * B.N + 1))) return rc;
        if ((rc = galloc(g, &g->Ainv, (size_t)ntot * ntot + 1))) return rc;
        if ((rc = galloc(g, &g->Awork, (size_t)ntot * ntot + 1))) return rc;
        if ((rc = galloc(g, &g->bwork, (size_t)ntot + 1))) return rc;
    }
    g->nfree = nfree;
    g->ntot = ntot;
    if (nfree > 0)
        CUDA_TRY(ctx, cudaMemcpyAsync(g->dofs, dofs.data(), sizeof(int) * nfree, cudaMemcpyHostToDevice, ctx->stream));
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return ELAS_OK;
}

int copy_in(elas_ctx c, double* dst, const double* src, size_t count, int memspace) {
    CUDA_TRY(c, cudaMemcpyAsync(dst, src, sizeof(double) * count,
                                memspace == ELAS_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return ELAS_OK;
}

}  // namespace

namespace {
void plan_free(elas_ctx c, BatchPlan* p);
bool plan_has_member(const BatchPlan* p, elas_grid g);
bool batch_engine_applies(elas_grid* grids, int n, const elas_solve_opts* o);
int batch_engine(elas_grid* grids, int n, const elas_solve_opts* o, elas_solve_info* info,
                 std::chrono::steady_clock::time_point t0);
}  // namespace

// ======================================================================================
// C ABI
// ======================================================================================
extern "C" {

int elas_ctx_create(elas_ctx* out, int device, size_t hbm_budget_bytes, const elas_allocator* alloc, void* stream) {
    if (!out) return ELAS_ERR_INVALID_ARG;
    elas_ctx c = new elas_ctx_s();
    c->device = device;
    c->budget = hbm_budget_bytes;
    if (alloc && alloc->alloc && alloc->free) {
        c->alloc = *alloc;
        c->has_alloc = true;
    }
    if (cudaSetDevice(device) != cudaSuccess) {
        delete c;
        return ELAS_ERR_DEVICE;
    }
    if (stream) {
        c->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return ELAS_ERR_DEVICE;
        }
        c->own_stream = true;
    }
    if (cudaMallocHost(&c->host_status, 64 * sizeof(double)) != cudaSuccess) {
        delete c;
        return ELAS_ERR_DEVICE;
    }
    *out = c;
    return ELAS_OK;
}

int elas_ctx_destroy(elas_ctx c) {
    if (!c) return ELAS_ERR_INVALID_ARG;
    if (!c->servers.empty()) return set_err(c, ELAS_ERR_STATE, "the context has live servers");
    cudaStreamSynchronize(c->stream);
    plan_free(c, c->plan);
    c->plan = nullptr;
    for (auto e : c->pool) cudaEventDestroy(e);
    for (auto st : c->branch) cudaStreamDestroy(st);
    for (auto e : c->branch_ev) cudaEventDestroy(e);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    if (c->host_status) cudaFreeHost(c->host_status);
    delete c;
    return ELAS_OK;
}

const char* elas_last_error(elas_ctx c) { return c ? c->err.c_str() : "null context"; }
size_t elas_ctx_bytes_in_use(elas_ctx c) { return c ? c->in_use : 0; }

size_t elas_grid_bytes_estimate(const elas_grid_desc* d) {
    if (!d) return 0;
    const int K = d->moduli_kind;
    size_t total = 0;
    const auto dims = level_dims(*d);
    for (auto& n : dims) {
        const size_t N = (size_t)n[0] * n[1] * n[2];
        total += N * 8 * (K + 12 + (K == 21 ? 18 : 0));
        if (d->mixed) {
            const bool split = !d->half_moduli && split_layout_applies(n.data(), K);
            total += (d->half_moduli ? 2 : 4) * (split ? split_entries((int)N) : moduli_copy_entries((int)N, K, d->half_moduli)) +
                     N * 48;
        }
        // stored rows: edges and corners, and the x faces
        auto stored_for = [&](int fm) {
            return (size_t)4 * (n[0] + n[1] + n[2]) + ((fm & 1) ? (size_t)2 * n[1] * n[2] : 0) +
                   ((fm & 2) ? (size_t)2 * n[0] * n[2] : 0) + ((fm & 4) ? (size_t)2 * n[0] * n[1] : 0);
        };
        const size_t stored = stored_for(face_list_mask(n.data(), d->periodic, false, K == 21));
        total += stored * kEdgeCoef * 8;
        if (d->mixed) total += stored_for(face_list_mask(n.data(), d->periodic, true, K == 21)) * kEdgeCoef * 4;
        if (d->mixed && d->max_levels != 1 && &n == &dims.front())   // double-float copies of the finest level
            total += 8 * (N * ((K == 21 ? 39 : 2) + 6) + stored * kEdgeCoef);
    }
    const size_t N0 = (size_t)d->n[0] * d->n[1] * d->n[2];
    total += N0 * 8 * 9;   // eigenstrain + body force when given
    return total;
}

int elas_grid_create(elas_ctx c, const elas_grid_desc* d, elas_grid* out) {
    if (!c || !d || !out) return ELAS_ERR_INVALID_ARG;
    if (d->moduli_kind != ELAS_MODULI_ISO && d->moduli_kind != ELAS_MODULI_GEN21)
        return set_err(c, ELAS_ERR_INVALID_ARG, "moduli_kind must be 2 or 21");
    for (int k = 0; k < 3; ++k) {
        if (d->periodic[k] ? d->n[k] < 4 : d->n[k] < 3)
            return set_err(c, ELAS_ERR_INVALID_ARG, "too few nodes in a direction");
        if (!(d->hi[k] > d->lo[k])) return set_err(c, ELAS_ERR_INVALID_ARG, "empty domain");
    }
    const double N0 = (double)d->n[0] * d->n[1] * d->n[2];
    if (N0 * mod_record(d->moduli_kind) >= 2147483647.0 || 3.0 * N0 >= 2147483647.0)
        return set_err(c, ELAS_ERR_INVALID_ARG, "grid too large for 32-bit plane indexing");
    cudaSetDevice(c->device);
    elas_grid g = new elas_grid_s();
    g->ctx = c;
    g->desc = *d;
    g->K = d->moduli_kind;
    for (int f = 0; f < 6; ++f)
        for (int k = 0; k < 3; ++k) {
            g->bc_type[f][k] = ELAS_BC_DIRICHLET;
            g->bc_val[f][k] = 0.0;
        }
    auto dims = level_dims(*d);
    g->lv.resize(dims.size());
    int rc = ELAS_OK;
    for (size_t l = 0; l < dims.size(); ++l) {
        Level& v = g->lv[l];
        for (int k = 0; k < 3; ++k) v.n[k] = dims[l][k];
        v.N = v.n[0] * v.n[1] * v.n[2];
        if ((rc = level_alloc(g, v, d->mixed != 0))) break;
    }
    // reduction blocks of one residual launch set: interior + faces (each at most one
    // block per 256 nodes) + edges/corners (one warp per node)
    size_t maxblocks = 0;
    for (auto& v : g->lv) {
        const size_t nbl = (size_t)(v.nbnd > v.nbnd32 ? v.nbnd : v.nbnd32);
        const size_t nb = 2 * (size_t)((v.N + kBlock - 1) / kBlock) + (nbl * 32 + kBlock - 1) / kBlock + 8;
        maxblocks = nb > maxblocks ? nb : maxblocks;
    }
    const size_t nparts = maxblocks * kPartialStride + 64;
    if (!rc) rc = galloc(g, &g->partials, nparts);
    if (!rc) rc = galloc(g, &g->status, 64);
    if (!rc) rc = galloc(g, &g->G, 36);
    if (!rc) rc = galloc(g, &g->Ginv, 36);
    if (!rc) rc = galloc(g, &g->lam, 8);
    if (!rc) rc = galloc(g, &g->dlam, 8);
    if (!rc) rc = galloc(g, &g->alam, kLoadDoubles);
    if (!rc) rc = galloc(g, &g->adlam, kLoadDoubles);
    if (!rc) rc = galloc(g, &g->flag, 4);
    if (!rc) {
        refresh_lv(g);
        rc = rebuild_bottom_dofs(g);
    }
    if (rc) {
        elas_grid_destroy(g);
        return rc;
    }
    cudaMemsetAsync(g->lv[0].u, 0, sizeof(double) * 3 * (size_t)g->lv[0].N, c->stream);
    cudaMemsetAsync(g->lam, 0, sizeof(double) * 8, c->stream);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
        elas_grid_destroy(g);
        return set_err(c, ELAS_ERR_DEVICE, "grid initialisation failed");
    }
    *out = g;
    return ELAS_OK;
}

int elas_grid_destroy(elas_grid g) {
    if (!g) return ELAS_ERR_INVALID_ARG;
    elas_ctx c = g->ctx;
    if (server_holds(c, g, nullptr))
        return set_err(c, ELAS_ERR_STATE, "grid has a waiting or active server request");
    if (g->amr_refs > 0) return set_err(c, ELAS_ERR_STATE, "grid is a level of a live AMR layout");
    cudaStreamSynchronize(c->stream);
    if (plan_has_member(c->plan, g)) {
        plan_free(c, c->plan);
        c->plan = nullptr;
    }
    cycle_graphs_free(g);
    for (auto& a : g->allocs) ctx_free(c, a.first, a.second);
    cudaStreamSynchronize(c->stream);
    delete g;
    return ELAS_OK;
}

int elas_grid_levels(elas_grid g, int* nlevels) {
    if (!g || !nlevels) return ELAS_ERR_INVALID_ARG;
    *nlevels = (int)g->lv.size();
    return ELAS_OK;
}

int elas_grid_level_dims(elas_grid g, int level, int n[3]) {
    if (!g || !n || level < 0 || level >= (int)g->lv.size()) return ELAS_ERR_INVALID_ARG;
    for (int k = 0; k < 3; ++k) n[k] = g->lv[level].n[k];
    return ELAS_OK;
}

size_t elas_grid_bytes(elas_grid g) {
    if (!g) return 0;
    size_t t = 0;
    for (auto& a : g->allocs) t += a.second;
    return t;
}

int elas_set_moduli(elas_grid g, const double* comps, int memspace) {
    if (!g || !comps || (memspace != ELAS_HOST && memspace != ELAS_DEVICE)) return ELAS_ERR_INVALID_ARG;
    if (int rc = refuse_if_served(g)) return rc;
    int rc = copy_in(g->ctx, g->lv[0].mod64, comps, (size_t)g->K * g->lv[0].N, memspace);
    if (rc) return rc;
    g->moduli_set = true;
    g->dirty = true;
    return ELAS_OK;
}

// Set (src non-null) or clear one finest-level input.  A cleared input's buffer stays with
// the grid and serves the next set of the same input, so clearing and setting again
// allocates nothing.
static int set_field(elas_grid g, double** slot, const double* src, size_t count, int memspace) {
    if (src && memspace != ELAS_HOST && memspace != ELAS_DEVICE) return ELAS_ERR_INVALID_ARG;
    if (int rc = refuse_if_served(g)) return rc;
    g->rhs_dirty = true;
    if (!src) {
        if (*slot) g->kept[slot] = *slot;
        *slot = nullptr;
        return ELAS_OK;
    }
    if (!*slot) {
        auto it = g->kept.find(slot);
        if (it != g->kept.end()) {
            *slot = it->second;
            g->kept.erase(it);
        } else {
            int rc = galloc(g, slot, count);
            if (rc) return rc;
        }
    }
    return copy_in(g->ctx, *slot, src, count, memspace);
}

int elas_set_eigenstrain(elas_grid g, const double* eps6, int memspace) {
    if (!g) return ELAS_ERR_INVALID_ARG;
    return set_field(g, &g->eps0, eps6, (size_t)6 * g->lv[0].N, memspace);
}

int elas_set_body_force(elas_grid g, const double* b3, int memspace) {
    if (!g) return ELAS_ERR_INVALID_ARG;
    return set_field(g, &g->body, b3, (size_t)3 * g->lv[0].N, memspace);
}

int elas_set_mean_strain(elas_grid g, const double eps6[6]) {
    if (!g || !eps6) return ELAS_ERR_INVALID_ARG;
    if (int rc = refuse_if_served(g)) return rc;
    if (!(g->desc.periodic[0] && g->desc.periodic[1] && g->desc.periodic[2]))
        return set_err(g->ctx, ELAS_ERR_INVALID_ARG, "mean strain needs a fully periodic grid");
    for (int k = 0; k < 6; ++k) g->mean[k] = eps6[k];
    g->has_mean = 1;
    g->rhs_dirty = true;
    return ELAS_OK;
}

int elas_set_bc(elas_grid g, int face, int comp, int type, double value) {
    if (!g || face < 0 || face > 5 || comp < 0 || comp > 2) return ELAS_ERR_INVALID_ARG;
    if (int rc = refuse_if_served(g)) return rc;
    if (type != ELAS_BC_DIRICHLET && type != ELAS_BC_TRACTION && type != ELAS_BC_NEUMANN)
        return set_err(g->ctx, ELAS_ERR_INVALID_ARG, "unknown boundary type");
    const bool changed = g->bc_type[face][comp] != type;
    g->bc_type[face][comp] = type;
    g->bc_val[face][comp] = value;
    if (changed) g->dirty = true;
    else g->rhs_dirty = true;
    if (changed) {
        g->gram_valid = false;
        refresh_lv(g);
        return rebuild_bottom_dofs(g);
    }
    return ELAS_OK;
}

int elas_set_face_values(elas_grid g, int face, const double* values, int memspace) {
    if (!g || face < 0 || face > 5) return ELAS_ERR_INVALID_ARG;
    return set_field(g, &g->face[face], values, (size_t)3 * g->lv[0].N, memspace);
}

void elas_solve_opts_default(elas_solve_opts* o) {
    if (!o) return;
    o->precision = ELAS_PRECISION_FP64;
    o->rel_tol = 1e-8;
    o->max_cycles = 100;
    o->nu1 = 2;
    o->nu2 = 2;
    o->warm_start = 0;
    o->fixed_cycles = 0;
    o->use_graph = 0;
    o->inner_cycles = 1;
    o->smoother = ELAS_SMOOTH_RB;
    o->cycle = ELAS_CYCLE_V;
    o->omega = 2.0 / 3.0;
    o->outer_residual = ELAS_OUTER_AUTO;
}

namespace {
// Take the smoother and cycle of a solve's options onto the grid (checked).
int take_cycle_opts(elas_grid g, const elas_solve_opts* o) {
    if (o->smoother < ELAS_SMOOTH_RB || o->smoother > ELAS_SMOOTH_JACOBI || (o->cycle != ELAS_CYCLE_V && o->cycle != ELAS_CYCLE_F))
        return set_err(g->ctx, ELAS_ERR_INVALID_ARG, "unknown smoother or cycle");
    if (o->smoother == ELAS_SMOOTH_JACOBI && !(o->omega > 0.0 && o->omega <= 1.0))
        return set_err(g->ctx, ELAS_ERR_INVALID_ARG, "Jacobi damping must lie in (0, 1]");
    if (o->outer_residual < ELAS_OUTER_AUTO || o->outer_residual > ELAS_OUTER_DF)
        return set_err(g->ctx, ELAS_ERR_INVALID_ARG, "unknown outer residual arithmetic");
    g->smoother = o->smoother;
    g->cycle = o->cycle;
    g->omega = o->omega;
    return ELAS_OK;
}
}  // namespace

int elas_solve(elas_grid g, const elas_solve_opts* opts, elas_solve_info* info) {
    if (!g || !opts || !info) return ELAS_ERR_INVALID_ARG;
    if (int rc = refuse_if_served(g)) return rc;
    elas_ctx c = g->ctx;
    cudaSetDevice(c->device);
    std::memset(info, 0, sizeof(*info));
    const bool mixed = opts->precision == ELAS_PRECISION_MIXED;
    if (mixed && !g->desc.mixed) return set_err(c, ELAS_ERR_STATE, "grid was created without the FP32 hierarchy");
    if (g->desc.max_levels == 1) return set_err(c, ELAS_ERR_STATE, "grid has no multigrid hierarchy (AMR level)");
    if (mixed && opts->use_graph) return elas_batch_solve(&g, 1, opts, info);   // graph replay, one member
    const auto t0 = std::chrono::steady_clock::now();
    int rc = take_cycle_opts(g, opts);
    if (rc) return rc;
    rc = setup(g);
    if (rc) return rc;
    if (mixed && outer_df(g, opts) && (rc = df_prepare(g))) return rc;
    cudaStream_t s = c->stream;
    Level& L0 = g->lv[0];
    const NullInfo* nf0 = L0.nf.m > 0 ? &L0.nf : nullptr;
    launch_dirichlet(L0.L64, boundary_data(g), L0.u, opts->warm_start ? 1 : 0, s);
    const bool df = mixed && outer_df(g, opts);
    outer_begin(g, df, s);
    CHECK_LAUNCH(c);
    CUDA_TRY(c, cudaMemsetAsync(g->lam, 0, sizeof(double) * 8, s));
    CUDA_TRY(c, cudaMemsetAsync(g->alam, 0, sizeof(double) * kLoadDoubles, s));
    CUDA_TRY(c, cudaMemsetAsync(g->adlam, 0, sizeof(double) * kLoadDoubles, s));
    const double* load = nf0 ? g->alam : nullptr;     // current equilibrating load
    const double* dload = nf0 ? g->adlam : nullptr;   // its latest increment
    info->r0 = g->r0;
    info->nlam = L0.nf.m;
    const int nu1 = opts->nu1 < 0 ? 0 : opts->nu1, nu2 = opts->nu2 < 0 ? 0 : opts->nu2;
    int cycles = 0;
    double rel = 0.0, rinf = 0.0;
    int status = ELAS_OK;
    int hist = 0;
    for (;;) {
        int nb = 0;
        if (!mixed) smooth<double>(g, 0, nu1, nf0, load);
        const size_t ev = prof_begin(c, ELAS_PROF_RESID64_L0);
        if (!mixed) launch_residual<double, double>(L0.L64, L0.u, L0.f, nf0, load, L0.r, g->partials, &nb, s);
        else outer_residual(g, df, nf0, load, &nb, s);
        prof_end(c, ev);
        CHECK_LAUNCH(c);
        launch_finalize(g->partials, nb, L0.nf, g->Ginv, g->G, g->lam, g->dlam, g->alam, g->adlam, g->status, 1, s);
        CHECK_LAUNCH(c);
        double st[2];
        rc = read_status(g, st, 2);
        if (rc) return rc;
        prof_collect(c);
        rel = g->r0 > 0 ? std::sqrt(st[0]) / g->r0 : 0.0;
        rinf = st[1];
        if (hist < ELAS_HISTORY) info->rel_history[hist++] = rel;
        if (!std::isfinite(rel) || rel > 1e12) {
            status = ELAS_ERR_DIVERGED;
            break;
        }
        if (opts->fixed_cycles > 0) {
            if (cycles >= opts->fixed_cycles) break;
        } else {
            if (rel <= opts->rel_tol) break;
            if (cycles >= opts->max_cycles) {
                status = ELAS_ERR_NOT_CONVERGED;
                break;
            }
        }
        if (!mixed && g->lv.size() == 1) {
            // single level: exact (bordered) solve of the correction; any rigid-mode
            // part of r is absorbed by the bordering, so r needs no equilibration here
            launch_bottom_solve<double>(L0.L64, g->dofs, g->nfree, g->ntot, g->Ainv, L0.r, L0.ua, g->bwork, s);
            launch_add_correction64(L0.L64, L0.u, L0.ua, s);
            smooth<double>(g, 0, nu2, nf0, load);
        } else if (!mixed) {
            Level& L1 = g->lv[1];
            launch_restrict<double>(L0.L64, L1.L64, L0.r, L1.f, nf0, dload, s);
            if (g->cycle == ELAS_CYCLE_F) {
                run_cycle<double>(g, 1, nu1, nu2, nullptr, nullptr, true, ELAS_CYCLE_F);
                run_cycle<double>(g, 1, nu1, nu2, nullptr, nullptr, false, ELAS_CYCLE_V);
            } else {
                run_cycle<double>(g, 1, nu1, nu2, nullptr, nullptr, true, ELAS_CYCLE_V);
            }
            launch_prolong_add<double>(L0.L64, L1.L64, L1.u, L0.u, s);
            smooth<double>(g, 0, nu2, nf0, load);
        } else {
            // FP32 V-cycles on the correction equation, the first from zero
            const int inner = opts->inner_cycles > 1 ? opts->inner_cycles : 1;
            for (int k = 0; k < inner; ++k) vcycle<float>(g, 0, nu1, nu2, nf0, dload, k == 0, g->cycle);
            outer_correct(g, df, s);
        }
        CHECK_LAUNCH(c);
        ++cycles;
    }
    rc = remove_rigid(g);
    if (rc) return rc;
    double lam[8] = {0};
    if (L0.nf.m > 0) {
        CUDA_TRY(c, cudaMemcpyAsync(c->host_status, g->lam, sizeof(double) * L0.nf.m, cudaMemcpyDeviceToHost, s));
    }
    CUDA_TRY(c, cudaStreamSynchronize(s));
    for (int q = 0; q < L0.nf.m; ++q) lam[q] = c->host_status[q];
    for (int q = 0; q < 6; ++q) info->lam[q] = lam[q];
    info->cycles = cycles;
    info->rel_residual = rel;
    info->residual_inf = rinf;
    info->rel_residual_inf = g->r0inf > 0 ? rinf / g->r0inf : 0.0;
    info->status = status;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (status == ELAS_ERR_NOT_CONVERGED) set_err(c, status, "maximum cycles reached above the tolerance");
    if (status == ELAS_ERR_DIVERGED) set_err(c, status, "residual diverged");
    return status;
}

int elas_get_displacement(elas_grid g, double* out, int memspace) {
    if (!g || !out || (memspace != ELAS_HOST && memspace != ELAS_DEVICE)) return ELAS_ERR_INVALID_ARG;
    elas_ctx c = g->ctx;
    CUDA_TRY(c, cudaMemcpyAsync(out, g->lv[0].u, sizeof(double) * 3 * (size_t)g->lv[0].N,
                                memspace == ELAS_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return ELAS_OK;
}

int elas_get_stress(elas_grid g, double* out, int memspace) {
    if (!g || !out || (memspace != ELAS_HOST && memspace != ELAS_DEVICE)) return ELAS_ERR_INVALID_ARG;
    if (int rc = refuse_if_served(g)) return rc;
    elas_ctx c = g->ctx;
    cudaSetDevice(c->device);
    if (!g->moduli_set) return set_err(c, ELAS_ERR_STATE, "moduli not set");
    Level& L0 = g->lv[0];
    const size_t count = (size_t)6 * L0.N;
    double* dst = (double*)out;
    void* tmp = nullptr;
    if (memspace == ELAS_HOST) {
        tmp = ctx_alloc(c, sizeof(double) * count);
        if (!tmp) return set_err(c, ELAS_ERR_ALLOC, "stress output buffer: allocation failed");
        dst = (double*)tmp;
    }
    MeanStrain ms{};
    if (g->has_mean)
        for (int k = 0; k < 6; ++k) ms.e[k] = g->mean[k];
    launch_stress(L0.L64, L0.u, g->eps0, ms, dst, c->stream);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && tmp)
        e = cudaMemcpyAsync(out, tmp, sizeof(double) * count, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (tmp) ctx_free(c, tmp, sizeof(double) * count);
    if (e != cudaSuccess) return set_err(c, ELAS_ERR_DEVICE, std::string("stress: ") + cudaGetErrorString(e));
    return ELAS_OK;
}

int elas_set_displacement(elas_grid g, const double* in, int memspace) {
    if (!g || !in || (memspace != ELAS_HOST && memspace != ELAS_DEVICE)) return ELAS_ERR_INVALID_ARG;
    if (int rc = refuse_if_served(g)) return rc;
    return copy_in(g->ctx, g->lv[0].u, in, (size_t)3 * g->lv[0].N, memspace);
}

int elas_query_residual(elas_grid g, double* rel_l2, double* abs_l2) {
    if (!g) return ELAS_ERR_INVALID_ARG;
    if (int rc = refuse_if_served(g)) return rc;
    int rc = setup(g);
    if (rc) return rc;
    elas_ctx c = g->ctx;
    Level& L0 = g->lv[0];
    const NullInfo* nf0 = L0.nf.m > 0 ? &L0.nf : nullptr;
    int nb = 0;
    launch_residual<double, double>(L0.L64, L0.u, L0.f, nf0, nf0 ? g->alam : nullptr, L0.r, g->partials, &nb,
                                    c->stream);
    CHECK_LAUNCH(c);
    launch_finalize(g->partials, nb, L0.nf, g->Ginv, g->G, g->lam, g->dlam, g->alam, g->adlam, g->status, 0,
                    c->stream);
    CHECK_LAUNCH(c);
    double st[1];
    rc = read_status(g, st, 1);
    if (rc) return rc;
    if (abs_l2) *abs_l2 = std::sqrt(st[0]);
    if (rel_l2) *rel_l2 = g->r0 > 0 ? std::sqrt(st[0]) / g->r0 : 0.0;
    return ELAS_OK;
}

int elas_query_residual_inf(elas_grid g, double* rel_inf, double* abs_inf) {
    if (!g) return ELAS_ERR_INVALID_ARG;
    if (int rc = refuse_if_served(g)) return rc;
    int rc = setup(g);
    if (rc) return rc;
    elas_ctx c = g->ctx;
    Level& L0 = g->lv[0];
    const NullInfo* nf0 = L0.nf.m > 0 ? &L0.nf : nullptr;
    int nb = 0;
    launch_residual<double, double>(L0.L64, L0.u, L0.f, nf0, nf0 ? g->alam : nullptr, L0.r, g->partials, &nb,
                                    c->stream);
    CHECK_LAUNCH(c);
    launch_finalize(g->partials, nb, L0.nf, g->Ginv, g->G, g->lam, g->dlam, g->alam, g->adlam, g->status, 0,
                    c->stream);
    CHECK_LAUNCH(c);
    double st[2];
    rc = read_status(g, st, 2);
    if (rc) return rc;
    if (abs_inf) *abs_inf = st[1];
    if (rel_inf) *rel_inf = g->r0inf > 0 ? st[1] / g->r0inf : 0.0;
    return ELAS_OK;
}

// ---- single operations ----------------------------------------------------------------
static int check_level(elas_grid g, int level, int precision, bool allow_df = false) {
    if (!g) return ELAS_ERR_INVALID_ARG;
    if (int rc = refuse_if_served(g)) return rc;
    if (level < 0 || level >= (int)g->lv.size()) return set_err(g->ctx, ELAS_ERR_INVALID_ARG, "bad level");
    if (precision < 0 || precision > (allow_df ? ELAS_OP_DF : 1))
        return set_err(g->ctx, ELAS_ERR_INVALID_ARG, "bad precision");
    if (precision == 1 && !g->desc.mixed) return set_err(g->ctx, ELAS_ERR_STATE, "no FP32 hierarchy");
    return setup(g);
}

int elas_op_apply(elas_grid g, int level, int precision, const void* u, void* out) {
    if (!g || !u || !out) return ELAS_ERR_INVALID_ARG;
    int rc = check_level(g, level, precision);
    if (rc) return rc;
    Level& v = g->lv[level];
    if (precision == 0) launch_apply<double>(v.L64, (const double*)u, (double*)out, g->ctx->stream);
    else launch_apply<float>(v.L32, (const float*)u, (float*)out, g->ctx->stream);
    CHECK_LAUNCH(g->ctx);
    CUDA_TRY(g->ctx, cudaStreamSynchronize(g->ctx->stream));
    return ELAS_OK;
}

int elas_op_residual(elas_grid g, int level, int precision, const void* u, const void* f, void* r, double* sumsq) {
    if (!g || !u || !f || !r) return ELAS_ERR_INVALID_ARG;
    int rc = check_level(g, level, precision, true);
    if (rc) return rc;
    Level& v = g->lv[level];
    int nb = 0;
    if (precision == ELAS_OP_DF) {
        // double-float residual of the finest level of a mixed grid (the refinement residual)
        elas_solve_opts o;
        elas_solve_opts_default(&o);
        o.outer_residual = ELAS_OUTER_DF;
        if (level != 0 || !outer_df(g, &o))
            return set_err(g->ctx, ELAS_ERR_STATE, "double-float residual: finest level of a mixed grid with a hierarchy only");
        if ((rc = df_prepare(g))) return rc;
        launch_split_df((const double*)u, v.u2, 3 * (size_t)v.N, g->ctx->stream);
        launch_split_df((const double*)f, v.f2, 3 * (size_t)v.N, g->ctx->stream);
        launch_residual_df(df_view(v), v.u2, v.f2, nullptr, nullptr, (float*)r, g->partials, &nb, g->ctx->stream);
    } else if (precision == 0)
        launch_residual<double, double>(v.L64, (const double*)u, (const double*)f, nullptr, nullptr, (double*)r,
                                        g->partials, &nb, g->ctx->stream);
    else
        launch_residual<float, float>(v.L32, (const float*)u, (const float*)f, nullptr, nullptr, (float*)r,
                                      g->partials, &nb, g->ctx->stream);
    CHECK_LAUNCH(g->ctx);
    launch_sum_partials(g->partials, nb, 1, g->status, g->ctx->stream);
    double st[1];
    rc = read_status(g, st, 1);
    if (rc) return rc;
    if (sumsq) *sumsq = st[0];
    return ELAS_OK;
}

// ---- residual without allocation: reduction scratch in a file-scope device array ----
static __device__ __align__(256) double g_noalloc_scratch[ELAS_NOALLOC_SCRATCH_DOUBLES];

// Device address of the scratch array, looked up once per device with that device
// current (a host-side use of the symbol itself would not be a device address).
static double* noalloc_scratch(elas_ctx c) {
    static std::mutex mu;
    static std::map<int, double*> addr;
    std::lock_guard<std::mutex> lk(mu);
    auto it = addr.find(c->device);
    if (it != addr.end()) return it->second;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return nullptr;
    if (cur != c->device && cudaSetDevice(c->device) != cudaSuccess) return nullptr;
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (cur != c->device) cudaSetDevice(cur);
    if (e != cudaSuccess || !p) return nullptr;
    addr[c->device] = (double*)p;
    return (double*)p;
}

int elas_op_residual_noalloc(elas_grid g, int level, int precision, const void* u, const void* f, void* r,
                             double* sumsq) {
    if (!g || !u || !f || !r) return ELAS_ERR_INVALID_ARG;
    elas_ctx c = g->ctx;
    // the grid's set-up (after new moduli, boundary types or loads) may allocate, so this
    // entry point refuses to run it
    if (g->dirty || g->rhs_dirty)
        return set_err(c, ELAS_ERR_STATE, "grid set-up pending: call a solve or elas_op_residual first");
    int rc = check_level(g, level, precision);
    if (rc) return rc;
    Level& v = g->lv[level];
    // blocks of one residual launch set (interior, faces, edges), as sized at grid creation
    const size_t nb_max =
        2 * (size_t)((v.N + kBlock - 1) / kBlock) + ((size_t)(precision == 0 ? v.nbnd : v.nbnd32) * 32 + kBlock - 1) / kBlock + 8;
    if (nb_max * kPartialStride + 8 > (size_t)ELAS_NOALLOC_SCRATCH_DOUBLES)
        return set_err(c, ELAS_ERR_INVALID_ARG, "level too large for the no-allocation residual's static scratch");
    double* scratch = noalloc_scratch(c);
    if (!scratch) return set_err(c, ELAS_ERR_DEVICE, "cudaGetSymbolAddress of the static scratch failed");
    double* out = scratch + (ELAS_NOALLOC_SCRATCH_DOUBLES - 8);   // the final sum's slot
    int nb = 0;
    if (precision == 0)
        launch_residual<double, double>(v.L64, (const double*)u, (const double*)f, nullptr, nullptr, (double*)r,
                                        scratch, &nb, c->stream);
    else
        launch_residual<float, float>(v.L32, (const float*)u, (const float*)f, nullptr, nullptr, (float*)r, scratch,
                                      &nb, c->stream);
    CHECK_LAUNCH(c);
    launch_sum_partials(scratch, nb, 1, out, c->stream);
    CHECK_LAUNCH(c);
    double h = 0.0;
    CUDA_TRY(c, cudaMemcpyAsync(&h, out, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (sumsq) *sumsq = h;
    return ELAS_OK;
}

int elas_op_sweep(elas_grid g, int level, int precision, void* u, const void* f) {
    if (!g || !u || !f) return ELAS_ERR_INVALID_ARG;
    int rc = check_level(g, level, precision);
    if (rc) return rc;
    Level& v = g->lv[level];
    cudaStream_t s = g->ctx->stream;
    if (precision == 0) {
        launch_half_sweep<double>(v.L64, (const double*)u, v.ua, (const double*)f, 0, nullptr, nullptr, s);
        launch_half_sweep<double>(v.L64, v.ua, (double*)u, (const double*)f, 1, nullptr, nullptr, s);
    } else {
        launch_half_sweep<float>(v.L32, (const float*)u, v.ua32, (const float*)f, 0, nullptr, nullptr, s);
        launch_half_sweep<float>(v.L32, v.ua32, (float*)u, (const float*)f, 1, nullptr, nullptr, s);
    }
    CHECK_LAUNCH(g->ctx);
    CUDA_TRY(g->ctx, cudaStreamSynchronize(s));
    return ELAS_OK;
}

int elas_op_smooth(elas_grid g, int level, int precision, int smoother, double omega, void* u, const void* f) {
    if (!g || !u || !f) return ELAS_ERR_INVALID_ARG;
    int rc = check_level(g, level, precision);
    if (rc) return rc;
    if (smoother < ELAS_SMOOTH_RB || smoother > ELAS_SMOOTH_JACOBI)
        return set_err(g->ctx, ELAS_ERR_INVALID_ARG, "unknown smoother");
    Level& v = g->lv[level];
    if (precision == 0) smooth_with<double>(g, level, 1, smoother, omega, (double*)u, v.ua, (const double*)f, nullptr, nullptr);
    else smooth_with<float>(g, level, 1, smoother, omega, (float*)u, v.ua32, (const float*)f, nullptr, nullptr);
    CHECK_LAUNCH(g->ctx);
    CUDA_TRY(g->ctx, cudaStreamSynchronize(g->ctx->stream));
    return ELAS_OK;
}

int elas_op_restrict(elas_grid g, int level, int precision, const void* r, void* fc) {
    if (!g || !r || !fc) return ELAS_ERR_INVALID_ARG;
    int rc = check_level(g, level, precision);
    if (rc) return rc;
    if (level + 1 >= (int)g->lv.size()) return set_err(g->ctx, ELAS_ERR_INVALID_ARG, "no coarser level");
    Level& v = g->lv[level];
    Level& w = g->lv[level + 1];
    if (precision == 0)
        launch_restrict<double>(v.L64, w.L64, (const double*)r, (double*)fc, nullptr, nullptr, g->ctx->stream);
    else
        launch_restrict<float>(v.L32, w.L32, (const float*)r, (float*)fc, nullptr, nullptr, g->ctx->stream);
    CHECK_LAUNCH(g->ctx);
    CUDA_TRY(g->ctx, cudaStreamSynchronize(g->ctx->stream));
    return ELAS_OK;
}

int elas_op_prolong_add(elas_grid g, int level, int precision, const void* ec, void* u) {
    if (!g || !ec || !u) return ELAS_ERR_INVALID_ARG;
    int rc = check_level(g, level, precision);
    if (rc) return rc;
    if (level + 1 >= (int)g->lv.size()) return set_err(g->ctx, ELAS_ERR_INVALID_ARG, "no coarser level");
    Level& v = g->lv[level];
    Level& w = g->lv[level + 1];
    if (precision == 0) launch_prolong_add<double>(v.L64, w.L64, (const double*)ec, (double*)u, g->ctx->stream);
    else launch_prolong_add<float>(v.L32, w.L32, (const float*)ec, (float*)u, g->ctx->stream);
    CHECK_LAUNCH(g->ctx);
    CUDA_TRY(g->ctx, cudaStreamSynchronize(g->ctx->stream));
    return ELAS_OK;
}

int elas_op_rhs(elas_grid g, double* f_out) {
    if (!g || !f_out) return ELAS_ERR_INVALID_ARG;
    int rc = check_level(g, 0, 0);
    if (rc) return rc;
    CUDA_TRY(g->ctx, cudaMemcpyAsync(f_out, g->lv[0].f, sizeof(double) * 3 * (size_t)g->lv[0].N,
                                     cudaMemcpyDeviceToDevice, g->ctx->stream));
    CUDA_TRY(g->ctx, cudaStreamSynchronize(g->ctx->stream));
    return ELAS_OK;
}

int elas_op_bottom(elas_grid g, int precision, const void* f, void* u) {
    if (!g || !f || !u) return ELAS_ERR_INVALID_ARG;
    const int l = (int)g->lv.size() - 1;
    int rc = check_level(g, l, precision);
    if (rc) return rc;
    Level& v = g->lv[l];
    if (precision == 0)
        launch_bottom_solve<double>(v.L64, g->dofs, g->nfree, g->ntot, g->Ainv, (const double*)f, (double*)u, g->bwork,
                                    g->ctx->stream);
    else
        launch_bottom_solve<float>(v.L32, g->dofs, g->nfree, g->ntot, g->Ainv, (const float*)f, (float*)u, g->bwork,
                                   g->ctx->stream);
    CHECK_LAUNCH(g->ctx);
    CUDA_TRY(g->ctx, cudaStreamSynchronize(g->ctx->stream));
    return ELAS_OK;
}

int elas_measure_fma_peak(int device, int precision, double* tflops) {
    if (!tflops || (precision != 0 && precision != 1)) return ELAS_ERR_INVALID_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return ELAS_ERR_DEVICE;
    cudaStream_t s = nullptr;
    void* out = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return ELAS_ERR_DEVICE;
    if (cudaMalloc(&out, 256 * sizeof(double)) != cudaSuccess) {
        cudaStreamDestroy(s);
        return ELAS_ERR_DEVICE;
    }
    // size the launch to about 20 ms from a short probe, then keep the best of three
    float ms = 0.f;
    int iters = precision == 0 ? 256 : 4096;
    double flops = measure_fma_flops(precision, iters, &ms, out, s);
    if (ms > 0.f) {
        const double scale = 20.0 / ms;
        const double it = scale * iters;
        iters = it > 2e8 ? 200000000 : (it < 4 ? 4 : (int)it);
        iters -= iters % 4;
    }
    double best = 0.0;
    for (int r = 0; r < 4; ++r) {
        flops = measure_fma_flops(precision, iters, &ms, out, s);
        if (r > 0 && ms > 0.f) best = std::max(best, flops / (ms * 1e-3) / 1e12);
    }
    const cudaError_t e = cudaGetLastError();
    cudaFree(out);
    cudaStreamDestroy(s);
    if (e != cudaSuccess) return ELAS_ERR_DEVICE;
    *tflops = best;
    return ELAS_OK;
}

int elas_profile_enable(elas_ctx c, int enable) {
    if (!c) return ELAS_ERR_INVALID_ARG;
    cudaStreamSynchronize(c->stream);
    c->pending.clear();
    c->pool_used = 0;
    c->profile = enable != 0;
    for (int k = 0; k < ELAS_PROF_CLASSES; ++k) {
        c->prof_ms[k] = 0.0;
        c->prof_count[k] = 0;
    }
    return ELAS_OK;
}

int elas_profile_read(elas_ctx c, int cls, double* total_ms, long long* launches) {
    if (!c || cls < 0 || cls >= ELAS_PROF_CLASSES) return ELAS_ERR_INVALID_ARG;
    cudaStreamSynchronize(c->stream);
    prof_collect(c);
    if (total_ms) *total_ms = c->prof_ms[cls];
    if (launches) *launches = c->prof_count[cls];
    return ELAS_OK;
}

unsigned long long elas_launch_count(void) { return elas::launch_count(); }

int elas_autotune(elas_grid g, float* times_ms, int ntimes) {
    if (!g) return ELAS_ERR_INVALID_ARG;
    if (int rc = refuse_if_served(g)) return rc;
    int rc = setup(g);
    if (rc) return rc;
    elas_ctx c = g->ctx;
    for (size_t l = 0; l < g->lv.size(); ++l) {
        Level& v = g->lv[l];
        float ms[kNumSweepVariants];
        if (g->desc.mixed) {
            cudaMemsetAsync(v.u32, 0, sizeof(float) * 3 * (size_t)v.N, c->stream);
            cudaMemsetAsync(v.f32, 0, sizeof(float) * 3 * (size_t)v.N, c->stream);
            tune_sweep<float>(v.L32, v.u32, v.ua32, v.f32, c->stream, ms);
            if (l == 0 && times_ms)
                for (int k = 0; k < kNumSweepVariants && k < ntimes; ++k) times_ms[k] = ms[k];
        }
        tune_sweep<double>(v.L64, v.u, v.ua, v.f, c->stream, nullptr);
    }
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    CHECK_LAUNCH(c);
    return ELAS_OK;
}

int elas_autotune_dump(char* buf, int cap) { return tune_table_dump(buf, cap); }
int elas_autotune_load(const char* text) { return text ? tune_table_load(text) : 0; }

}  // extern "C"
namespace {
int batch_run(elas_grid* grids, int n, const elas_solve_opts* opts, elas_solve_info* info, void* mem,
              std::chrono::steady_clock::time_point t0);
}  // namespace
extern "C" {

int elas_batch_solve(elas_grid* grids, int n, const elas_solve_opts* opts, elas_solve_info* info) {
    if (!grids || n < 0 || !opts || !info) return ELAS_ERR_INVALID_ARG;
    if (n == 0) return ELAS_OK;
    for (int i = 0; i < n; ++i)
        if (!grids[i]) return ELAS_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i)
        if (int rc = refuse_if_served(grids[i])) return rc;
    elas_ctx c = grids[0]->ctx;
    {
        // members share nothing: a grid listed twice would have two solves in its buffers
        std::vector<elas_grid> sorted(grids, grids + n);
        std::sort(sorted.begin(), sorted.end());
        if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end())
            return set_err(c, ELAS_ERR_INVALID_ARG, "a grid appears twice in the batch");
    }
    bool batched = opts->precision == ELAS_PRECISION_MIXED && (n > 1 || opts->use_graph);
    for (int i = 0; i < n; ++i)
        if (grids[i]->ctx != c || !grids[i]->desc.mixed || grids[i]->desc.max_levels == 1) batched = false;
    if (!batched) {
        int worst = ELAS_OK;
        elas_solve_opts one = *opts;
        one.use_graph = 0;
        for (int i = 0; i < n; ++i) {
            const int rc = elas_solve(grids[i], &one, &info[i]);
            if (rc != ELAS_OK && worst == ELAS_OK) worst = rc;
        }
        return worst;
    }
    cudaSetDevice(c->device);
    const auto t0 = std::chrono::steady_clock::now();
    for (int i = 0; i < n; ++i) {
        std::memset(&info[i], 0, sizeof(info[i]));
        int rc = take_cycle_opts(grids[i], opts);
        if (!rc) rc = setup(grids[i]);
        if (!rc && outer_df(grids[i], opts)) rc = df_prepare(grids[i]);
        if (rc) return rc;
    }
    if (batch_engine_applies(grids, n, opts)) {
        const int rc = batch_engine(grids, n, opts, info, t0);
        for (int i = 0; i < n; ++i)
            for (auto& v : grids[i]->lv) {
                v.L64.active = nullptr;
                v.L32.active = nullptr;
            }
        return rc;
    }
    // per-member flags, counters and histories; every exit of the run clears the members'
    // flag pointers and frees them
    const size_t bytes = n * (2 * sizeof(int)) + 256 + n * (size_t)ELAS_HISTORY * sizeof(double);
    void* mem = ctx_alloc(c, bytes);
    if (!mem) return set_err(c, ELAS_ERR_ALLOC, "batch work arrays: allocation failed");
    const int rc = batch_run(grids, n, opts, info, mem, t0);
    for (int i = 0; i < n; ++i)
        for (auto& v : grids[i]->lv) {
            v.L64.active = nullptr;
            v.L32.active = nullptr;
        }
    cudaStreamSynchronize(c->stream);
    ctx_free(c, mem, bytes);
    return rc;
}

}  // extern "C"

// ---- batched engine: per-phase launches over a work list, one captured graph per plan ----
struct BatchPlan {
    std::vector<elas_grid> members;
    std::vector<unsigned long long> gen;
    std::vector<double> r0;
    int nu1 = 0, nu2 = 0, inner = 1, cycle = 0, max_cycles = 0, fixed = 0;
    bool df = false;   // double-float refinement residual
    double tol = 0.0;
    void* mem = nullptr;
    size_t bytes = 0;
    int* flags = nullptr;
    int* counts = nullptr;
    double* hist = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned long long per_replay = 0;
    int steps_per_replay = 2;
};

namespace {

bool plan_has_member(const BatchPlan* p, elas_grid g) {
    if (!p) return false;
    for (auto m : p->members)
        if (m == g) return true;
    return false;
}

void plan_free(elas_ctx c, BatchPlan* p) {
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->mem) ctx_free(c, p->mem, p->bytes);
    delete p;
}

// Task arrays of the plan: host bytes laid out as in the device arena.
struct Arena {
    std::vector<char> host;
    size_t push(const void* data, size_t bytes) {
        const size_t off = (host.size() + 255) & ~size_t(255);
        host.resize(off + bytes);
        std::memcpy(host.data() + off, data, bytes);
        return off;
    }
};
struct PhaseRef {   // a phase before upload: arena offsets of its tasks and block map
    BatchPhase ph;
    size_t tasks_off = 0, bmap_off = 0;
};

template <typename Task>
PhaseRef make_phase(Arena& ar, int kind, const std::vector<Task>& tasks, int K, int ml, int colour = 0) {
    PhaseRef r;
    r.ph.kind = kind;
    r.ph.n = (int)tasks.size();
    r.ph.K = K;
    r.ph.ml = ml;
    r.ph.colour = colour;
    if (tasks.empty()) return r;
    std::vector<int2> bmap;
    for (size_t i = 0; i < tasks.size(); ++i) {
        const int nb = batch_task_blocks(kind, &tasks[i]);
        for (int b = 0; b < nb; ++b) bmap.push_back(make_int2((int)i, b));
    }
    r.ph.blocks = (int)bmap.size();
    r.tasks_off = ar.push(tasks.data(), sizeof(Task) * tasks.size());
    r.bmap_off = ar.push(bmap.data(), sizeof(int2) * bmap.size());
    return r;
}

// Whether the grids can share the per-phase kernels: mixed, one moduli kind and one FP32
// moduli layout on every level, the red-black smoother.
bool batch_engine_applies(elas_grid* grids, int n, const elas_solve_opts* o) {
    if (o->smoother != ELAS_SMOOTH_RB) return false;
    const int K = grids[0]->K;
    const int ml = grids[0]->lv[0].L32.mlay;
    for (int i = 0; i < n; ++i) {
        elas_grid g = grids[i];
        if (g->K != K || g->desc.half_moduli || !g->desc.mixed) return false;
        for (auto& v : g->lv)
            if (v.L32.mlay != ml) return false;
    }
    return ml == kModBlocked || ml == kModSplit;
}

bool plan_matches(const BatchPlan* p, elas_grid* grids, int n, const elas_solve_opts* o) {
    if (!p || (int)p->members.size() != n) return false;
    if (p->nu1 != o->nu1 || p->nu2 != o->nu2 || p->inner != (o->inner_cycles > 1 ? o->inner_cycles : 1) ||
        p->cycle != o->cycle || p->tol != o->rel_tol ||
        p->max_cycles != (o->fixed_cycles > 0 ? o->fixed_cycles : o->max_cycles) || p->fixed != o->fixed_cycles ||
        p->df != batch_df(grids, n, o))
        return false;
    for (int i = 0; i < n; ++i)
        if (p->members[i] != grids[i] || p->gen[i] != grids[i]->gen || p->r0[i] != grids[i]->r0) return false;
    return true;
}

// Build the task arrays of one refinement step of every member (FP64 or double-float residual, the
// load update and convergence test, `inner` FP32 V-cycles level by level, the FP64
// correction), upload them, and capture two steps as a graph.
int plan_build(elas_grid* grids, int n, const elas_solve_opts* o, BatchPlan** out) {
    elas_ctx c = grids[0]->ctx;
    BatchPlan* p = new BatchPlan();
    p->nu1 = o->nu1;
    p->nu2 = o->nu2;
    p->inner = o->inner_cycles > 1 ? o->inner_cycles : 1;
    p->cycle = o->cycle;
    p->tol = o->rel_tol;
    p->fixed = o->fixed_cycles;
    p->max_cycles = o->fixed_cycles > 0 ? o->fixed_cycles : o->max_cycles;
    p->df = batch_df(grids, n, o);
    const int H = ELAS_HISTORY;
    const size_t flag_bytes = ((size_t)2 * n * sizeof(int) + 255) & ~size_t(255);
    const size_t hist_bytes = ((size_t)n * H * sizeof(double) + 255) & ~size_t(255);
    const int K = grids[0]->K;
    const int ml = grids[0]->lv[0].L32.mlay == kModSplit ? kMlSplit : kMlDefault;
    int depth = 0;
    for (int i = 0; i < n; ++i) depth = std::max(depth, (int)grids[i]->lv.size());
    // flags live at the start of the arena; the tasks point at them through each level's
    // active pointer, so the arena's device address is needed first: allocate for the
    // task bytes measured on a dry build, then build for real
    Arena ar;
    std::vector<PhaseRef> phases;
    auto build = [&](char* dev_base) {
        ar.host.assign(flag_bytes + hist_bytes, 0);
        phases.clear();
        int* flags = (int*)dev_base;
        int* counts = flags + n;
        double* hist = (double*)(dev_base + flag_bytes);
        for (int i = 0; i < n; ++i)
            for (auto& v : grids[i]->lv) v.L64.active = v.L32.active = flags + i;
        NullInfo none{};
        // FP64 or double-float residual (written as FP32 into the level-0 right-hand side)
        // and finalize
        std::vector<ResidTask<double, float>> r64;
        std::vector<ResidTask<dfloat, float>> rdf;
        std::vector<FinalizeTask> fin;
        std::vector<CorrTask> corr;
        for (int i = 0; i < n; ++i) {
            elas_grid g = grids[i];
            Level& L0 = g->lv[0];
            const bool rm = L0.nf.m > 0;
            FinalizeTask ft{};
            if (p->df) {
                ResidTask<dfloat, float> t{df_view(L0), L0.u2, L0.f2, rm ? L0.nf : none, rm ? g->alam : nullptr,
                                           L0.f32, g->partials};
                rdf.push_back(t);
                ft.nblocks = batch_task_blocks(kPhaseResidDf, &t);
            } else {
                ResidTask<double, float> t{L0.L64, L0.u, L0.f, rm ? L0.nf : none, rm ? g->alam : nullptr, L0.f32,
                                           g->partials};
                r64.push_back(t);
                ft.nblocks = batch_task_blocks(kPhaseResid64, &t);
            }
            ft.partials = g->partials;
            ft.nf = L0.nf;
            ft.Ginv = g->Ginv;
            ft.G = g->G;
            ft.lam = g->lam;
            ft.dlam = g->dlam;
            ft.alam = g->alam;
            ft.adlam = g->adlam;
            ft.out = g->status;
            ft.bf = BatchFlags{flags + i, counts + i, hist + (size_t)i * H, H, g->r0, o->rel_tol, p->max_cycles};
            fin.push_back(ft);
            corr.push_back(CorrTask{L0.L64, L0.u, L0.u32, p->df ? L0.u2 : nullptr});
        }
        const PhaseRef ph_r64 = p->df ? make_phase(ar, kPhaseResidDf, rdf, K, ml) : make_phase(ar, kPhaseResid64, r64, K, ml);
        PhaseRef ph_fin;
        ph_fin.ph.kind = kPhaseFinalize;
        ph_fin.ph.n = n;
        ph_fin.ph.blocks = n;
        ph_fin.tasks_off = ar.push(fin.data(), sizeof(FinalizeTask) * fin.size());
        const PhaseRef ph_corr = make_phase(ar, kPhaseCorr, corr, K, ml);
        // per-depth task arrays of the FP32 V-cycle
        struct Depth {
            PhaseRef zero, red, black, res, restr, prol, bzero, gather, matvec;
        };
        std::vector<Depth> D(depth);
        for (int d = 0; d < depth; ++d) {
            std::vector<ZeroTask<float>> zv, zb;
            std::vector<SweepTask<float>> sr, sb;
            std::vector<ResidTask<float, float>> rs;
            std::vector<RestrictTask<float>> re;
            std::vector<ProlongTask<float>> pr;
            std::vector<BottomTask<float>> bt;
            for (int i = 0; i < n; ++i) {
                elas_grid g = grids[i];
                const int nl = (int)g->lv.size();
                if (d >= nl) continue;
                Level& v = g->lv[d];
                const size_t n3 = (size_t)3 * v.N;
                const bool rm = d == 0 && g->lv[0].nf.m > 0;
                const NullInfo& nf = rm ? g->lv[0].nf : none;
                const double* lam = rm ? g->adlam : nullptr;
                if (d == nl - 1) {
                    zb.push_back(ZeroTask<float>{v.u32, n3, flags + i});
                    bt.push_back(BottomTask<float>{v.L32, g->dofs, g->nfree, g->ntot, g->Ainv, v.f32, v.u32, g->bwork});
                    continue;
                }
                Level& w = g->lv[d + 1];
                zv.push_back(ZeroTask<float>{v.u32, n3, flags + i});
                sr.push_back(SweepTask<float>{v.L32, v.u32, v.ua32, v.f32, nf, lam});
                sb.push_back(SweepTask<float>{v.L32, v.ua32, v.u32, v.f32, nf, lam});
                rs.push_back(ResidTask<float, float>{v.L32, v.u32, v.f32, nf, lam, v.r32, nullptr});
                re.push_back(RestrictTask<float>{v.L32, w.L32, v.r32, w.f32, none, nullptr});
                pr.push_back(ProlongTask<float>{v.L32, w.L32, w.u32, v.u32});
            }
            D[d].zero = make_phase(ar, kPhaseZero, zv, K, ml);
            D[d].red = make_phase(ar, kPhaseSweep, sr, K, ml, 0);
            D[d].black = make_phase(ar, kPhaseSweep, sb, K, ml, 1);
            D[d].res = make_phase(ar, kPhaseResid32, rs, K, ml);
            D[d].restr = make_phase(ar, kPhaseRestrict, re, K, ml);
            D[d].prol = make_phase(ar, kPhaseProlong, pr, K, ml);
            D[d].bzero = make_phase(ar, kPhaseZero, zb, K, ml);
            D[d].gather = make_phase(ar, kPhaseGather, bt, K, ml);
            D[d].matvec = make_phase(ar, kPhaseMatvec, bt, K, ml);
        }
        // one refinement step as a sequence of phases
        auto smooth = [&](int d, int sweeps) {
            for (int k = 0; k < sweeps; ++k) {
                phases.push_back(D[d].red);
                phases.push_back(D[d].black);
            }
        };
        // the FP32 cycle of depth d (V, or F: the next depth's correction F then V)
        std::function<void(int, bool, int)> cyc = [&](int d, bool zero, int kind) {
            if (d >= depth) return;
            phases.push_back(D[d].bzero);
            phases.push_back(D[d].gather);
            phases.push_back(D[d].matvec);
            if (zero) phases.push_back(D[d].zero);
            smooth(d, o->nu1);
            phases.push_back(D[d].res);
            phases.push_back(D[d].restr);
            if (kind == ELAS_CYCLE_F) {
                cyc(d + 1, true, ELAS_CYCLE_F);
                cyc(d + 1, false, ELAS_CYCLE_V);
            } else {
                cyc(d + 1, true, ELAS_CYCLE_V);
            }
            phases.push_back(D[d].prol);
            smooth(d, o->nu2);
        };
        phases.push_back(ph_r64);
        phases.push_back(ph_fin);
        for (int k = 0; k < p->inner; ++k) cyc(0, k == 0, o->cycle);
        phases.push_back(ph_corr);
    };
    build(nullptr);
    p->bytes = ar.host.size();
    p->mem = ctx_alloc(c, p->bytes);
    if (!p->mem) {
        delete p;
        return set_err(c, ELAS_ERR_ALLOC, "batch plan: allocation failed");
    }
    build((char*)p->mem);
    p->flags = (int*)p->mem;
    p->counts = p->flags + n;
    p->hist = (double*)((char*)p->mem + flag_bytes);
    for (int i = 0; i < n; ++i) {
        p->members.push_back(grids[i]);
        p->gen.push_back(grids[i]->gen);
        p->r0.push_back(grids[i]->r0);
    }
    cudaStream_t main = c->stream;
    cudaError_t ce = cudaMemcpyAsync(p->mem, ar.host.data(), p->bytes, cudaMemcpyHostToDevice, main);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(main);
    // capture two refinement steps
    const unsigned long long l0 = launch_count();
    if (ce == cudaSuccess) ce = cudaStreamBeginCapture(main, cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess) {
        for (int rep = 0; rep < p->steps_per_replay; ++rep)
            for (auto& r : phases) {
                BatchPhase ph = r.ph;
                ph.tasks = (const char*)p->mem + r.tasks_off;
                ph.bmap = (const int2*)((const char*)p->mem + r.bmap_off);
                batch_phase_launch(ph, main);
            }
        ce = cudaStreamEndCapture(main, &p->graph);
    }
    p->per_replay = launch_count() - l0;
    count_launch(-(int)p->per_replay);
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&p->exec, p->graph, 0);
    if (ce != cudaSuccess) {
        plan_free(c, p);
        return set_err(c, ELAS_ERR_DEVICE, std::string("batch plan graph: ") + cudaGetErrorString(ce));
    }
    *out = p;
    return ELAS_OK;
}

// Run a batch through the engine: per-call initial state, graph replays until every
// member stops, results.
int batch_engine(elas_grid* grids, int n, const elas_solve_opts* o, elas_solve_info* info,
                 std::chrono::steady_clock::time_point t0) {
    elas_ctx c = grids[0]->ctx;
    cudaStream_t main = c->stream;
    const bool prof = c->profile;
    c->profile = false;
    if (!plan_matches(c->plan, grids, n, o)) {
        plan_free(c, c->plan);
        c->plan = nullptr;
        int rc = plan_build(grids, n, o, &c->plan);
        if (rc) {
            c->profile = prof;
            return rc;
        }
    }
    BatchPlan* p = c->plan;
    for (int i = 0; i < n; ++i)
        for (auto& v : grids[i]->lv) v.L64.active = v.L32.active = p->flags + i;
    std::vector<int> h_flags(n, 1), h_counts(n, 0);
    CUDA_TRY(c, cudaMemcpyAsync(p->flags, h_flags.data(), sizeof(int) * n, cudaMemcpyHostToDevice, main));
    CUDA_TRY(c, cudaMemcpyAsync(p->counts, h_counts.data(), sizeof(int) * n, cudaMemcpyHostToDevice, main));
    for (int i = 0; i < n; ++i) {
        elas_grid g = grids[i];
        Level& L0 = g->lv[0];
        launch_dirichlet(L0.L64, boundary_data(g), L0.u, o->warm_start ? 1 : 0, main);
        outer_begin(g, p->df, main);
        cudaMemsetAsync(g->lam, 0, sizeof(double) * 8, main);
        cudaMemsetAsync(g->alam, 0, sizeof(double) * kLoadDoubles, main);
        cudaMemsetAsync(g->adlam, 0, sizeof(double) * kLoadDoubles, main);
    }
    CHECK_LAUNCH(c);
    const int max_replays = p->max_cycles / p->steps_per_replay + 2;
    cudaError_t ce = cudaSuccess;
    for (int r = 0; r < max_replays; ++r) {
        ce = cudaGraphLaunch(p->exec, main);
        if (ce != cudaSuccess) break;
        count_launch((int)p->per_replay);
        cudaMemcpyAsync(h_flags.data(), p->flags, sizeof(int) * n, cudaMemcpyDeviceToHost, main);
        ce = cudaStreamSynchronize(main);
        if (ce != cudaSuccess) break;
        bool any = false;
        for (int i = 0; i < n; ++i) any |= h_flags[i] != 0;
        if (!any) break;
    }
    c->profile = prof;
    if (ce != cudaSuccess) return set_err(c, ELAS_ERR_DEVICE, std::string("batch replay: ") + cudaGetErrorString(ce));
    const int H = ELAS_HISTORY;
    std::vector<double> h_hist((size_t)n * H);
    CUDA_TRY(c, cudaMemcpyAsync(h_counts.data(), p->counts, sizeof(int) * n, cudaMemcpyDeviceToHost, main));
    CUDA_TRY(c, cudaMemcpyAsync(h_hist.data(), p->hist, sizeof(double) * n * H, cudaMemcpyDeviceToHost, main));
    std::vector<double> h_inf(n);
    for (int i = 0; i < n; ++i)
        CUDA_TRY(c, cudaMemcpyAsync(&h_inf[i], grids[i]->status + 1, sizeof(double), cudaMemcpyDeviceToHost, main));
    for (int i = 0; i < n; ++i) {
        const int rr = remove_rigid(grids[i]);
        if (rr) return rr;
    }
    CUDA_TRY(c, cudaStreamSynchronize(main));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    int worst = ELAS_OK;
    for (int i = 0; i < n; ++i) {
        const int cnt = h_counts[i] < H ? h_counts[i] : H;
        for (int k = 0; k < cnt; ++k) info[i].rel_history[k] = h_hist[(size_t)i * H + k];
        info[i].cycles = h_counts[i] > 0 ? h_counts[i] - 1 : 0;
        info[i].rel_residual = cnt > 0 ? h_hist[(size_t)i * H + cnt - 1] : 0.0;
        info[i].residual_inf = h_inf[i];
        info[i].rel_residual_inf = grids[i]->r0inf > 0 ? h_inf[i] / grids[i]->r0inf : 0.0;
        info[i].r0 = grids[i]->r0;
        info[i].nlam = grids[i]->lv[0].nf.m;
        info[i].seconds = secs;
        const bool ok = o->fixed_cycles > 0 ? true : info[i].rel_residual <= o->rel_tol;
        info[i].status = ok ? ELAS_OK : ELAS_ERR_NOT_CONVERGED;
        if (!ok && worst == ELAS_OK) worst = ELAS_ERR_NOT_CONVERGED;
    }
    if (worst) set_err(c, worst, "a batch member did not reach the tolerance");
    return worst;
}

}  // namespace

namespace {
int batch_run(elas_grid* grids, int n, const elas_solve_opts* opts, elas_solve_info* info, void* mem,
              std::chrono::steady_clock::time_point t0) {
    elas_ctx c = grids[0]->ctx;
    cudaStream_t main = c->stream;
    const size_t hist_len = ELAS_HISTORY;
    int* flags = (int*)mem;
    int* counts = flags + n;
    double* hist = (double*)((char*)mem + (((size_t)2 * n * sizeof(int) + 255) & ~size_t(255)));
    std::vector<int> h_flags(n, 1), h_counts(n, 0);
    CUDA_TRY(c, cudaMemcpyAsync(flags, h_flags.data(), sizeof(int) * n, cudaMemcpyHostToDevice, main));
    CUDA_TRY(c, cudaMemcpyAsync(counts, h_counts.data(), sizeof(int) * n, cudaMemcpyHostToDevice, main));
    const bool dfb = batch_df(grids, n, opts);
    for (int i = 0; i < n; ++i) {
        elas_grid g = grids[i];
        Level& L0 = g->lv[0];
        launch_dirichlet(L0.L64, boundary_data(g), L0.u, opts->warm_start ? 1 : 0, main);
        outer_begin(g, dfb, main);
        cudaMemsetAsync(g->lam, 0, sizeof(double) * 8, main);
        cudaMemsetAsync(g->alam, 0, sizeof(double) * kLoadDoubles, main);
        cudaMemsetAsync(g->adlam, 0, sizeof(double) * kLoadDoubles, main);
        for (auto& v : g->lv) {
            v.L64.active = flags + i;
            v.L32.active = flags + i;
        }
    }
    CHECK_LAUNCH(c);
    CUDA_TRY(c, cudaStreamSynchronize(main));
    // branches of the graph
    const int S = n < 32 ? n : 32;
    while ((int)c->branch.size() < S) {
        cudaStream_t st;
        cudaEvent_t ev;
        CUDA_TRY(c, cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        CUDA_TRY(c, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        c->branch.push_back(st);
        c->branch_ev.push_back(ev);
    }
    cudaEvent_t fork;
    CUDA_TRY(c, cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    const bool prof = c->profile;
    c->profile = false;
    const int nu1 = opts->nu1 < 0 ? 0 : opts->nu1, nu2 = opts->nu2 < 0 ? 0 : opts->nu2;
    const int K = 2;   // refinement steps per graph replay
    const unsigned long long launches0 = launch_count();
    cudaGraph_t graph = nullptr;
    CUDA_TRY(c, cudaStreamBeginCapture(main, cudaStreamCaptureModeThreadLocal));
    cudaEventRecord(fork, main);
    for (int b = 0; b < S; ++b) cudaStreamWaitEvent(c->branch[b], fork, 0);
    for (int it = 0; it < K; ++it) {
        for (int i = 0; i < n; ++i) {
            elas_grid g = grids[i];
            Level& L0 = g->lv[0];
            c->stream = c->branch[i % S];
            const NullInfo* nf0 = L0.nf.m > 0 ? &L0.nf : nullptr;
            int nb = 0;
            outer_residual(g, dfb, nf0, nf0 ? g->alam : nullptr, &nb, c->stream);
            BatchFlags bfl{flags + i, counts + i, hist + (size_t)i * hist_len, (int)hist_len, g->r0, opts->rel_tol,
                           opts->fixed_cycles > 0 ? opts->fixed_cycles : opts->max_cycles};
            launch_finalize(g->partials, nb, L0.nf, g->Ginv, g->G, g->lam, g->dlam, g->alam, g->adlam, g->status, 1,
                            c->stream, bfl);
            for (int k = 0; k < (opts->inner_cycles > 1 ? opts->inner_cycles : 1); ++k)
                vcycle<float>(g, 0, nu1, nu2, nf0, nf0 ? g->adlam : nullptr, k == 0, opts->cycle);
            outer_correct(g, dfb, c->stream);
        }
    }
    for (int b = 0; b < S; ++b) {
        cudaEventRecord(c->branch_ev[b], c->branch[b]);
        cudaStreamWaitEvent(main, c->branch_ev[b], 0);
    }
    c->stream = main;
    cudaError_t ce = cudaStreamEndCapture(main, &graph);
    c->profile = prof;
    const unsigned long long per_replay = launch_count() - launches0;
    count_launch(-(int)per_replay);   // captured, not launched: counted per replay below
    cudaGraphExec_t exec = nullptr;
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&exec, graph, 0);
    int rc = ELAS_OK;
    if (ce != cudaSuccess) {
        rc = set_err(c, ELAS_ERR_DEVICE, std::string("batched graph: ") + cudaGetErrorString(ce));
    } else {
        const int max_replays = (opts->fixed_cycles > 0 ? opts->fixed_cycles : opts->max_cycles) / K + 2;
        for (int r = 0; r < max_replays; ++r) {
            ce = cudaGraphLaunch(exec, main);
            if (ce != cudaSuccess) break;
            count_launch((int)per_replay);
            cudaMemcpyAsync(h_flags.data(), flags, sizeof(int) * n, cudaMemcpyDeviceToHost, main);
            ce = cudaStreamSynchronize(main);
            if (ce != cudaSuccess) break;
            bool any = false;
            for (int i = 0; i < n; ++i) any |= h_flags[i] != 0;
            if (!any) break;
        }
        if (ce != cudaSuccess) rc = set_err(c, ELAS_ERR_DEVICE, std::string("batched replay: ") + cudaGetErrorString(ce));
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaEventDestroy(fork);
    if (rc) return rc;
    std::vector<double> h_hist((size_t)n * hist_len);
    CUDA_TRY(c, cudaMemcpyAsync(h_counts.data(), counts, sizeof(int) * n, cudaMemcpyDeviceToHost, main));
    CUDA_TRY(c, cudaMemcpyAsync(h_hist.data(), hist, sizeof(double) * n * hist_len, cudaMemcpyDeviceToHost, main));
    std::vector<double> h_inf(n);
    for (int i = 0; i < n; ++i)
        CUDA_TRY(c, cudaMemcpyAsync(&h_inf[i], grids[i]->status + 1, sizeof(double), cudaMemcpyDeviceToHost, main));
    int worst = ELAS_OK;
    for (int i = 0; i < n; ++i) {
        const int rr = remove_rigid(grids[i]);
        if (rr) return rr;
    }
    CUDA_TRY(c, cudaStreamSynchronize(main));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (int i = 0; i < n; ++i) {
        const int cnt = h_counts[i] < (int)hist_len ? h_counts[i] : (int)hist_len;
        for (int k = 0; k < cnt; ++k) info[i].rel_history[k] = h_hist[(size_t)i * hist_len + k];
        info[i].cycles = h_counts[i] > 0 ? h_counts[i] - 1 : 0;
        info[i].rel_residual = cnt > 0 ? h_hist[(size_t)i * hist_len + cnt - 1] : 0.0;
        info[i].residual_inf = h_inf[i];
        info[i].rel_residual_inf = grids[i]->r0inf > 0 ? h_inf[i] / grids[i]->r0inf : 0.0;
        info[i].r0 = grids[i]->r0;
        info[i].nlam = grids[i]->lv[0].nf.m;
        info[i].seconds = secs;
        const bool ok = opts->fixed_cycles > 0 ? true : info[i].rel_residual <= opts->rel_tol;
        info[i].status = ok ? ELAS_OK : ELAS_ERR_NOT_CONVERGED;
        if (!ok && worst == ELAS_OK) worst = ELAS_ERR_NOT_CONVERGED;
    }
    if (worst) set_err(c, worst, "a batch member did not reach the tolerance");
    return worst;
}
}  // namespace

// ======================================================================================
// block-structured AMR: composite reflux-free cycle
// ======================================================================================
struct elas_amr_s {
    std::vector<elas_grid> g;
    std::vector<AmrBox> box;    // valid boxes
    std::vector<AmrBox> rbox;   // relaxed boxes: the valid box (R1), grown by the inner ghost layer (R2)
    int reading = ELAS_AMR_R1;
    std::vector<double*> res, rpass, cor, cora, tmp;
    std::vector<float*> res32, rpass32, cor32, cora32, tmp32;   // mixed solves (allocated on first use)
    std::vector<std::pair<void*, size_t>> allocs;
    double* partials = nullptr;
    size_t npart = 0;
    bool holds_refs = false;   // counted in its grids' amr_refs (from a successful create)
};

namespace {

struct LevelSwap {
    Level& v;
    double *u, *ua, *f, *r;
    LevelSwap(Level& lv, double* nu, double* nua, double* nf, double* nr) : v(lv), u(lv.u), ua(lv.ua), f(lv.f), r(lv.r) {
        v.u = nu;
        v.ua = nua;
        v.f = nf;
        v.r = nr;
    }
    ~LevelSwap() {
        v.u = u;
        v.ua = ua;
        v.f = f;
        v.r = r;
    }
};

int amr_composite_residual(elas_amr a) {
    const int nl = (int)a->g.size();
    elas_ctx c = a->g[0]->ctx;
    cudaStream_t s = c->stream;
    for (int l = nl - 1; l >= 1; --l)
        launch_amr_interp(a->g[l]->lv[0].L64, a->box[l], a->g[l - 1]->lv[0].L64, a->box[l - 1], a->g[l - 1]->lv[0].u,
                          a->g[l]->lv[0].u, 0, s);
    for (int l = 0; l < nl; ++l) {
        Level& v = a->g[l]->lv[0];
        launch_residual<double, double>(v.L64, v.u, v.f, nullptr, nullptr, a->res[l], nullptr, nullptr, s);
    }
    for (int l = nl - 1; l >= 1; --l)
        launch_amr_restrict(a->g[l]->lv[0].L64, a->rbox[l], a->g[l - 1]->lv[0].L64, a->box[l - 1], a->res[l],
                            a->res[l - 1], 3, 1, s);
    CHECK_LAUNCH(c);
    return ELAS_OK;
}

// Covered coarse nodes from the fine solution: injection (R1), or the full-weighting
// restriction over the relaxed fine nodes, Dirichlet rows kept (R2).
void amr_sync(elas_amr a, int l, const double* ffield, double* cfield) {
    cudaStream_t s = a->g[0]->ctx->stream;
    const Lv<double>& Lf = a->g[l]->lv[0].L64;
    const Lv<double>& Lc = a->g[l - 1]->lv[0].L64;
    if (a->reading == ELAS_AMR_R2) launch_amr_restrict(Lf, a->rbox[l], Lc, a->box[l - 1], ffield, cfield, 3, 2, s);
    else launch_amr_inject(Lf, a->box[l], Lc, a->box[l - 1], ffield, cfield, s);
}

// Sum of the squared composite residual into g[0]->status[0] (enqueued only).
int amr_norm_enqueue(elas_amr a) {
    const int nl = (int)a->g.size();
    elas_ctx c = a->g[0]->ctx;
    cudaStream_t s = c->stream;
    int off = 0;
    for (int l = 0; l < nl; ++l)
        off += launch_amr_norm(a->g[l]->lv[0].L64, a->box[l], l + 1 < nl ? &a->box[l + 1] : nullptr, a->res[l],
                               a->partials + (size_t)off * kPartialStride, s);
    launch_sum_partials(a->partials, off, 1, a->g[0]->status, s);
    CHECK_LAUNCH(c);
    return ELAS_OK;
}

int amr_norm(elas_amr a, double* out) {
    int rc = amr_norm_enqueue(a);
    if (rc) return rc;
    double st[1];
    rc = read_status(a->g[0], st, 1);
    if (rc) return rc;
    *out = std::sqrt(st[0]);
    return ELAS_OK;
}

struct LevelSwap32 {
    Level& v;
    float *u, *ua, *f, *r;
    LevelSwap32(Level& lv, float* nu, float* nua, float* nf, float* nr)
        : v(lv), u(lv.u32), ua(lv.ua32), f(lv.f32), r(lv.r32) {
        v.u32 = nu;
        v.ua32 = nua;
        v.f32 = nf;
        v.r32 = nr;
    }
    ~LevelSwap32() {
        v.u32 = u;
        v.ua32 = ua;
        v.f32 = f;
        v.r32 = r;
    }
};

// The composite correction cycle of a mixed solve in FP32 (the same steps as amr_cycle,
// on FP32 copies of the residuals, corrections and moduli); the corrections are left in
// cor32 for the FP64 update.
void amr_cycle32(elas_amr a, int nu1, int nu2) {
    const int nl = (int)a->g.size();
    cudaStream_t s = a->g[0]->ctx->stream;
    for (int l = 0; l < nl; ++l) {
        const size_t bytes = sizeof(float) * 3 * (size_t)a->g[l]->lv[0].N;
        cudaMemcpyAsync(a->rpass32[l], a->res32[l], bytes, cudaMemcpyDeviceToDevice, s);
    }
    for (int l = nl - 1; l >= 1; --l) {
        elas_grid gl = a->g[l];
        Level& v = gl->lv[0];
        cudaMemsetAsync(a->cor32[l], 0, sizeof(float) * 3 * (size_t)v.N, s);
        {
            LevelSwap32 sw(v, a->cor32[l], a->cora32[l], a->res32[l], a->tmp32[l]);
            smooth<float>(gl, 0, nu1, nullptr, nullptr);
            launch_residual<float, float>(v.L32, v.u32, v.f32, nullptr, nullptr, a->rpass32[l], nullptr, nullptr, s);
        }
        launch_amr_restrict<float>(v.L32, a->rbox[l], a->g[l - 1]->lv[0].L32, a->box[l - 1], a->rpass32[l],
                                   a->rpass32[l - 1], 3, 1, s);
        if (l - 1 >= 1)
            cudaMemcpyAsync(a->res32[l - 1], a->rpass32[l - 1], sizeof(float) * 3 * (size_t)a->g[l - 1]->lv[0].N,
                            cudaMemcpyDeviceToDevice, s);
    }
    {
        Level& v0 = a->g[0]->lv[0];
        LevelSwap32 sw(v0, a->cor32[0], a->cora32[0], nl > 1 ? a->rpass32[0] : a->res32[0], a->tmp32[0]);
        vcycle<float>(a->g[0], 0, nu1, nu2, nullptr, nullptr);
    }
    for (int l = 1; l < nl; ++l) {
        elas_grid gl = a->g[l];
        Level& v = gl->lv[0];
        const Lv<float>& Lc = a->g[l - 1]->lv[0].L32;
        launch_amr_interp<float>(v.L32, a->box[l], Lc, a->box[l - 1], a->cor32[l - 1], a->cor32[l], 1, s);
        launch_amr_interp<float>(v.L32, a->box[l], Lc, a->box[l - 1], a->cor32[l - 1], a->cor32[l], 0, s);
        LevelSwap32 sw(v, a->cor32[l], a->cora32[l], a->res32[l], a->tmp32[l]);
        smooth<float>(gl, 0, nu2, nullptr, nullptr);
    }
}

// FP32 work arrays of the mixed composite solve (once).
int amr_alloc32(elas_amr a) {
    if (!a->res32.empty()) return ELAS_OK;
    elas_ctx c = a->g[0]->ctx;
    for (auto g : a->g)
        if (!g->desc.mixed) return set_err(c, ELAS_ERR_STATE, "mixed AMR solve needs every level created with mixed = 1");
    for (auto g : a->g) {
        const size_t bytes = sizeof(float) * 3 * (size_t)g->lv[0].N;
        float* p[5];
        for (int k = 0; k < 5; ++k) {
            p[k] = (float*)ctx_alloc(c, bytes);
            if (!p[k]) return set_err(c, ELAS_ERR_ALLOC, "AMR FP32 work arrays: allocation failed");
            a->allocs.push_back({p[k], bytes});
        }
        a->res32.push_back(p[0]);
        a->rpass32.push_back(p[1]);
        a->cor32.push_back(p[2]);
        a->cora32.push_back(p[3]);
        a->tmp32.push_back(p[4]);
    }
    return ELAS_OK;
}

void amr_cycle(elas_amr a, int nu1, int nu2) {
    const int nl = (int)a->g.size();
    cudaStream_t s = a->g[0]->ctx->stream;
    for (int l = 0; l < nl; ++l) {
        const size_t bytes = sizeof(double) * 3 * (size_t)a->g[l]->lv[0].N;
        cudaMemcpyAsync(a->rpass[l], a->res[l], bytes, cudaMemcpyDeviceToDevice, s);
    }
    for (int l = nl - 1; l >= 1; --l) {
        elas_grid gl = a->g[l];
        Level& v = gl->lv[0];
        cudaMemsetAsync(a->cor[l], 0, sizeof(double) * 3 * (size_t)v.N, s);
        {
            LevelSwap sw(v, a->cor[l], a->cora[l], a->res[l], a->tmp[l]);
            smooth<double>(gl, 0, nu1, nullptr, nullptr);
            launch_residual<double, double>(v.L64, v.u, v.f, nullptr, nullptr, a->rpass[l], nullptr, nullptr, s);
        }
        launch_amr_restrict(v.L64, a->rbox[l], a->g[l - 1]->lv[0].L64, a->box[l - 1], a->rpass[l], a->rpass[l - 1], 3,
                            1, s);
        if (l - 1 >= 1)
            cudaMemcpyAsync(a->res[l - 1], a->rpass[l - 1], sizeof(double) * 3 * (size_t)a->g[l - 1]->lv[0].N,
                            cudaMemcpyDeviceToDevice, s);
    }
    {
        Level& v0 = a->g[0]->lv[0];
        LevelSwap sw(v0, a->cor[0], a->cora[0], nl > 1 ? a->rpass[0] : a->res[0], a->tmp[0]);
        vcycle<double>(a->g[0], 0, nu1, nu2, nullptr, nullptr);
    }
    for (int l = 1; l < nl; ++l) {
        elas_grid gl = a->g[l];
        Level& v = gl->lv[0];
        const Lv<double>& Lc = a->g[l - 1]->lv[0].L64;
        launch_amr_interp(v.L64, a->box[l], Lc, a->box[l - 1], a->cor[l - 1], a->cor[l], 1, s);
        launch_amr_interp(v.L64, a->box[l], Lc, a->box[l - 1], a->cor[l - 1], a->cor[l], 0, s);
        LevelSwap sw(v, a->cor[l], a->cora[l], a->res[l], a->tmp[l]);
        smooth<double>(gl, 0, nu2, nullptr, nullptr);
    }
    for (int l = 0; l < nl; ++l) launch_amr_add(a->g[l]->lv[0].L64, a->box[l], a->g[l]->lv[0].u, a->cor[l], s);
    for (int l = nl - 1; l >= 1; --l) amr_sync(a, l, a->g[l]->lv[0].u, a->g[l - 1]->lv[0].u);
}

}  // namespace

extern "C" {

int elas_amr_create(elas_grid* grids, const elas_amr_level* levels, int nlevels, elas_amr* out) {
    if (!grids || !levels || nlevels < 1 || !out) return ELAS_ERR_INVALID_ARG;
    for (int l = 0; l < nlevels; ++l)
        if (!grids[l]) return ELAS_ERR_INVALID_ARG;
    elas_ctx c = grids[0]->ctx;
    for (int l = 0; l < nlevels; ++l)
        for (int k = 0; k < l; ++k)
            if (grids[k] == grids[l]) return set_err(c, ELAS_ERR_INVALID_ARG, "one grid given for two AMR levels");
    for (int l = 0; l < nlevels; ++l) {
        if (grids[l]->ctx != c) return set_err(c, ELAS_ERR_INVALID_ARG, "AMR grids must share a context");
        if (grids[l]->K != grids[0]->K) return set_err(c, ELAS_ERR_INVALID_ARG, "AMR levels need one moduli kind");
        if (l > 0 && grids[l]->desc.max_levels != 1)
            return set_err(c, ELAS_ERR_INVALID_ARG, "AMR levels above 0 must be created with max_levels = 1");
    }
    elas_amr a = new elas_amr_s();
    size_t parts = 64;
    for (int l = 0; l < nlevels; ++l) {
        elas_grid g = grids[l];
        AmrBox b{};
        for (int d = 0; d < 3; ++d) {
            b.grid_lo[d] = levels[l].grid_lo[d];
            b.valid_lo[d] = levels[l].valid_lo[d];
            b.valid_hi[d] = levels[l].valid_hi[d];
            b.count[d] = (grids[0]->desc.n[d] - 1) * (1 << l) + 1;
            const int glo = b.grid_lo[d], ghi = glo + g->desc.n[d] - 1;
            if (b.valid_lo[d] < glo || b.valid_hi[d] > ghi || b.valid_lo[d] > b.valid_hi[d] ||
                (l > 0 && ((b.valid_lo[d] & 1) || (b.valid_hi[d] & 1)))) {
                delete a;
                return set_err(c, ELAS_ERR_INVALID_ARG, "AMR valid box outside its grid or not coarse-aligned");
            }
        }
        for (int f = 0; f < 6; ++f) b.ghost[f] = levels[l].ghost[f];
        a->g.push_back(g);
        a->box.push_back(b);
        a->rbox.push_back(b);
        parts += (size_t)((g->lv[0].N + kBlock - 1) / kBlock) * kPartialStride;
    }
    auto alloc = [&](double** p, size_t count) -> int {
        const size_t bytes = count * sizeof(double);
        void* q = ctx_alloc(c, bytes);
        if (!q) return set_err(c, ELAS_ERR_ALLOC, "AMR work arrays: allocation failed");
        a->allocs.push_back({q, bytes});
        *p = (double*)q;
        return ELAS_OK;
    };
    int rc = alloc(&a->partials, parts);
    for (int l = 0; l < nlevels && !rc; ++l) {
        const size_t n3 = 3 * (size_t)grids[l]->lv[0].N;
        double *r1, *r2, *r3, *r4, *r5;
        if ((rc = alloc(&r1, n3)) || (rc = alloc(&r2, n3)) || (rc = alloc(&r3, n3)) || (rc = alloc(&r4, n3)) ||
            (rc = alloc(&r5, n3)))
            break;
        a->res.push_back(r1);
        a->rpass.push_back(r2);
        a->cor.push_back(r3);
        a->cora.push_back(r4);
        a->tmp.push_back(r5);
    }
    if (rc) {
        elas_amr_destroy(a);
        return rc;
    }
    for (auto g : a->g) ++g->amr_refs;
    a->holds_refs = true;
    *out = a;
    return ELAS_OK;
}

int elas_amr_set_reading(elas_amr a, int reading) {
    if (!a) return ELAS_ERR_INVALID_ARG;
    elas_ctx c = a->g[0]->ctx;
    if (reading != ELAS_AMR_R1 && reading != ELAS_AMR_R2) return set_err(c, ELAS_ERR_INVALID_ARG, "unknown AMR reading");
    const int nl = (int)a->g.size();
    for (int l = 0; l < nl; ++l) {
        AmrBox rb = a->box[l];
        if (reading == ELAS_AMR_R2 && l > 0) {
            for (int d = 0; d < 3; ++d) {
                const int glo = rb.grid_lo[d], ghi = glo + a->g[l]->desc.n[d] - 1;
                if (rb.ghost[2 * d]) {
                    if (rb.valid_lo[d] - glo < 2) return set_err(c, ELAS_ERR_INVALID_ARG, "reading R2 needs two ghost layers");
                    rb.valid_lo[d] -= 1;
                }
                if (rb.ghost[2 * d + 1]) {
                    if (ghi - rb.valid_hi[d] < 2) return set_err(c, ELAS_ERR_INVALID_ARG, "reading R2 needs two ghost layers");
                    rb.valid_hi[d] += 1;
                }
            }
        }
        a->rbox[l] = rb;
    }
    a->reading = reading;
    for (auto g : a->g) g->dirty = true;   // covered coarse moduli follow the reading
    return ELAS_OK;
}

int elas_amr_destroy(elas_amr a) {
    if (!a) return ELAS_ERR_INVALID_ARG;
    if (!a->g.empty() && server_holds(a->g[0]->ctx, nullptr, a))
        return set_err(a->g[0]->ctx, ELAS_ERR_STATE, "AMR layout has a waiting or active server request");
    if (!a->g.empty()) {
        elas_ctx c = a->g[0]->ctx;
        cudaStreamSynchronize(c->stream);
        for (auto& p : a->allocs) ctx_free(c, p.first, p.second);
        cudaStreamSynchronize(c->stream);
    }
    if (a->holds_refs)
        for (auto g : a->g) --g->amr_refs;
    delete a;
    return ELAS_OK;
}

}  // extern "C"

namespace {
// Set-up of a composite solve: covered coarse moduli (after changes), every level's
// set-up, the initial state (Dirichlet data; the free values kept for a warm start) and
// the covered coarse nodes from the fine ones.
int amr_prepare(elas_amr a, bool warm) {
    const int nl = (int)a->g.size();
    elas_ctx c = a->g[0]->ctx;
    cudaStream_t s = c->stream;
    bool dirty = false;
    for (auto g : a->g) dirty |= g->dirty;
    if (dirty) {
        for (int l = nl - 1; l >= 1; --l) {
            if (!a->g[l]->moduli_set || !a->g[l - 1]->moduli_set) return set_err(c, ELAS_ERR_STATE, "moduli not set");
            launch_amr_restrict(a->g[l]->lv[0].L64, a->rbox[l], a->g[l - 1]->lv[0].L64, a->box[l - 1],
                                a->g[l]->lv[0].mod64, a->g[l - 1]->lv[0].mod64, a->g[l]->K, 0, s);
            a->g[l - 1]->dirty = true;
        }
        CHECK_LAUNCH(c);
    }
    for (auto g : a->g) {
        // the composite cycle smooths with the red-black smoother in V-cycles
        g->smoother = ELAS_SMOOTH_RB;
        g->cycle = ELAS_CYCLE_V;
        int rc = setup(g);
        if (rc) return rc;
    }
    if (a->g[0]->lv[0].nf.m > 0) return set_err(c, ELAS_ERR_STATE, "AMR solve needs a problem without free rigid modes");
    for (int l = 0; l < nl; ++l)
        launch_dirichlet(a->g[l]->lv[0].L64, boundary_data(a->g[l]), a->g[l]->lv[0].u, warm ? 1 : 0, s);
    for (int l = nl - 1; l >= 1; --l) amr_sync(a, l, a->g[l]->lv[0].u, a->g[l - 1]->lv[0].u);
    CHECK_LAUNCH(c);
    return ELAS_OK;
}
}  // namespace

extern "C" {

int elas_amr_solve(elas_amr a, const elas_solve_opts* opts, elas_solve_info* info) {
    if (!a || !opts || !info) return ELAS_ERR_INVALID_ARG;
    elas_ctx c = a->g[0]->ctx;
    if (server_holds(c, nullptr, a))
        return set_err(c, ELAS_ERR_STATE, "AMR layout has a waiting or active server request");
    for (auto lg : a->g)
        if (int rc = refuse_if_served(lg)) return rc;
    cudaSetDevice(c->device);
    std::memset(info, 0, sizeof(*info));
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = c->stream;
    const bool mixed = opts->precision == ELAS_PRECISION_MIXED;
    const int nl = (int)a->g.size();
    int rc = mixed ? amr_alloc32(a) : ELAS_OK;
    if (rc) return rc;
    rc = amr_prepare(a, opts->warm_start != 0);
    if (rc) return rc;
    rc = amr_composite_residual(a);
    if (rc) return rc;
    double r0 = 0.0;
    if ((rc = amr_norm(a, &r0))) return rc;
    info->r0 = r0;
    const int nu1 = opts->nu1 < 0 ? 0 : opts->nu1, nu2 = opts->nu2 < 0 ? 0 : opts->nu2;
    int cycles = 0, hist = 0, status = ELAS_OK;
    double rel = 0.0;
    for (;;) {
        double nr = 0.0;
        if (cycles > 0) {
            if ((rc = amr_composite_residual(a))) return rc;
            if ((rc = amr_norm(a, &nr))) return rc;
        } else {
            nr = r0;
        }
        rel = r0 > 0 ? nr / r0 : 0.0;
        if (hist < ELAS_HISTORY) info->rel_history[hist++] = rel;
        if (!std::isfinite(rel) || rel > 1e12) {
            status = ELAS_ERR_DIVERGED;
            break;
        }
        if (opts->fixed_cycles > 0) {
            if (cycles >= opts->fixed_cycles) break;
        } else {
            if (rel <= opts->rel_tol) break;
            if (cycles >= opts->max_cycles) {
                status = ELAS_ERR_NOT_CONVERGED;
                break;
            }
        }
        if (mixed) {
            // FP32 composite cycle on the FP64 composite residual, FP64 update
            for (int l = 0; l < nl; ++l)
                launch_cast<float, double>(a->res32[l], a->res[l], (size_t)3 * a->g[l]->lv[0].N, s);
            amr_cycle32(a, nu1, nu2);
            for (int l = 0; l < nl; ++l)
                launch_amr_add<double, float>(a->g[l]->lv[0].L64, a->box[l], a->g[l]->lv[0].u, a->cor32[l], s);
            for (int l = nl - 1; l >= 1; --l) amr_sync(a, l, a->g[l]->lv[0].u, a->g[l - 1]->lv[0].u);
        } else {
            amr_cycle(a, nu1, nu2);
        }
        CHECK_LAUNCH(c);
        ++cycles;
    }
    CUDA_TRY(c, cudaStreamSynchronize(s));
    info->cycles = cycles;
    info->rel_residual = rel;
    info->residual_inf = -1.0;   // composite norms: the 2-norm only
    info->rel_residual_inf = -1.0;
    info->status = status;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (status == ELAS_ERR_NOT_CONVERGED) set_err(c, status, "maximum cycles reached above the tolerance");
    if (status == ELAS_ERR_DIVERGED) set_err(c, status, "residual diverged");
    return status;
}

}  // extern "C"

// ======================================================================================
// serving: continuous batching at refinement-step granularity
// ======================================================================================
namespace {
struct ServerReq {
    long long ticket;
    elas_grid g;
    elas_amr a = nullptr;       // composite AMR request (g = its level-0 grid)
    elas_solve_opts opts;
    int slot = -1;
    std::chrono::steady_clock::time_point t_submit;
    // AMR requests: convergence is followed on the host
    bool started = false;
    int cycles = 0;
    double r0 = 0.0;
    std::vector<double> hist;
};
struct ServerDone {
    elas_solve_info info;
    double latency;
};
}  // namespace

struct elas_server_s {
    elas_ctx ctx;
    int max_active;
    long long next = 1;
    std::deque<ServerReq> waiting;
    std::vector<ServerReq> active;
    std::vector<int> free_slots;
    std::map<long long, ServerDone> done;
    int* flags = nullptr;
    int* counts = nullptr;
    double* hist = nullptr;
    void* mem = nullptr;
    size_t bytes = 0;
    std::vector<int> h_flags, h_counts;
    double* h_norm = nullptr;   // pinned: the composite residual norms of AMR requests, per slot
};

bool server_holds(elas_ctx c, elas_grid g, elas_amr a) {
    auto holds = [&](const ServerReq& r) {
        if (a && r.a == a) return true;
        if (!g) return false;
        if (r.g == g) return true;
        if (r.a)
            for (auto lg : r.a->g)
                if (lg == g) return true;
        return false;
    };
    for (auto s : c->servers) {
        for (const auto& r : s->waiting)
            if (holds(r)) return true;
        for (const auto& r : s->active)
            if (holds(r)) return true;
    }
    return false;
}

extern "C" {

int elas_server_create(elas_ctx c, int max_active, elas_server* out) {
    if (!c || max_active < 1 || !out) return ELAS_ERR_INVALID_ARG;
    elas_server s = new elas_server_s();
    s->ctx = c;
    s->max_active = max_active;
    s->bytes = (size_t)max_active * 2 * sizeof(int) + 256 + (size_t)max_active * ELAS_HISTORY * sizeof(double);
    s->mem = ctx_alloc(c, s->bytes);
    if (!s->mem) {
        delete s;
        return set_err(c, ELAS_ERR_ALLOC, "server work arrays: allocation failed");
    }
    s->flags = (int*)s->mem;
    s->counts = s->flags + max_active;
    s->hist = (double*)((char*)s->mem + (((size_t)2 * max_active * sizeof(int) + 255) & ~size_t(255)));
    for (int i = max_active - 1; i >= 0; --i) s->free_slots.push_back(i);
    s->h_flags.assign(max_active, 0);
    s->h_counts.assign(max_active, 0);
    if (cudaMallocHost(&s->h_norm, sizeof(double) * max_active) != cudaSuccess) {
        ctx_free(c, s->mem, s->bytes);
        delete s;
        return set_err(c, ELAS_ERR_DEVICE, "server: pinned host buffer");
    }
    c->servers.push_back(s);
    *out = s;
    return ELAS_OK;
}

int elas_server_destroy(elas_server s) {
    if (!s) return ELAS_ERR_INVALID_ARG;
    cudaStreamSynchronize(s->ctx->stream);
    for (auto& r : s->active)
        for (auto& v : r.g->lv) v.L64.active = v.L32.active = nullptr;
    ctx_free(s->ctx, s->mem, s->bytes);
    if (s->h_norm) cudaFreeHost(s->h_norm);
    auto& sv = s->ctx->servers;
    sv.erase(std::remove(sv.begin(), sv.end(), s), sv.end());
    delete s;
    return ELAS_OK;
}

int elas_server_submit_amr(elas_server s, elas_amr a, const elas_solve_opts* opts, long long* ticket) {
    if (!s || !a || !opts || !ticket) return ELAS_ERR_INVALID_ARG;
    if (a->g[0]->ctx != s->ctx) return set_err(s->ctx, ELAS_ERR_INVALID_ARG, "AMR request of another context");
    for (const auto& w : s->waiting)
        if (w.a == a) return set_err(s->ctx, ELAS_ERR_STATE, "composite solve already has a waiting request");
    for (const auto& r : s->active)
        if (r.a == a) return set_err(s->ctx, ELAS_ERR_STATE, "composite solve already has an active request");
    ServerReq r;
    r.ticket = s->next++;
    r.g = a->g[0];
    r.a = a;
    r.opts = *opts;
    r.t_submit = std::chrono::steady_clock::now();
    s->waiting.push_back(r);
    *ticket = r.ticket;
    return ELAS_OK;
}

int elas_server_submit(elas_server s, elas_grid g, const elas_solve_opts* opts, long long* ticket) {
    if (!s || !g || !opts || !ticket) return ELAS_ERR_INVALID_ARG;
    if (g->ctx != s->ctx || !g->desc.mixed || g->desc.max_levels == 1)
        return set_err(s->ctx, ELAS_ERR_INVALID_ARG, "server requests need grids of its context with mixed = 1");
    // one request per grid at a time: two would share its residual partials, levels and flags
    for (const auto& w : s->waiting)
        if (w.g == g) return set_err(s->ctx, ELAS_ERR_STATE, "grid already has a waiting request");
    for (const auto& a : s->active)
        if (a.g == g) return set_err(s->ctx, ELAS_ERR_STATE, "grid already has an active request");
    ServerReq r;
    r.ticket = s->next++;
    r.g = g;
    r.opts = *opts;
    r.t_submit = std::chrono::steady_clock::now();
    s->waiting.push_back(r);
    *ticket = r.ticket;
    return ELAS_OK;
}

int elas_server_step(elas_server s, int* n_active, int* n_waiting) {
    if (!s) return ELAS_ERR_INVALID_ARG;
    elas_ctx c = s->ctx;
    cudaSetDevice(c->device);
    cudaStream_t main = c->stream;
    // admit: set the grid up first; a request whose set-up fails retires at once with
    // that error as its status and takes no slot
    while (!s->waiting.empty() && !s->free_slots.empty()) {
        ServerReq r = s->waiting.front();
        s->waiting.pop_front();
        elas_grid g = r.g;
        int rc = ELAS_OK;
        if (r.a) {
            if (r.opts.precision == ELAS_PRECISION_MIXED) rc = amr_alloc32(r.a);
            if (!rc) rc = amr_prepare(r.a, r.opts.warm_start != 0);
        } else {
            rc = take_cycle_opts(g, &r.opts);
            if (!rc) rc = setup(g);
            if (!rc && outer_df(g, &r.opts)) rc = df_prepare(g);
        }
        if (rc) {
            ServerDone d{};
            d.info.status = rc;
            d.latency = std::chrono::duration<double>(std::chrono::steady_clock::now() - r.t_submit).count();
            d.info.seconds = d.latency;
            s->done[r.ticket] = d;
            continue;
        }
        r.slot = s->free_slots.back();
        s->free_slots.pop_back();
        if (r.a) {
            s->active.push_back(r);
            continue;
        }
        Level& L0 = g->lv[0];
        launch_dirichlet(L0.L64, boundary_data(g), L0.u, r.opts.warm_start ? 1 : 0, main);
        outer_begin(g, outer_df(g, &r.opts), main);
        cudaMemsetAsync(g->lam, 0, sizeof(double) * 8, main);
        cudaMemsetAsync(g->alam, 0, sizeof(double) * kLoadDoubles, main);
        cudaMemsetAsync(g->adlam, 0, sizeof(double) * kLoadDoubles, main);
        const int one = 1, zero = 0;
        cudaMemcpyAsync(s->flags + r.slot, &one, sizeof(int), cudaMemcpyHostToDevice, main);
        cudaMemcpyAsync(s->counts + r.slot, &zero, sizeof(int), cudaMemcpyHostToDevice, main);
        CUDA_TRY(c, cudaStreamSynchronize(main));
        for (auto& v : g->lv) v.L64.active = v.L32.active = s->flags + r.slot;
        s->active.push_back(r);
    }
    if (!s->active.empty()) {
        // one refinement step of every active request, interleaved on branch streams
        const int S = (int)s->active.size() < 32 ? (int)s->active.size() : 32;
        while ((int)c->branch.size() < S) {
            cudaStream_t st;
            cudaEvent_t ev;
            CUDA_TRY(c, cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
            CUDA_TRY(c, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
            c->branch.push_back(st);
            c->branch_ev.push_back(ev);
        }
        cudaEvent_t fork = c->branch_ev[0];
        CUDA_TRY(c, cudaEventRecord(fork, main));
        for (int b = 0; b < S; ++b) cudaStreamWaitEvent(c->branch[b], fork, 0);
        const bool prof = c->profile;
        c->profile = false;
        for (size_t k = 0; k < s->active.size(); ++k) {
            ServerReq& r = s->active[k];
            elas_grid g = r.g;
            Level& L0 = g->lv[0];
            c->stream = c->branch[k % S];
            if (r.a) {
                // one composite cycle (the first step only evaluates the initial residual),
                // then the composite residual and its norm; mixed: the FP32 correction cycle
                // on the FP64 residual, as elas_amr_solve does
                if (r.started) {
                    if (r.opts.precision == ELAS_PRECISION_MIXED) {
                        elas_amr a = r.a;
                        const int nl = (int)a->g.size();
                        for (int l = 0; l < nl; ++l)
                            launch_cast<float, double>(a->res32[l], a->res[l], (size_t)3 * a->g[l]->lv[0].N, c->stream);
                        amr_cycle32(a, r.opts.nu1, r.opts.nu2);
                        for (int l = 0; l < nl; ++l)
                            launch_amr_add<double, float>(a->g[l]->lv[0].L64, a->box[l], a->g[l]->lv[0].u, a->cor32[l],
                                                          c->stream);
                        for (int l = nl - 1; l >= 1; --l) amr_sync(a, l, a->g[l]->lv[0].u, a->g[l - 1]->lv[0].u);
                    } else {
                        amr_cycle(r.a, r.opts.nu1, r.opts.nu2);
                    }
                }
                amr_composite_residual(r.a);
                amr_norm_enqueue(r.a);
                cudaMemcpyAsync(s->h_norm + r.slot, g->status, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
                continue;
            }
            const NullInfo* nf0 = L0.nf.m > 0 ? &L0.nf : nullptr;
            int nb = 0;
            outer_residual(g, outer_df(g, &r.opts), nf0, nf0 ? g->alam : nullptr, &nb, c->stream);
            BatchFlags bfl{s->flags + r.slot, s->counts + r.slot, s->hist + (size_t)r.slot * ELAS_HISTORY,
                           ELAS_HISTORY, g->r0, r.opts.rel_tol,
                           r.opts.fixed_cycles > 0 ? r.opts.fixed_cycles : r.opts.max_cycles};
            launch_finalize(g->partials, nb, L0.nf, g->Ginv, g->G, g->lam, g->dlam, g->alam, g->adlam, g->status, 1,
                            c->stream, bfl);
            for (int k = 0; k < (r.opts.inner_cycles > 1 ? r.opts.inner_cycles : 1); ++k)
                vcycle<float>(g, 0, r.opts.nu1, r.opts.nu2, nf0, nf0 ? g->adlam : nullptr, k == 0, r.opts.cycle);
            outer_correct(g, outer_df(g, &r.opts), c->stream);
        }
        c->stream = main;
        c->profile = prof;
        for (int b = 0; b < S; ++b) {
            cudaEventRecord(c->branch_ev[b], c->branch[b]);
            cudaStreamWaitEvent(main, c->branch_ev[b], 0);
        }
        CHECK_LAUNCH(c);
        CUDA_TRY(c, cudaMemcpyAsync(s->h_flags.data(), s->flags, sizeof(int) * s->max_active, cudaMemcpyDeviceToHost, main));
        CUDA_TRY(c, cudaMemcpyAsync(s->h_counts.data(), s->counts, sizeof(int) * s->max_active, cudaMemcpyDeviceToHost,
                                    main));
        CUDA_TRY(c, cudaStreamSynchronize(main));
        // retire
        std::vector<ServerReq> keep;
        for (auto& r : s->active) {
            if (r.a) {
                const double nr = std::sqrt(s->h_norm[r.slot]);
                if (!r.started) {
                    r.started = true;
                    r.r0 = nr;
                } else {
                    ++r.cycles;
                }
                const double rel = r.r0 > 0 ? nr / r.r0 : 0.0;
                r.hist.push_back(rel);
                const int maxc = r.opts.fixed_cycles > 0 ? r.opts.fixed_cycles : r.opts.max_cycles;
                const bool bad = !std::isfinite(rel) || rel > 1e12;
                const bool stop = bad || r.cycles >= maxc || (r.opts.fixed_cycles <= 0 && rel <= r.opts.rel_tol);
                if (!stop) {
                    keep.push_back(r);
                    continue;
                }
                ServerDone d{};
                const int cnt = (int)r.hist.size() < ELAS_HISTORY ? (int)r.hist.size() : ELAS_HISTORY;
                for (int k = 0; k < cnt; ++k) d.info.rel_history[k] = r.hist[k];
                d.info.cycles = r.cycles;
                d.info.rel_residual = rel;
                d.info.residual_inf = -1.0;   // composite norms: the 2-norm only
                d.info.rel_residual_inf = -1.0;
                d.info.r0 = r.r0;
                const bool ok = r.opts.fixed_cycles > 0 || rel <= r.opts.rel_tol;
                d.info.status = bad ? ELAS_ERR_DIVERGED : (ok ? ELAS_OK : ELAS_ERR_NOT_CONVERGED);
                d.latency = std::chrono::duration<double>(std::chrono::steady_clock::now() - r.t_submit).count();
                d.info.seconds = d.latency;
                s->done[r.ticket] = d;
                s->free_slots.push_back(r.slot);
                continue;
            }
            if (s->h_flags[r.slot]) {
                keep.push_back(r);
                continue;
            }
            elas_grid g = r.g;
            for (auto& v : g->lv) v.L64.active = v.L32.active = nullptr;
            int rc = remove_rigid(g);
            if (rc) return rc;
            ServerDone d{};
            const int cnt = s->h_counts[r.slot] < ELAS_HISTORY ? s->h_counts[r.slot] : ELAS_HISTORY;
            std::vector<double> h(cnt > 0 ? cnt : 1);
            if (cnt > 0)
                CUDA_TRY(c, cudaMemcpyAsync(h.data(), s->hist + (size_t)r.slot * ELAS_HISTORY, sizeof(double) * cnt,
                                            cudaMemcpyDeviceToHost, main));
            double rinf = 0.0;
            CUDA_TRY(c, cudaMemcpyAsync(&rinf, g->status + 1, sizeof(double), cudaMemcpyDeviceToHost, main));
            CUDA_TRY(c, cudaStreamSynchronize(main));
            d.info.residual_inf = rinf;
            d.info.rel_residual_inf = g->r0inf > 0 ? rinf / g->r0inf : 0.0;
            for (int k = 0; k < cnt; ++k) d.info.rel_history[k] = h[k];
            d.info.cycles = s->h_counts[r.slot] > 0 ? s->h_counts[r.slot] - 1 : 0;
            d.info.rel_residual = cnt > 0 ? h[cnt - 1] : 0.0;
            d.info.r0 = g->r0;
            d.info.nlam = g->lv[0].nf.m;
            const bool ok = r.opts.fixed_cycles > 0 || d.info.rel_residual <= r.opts.rel_tol;
            d.info.status = ok ? ELAS_OK : ELAS_ERR_NOT_CONVERGED;
            d.latency = std::chrono::duration<double>(std::chrono::steady_clock::now() - r.t_submit).count();
            d.info.seconds = d.latency;
            s->done[r.ticket] = d;
            s->free_slots.push_back(r.slot);
        }
        s->active.swap(keep);
    }
    if (n_active) *n_active = (int)s->active.size();
    if (n_waiting) *n_waiting = (int)s->waiting.size();
    return ELAS_OK;
}

int elas_server_poll(elas_server s, long long ticket, elas_solve_info* info, double* latency_s) {
    if (!s) return ELAS_ERR_INVALID_ARG;
    auto it = s->done.find(ticket);
    if (it == s->done.end()) return 0;
    if (info) *info = it->second.info;
    if (latency_s) *latency_s = it->second.latency;
    s->done.erase(it);
    return 1;
}

}  // extern "C"
