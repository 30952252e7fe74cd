/*
 * elas.h -- C ABI of the GB300 matrix-free geometric-multigrid elasticity solver.
 *
 * Solves the node-centred finite-difference form of static linear elasticity
 * with eigenstrain (Runnels et al., "Massively parallel finite difference
 * elasticity using block-structured adaptive mesh refinement with a geometric
 * multigrid solver", Section 2.1, Eq. 1a-1d):
 *
 *     d/dx_j [ C_ijkl(x) (du_k/dx_l - eps0_kl) ] = -b_i        in the interior
 *     u_i = u0_i                                               (Dirichlet, Eq. 1b)
 *     C_ijkl (du_k/dx_l - eps0_kl) n_j = t0_i                  (traction,  Eq. 1c)
 *     du_i/dx_j n_j = du0_i                                    (Neumann,   Eq. 1d)
 *
 * with the product-rule split of Section 2.1.1, the homogeneous/inhomogeneous
 * split D_H(u) = D(u) - D(0), boundary conditions as boundary-operator rows whose
 * data enter only through the right-hand side (Section 2.1), and a geometric
 * multigrid V-cycle over coarsened levels (Section 3.1) with trilinear
 * interpolation and power-of-two restriction (Section 3.2).
 *
 * Conventions shared by every call:
 *   - A grid has n[0] x n[1] x n[2] nodes, x fastest: node p = i + n0 (j + n1 k).
 *     A non-periodic direction includes both boundary planes, h = (hi-lo)/(n-1);
 *     a periodic direction counts unique nodes, h = (hi-lo)/n.
 *   - Vector fields are 3 planes of N doubles (structure of arrays): u_x, u_y, u_z.
 *   - Isotropic moduli (kind 2): 2 planes lambda, mu.  General moduli (kind 21):
 *     the 21 upper-triangle entries of the 6x6 Voigt matrix in Voigt order
 *     11,22,33,23,31,12, row by row (C11 C12 .. C16 C22 .. C66), one plane each.
 *   - Symmetric tensors (eigenstrain, mean strain): 6 tensor components
 *     11,22,33,23,31,12 (shears not doubled).
 *   - Faces 0..5 = -x,+x,-y,+y,-z,+z.  Boundary types per (face, component):
 *     ELAS_BC_DIRICHLET, ELAS_BC_TRACTION, ELAS_BC_NEUMANN; periodic directions
 *     have no faces.
 *   - memspace: ELAS_HOST for host pointers (copied during the call),
 *     ELAS_DEVICE for device pointers on the context's device (read during the
 *     call only, ordered on the context's stream); any other value is
 *     ELAS_ERR_INVALID_ARG.
 *   - Every function returns ELAS_OK (0) or a negative error code; the message of
 *     the last error on a context is returned by elas_last_error.
 *   - The library owns all device memory it allocates, through the allocator
 *     given at context creation (cudaMallocAsync on the context's stream when
 *     none is given).  Caller buffers are never retained after a call returns.
 *   - All device work is ordered on the context's stream; calls return after
 *     that work has completed unless stated otherwise.  A grid must not be used
 *     from two host threads at once; separate contexts are independent.
 */
#ifndef ELAS_H
#define ELAS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* error codes */
#define ELAS_OK                 0
#define ELAS_ERR_INVALID_ARG   -1
#define ELAS_ERR_OUT_OF_BUDGET -2   /* HBM budget of the context would be exceeded */
#define ELAS_ERR_NOT_CONVERGED -3   /* max_cycles reached above the tolerance */
#define ELAS_ERR_DIVERGED      -4   /* non-finite or exploding residual */
#define ELAS_ERR_DEVICE        -5   /* a CUDA call failed */
#define ELAS_ERR_ALLOC         -6   /* the allocator returned NULL */
#define ELAS_ERR_STATE         -7   /* call out of order (e.g. solve before moduli) */

#define ELAS_HOST   0
#define ELAS_DEVICE 1

#define ELAS_BC_DIRICHLET 1
#define ELAS_BC_TRACTION  2
#define ELAS_BC_NEUMANN   3

#define ELAS_MODULI_ISO   2
#define ELAS_MODULI_GEN21 21

#define ELAS_PRECISION_FP64  0   /* every level in FP64 */
#define ELAS_PRECISION_MIXED 1   /* FP32 V-cycle inside FP64 iterative refinement */

/* Smoothers (Section 3.1 smooths with Jacobi iterations; the default here is red-black).
 * One sweep of each: ELAS_SMOOTH_RB, red then black nodes ((i+j+k) even first), each
 * colour updated from the values before it (u <- u + B^-1 r with B the node's 3x3
 * diagonal block); ELAS_SMOOTH_GS8, the eight colours (i mod 2) + 2 (j mod 2) + 4 (k mod 2)
 * in that order, likewise (block Gauss-Seidel on interior rows, whose stencil never
 * joins two nodes of one colour); ELAS_SMOOTH_JACOBI, u <- u + omega B^-1 r on every node. */
#define ELAS_SMOOTH_RB     0
#define ELAS_SMOOTH_GS8    1
#define ELAS_SMOOTH_JACOBI 2
/* Cycles: V, or F (Section 3.1, the paper's runs): the coarse-grid correction of a level
 * is an F-cycle on the next level followed by a V-cycle from its result. */
#define ELAS_CYCLE_V 0
#define ELAS_CYCLE_F 1

typedef struct elas_ctx_s*  elas_ctx;
typedef struct elas_grid_s* elas_grid;

/* Device-memory allocator.  alloc returns a device pointer aligned to at least
 * 256 bytes, or NULL; free releases it.  Both receive the context's stream. */
typedef struct {
    void* (*alloc)(size_t bytes, void* user, void* stream);
    void  (*free)(void* ptr, size_t bytes, void* user, void* stream);
    void* user;
} elas_allocator;

/* Create a context on CUDA device `device`.  hbm_budget_bytes caps the device
 * memory the context may hold (0 = no cap); grid creation fails with
 * ELAS_ERR_OUT_OF_BUDGET beyond it.  alloc may be NULL.  stream is a
 * cudaStream_t (NULL = a stream created and owned by the context). */
int  elas_ctx_create(elas_ctx* out, int device, size_t hbm_budget_bytes,
                     const elas_allocator* alloc, void* stream);
/* Destroy the context's servers, AMR layouts and grids first: ELAS_ERR_STATE while a
 * server of the context is alive. */
int  elas_ctx_destroy(elas_ctx ctx);
const char* elas_last_error(elas_ctx ctx);
/* Bytes currently held by the context. */
size_t elas_ctx_bytes_in_use(elas_ctx ctx);

typedef struct {
    int    n[3];          /* nodes per direction (see conventions)          */
    int    periodic[3];   /* 1 = periodic direction                          */
    double lo[3], hi[3];  /* domain corners                                  */
    int    moduli_kind;   /* ELAS_MODULI_ISO or ELAS_MODULI_GEN21            */
    int    mixed;         /* 1 = also allocate the FP32 hierarchy            */
    int    max_levels;    /* 0 = coarsen automatically; 1 = this level only (AMR
                             fine levels: smoothed, never solved on their own)  */
    int    half_moduli;   /* mixed grids: the FP32 V-cycle reads FP16 moduli (half
                             the bytes); the FP64 refinement keeps FP64 moduli   */
} elas_grid_desc;

/* Create a grid and its multigrid hierarchy (Section 3.1: levels below 0,
 * coarsened by 2 while every direction stays coarsenable and some direction has
 * more than 5 nodes).  Requires n >= 3 per non-periodic direction, n >= 4 per
 * periodic one, and (unless max_levels == 1) node counts that coarsen down to a
 * bottom level of at most 6000 unknowns (e.g. n = 2^k m + 1 with small m).  All
 * boundary types default to Dirichlet 0. */
int  elas_grid_create(elas_ctx ctx, const elas_grid_desc* desc, elas_grid* out);
/* ELAS_ERR_STATE while a server holds a waiting or active request on the grid (as the
 * request's grid or a level of its AMR layout) or while a live AMR layout holds it as a
 * level (destroy the layout first); the grid then stays valid. */
int  elas_grid_destroy(elas_grid g);
/* Number of multigrid levels and the node counts of one of them. */
int  elas_grid_levels(elas_grid g, int* nlevels);
int  elas_grid_level_dims(elas_grid g, int level, int n[3]);
/* Device bytes the grid holds. */
size_t elas_grid_bytes(elas_grid g);
/* Device bytes a grid with this descriptor would hold (for admission control). */
size_t elas_grid_bytes_estimate(const elas_grid_desc* desc);

/* Moduli of the finest level: kind x N doubles (Section 2.1.1; general moduli as
 * stored per point in Section 4.3).  Coarse levels take the restriction of the
 * stored components. */
int  elas_set_moduli(elas_grid g, const double* comps, int memspace);
/* Eigenstrain eps0 (Eq. 1a), 6 x N doubles, or NULL for none.  The grid copies the
 * data into its own buffer; clearing with NULL keeps that buffer for the next set
 * (the same holds for the body force and the face values). */
int  elas_set_eigenstrain(elas_grid g, const double* eps6, int memspace);
/* Body force b (Eq. 1a), 3 x N doubles, or NULL for none. */
int  elas_set_body_force(elas_grid g, const double* b3, int memspace);
/* Mean strain E of a fully periodic grid: u = E x + u~, u~ periodic. */
int  elas_set_mean_strain(elas_grid g, const double eps6[6]);
/* Boundary type and uniform datum of (face, component): the prescribed
 * displacement (Eq. 1b), traction (Eq. 1c) or normal derivative (Eq. 1d). */
int  elas_set_bc(elas_grid g, int face, int comp, int type, double value);
/* Per-node boundary data of a face: 3 x N doubles over the whole grid, read on
 * that face only; NULL restores the uniform values. */
int  elas_set_face_values(elas_grid g, int face, const double* values, int memspace);

typedef struct {
    int    precision;     /* ELAS_PRECISION_FP64 or ELAS_PRECISION_MIXED          */
    double rel_tol;       /* stop when ||r||_2 / ||r_0||_2 <= rel_tol               */
    int    max_cycles;    /* V-cycles (FP64) or refinement steps (mixed)           */
    int    nu1, nu2;      /* pre / post smoothing sweeps (one sweep = red + black) */
    int    warm_start;    /* 1 = start from the current displacement              */
    int    fixed_cycles;  /* > 0: run exactly this many cycles, ignore rel_tol     */
    int    use_graph;     /* mixed: replay refinement steps as a captured CUDA graph
                             with device-side stopping (batched solves always do)  */
    int    inner_cycles;  /* mixed: FP32 V-cycles per FP64 refinement step (>= 1)  */
    int    smoother;      /* ELAS_SMOOTH_RB (default), ELAS_SMOOTH_GS8 or
                             ELAS_SMOOTH_JACOBI; nu1, nu2 count its sweeps         */
    int    cycle;         /* ELAS_CYCLE_V (default) or ELAS_CYCLE_F                 */
    double omega;         /* damping of ELAS_SMOOTH_JACOBI, in (0, 1] (default 2/3) */
    int    outer_residual;/* mixed: arithmetic of the refinement residual,
                             ELAS_OUTER_AUTO (default), ELAS_OUTER_FP64 or
                             ELAS_OUTER_DF                                         */
} elas_solve_opts;

/* Arithmetic of the refinement residual r = f - D_H(u) of a mixed solve.  FP64: plain
 * FP64 operations.  DF: double-float, every operation on an unevaluated FP32 pair
 * hi + lo (about 48 bits; rounding error a few 2^-47 of the operands' magnitudes) on
 * the FP32 pipes, from double-float copies of u, f and the moduli that the grid keeps
 * beside the FP64 ones (8 bytes per value); its residual floor lies near 1e-12 of the
 * load.  AUTO: DF when rel_tol >= 1e-11 or fixed_cycles > 0, else FP64.  The solution
 * stays an FP64 field either way; info->rel_residual is the norm of the residual so
 * evaluated. */
#define ELAS_OUTER_AUTO 0
#define ELAS_OUTER_FP64 1
#define ELAS_OUTER_DF   2

#define ELAS_HISTORY 128
typedef struct {
    int    status;                     /* ELAS_OK, ELAS_ERR_NOT_CONVERGED, ...        */
    int    cycles;                     /* coarse-grid corrections performed           */
    double rel_residual;               /* final ||r||/||r_0|| (FP64, or the refinement
                                          residual's double-float for mixed solves)     */
    double r0;                         /* ||r_0||: residual of the Dirichlet-only field */
    int    nlam;                       /* number of free rigid modes                  */
    double lam[6];                     /* equilibrating-load coefficients             */
    double seconds;                    /* wall time of the solve                      */
    double rel_history[ELAS_HISTORY];  /* relative residual before each correction    */
    double residual_inf;               /* ||r||_inf of the last residual evaluated (the
                                          refinement residual's arithmetic); -1 for
                                          composite AMR solves                          */
    double rel_residual_inf;           /* the same over ||r_0||_inf                     */
} elas_solve_info;

void elas_solve_opts_default(elas_solve_opts* o);

/* Solve D_H(u) = -(D(0) + b) with the boundary rows (Section 2.1.1).  Each cycle:
 * nu1 red-black block sweeps, the FP64 residual and its norm, stop if small
 * enough, restriction, recursive cycle, trilinear correction, nu2 sweeps
 * (Section 3.1).  Problems with free rigid modes get an equilibrating load
 * lambda W (W = the free rigid modes) and u has its rigid part removed.
 * Returns info->status. */
int  elas_solve(elas_grid g, const elas_solve_opts* opts, elas_solve_info* info);

/* Displacement of the finest level, 3 x N doubles (the fluctuation u~ on a
 * periodic grid with mean strain). */
int  elas_get_displacement(elas_grid g, double* out, int memspace);
int  elas_set_displacement(elas_grid g, const double* in, int memspace);
/* Stress of the current displacement of the finest level (the stress of Eq. 1c):
 * sigma = C : (grad u + E - eps0), E the mean strain of a periodic grid (else 0), eps0 the
 * eigenstrain (if set); first derivatives central, one-sided second order on the
 * boundary planes of a non-periodic direction.  out: 6 x N doubles, tensor components
 * 11, 22, 33, 23, 31, 12 (HOST or DEVICE per memspace; a HOST call allocates and frees a
 * 6 x N device buffer through the context's allocator). */
int  elas_get_stress(elas_grid g, double* out, int memspace);
/* FP64 residual of the current displacement: ||r||_2 / ||r_0||_2 and ||r||_2. */
int  elas_query_residual(elas_grid g, double* rel_l2, double* abs_l2);
/* The same residual's max norm: ||r||_inf / ||r_0||_inf and ||r||_inf (largest |r_i|
 * over all rows and components, the equilibrating load of the last solve applied). */
int  elas_query_residual_inf(elas_grid g, double* rel_inf, double* abs_inf);

/* ---- single operations of the path, for testing and benchmarking --------------
 * All take DEVICE pointers to FP64 (precision 0) or FP32 (precision 1) arrays of
 * the named level (3 x N_level unless stated) and run on the context's stream.  A
 * NULL grid or array pointer is ELAS_ERR_INVALID_ARG; the arrays' extent and element
 * type cannot be checked through a raw pointer and are the caller's to get right. */

/* out = A u on every row of `level`: interior and traction rows (Section 2.1.1
 * product rule, half-cell closure of Eq. 1c), Neumann rows, u itself on
 * Dirichlet rows. */
int  elas_op_apply(elas_grid g, int level, int precision, const void* u, void* out);
/* r = f - A u (0 on Dirichlet rows); *sumsq = sum r^2 (FP64 reduction).  precision
 * ELAS_OP_DF: the refinement residual of a mixed solve, in double-float arithmetic
 * from FP64 u and f, r written as FP32 (level 0 of a mixed grid with a hierarchy;
 * sumsq then sums the FP32 values of r). */
#define ELAS_OP_DF 2
int  elas_op_residual(elas_grid g, int level, int precision, const void* u, const void* f,
                      void* r, double* sumsq);
/* One red-black sweep (red then black, Jacobi within a colour), in place on u. */
int  elas_op_sweep(elas_grid g, int level, int precision, void* u, const void* f);
/* One sweep of the given smoother (ELAS_SMOOTH_*; omega for Jacobi), in place on u. */
int  elas_op_smooth(elas_grid g, int level, int precision, int smoother, double omega, void* u,
                    const void* f);
/* fc = R r: volume-weighted full weighting to level+1 (Section 3.2); 0 on
 * Dirichlet rows of the coarse level. */
int  elas_op_restrict(elas_grid g, int level, int precision, const void* r, void* fc);
/* u += P e: trilinear interpolation of the level+1 correction (Section 3.2),
 * added on non-Dirichlet rows. */
int  elas_op_prolong_add(elas_grid g, int level, int precision, const void* ec, void* u);
/* Right-hand side of the finest level (FP64, 3 x N) from moduli, eigenstrain,
 * body force, mean strain and boundary data. */
int  elas_op_rhs(elas_grid g, double* f_out);
/* Exact solve of the coarsest level (dense FP64 inverse built at setup). */
int  elas_op_bottom(elas_grid g, int precision, const void* f, void* u);

/* The residual of elas_op_residual, for callers that cannot allocate device memory
 * while they run: a host that has handed all of its memory to another runtime, code
 * running between the phases of a memory pool it does not own, or an embedding that
 * forbids cudaMalloc on its hot path.  This call allocates nothing: no cudaMalloc or
 * cudaFree, no allocator callback, no library routine that allocates.  Its reduction
 * scratch is one file-scope device array of ELAS_NOALLOC_SCRATCH_DOUBLES doubles that
 * every GPU loading this library holds until the process exits.  (The paper has no
 * counterpart; this is an interface for such callers only.)
 *   - Same arguments and results as elas_op_residual (device pointers u, f, r of the
 *     named level; *sumsq receives sum r^2).  The grid's own buffers are not used.
 *   - The grid must be set up: after new moduli, boundary types or loads the set-up
 *     (which may allocate) runs in the next solve or elas_op_residual; until then this
 *     call returns ELAS_ERR_STATE and does nothing.
 *   - A level whose reduction needs more blocks than the array holds is rejected with
 *     ELAS_ERR_INVALID_ARG (levels above about 33 million nodes with the default size:
 *     the bound counts two blocks of 256 per 256 nodes, covering the boundary blocks).
 *   - The first call on a device looks up the array's device address with that device
 *     current; make that first call before any stream capture.
 *   - All calls share the array and it keeps the last call's contents; every slot a
 *     call reads is written earlier in the same call, so nothing needs clearing, but
 *     calls that overlap on the GPU (other streams, other host threads) race. */
#define ELAS_NOALLOC_SCRATCH_DOUBLES (1 << 21)
int  elas_op_residual_noalloc(elas_grid g, int level, int precision, const void* u, const void* f,
                              void* r, double* sumsq);

/* ---- measurement -------------------------------------------------------------
 * With profiling enabled, every finest-level launch of the smoother and of the
 * residual inside elas_solve is bracketed by CUDA events on the context's stream;
 * elas_profile_read returns the summed device time and the launch count per
 * kernel class since the last enable.  elas_launch_count counts every kernel this
 * library has launched since it was loaded (all contexts). */
#define ELAS_PROF_SWEEP64_L0 0   /* FP64 red or black half-sweep, finest level   */
#define ELAS_PROF_SWEEP32_L0 1   /* FP32 half-sweep, finest level (mixed path)    */
#define ELAS_PROF_RESID64_L0 2   /* FP64 residual + norms, finest level           */
#define ELAS_PROF_RESID32_L0 3   /* FP32 residual, finest level (mixed path)      */
#define ELAS_PROF_CLASSES    4
/* ALU peak of the device, measured: a launch of independent fused multiply-add chains
 * on every SM (FP64 for precision 0, FP32 for precision 1), sized to about 20 ms, best
 * of three timed with CUDA events; *tflops receives FLOP/s / 1e12 (an FMA counts two).
 * The roofline of a kernel bound by arithmetic is stated against this number.  Allocates
 * and frees a 2 KB device buffer and a stream of its own. */
int  elas_measure_fma_peak(int device, int precision, double* tflops);
int  elas_profile_enable(elas_ctx ctx, int enable);
int  elas_profile_read(elas_ctx ctx, int kernel_class, double* total_ms, long long* launches);
unsigned long long elas_launch_count(void);

/* ---- autotuner ---------------------------------------------------------------
 * The interior smoother has several launch shapes: 0-4 are one thread per x-pair
 * of interior nodes with (threads per block, minimum resident blocks per SM) =
 * (256,1) (256,2) (256,3) (256,4) (128,8), the second number bounding registers per
 * thread (levels with FP16 moduli use shapes 1 and 2 only); 5 and 6 stage moduli and
 * displacement planes of a 32 x 16 (resp. 32 x 8) tile in shared memory and march
 * through z (FP32 levels with blocked FP32 moduli); 7 and 8 march 32 x 16 (resp. 32 x 8)
 * tiles through z with every global read an asynchronous copy one plane ahead (FP32
 * levels with colour-split moduli).  The arithmetic is identical, so every shape gives
 * bitwise-equal results.  elas_autotune
 * times each shape on every level of the grid, in FP32 (mixed grids) and FP64,
 * and keeps the fastest per (level dimensions, moduli kind, precision) in a
 * process-wide table used by every later launch.  times_ms (optional) receives
 * the FP32 timings of the finest level, one per shape (-1 where a shape does not
 * apply).  The table can be saved
 * and restored as text: one "nx ny nz kind bytes layout shape" line per entry, bytes the
 * element size (4 or 8), layout 0 for moduli stored plainly, 1 with the precomputed
 * modulus divergence, 2 for colour-split records.  A line naming an unknown shape is
 * skipped. */
int  elas_autotune(elas_grid g, float* times_ms, int ntimes);
int  elas_autotune_dump(char* buf, int cap);   /* returns the text length */
int  elas_autotune_load(const char* text);     /* returns the entries read */

/* ---- block-structured AMR (Section 3.1, reflux-free coarse/fine, Section 3.2,
 * Appendix A) ------------------------------------------------------------------
 * nlevels grids of one context: level 0 covers the domain (with its multigrid
 * hierarchy); level l >= 1 is one box at half the spacing of level l-1, created
 * with max_levels = 1.  Placement: node i of level l's global index space sits at
 * lo + i h_0 / 2^l; grid_lo is the global index of the grid's first node, the valid
 * box [valid_lo, valid_hi] is the part it solves for, and ghost[f] marks a
 * coarse/fine face carrying one ghost layer (set that face's boundary type to
 * Dirichlet).  The caller creates, loads and destroys the grids; elas_amr holds
 * work arrays only.  Covered coarse moduli are replaced by the restriction of the
 * finer level's (operator equivalence across levels).  Solve: the composite cycle
 * (ghosts by trilinear interpolation of the coarser level, covered coarse nodes by
 * injection, restricted fine residuals on covered nodes, level-0 V-cycle); the
 * problem must have no free rigid modes.  opts->precision ELAS_PRECISION_FP64: FP64
 * composite cycles; ELAS_PRECISION_MIXED (every level's grid created with mixed = 1):
 * each refinement step casts the FP64 composite residual to FP32, runs one composite
 * correction cycle in FP32 (FP32 fine-level smoothing, FP32 level-0 V-cycle) and adds the
 * corrections to the FP64 levels; convergence is tested on the FP64 composite residual.
 * Level solutions are read with elas_get_displacement on each grid. */
typedef struct elas_amr_s* elas_amr;
typedef struct {
    int grid_lo[3];
    int valid_lo[3];
    int valid_hi[3];
    int ghost[6];
} elas_amr_level;
int  elas_amr_create(elas_grid* grids, const elas_amr_level* levels, int nlevels, elas_amr* out);
/* Which reading of the reflux-free treatment (Section 3.2) the composite cycle uses.
 * ELAS_AMR_R1 (default): valid fine nodes include the coarse/fine boundary, one ghost
 * layer (Dirichlet, interpolated), covered coarse nodes take the coincident fine value,
 * fine residuals and moduli pass down with the restriction weights truncated to valid
 * nodes and renormalised.  ELAS_AMR_R2 (the "N + 1 ghost nodes" of Section 3.2, N = 1):
 * fine grids carry two ghost layers on each coarse/fine face (grid_lo two nodes before
 * valid_lo there); the inner layer is relaxed with the valid nodes, the outer one is the
 * interpolated Dirichlet layer; residuals, moduli and the solution pass down by the
 * untruncated full-weighting restriction (covered Dirichlet coarse rows keep their
 * values).  ELAS_ERR_INVALID_ARG if a grid lacks the second layer.  The composite norm
 * counts valid fine rows and uncovered coarse rows in both readings. */
#define ELAS_AMR_R1 1
#define ELAS_AMR_R2 2
int  elas_amr_set_reading(elas_amr a, int reading);
/* Releases the layout's own buffers (not its grids); ELAS_ERR_STATE while a server holds
 * a waiting or active request on it. */
int  elas_amr_destroy(elas_amr a);
int  elas_amr_solve(elas_amr a, const elas_solve_opts* opts, elas_solve_info* info);

/* ---- batches ---------------------------------------------------------------
 * Solve n independent grids of the same context (mixed precision), all in flight at
 * once on the context's stream.  When every grid has one moduli kind and one FP32
 * moduli layout (and the red-black smoother is chosen), each phase of the cycle -- a
 * half-sweep of one level, a residual, a restriction, a prolongation, the bottom solve,
 * the load update, the FP64 correction -- is ONE launch over a device work list of the
 * members taking part (a block reads its member and its block within it from a block map),
 * so launches per refinement step depend on the number of levels, not of members.  Two
 * refinement steps are captured as a CUDA graph once per batch composition and options
 * (cached on the context until a member is destroyed, set up anew, or gets new loads)
 * and replayed until every member has stopped on its own tolerance (device-side flags).
 * Other batches run each member's own launches as parallel graph branches.  Every member
 * computes exactly what its lone elas_solve computes.  info has n entries.  A grid listed
 * twice is ELAS_ERR_INVALID_ARG. */
int  elas_batch_solve(elas_grid* grids, int n, const elas_solve_opts* opts,
                      elas_solve_info* info);

/* ---- serving: continuous batching at refinement-step granularity -----------------
 * A server owns no grids: the caller keeps hierarchies resident and submits solves
 * of them (typically warm-started).  elas_server_step admits waiting requests into
 * free slots (at most max_active), advances every active request by one
 * refinement step (FP64 residual, FP32 V-cycle, FP64 update; mixed precision,
 * grids created with mixed = 1), all members' kernels interleaved on parallel
 * streams, and retires the ones that reached their tolerance.  elas_server_submit
 * refuses (ELAS_ERR_STATE) a grid that already has a waiting or active request.  A
 * request whose set-up fails at admission (e.g. no moduli set) takes no slot: it
 * retires at once and polls as done with that error in info->status.  Results are the
 * same as a lone elas_solve with the same options (same kernels in the same
 * order per grid).  While a request on a grid (or on an AMR layout holding it) waits or
 * runs, calls that launch on that grid or change it -- solves, batches, single
 * operations, setters, residual queries, stress, autotune, destroy -- return
 * ELAS_ERR_STATE; reading its displacement stays allowed. */
typedef struct elas_server_s* elas_server;
int  elas_server_create(elas_ctx ctx, int max_active, elas_server* out);
int  elas_server_destroy(elas_server s);
int  elas_server_submit(elas_server s, elas_grid g, const elas_solve_opts* opts, long long* ticket);
/* A composite AMR solve as a request (Section 3.2, reading as set on the elas_amr):
 * admitted into a free slot like a grid request; each server step runs one composite
 * cycle of it (FP64, or for opts->precision ELAS_PRECISION_MIXED one FP32 correction cycle
 * on the FP64 composite residual, as in elas_amr_solve), interleaved with the other
 * requests, and it retires at opts->rel_tol (composite norm) or max_cycles.  warm_start
 * keeps the levels' current displacements.  Results are the same as elas_amr_solve's
 * (same kernels, same order). */
int  elas_server_submit_amr(elas_server s, elas_amr a, const elas_solve_opts* opts, long long* ticket);
/* One step; *active and *waiting receive the counts after it. */
int  elas_server_step(elas_server s, int* active, int* waiting);
/* 1 when the request is done (info filled, latency from submit to retirement in
 * seconds; info->status is negative if it failed), 0 while pending or unknown,
 * negative on a bad argument. */
int  elas_server_poll(elas_server s, long long ticket, elas_solve_info* info, double* latency_s);

#ifdef __cplusplus
}
#endif
#endif /* ELAS_H */
