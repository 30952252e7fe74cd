// Device code of the matrix-free multigrid path (sm_103a), shared by the translation
// units that instantiate its launchers (elas_kernels.cu, elas_residual.cu and the two
// smoother units), so that they compile in parallel.  Kernels that are not templates
// are compiled only in elas_kernels.cu (ELAS_KERNELS_TU), which launches them.
//
// One thread per node (per node pair in the smoother).  Fields are structure of
// arrays, so every warp reads and writes contiguous x-runs of each plane; the
// stencil's neighbour reuse is served by L1/L2.  Reductions are deterministic:
// warp shuffles, one partial per block, then a single-block fixed-order sum.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "elas_internal.h"

namespace elas {
namespace {

inline int blocks_for(size_t n) { return (int)((n + kBlock - 1) / kBlock); }

__device__ __forceinline__ void coords_of(int p, const int n[3], int c[3]) {
    c[0] = p % n[0];
    const int r = p / n[0];
    c[1] = r % n[1];
    c[2] = r / n[1];
}

// Block-wide sum of `width` doubles per thread into partials[bid * kPartialStride + w].
template <int MAXW>
__device__ __forceinline__ void block_reduce_store_at(double (&v)[MAXW], int width, double* partials, int bid) {
    __shared__ double sm[kBlock / 32][MAXW];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int w = 0; w < MAXW; ++w) {
        if (w >= width) break;
        double x = v[w];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sm[warp][w] = x;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
#pragma unroll
        for (int w = 0; w < MAXW; ++w) {
            if (w >= width) break;
            double x = (lane < kBlock / 32) ? sm[lane][w] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if (lane == 0) partials[(size_t)bid * kPartialStride + w] = x;
        }
    }
}

template <int MAXW>
__device__ __forceinline__ void block_reduce_store(double (&v)[MAXW], int width, double* partials) {
    block_reduce_store_at<MAXW>(v, width, partials, blockIdx.x);
}

// Residual norms of a block: the sums v[0 .. width) (sum r^2, the rigid moments) and the
// maximum v[7] of |r| into partials[bid * kPartialStride + 0 .. width) and [+ 7].
__device__ __forceinline__ void block_reduce_norms_at(double (&v)[8], int width, double* partials, int bid) {
    double sums[7];
#pragma unroll
    for (int w = 0; w < 7; ++w) sums[w] = v[w];
    block_reduce_store_at<7>(sums, width, partials, bid);
    __shared__ double smax[kBlock / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double x = v[7];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_down_sync(0xffffffffu, x, o));
    if (lane == 0) smax[warp] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
        x = lane < kBlock / 32 ? smax[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_down_sync(0xffffffffu, x, o));
        if (lane == 0) partials[(size_t)bid * kPartialStride + 7] = x;
    }
}

// Fixed-order sum of the 7-wide block partials by one block of kSumThreads threads:
// each thread keeps four records in flight per step (the loads are independent, so the
// sum is limited by bandwidth rather than by one load's latency), then a warp-shuffle
// tree and a second one over the warps.  The result lands in sm[0][0..6]; sm[0][7] is the
// maximum of the records' slot 7 (max |r| where a residual wrote them).
constexpr int kSumThreads = 512;
__device__ __forceinline__ void sum_partials_block(const double* __restrict__ partials, int nblocks,
                                                   double (&sm)[kSumThreads / 32][8]) {
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b0 = threadIdx.x; b0 < nblocks; b0 += 4 * kSumThreads) {
        double v[4][8];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int b = b0 + k * kSumThreads;
#pragma unroll
            for (int w = 0; w < 8; ++w) v[k][w] = b < nblocks ? partials[(size_t)b * kPartialStride + w] : 0.0;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
#pragma unroll
            for (int w = 0; w < 7; ++w) acc[w] += v[k][w];
            acc[7] = fmax(acc[7], v[k][7]);
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        double x = acc[w];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double y = __shfl_down_sync(0xffffffffu, x, o);
            x = w == 7 ? fmax(x, y) : x + y;
        }
        if (lane == 0) sm[warp][w] = x;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            double x = lane < kSumThreads / 32 ? sm[lane][w] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double y = __shfl_down_sync(0xffffffffu, x, o);
                x = w == 7 ? fmax(x, y) : x + y;
            }
            if (lane == 0) sm[0][w] = x;
        }
    }
    __syncthreads();
}

template <typename T>
__device__ __forceinline__ T face_datum(const BoundaryData& bd, int f, int c, int p, int N) {
    return bd.face[f] ? T(bd.face[f][c * N + p]) : T(bd.uniform[f][c]);
}

// ---------------------------------------------------------------------------
// right-hand side (setup, FP64)
// ---------------------------------------------------------------------------
template <int KIND>
__global__ void k_rhs(Lv<double> L, RhsInputs in, BoundaryData bd, double* __restrict__ f) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= L.N) return;
    int c[3];
    coords_of(p, L.n, c);
    const NodeInfo ni = node_info(L, c[0], c[1], c[2]);
    const int N = L.N;
    auto eps = [&](int k, int l, int q) -> double {
        return in.eps0 ? in.eps0[voigt(k, l) * N + q] : 0.0;
    };
    // with no eigenstrain and no mean strain the source terms vanish: only body force and
    // boundary data remain
    const bool source = in.eps0 || in.has_mean_strain;
    for (int i = 0; i < 3; ++i) {
        const int t = row_type(L, ni, i);
        double v = 0.0;
        if (t == ROW_INTERIOR || t == ROW_TRACTION) {
            if (in.body) v -= in.body[i * N + p];
            for (int j = 0; j < 3 && source; ++j) {
                if (ni.side[j] != 0) continue;
                int cp[3] = {c[0], c[1], c[2]}, cm[3] = {c[0], c[1], c[2]};
                cp[j] = wrapc(L, j, c[j] + 1);
                cm[j] = wrapc(L, j, c[j] - 1);
                const int qp = lin(L, cp[0], cp[1], cp[2]), qm = lin(L, cm[0], cm[1], cm[2]);
                for (int k = 0; k < 3; ++k)
                    for (int l = 0; l < 3; ++l) {
                        const double C0 = (KIND == 2) ? Cm<double, 2>(L, p, i, j, k, l) : Cm<double, 21>(L, p, i, j, k, l);
                        const double Cp = (KIND == 2) ? Cm<double, 2>(L, qp, i, j, k, l) : Cm<double, 21>(L, qp, i, j, k, l);
                        const double Cn = (KIND == 2) ? Cm<double, 2>(L, qm, i, j, k, l) : Cm<double, 21>(L, qm, i, j, k, l);
                        const double ebar = in.has_mean_strain ? in.mean_strain[voigt(k, l)] : 0.0;
                        v += (Cp - Cn) * L.inv2h[j] * (eps(k, l, p) - ebar) +
                             C0 * (eps(k, l, qp) - eps(k, l, qm)) * L.inv2h[j];
                    }
            }
            if (t == ROW_TRACTION) {
                for (int a = 0; a < 3; ++a) {
                    if (ni.side[a] == 0) continue;
                    const int fc = 2 * a + (ni.side[a] > 0 ? 1 : 0);
                    const double s = ni.side[a];
                    int cn[3] = {c[0], c[1], c[2]};
                    cn[a] -= ni.side[a];
                    const int qn = lin(L, cn[0], cn[1], cn[2]);
                    double acc = 0.0;
                    for (int k = 0; k < 3 && in.eps0; ++k)
                        for (int l = 0; l < 3; ++l) {
                            const double Ca = (KIND == 2) ? Cm<double, 2>(L, p, i, a, k, l) : Cm<double, 21>(L, p, i, a, k, l);
                            const double Cb = (KIND == 2) ? Cm<double, 2>(L, qn, i, a, k, l) : Cm<double, 21>(L, qn, i, a, k, l);
                            acc += 0.5 * (Ca + Cb) * 0.5 * (eps(k, l, p) + eps(k, l, qn));
                        }
                    v -= (2.0 * L.invh[a]) * (face_datum<double>(bd, fc, i, p, N) + s * acc);
                }
            }
        } else if (t == ROW_NEUMANN) {
            for (int a = 0; a < 3; ++a) {
                if (ni.side[a] == 0) continue;
                const int fc = 2 * a + (ni.side[a] > 0 ? 1 : 0);
                if (L.bc[fc][i] != ROW_NEUMANN) continue;
                const double C = (KIND == 2) ? Cm<double, 2>(L, p, i, a, i, a) : Cm<double, 21>(L, p, i, a, i, a);
                v += -(2.0 * L.invh[a]) * C * face_datum<double>(bd, fc, i, p, N);
            }
        }
        f[i * N + p] = v;
    }
}

#ifdef ELAS_KERNELS_TU
__global__ void k_dirichlet(Lv<double> L, BoundaryData bd, double* __restrict__ u, int keep_free) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= L.N) return;
    int c[3];
    coords_of(p, L.n, c);
    const NodeInfo ni = node_info(L, c[0], c[1], c[2]);
    for (int i = 0; i < 3; ++i) {
        const int t = row_type(L, ni, i);
        if (t == ROW_DIRICHLET) {
            // lowest-numbered Dirichlet face of this node wins
            double v = 0.0;
            for (int f = 5; f >= 0; --f) {
                const int d = f / 2;
                const int on = (f % 2 == 0) ? (ni.side[d] < 0) : (ni.side[d] > 0);
                if (on && L.bc[f][i] == ROW_DIRICHLET) v = face_datum<double>(bd, f, i, p, L.N);
            }
            u[i * L.N + p] = v;
        } else if (!keep_free) {
            u[i * L.N + p] = 0.0;
        }
    }
}
#endif

// ---------------------------------------------------------------------------
// operator, residual, smoother.  Each comes as an interior kernel over the box of
// nodes on no boundary plane (the fast stencil, no divergence) and a boundary
// kernel over the level's list of boundary-plane nodes (generic rows).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void interior_box(const Lv<T>& L, int lo[3], int cnt[3]) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        lo[d] = L.per[d] ? 0 : 1;
        cnt[d] = L.per[d] ? L.n[d] : L.n[d] - 2;
    }
}

template <typename T>
__host__ __device__ inline size_t interior_count(const Lv<T>& L) {
    size_t c = 1;
    for (int d = 0; d < 3; ++d) c *= (size_t)(L.per[d] ? L.n[d] : L.n[d] - 2);
    return c;
}

template <typename T>
__host__ __device__ inline size_t interior_pairs(const Lv<T>& L) {
    const int cx = L.per[0] ? L.n[0] : L.n[0] - 2;
    const int cy = L.per[1] ? L.n[1] : L.n[1] - 2;
    const int cz = L.per[2] ? L.n[2] : L.n[2] - 2;
    return (size_t)((cx + 1) / 2) * cy * cz;
}

template <typename T, int KIND, bool HM>
__global__ void __launch_bounds__(kBlock) k_apply_int(Lv<T> L, const T* __restrict__ u, T* __restrict__ out) {
    int lo[3], cnt[3];
    interior_box(L, lo, cnt);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cnt[0] * cnt[1] * cnt[2]) return;
    const int x = lo[0] + t % cnt[0], y = lo[1] + (t / cnt[0]) % cnt[1], z = lo[2] + t / (cnt[0] * cnt[1]);
    T v[3];
    interior_rows<T, KIND, HM>(L, u, x, y, z, v);
    const int p = lin(L, x, y, z);
    for (int i = 0; i < 3; ++i) out[i * L.N + p] = v[i];
}

// Edge and corner nodes: one warp per node, lanes 0-2 evaluate its three rows.
template <typename T, int KIND>
__global__ void __launch_bounds__(kBlock) k_apply_bnd(Lv<T> L, const T* __restrict__ u, T* __restrict__ out) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= L.nbnd || lane >= 3) return;
    const int p = L.bnodes[w];
    int c[3];
    coords_of(p, L.n, c);
    const NodeInfo ni = node_info(L, c[0], c[1], c[2]);
    UField<T> uf{u, L.N, L.n[0], L.n[1]};
    out[lane * L.N + p] = boundary_row<T, KIND>(L, uf, ni, lane, row_type(L, ni, lane));
}

// r = f - load - A u on one node's rows (load = t + w x d, the equilibrating load);
// accumulates sum r^2 and the six rigid-motion moments sum r, sum d x r.
template <typename T, typename TR, bool NORM>
__device__ __forceinline__ void residual_store(const Lv<T>& L, const T* __restrict__ f, const NullInfo& nf,
                                               const double* __restrict__ load, const int c[3], int p,
                                               const int types[3], const T v[3], TR* __restrict__ r,
                                               double acc[8]) {
    T rr[3];
    for (int i = 0; i < 3; ++i) {
        T ri = T(0);
        if (types[i] != ROW_DIRICHLET) {
            T fi = f[i * L.N + p];
            if (load) fi -= rigid_load<T>(nf, load, i, c);
            ri = fi - v[i];
        }
        rr[i] = ri;
        r[i * L.N + p] = (TR)ri;
    }
    if (NORM) {
        const double r0 = (double)rr[0], r1 = (double)rr[1], r2 = (double)rr[2];
        acc[0] += r0 * r0 + r1 * r1 + r2 * r2;
        acc[7] = fmax(acc[7], fmax(fabs(r0), fmax(fabs(r1), fabs(r2))));
        if (nf.m > 0) {
            // FP64: the moments of r cancel strongly (they measure the small incompatible
            // part), so they are summed in full precision
            const double d0 = nf.off[0] + nf.h[0] * c[0];
            const double d1 = nf.off[1] + nf.h[1] * c[1];
            const double d2 = nf.off[2] + nf.h[2] * c[2];
            acc[1] += r0;
            acc[2] += r1;
            acc[3] += r2;
            acc[4] += d1 * r2 - d2 * r1;
            acc[5] += d2 * r0 - d0 * r2;
            acc[6] += d0 * r1 - d1 * r0;
        }
    }
}

// Residual bodies: one interior node per thread, one edge/corner node per warp, one
// face node per thread; each adds its node's contributions to the thread's sums.
template <typename T, typename TR, int KIND, bool NORM, bool HM, int ML>
__device__ __forceinline__ void residual_int_body(const Lv<T>& L, const T* __restrict__ u, const T* __restrict__ f,
                                                  const NullInfo& nf, const double* __restrict__ lam,
                                                  TR* __restrict__ r, int t, double acc[8]) {
    if constexpr (ML == kMlSplit) {
        // warps in pairs over 64 consecutive interior nodes, the first taking the even
        // offsets and the second the odd ones: within a row a warp's nodes then share a
        // colour, so each of its record loads is 32 consecutive entries of one colour half
        // (one 128-byte line) instead of 16 from each half
        const int w = t >> 5, lane = t & 31;
        t = ((w >> 1) << 6) + (lane << 1) + (w & 1);
    }
    int lo[3], cnt[3];
    interior_box(L, lo, cnt);
    if (t >= cnt[0] * cnt[1] * cnt[2]) return;
    const int c[3] = {lo[0] + t % cnt[0], lo[1] + (t / cnt[0]) % cnt[1], lo[2] + t / (cnt[0] * cnt[1])};
    T v[3];
    with_interior<T, KIND, ML>(L, u, c[0], c[1], c[2], [&](const auto& ua, const auto& ca, int p) {
        interior_rows_core<T, KIND, HM>(L, ua, ca, p, v);
    });
    const int types[3] = {ROW_INTERIOR, ROW_INTERIOR, ROW_INTERIOR};
    residual_store<T, TR, NORM>(L, f, nf, lam, c, lin(L, c[0], c[1], c[2]), types, v, r, acc);
}

// Rows of an edge or corner node from its stored coefficients (L.bcoef): lanes 0-26 take
// one slot each (three displacement loads, nine multiply-adds), then a fixed shuffle
// tree sums the lanes.  Every lane returns the three rows.
template <typename T>
__device__ __forceinline__ void edge_rows_coef(const Lv<T>& L, const T* __restrict__ u, const NodeInfo& ni,
                                               const T* __restrict__ cf, int lane, T v[3]) {
    T s0 = T(0), s1 = T(0), s2 = T(0);
    if (lane < 27) {
        int a[3];
        edge_slot_node(L, ni, lane, a);
        const int q = lin(L, a[0], a[1], a[2]);
        const T u0 = u[q], u1 = u[L.N + q], u2 = u[2 * L.N + q];
        const T* c0 = cf + 3 * lane;
        s0 = xfma(c0[2], u2, xfma(c0[1], u1, xmul(c0[0], u0)));
        s1 = xfma(c0[83], u2, xfma(c0[82], u1, xmul(c0[81], u0)));
        s2 = xfma(c0[164], u2, xfma(c0[163], u1, xmul(c0[162], u0)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s0 = xadd(s0, shfl_xor_all(s0, o));
        s1 = xadd(s1, shfl_xor_all(s1, o));
        s2 = xadd(s2, shfl_xor_all(s2, o));
    }
    v[0] = s0;
    v[1] = s1;
    v[2] = s2;
}

template <typename T, typename TR, int KIND, bool NORM>
__device__ __forceinline__ void residual_bnd_body(const Lv<T>& L, const T* __restrict__ u, const T* __restrict__ f,
                                                  const NullInfo& nf, const double* __restrict__ lam,
                                                  TR* __restrict__ r, int w, int lane, double acc[8]) {
    if (w >= L.nbnd) return;   // whole warp
    const int p = L.bnodes[w];
    int c[3];
    coords_of(p, L.n, c);
    const NodeInfo ni = node_info(L, c[0], c[1], c[2]);
    int types[3];
    for (int i = 0; i < 3; ++i) types[i] = row_type(L, ni, i);
    T v[3];
    edge_rows_coef<T>(L, u, ni, L.bcoef + (size_t)w * kEdgeCoef, lane, v);
    if (lane == 0) residual_store<T, TR, NORM>(L, f, nf, lam, c, p, types, v, r, acc);
}

// Red-black smoother, interior nodes: each thread owns the x-pair (x0, x0+1) of the
// interior box, updates the one of the active colour and copies the other; every
// row uses the values from before the half-sweep (Jacobi within the colour).
template <typename T, int KIND, bool HM, int ML>
__device__ __forceinline__ void sweep_pair_body(const Lv<T>& L, const T* __restrict__ u, T* __restrict__ uo,
                                                const T* __restrict__ f, int colour, const NullInfo& nf,
                                                const double* __restrict__ lam, int t) {
    int lo[3], cnt[3];
    interior_box(L, lo, cnt);
    const int npair = (cnt[0] + 1) >> 1;
    if (t >= npair * cnt[1] * cnt[2]) return;
    const int m = t % npair;
    const int yz = t / npair;
    const int y = lo[1] + yz % cnt[1], z = lo[2] + yz / cnt[1];
    const int x0 = lo[0] + 2 * m;
    const int xend = lo[0] + cnt[0];          // one past the last interior x
    const int N = L.N;
    auto copy = [&](int x) {
        const int q = lin(L, x, y, z);
        uo[q] = u[q];
        uo[N + q] = u[N + q];
        uo[2 * N + q] = u[2 * N + q];
    };
    // copy_dx: 0, or the x offset (+-1) of an inactive pair partner to copy with the update
    auto update = [&](int x, int copy_dx) {
        const int c[3] = {x, y, z};
        auto body = [&](const auto& ua, const auto& ca, int p) {
            T v[3], r[3], B[3][3], d[3];
            interior_rows_core<T, KIND, HM>(L, ua, ca, p, v);
            for (int i = 0; i < 3; ++i) {
                T fi = f[i * N + p];
                if (lam) fi = xsub(fi, rigid_load<T>(nf, lam, i, c));
                r[i] = xsub(fi, v[i]);
            }
            interior_block_acc<T, KIND>(L, ca, B);
            solve3(B, r, d);
            if (colour == kJacobiColour)
                for (int i = 0; i < 3; ++i) d[i] = xmul(L.omega, d[i]);
            for (int i = 0; i < 3; ++i) {
                if (copy_dx > 0) uo[i * N + p + 1] = ua(i, 1, 0, 0);
                else if (copy_dx < 0) uo[i * N + p - 1] = ua(i, -1, 0, 0);
                uo[i * N + p] = xadd(ua(i, 0, 0, 0), d[i]);
            }
        };
        with_interior<T, KIND, ML>(L, u, x, y, z, body);
    };
    if (colour < 2) {
        // red-black: exactly one node of the pair is active (the partner's copy goes
        // first: storing it beside the update measured slower)
        const int xa = x0 + ((x0 + y + z + colour) & 1);
        const int xi = (xa == x0) ? x0 + 1 : x0;
        if (xi < xend) copy(xi);
        if (xa < xend) update(xa, 0);
        return;
    }
    // eight colours or Jacobi: each node of the pair in turn
#pragma unroll 1
    for (int x = x0; x < x0 + 2 && x < xend; ++x) {
        if (sweep_active(colour, x, y, z)) update(x, 0);
        else copy(x);
    }
}

// ---- shared-memory tiled FP32 interior smoother --------------------------------------
// A block owns a 32 x TY tile of interior (x, y) nodes and marches through a chunk of
// interior z planes.  Moduli planes with a one-node x/y halo rotate through three shared
// buffers and displacement planes through four; plane z+2 streams in (cp.async) while
// plane z is computed, and the moduli of plane z-1 that the z-derivative needs are
// copied to registers before their buffer is refilled.  Each warp covers 16 x-pairs of
// two neighbouring rows: their active nodes have opposite x parity, so with an even row
// stride every shared load of the warp falls on 32 distinct banks.  The arithmetic is
// the same inlined stencil as the untiled kernel (same operations, same order).
constexpr int kTileX = 32;             // interior nodes per tile row
constexpr int kTileS = kTileX + 2;     // shared row stride (with halo), even

__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <int KIND, int TY>
struct TiledShape {
    static constexpr int KP = (KIND == 2) ? 2 : 21;
    static constexpr int R = TY + 2;                   // rows with halo
    static constexpr int PLANE = R * kTileS;           // one component of one plane
    static constexpr int CPL = KP * PLANE;             // floats per moduli plane
    static constexpr int UPL = 3 * PLANE;              // floats per displacement plane
    static constexpr int NPOS = (PLANE + 16 * TY - 1) / (16 * TY);   // positions per thread
    static constexpr size_t SMEM = sizeof(float) * (3 * CPL + 4 * UPL);
};

template <int KIND, int TY>
__global__ void __launch_bounds__(16 * TY, (TY <= 8) ? 2 : 1)
    k_half_sweep_tiled(Lv<float> L, const float* __restrict__ u, float* __restrict__ uo,
                       const float* __restrict__ f, int colour, NullInfo nf, const double* __restrict__ lam,
                       int zlen) {
    using S = TiledShape<KIND, TY>;
    constexpr int KP = S::KP, PLANE = S::PLANE, CPL = S::CPL, UPL = S::UPL, NPOS = S::NPOS;
    constexpr int NT = 16 * TY;
    extern __shared__ __align__(16) float sm[];
    float* const Cs = sm;                  // [3][KP][R][kTileS]
    float* const Us = sm + 3 * CPL;        // [4][3][R][kTileS]
    if (L.active && *L.active == 0) return;
    int lo[3], cnt[3];
    interior_box(L, lo, cnt);
    const int nx = L.n[0], ny = L.n[1], nz = L.n[2], N = L.N;
    const int xt0 = lo[0] + kTileX * blockIdx.x;
    const int yt0 = lo[1] + TY * blockIdx.y;
    const int z0 = lo[2] + zlen * blockIdx.z;
    const int zend = min(z0 + zlen, lo[2] + cnt[2]);
    if (z0 >= zend) return;
    const int xend = lo[0] + cnt[0], yend = lo[1] + cnt[1];

    // plane positions (row, column) this thread copies: in-plane global offset or -1
    int goff[NPOS];
#pragma unroll
    for (int j = 0; j < NPOS; ++j) {
        const int pos = threadIdx.x + NT * j;
        goff[j] = -1;
        if (pos < PLANE) {
            int x = xt0 - 1 + pos % kTileS, y = yt0 - 1 + pos / kTileS;
            if (x <= xend && y <= yend) {
                if (x < 0) x += nx;
                if (x >= nx) x -= nx;
                if (y < 0) y += ny;
                if (y >= ny) y -= ny;
                goff[j] = x + nx * y;
            }
        }
    }
    auto plane_base = [&](int z) -> int {
        if (z < 0) z += nz;
        if (z >= nz) z -= nz;
        return z * nx * ny;
    };
    // enqueue moduli and displacement of plane z into ring slot j (moduli: j % 3, u: j % 4)
    auto load_plane = [&](int z, int j) {
        const int zb = plane_base(z);
        float* cd = Cs + (j % 3) * CPL;
        float* ud = Us + (j & 3) * UPL;
#pragma unroll
        for (int q = 0; q < NPOS; ++q) {
            const int pos = threadIdx.x + NT * q;
            if (goff[q] < 0) continue;
            const int qn = zb + goff[q];
            const float* cs = L.mod + (size_t)(qn >> 5) * (32 * KP) + (qn & 31);   // blocked copy
#pragma unroll 7
            for (int c = 0; c < KP; ++c) cp_async4(cd + c * PLANE + pos, cs + 32 * c);
#pragma unroll
            for (int k = 0; k < 3; ++k) cp_async4(ud + k * PLANE + pos, u + (size_t)k * N + zb + goff[q]);
        }
        cp_async_commit();
    };

    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int y = yt0 + ty;
    const int x0 = xt0 + 2 * tx;
    const int yl = ty + 1;

    // prologue: planes z0-1, z0, z0+1 in slots 0, 1, 2
    load_plane(z0 - 1, 0);
    load_plane(z0, 1);
    load_plane(z0 + 1, 2);

    for (int z = z0; z < zend; ++z) {
        const int j = z - z0 + 1;          // ring index of the current plane
        const int xa = x0 + ((x0 + y + z + colour) & 1);
        const int xi = (xa == x0) ? x0 + 1 : x0;
        const int xla = xa - xt0 + 1, xli = xi - xt0 + 1;
        cp_async_wait_all();
        __syncthreads();
        // moduli of plane z-1 at the active node, before its slot is refilled
        float cprev[KP];
        {
            const float* cb = Cs + ((j + 2) % 3) * CPL + yl * kTileS + xla;
#pragma unroll
            for (int c = 0; c < KP; ++c) cprev[c] = cb[c * PLANE];
        }
        __syncthreads();
        if (z + 2 <= zend) load_plane(z + 2, j + 2);

        const float* const Cz = Cs + (j % 3) * CPL + yl * kTileS;
        const float* const Cn = Cs + ((j + 1) % 3) * CPL + yl * kTileS + xla;
        const float* const Um = Us + ((j + 3) & 3) * UPL + yl * kTileS + xla;
        const float* const U0 = Us + (j & 3) * UPL + yl * kTileS;
        const float* const Up = Us + ((j + 1) & 3) * UPL + yl * kTileS + xla;
        const int row = nx * (y + ny * z);
        if (y < yend && xi < xend) {
            const int q = xi + row;
#pragma unroll
            for (int k = 0; k < 3; ++k) uo[(size_t)k * N + q] = U0[k * PLANE + xli];
        }
        if (y < yend && xa < xend) {
            auto ua = [&](int k, int dx, int dy, int dz) -> float {
                const float* b = dz < 0 ? Um : (dz > 0 ? Up : U0 + xla);
                return b[k * PLANE + dy * kTileS + dx];
            };
            auto ca = [&](int c, int dx, int dy, int dz) -> float {
                if (dz < 0) return cprev[c];
                if (dz > 0) return Cn[c * PLANE];
                return Cz[c * PLANE + dy * kTileS + xla + dx];
            };
            const int p = xa + row;
            float v[3];
            interior_rows_core<float, KIND, false>(L, ua, ca, p, v);
            float r[3], B[3][3], d[3];
            const int c3[3] = {xa, y, z};
            for (int i = 0; i < 3; ++i) {
                float fi = f[(size_t)i * N + p];
                if (lam) fi = xsub(fi, rigid_load<float>(nf, lam, i, c3));
                r[i] = xsub(fi, v[i]);
            }
            interior_block_acc<float, KIND>(L, ca, B);
            solve3(B, r, d);
            for (int i = 0; i < 3; ++i) uo[(size_t)i * N + p] = xadd(ua(i, 0, 0, 0), d[i]);
        }
    }
    cp_async_wait_all();
}

// Red-black smoother, edge and corner nodes: one warp per node; lanes 0-8 compute
// the diagonal block entries, lanes 9-11 the rows, lane 0 solves and writes.
template <typename T, int KIND>
__device__ __forceinline__ void sweep_bnd_body(const Lv<T>& L, const T* __restrict__ u, T* __restrict__ uo,
                                               const T* __restrict__ f, int colour, const NullInfo& nf,
                                               const double* __restrict__ lam, int w, int lane) {
    if (w >= L.nbnd) return;   // whole warp
    const int p = L.bnodes[w];
    const int N = L.N;
    int c[3];
    coords_of(p, L.n, c);
    if (!sweep_active(colour, c[0], c[1], c[2])) {
        if (lane < 3) uo[lane * N + p] = u[lane * N + p];
        return;
    }
    const NodeInfo ni = node_info(L, c[0], c[1], c[2]);
    int types[3];
    for (int i = 0; i < 3; ++i) types[i] = row_type(L, ni, i);
    // stored rows (L.bcoef, set up with the moduli); the diagonal block is the node's own slot
    T B[3][3], v[3];
    const T* cf = L.bcoef + (size_t)w * kEdgeCoef;
    edge_rows_coef<T>(L, u, ni, cf, lane, v);
    if (lane != 0) return;
    const int cs = edge_center_slot(ni);
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) B[i][k] = cf[81 * i + 3 * cs + k];
    T r[3], d[3];
    for (int i = 0; i < 3; ++i) {
        if (types[i] == ROW_DIRICHLET) {
            r[i] = T(0);
        } else {
            T fi = f[i * N + p];
            if (lam) fi -= rigid_load<T>(nf, lam, i, c);
            r[i] = fi - v[i];
        }
    }
    solve3(B, r, d);
    if (colour == kJacobiColour)
        for (int i = 0; i < 3; ++i) d[i] *= L.omega;
    for (int i = 0; i < 3; ++i) uo[i * N + p] = u[i * N + p] + (types[i] == ROW_DIRICHLET ? T(0) : d[i]);
}

template <typename T, int KIND>
__global__ void __launch_bounds__(kBlock) k_half_sweep_bnd(Lv<T> L, const T* __restrict__ u, T* __restrict__ uo,
                                                          const T* __restrict__ f, int colour, NullInfo nf,
                                                          const double* __restrict__ lam) {
    if (L.active && *L.active == 0) return;
    sweep_bnd_body<T, KIND>(L, u, uo, f, colour, nf, lam, (blockIdx.x * blockDim.x + threadIdx.x) >> 5,
                            threadIdx.x & 31);
}

// ---------------------------------------------------------------------------
// face nodes: nodes on exactly one boundary plane, enumerated per direction A
// (both sides): thread -> (side, slow tangential, fast tangential)
// ---------------------------------------------------------------------------
template <typename T, int A>
__host__ __device__ inline void face_extent(const Lv<T>& L, int& n_fast, int& n_slow) {
    constexpr int ta = A == 0 ? 1 : 0;
    constexpr int tb = A == 2 ? 1 : 2;
    n_fast = L.per[ta] ? L.n[ta] : L.n[ta] - 2;
    n_slow = L.per[tb] ? L.n[tb] : L.n[tb] - 2;
}

template <typename T, int A>
__device__ __forceinline__ bool face_coords(const Lv<T>& L, int t, int c[3], int& side) {
    constexpr int ta = A == 0 ? 1 : 0;
    constexpr int tb = A == 2 ? 1 : 2;
    int nf, ns;
    face_extent<T, A>(L, nf, ns);
    if (t >= 2 * nf * ns) return false;
    const int i_fast = t % nf;
    const int rest = t / nf;
    const int i_slow = rest % ns;
    const int sd = rest / ns;
    c[ta] = (L.per[ta] ? 0 : 1) + i_fast;
    c[tb] = (L.per[tb] ? 0 : 1) + i_slow;
    c[A] = sd == 0 ? 0 : L.n[A] - 1;
    side = sd == 0 ? -1 : 1;
    return true;
}

template <typename T, int A>
__device__ __forceinline__ void face_types(const Lv<T>& L, int side, int types[3]) {
    const int f = 2 * A + (side > 0 ? 1 : 0);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int t = L.bc[f][i];
        types[i] = t == ROW_DIRICHLET ? ROW_DIRICHLET : (t == ROW_NEUMANN ? ROW_NEUMANN : ROW_TRACTION);
    }
}

template <typename T, int KIND, int A>
__global__ void __launch_bounds__(kBlock) k_apply_face(Lv<T> L, const T* __restrict__ u, T* __restrict__ out) {
    int c[3], side;
    if (!face_coords<T, A>(L, blockIdx.x * blockDim.x + threadIdx.x, c, side)) return;
    int types[3];
    face_types<T, A>(L, side, types);
    T v[3], B[3][3];
    face_node<T, KIND, A>(L, u, c, side, types, v, B, false);
    const int p = lin(L, c[0], c[1], c[2]);
    for (int i = 0; i < 3; ++i) out[i * L.N + p] = v[i];
}

template <typename T, typename TR, int KIND, int A, bool NORM>
__device__ __forceinline__ void residual_face_body(const Lv<T>& L, const T* __restrict__ u, const T* __restrict__ f,
                                                   const NullInfo& nf, const double* __restrict__ load,
                                                   TR* __restrict__ r, int t, double acc[8]) {
    int c[3], side;
    if (!face_coords<T, A>(L, t, c, side)) return;
    int types[3];
    face_types<T, A>(L, side, types);
    T v[3], B[3][3];
    face_node<T, KIND, A>(L, u, c, side, types, v, B, false);
    residual_store<T, TR, NORM>(L, f, nf, load, c, lin(L, c[0], c[1], c[2]), types, v, r, acc);
}

template <typename T, int KIND, int A>
__device__ __forceinline__ void sweep_face_body(const Lv<T>& L, const T* __restrict__ u, T* __restrict__ uo,
                                                const T* __restrict__ f, int colour, const NullInfo& nf,
                                                const double* __restrict__ load, int t) {
    int c[3], side;
    if (!face_coords<T, A>(L, t, c, side)) return;
    const int N = L.N;
    const int p = lin(L, c[0], c[1], c[2]);
    if (!sweep_active(colour, c[0], c[1], c[2])) {
        uo[p] = u[p];
        uo[N + p] = u[N + p];
        uo[2 * N + p] = u[2 * N + p];
        return;
    }
    int types[3];
    face_types<T, A>(L, side, types);
    T v[3], B[3][3], r[3], d[3];
    face_node<T, KIND, A>(L, u, c, side, types, v, B, true);
    for (int i = 0; i < 3; ++i) {
        if (types[i] == ROW_DIRICHLET) {
            r[i] = T(0);
        } else {
            T fi = f[i * N + p];
            if (load) fi -= rigid_load<T>(nf, load, i, c);
            r[i] = fi - v[i];
        }
    }
    solve3(B, r, d);
    if (colour == kJacobiColour)
        for (int i = 0; i < 3; ++i) d[i] *= L.omega;
    for (int i = 0; i < 3; ++i) uo[i * N + p] = u[i * N + p] + (types[i] == ROW_DIRICHLET ? T(0) : d[i]);
}

template <typename T, int KIND, int A>
__global__ void __launch_bounds__(kBlock) k_half_sweep_face(Lv<T> L, const T* __restrict__ u, T* __restrict__ uo,
                                                           const T* __restrict__ f, int colour, NullInfo nf,
                                                           const double* __restrict__ load) {
    if (L.active && *L.active == 0) return;
    sweep_face_body<T, KIND, A>(L, u, uo, f, colour, nf, load, blockIdx.x * blockDim.x + threadIdx.x);
}

template <typename T, int A>
__host__ __device__ inline size_t face_count(const Lv<T>& L) {
    if (L.per[A]) return 0;
    if ((L.xface_list >> A) & 1) return 0;   // these faces go with the stored-coefficient rows
    int nf, ns;
    face_extent<T, A>(L, nf, ns);
    return (size_t)2 * nf * ns;
}

// Coefficients of the edge and corner rows: entry e = (w, i, slot, k) is row i of node
// bnodes[w] applied to the unit vector of component k at the slot's node, i.e. the
// operator's matrix entry (the generic rows are linear in u).  Setup only.
template <typename T, int KIND>
__global__ void k_edge_coef(Lv<T> L, T* __restrict__ out) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)L.nbnd * kEdgeCoef) return;
    const int w = (int)(e / kEdgeCoef), rem = (int)(e % kEdgeCoef);
    const int i = rem / 81, slot = (rem % 81) / 3, k = rem % 3;
    int c[3];
    coords_of(L.bnodes[w], L.n, c);
    const NodeInfo ni = node_info(L, c[0], c[1], c[2]);
    UProbe<T> probe;
    probe.kk = k;
    edge_slot_node(L, ni, slot, probe.c0);
    out[e] = boundary_row<T, KIND>(L, probe, ni, i, row_type(L, ni, i));
}

// ---- one launch per half-sweep / residual ---------------------------------------------
// The grid's first blocks take the edge and corner nodes (a warp each), then the face
// nodes of directions 0, 1, 2 (a thread each), then the interior.  The boundary blocks
// are few and latency-bound; issued first, they run alongside the interior blocks
// instead of as four short launches of their own.  Block ranges are uniform per block.
struct BndSegs {
    int e, f0, f1, f2;   // one past the last block of the edge, x-, y- and z-face ranges
};

template <typename T>
__host__ __device__ inline BndSegs bnd_segs(const Lv<T>& L, int bs) {
    BndSegs g;
    g.e = (int)(((size_t)L.nbnd * 32 + bs - 1) / bs);
    g.f0 = g.e + (int)((face_count<T, 0>(L) + bs - 1) / bs);
    g.f1 = g.f0 + (int)((face_count<T, 1>(L) + bs - 1) / bs);
    g.f2 = g.f1 + (int)((face_count<T, 2>(L) + bs - 1) / bs);
    return g;
}

// Red-black smoother, all nodes of one colour (see the bodies above for each kind).
template <typename T, int KIND, bool HM, int ML, int BS, int MINB>
__global__ void __launch_bounds__(BS, MINB) k_half_sweep_int(Lv<T> L, const T* __restrict__ u, T* __restrict__ uo,
                                                          const T* __restrict__ f, int colour, NullInfo nf,
                                                          const double* __restrict__ lam, BndSegs sg) {
    if (L.active && *L.active == 0) return;
    const int b = blockIdx.x, tid = threadIdx.x;
    if (b < sg.f2) {
        if (b < sg.e) sweep_bnd_body<T, KIND>(L, u, uo, f, colour, nf, lam, (b * BS + tid) >> 5, tid & 31);
        else if (b < sg.f0) sweep_face_body<T, KIND, 0>(L, u, uo, f, colour, nf, lam, (b - sg.e) * BS + tid);
        else if (b < sg.f1) sweep_face_body<T, KIND, 1>(L, u, uo, f, colour, nf, lam, (b - sg.f0) * BS + tid);
        else sweep_face_body<T, KIND, 2>(L, u, uo, f, colour, nf, lam, (b - sg.f1) * BS + tid);
        return;
    }
    sweep_pair_body<T, KIND, HM, ML>(L, u, uo, f, colour, nf, lam, (b - sg.f2) * BS + tid);
}

// ---- z-marching tiled half-sweep of colour-split FP32 levels ---------------------------
// A block owns a 32 x TY tile of interior (x, y) nodes and a chunk of interior z planes.
// Every global read is an asynchronous copy issued one plane ahead (cp.async): the
// displacement planes, with a one-node x/y halo, rotate through four shared buffers
// (plane z+2 streams in while plane z is computed), and the active nodes' colour-split
// records (21 moduli + 18 divergence entries) and right-hand sides of plane z+1 fill the
// other half of a double buffer.  So each value comes from DRAM once per half-sweep and
// the stencil reads only shared memory, the 57 displacement reads at compile-time
// offsets.  Each warp covers 16 x-pairs of two neighbouring rows (active nodes of
// opposite x parity: conflict-free shared loads).  The first blocks of the launch take
// the edge, corner and face nodes, as in k_half_sweep_int.  Same stencil, same order of
// operations as the untiled kernel: identical bits.
template <int TY>
struct SplitTile {
    static constexpr int R = TY + 2;                   // rows with halo
    static constexpr int PLANE = R * kTileS;           // one component of one plane
    static constexpr int UPL = 3 * PLANE;              // floats per displacement plane
    static constexpr int NT = 16 * TY;
    static constexpr int NPOS = (PLANE + NT - 1) / NT; // positions per thread
    static constexpr int REC = kSplitK * NT;           // floats of one plane's records
    static constexpr int FRH = 3 * NT;                 // floats of one plane's right-hand sides
    static constexpr size_t SMEM = sizeof(float) * (4 * UPL + 2 * REC + 2 * FRH);
};

template <int TY, int MINB>
__global__ void __launch_bounds__(16 * TY, MINB)
    k_half_sweep_tiled_split(Lv<float> L, const float* __restrict__ u, float* __restrict__ uo,
                             const float* __restrict__ f, int colour, NullInfo nf, const double* __restrict__ lam,
                             BndSegs sg, int gx, int gy, int zlen) {
    using S = SplitTile<TY>;
    constexpr int PLANE = S::PLANE, UPL = S::UPL, NPOS = S::NPOS, NT = S::NT, REC = S::REC, FRH = S::FRH;
    extern __shared__ __align__(16) float sm[];
    float* const Us = sm;                          // [4][3][R][kTileS]
    float* const Rs = sm + 4 * UPL;                // [2][kSplitK][NT]
    float* const Fs = Rs + 2 * REC;                // [2][3][NT]
    if (L.active && *L.active == 0) return;
    const int b = blockIdx.x, tid = threadIdx.x;
    if (b < sg.f2) {
        if (b < sg.e) sweep_bnd_body<float, 21>(L, u, uo, f, colour, nf, lam, (b * NT + tid) >> 5, tid & 31);
        else if (b < sg.f0) sweep_face_body<float, 21, 0>(L, u, uo, f, colour, nf, lam, (b - sg.e) * NT + tid);
        else if (b < sg.f1) sweep_face_body<float, 21, 1>(L, u, uo, f, colour, nf, lam, (b - sg.f0) * NT + tid);
        else sweep_face_body<float, 21, 2>(L, u, uo, f, colour, nf, lam, (b - sg.f1) * NT + tid);
        return;
    }
    const int t = b - sg.f2;
    const int bx = t % gx, by = (t / gx) % gy, bz = t / (gx * gy);
    int lo[3], cnt[3];
    interior_box(L, lo, cnt);
    const int nx = L.n[0], ny = L.n[1], nz = L.n[2], N = L.N;
    const int xt0 = lo[0] + kTileX * bx;
    const int yt0 = lo[1] + TY * by;
    const int z0 = lo[2] + zlen * bz;
    const int zend = min(z0 + zlen, lo[2] + cnt[2]);
    if (z0 >= zend) return;
    const int xend = lo[0] + cnt[0], yend = lo[1] + cnt[1];

    // in-plane global offset of each shared position this thread copies, or -1
    int goff[NPOS];
#pragma unroll
    for (int j = 0; j < NPOS; ++j) {
        const int pos = tid + NT * j;
        goff[j] = -1;
        if (pos < PLANE) {
            int x = xt0 - 1 + pos % kTileS, y = yt0 - 1 + pos / kTileS;
            if (x <= xend && y <= yend) {
                if (x < 0) x += nx;
                if (x >= nx) x -= nx;
                if (y < 0) y += ny;
                if (y >= ny) y -= ny;
                goff[j] = x + nx * y;
            }
        }
    }
    const int tx = tid & 15, ty = tid >> 4;
    const int y = yt0 + ty;
    const int x0 = xt0 + 2 * tx;
    const int yl = ty + 1;
    auto active_x = [&](int z) { return x0 + ((x0 + y + z + colour) & 1); };
    // displacement plane z into ring slot j & 3
    auto load_u = [&](int z, int j) {
        if (z < 0) z += nz;
        if (z >= nz) z -= nz;
        const int zb = z * nx * ny;
        float* ud = Us + (j & 3) * UPL;
#pragma unroll
        for (int q = 0; q < NPOS; ++q) {
            if (goff[q] < 0) continue;
            const int pos = tid + NT * q;
#pragma unroll
            for (int k = 0; k < 3; ++k) cp_async4(ud + k * PLANE + pos, u + (size_t)k * N + zb + goff[q]);
        }
    };
    // this thread's active node of plane z: its record and right-hand side into buffer z & 1
    auto load_node = [&](int z) {
        const int xa = active_x(z);
        if (y >= yend || xa >= xend) return;
        const int p = xa + nx * (y + ny * z);
        const float* cb = L.mod + (p & 1) * L.msplit1 + (size_t)((p >> 1) >> 5) * (32 * kSplitK) + ((p >> 1) & 31);
        float* rd = Rs + (z & 1) * REC + tid;
#pragma unroll
        for (int c = 0; c < kSplitK; ++c) cp_async4(rd + c * NT, cb + 32 * c);
        float* fd = Fs + (z & 1) * FRH + tid;
#pragma unroll
        for (int k = 0; k < 3; ++k) cp_async4(fd + k * NT, f + (size_t)k * N + p);
    };
    load_u(z0 - 1, 0);
    load_u(z0, 1);
    load_u(z0 + 1, 2);
    load_node(z0);
    cp_async_commit();
    for (int z = z0; z < zend; ++z) {
        const int j = z - z0 + 1;          // ring slot of plane z
        cp_async_wait_all();
        __syncthreads();
        // one plane ahead: displacement plane z+2 (into the slot of plane z-2) and the
        // records of plane z+1 (into the buffer of plane z-1)
        if (z + 2 <= zend) load_u(z + 2, j + 2);
        if (z + 1 < zend) load_node(z + 1);
        cp_async_commit();
        const int xa = active_x(z);
        const int xi = (xa == x0) ? x0 + 1 : x0;
        const int xla = xa - xt0 + 1, xli = xi - xt0 + 1;
        const float* const Um = Us + ((j + 3) & 3) * UPL + yl * kTileS + xla;
        const float* const U0 = Us + (j & 3) * UPL + yl * kTileS;
        const float* const Up = Us + ((j + 1) & 3) * UPL + yl * kTileS + xla;
        const int row = nx * (y + ny * z);
        if (y < yend && xi < xend && xa >= xend) {
            const int q = xi + row;
#pragma unroll
            for (int k = 0; k < 3; ++k) uo[(size_t)k * N + q] = U0[k * PLANE + xli];
        }
        if (y < yend && xa < xend) {
            const int p = xa + row;
            const bool cp = xi < xend;
            const float* rb = Rs + (z & 1) * REC + tid;
            const float* fb = Fs + (z & 1) * FRH + tid;
            auto ua = [&](int k, int dx, int dy, int dz) -> float {
                const float* bp = dz < 0 ? Um : (dz > 0 ? Up : U0 + xla);
                return bp[k * PLANE + dy * kTileS + dx];
            };
            auto ca = [&](int c, int, int, int) -> float { return rb[c * NT]; };
            float v[3];
            interior_rows_core<float, 21, true>(L, ua, ca, p, v);
            float r[3], B[3][3], d[3];
            const int c3[3] = {xa, y, z};
            for (int i = 0; i < 3; ++i) {
                float fi = fb[i * NT];
                if (lam) fi = xsub(fi, rigid_load<float>(nf, lam, i, c3));
                r[i] = xsub(fi, v[i]);
            }
            interior_block_acc<float, 21>(L, ca, B);
            solve3(B, r, d);
            for (int i = 0; i < 3; ++i) {
                if (cp) uo[(size_t)i * N + xi + row] = U0[i * PLANE + xli];
                uo[(size_t)i * N + p] = xadd(ua(i, 0, 0, 0), d[i]);
            }
        }
    }
    cp_async_wait_all();
}

// ---- refinement residual in double-float arithmetic --------------------------------------
// r = f - load - A u of an FP64 level evaluated on the FP32 pipes: u, f, the moduli with
// their divergence and the stored rows are double-float planes split from the FP64 ones,
// every term of the operator is a double-float operation (the same stencil code as the
// FP64 kernel, instantiated for dfloat), and r is written as FP32 for the correction
// cycle.  Per block: sum r^2 in FP32 (the stopping test needs a few digits of the norm)
// and the six rigid moments in double-float (they cancel), stored as FP64 partials in
// the layout of k_residual.  Interior threads take NPT nodes each, which spreads the
// block reduction over NPT times more nodes.
struct DfAcc {
    float r2, rmax;
    dfloat m[6];
};

template <bool NORM>
__device__ __forceinline__ void residual_store_df(const Lv<dfloat>& L, const dfloat* __restrict__ f,
                                                  const NullInfo& nf, const double* __restrict__ load,
                                                  const int c[3], int p, const int types[3], const dfloat v[3],
                                                  float* __restrict__ r, DfAcc& acc) {
    dfloat rr[3];
    float rf[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        dfloat ri(0.f, 0.f);
        if (types[i] != ROW_DIRICHLET) {
            dfloat fi = f[(size_t)i * L.N + p];
            if (load) fi = df_sub(fi, dfloat(rigid_load<float>(nf, load, i, c)));
            ri = df_sub(fi, v[i]);
        }
        rr[i] = ri;
        rf[i] = df_to_float(ri);
        r[(size_t)i * L.N + p] = rf[i];
    }
    if (NORM) {
        acc.r2 = __fmaf_rn(rf[2], rf[2], __fmaf_rn(rf[1], rf[1], __fmaf_rn(rf[0], rf[0], acc.r2)));
        acc.rmax = fmaxf(acc.rmax, fmaxf(fabsf(rf[0]), fmaxf(fabsf(rf[1]), fabsf(rf[2]))));
        if (nf.m > 0) {
            const float d0 = xfma(nf.h32[0], float(c[0]), nf.off32[0]);
            const float d1 = xfma(nf.h32[1], float(c[1]), nf.off32[1]);
            const float d2 = xfma(nf.h32[2], float(c[2]), nf.off32[2]);
            acc.m[0] = df_add(acc.m[0], rr[0]);
            acc.m[1] = df_add(acc.m[1], rr[1]);
            acc.m[2] = df_add(acc.m[2], rr[2]);
            acc.m[3] = df_add(acc.m[3], df_sub(df_mul(rr[2], d1), df_mul(rr[1], d2)));
            acc.m[4] = df_add(acc.m[4], df_sub(df_mul(rr[0], d2), df_mul(rr[2], d0)));
            acc.m[5] = df_add(acc.m[5], df_sub(df_mul(rr[1], d0), df_mul(rr[0], d1)));
        }
    }
}

// Block sum of the accumulators into partials[bid * kPartialStride + 0 .. width), and the
// block's max |r| into [+ 7]
__device__ __forceinline__ void block_reduce_store_df(const DfAcc& a, int width, double* partials, int bid) {
    __shared__ float sr[kBlock / 32], sx[kBlock / 32];
    __shared__ dfloat sm[kBlock / 32][6];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float x = a.r2, mx = a.rmax;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x = __fadd_rn(x, shfl_xor_all(x, o));
        mx = fmaxf(mx, shfl_xor_all(mx, o));
    }
    if (lane == 0) {
        sr[warp] = x;
        sx[warp] = mx;
    }
    if (width > 1) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            dfloat y = a.m[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) y = df_add(y, shfl_xor_all(y, o));
            if (lane == 0) sm[warp][k] = y;
        }
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        x = lane < kBlock / 32 ? sr[lane] : 0.f;
        mx = lane < kBlock / 32 ? sx[lane] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            x = __fadd_rn(x, shfl_xor_all(x, o));
            mx = fmaxf(mx, shfl_xor_all(mx, o));
        }
        if (lane == 0) {
            partials[(size_t)bid * kPartialStride] = (double)x;
            partials[(size_t)bid * kPartialStride + 7] = (double)mx;
        }
        if (width > 1) {
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                dfloat y = lane < kBlock / 32 ? sm[lane][k] : dfloat(0.f, 0.f);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) y = df_add(y, shfl_xor_all(y, o));
                if (lane == 0) partials[(size_t)bid * kPartialStride + 1 + k] = (double)y.hi + (double)y.lo;
            }
        }
    }
}

template <int KIND, bool NORM>
__device__ __forceinline__ void residual_bnd_body_df(const Lv<dfloat>& L, const dfloat* __restrict__ u,
                                                     const dfloat* __restrict__ f, const NullInfo& nf,
                                                     const double* __restrict__ lam, float* __restrict__ r, int w,
                                                     int lane, DfAcc& acc) {
    if (w >= L.nbnd) return;   // whole warp
    const int p = L.bnodes[w];
    int c[3];
    coords_of(p, L.n, c);
    const NodeInfo ni = node_info(L, c[0], c[1], c[2]);
    int types[3];
    for (int i = 0; i < 3; ++i) types[i] = row_type(L, ni, i);
    dfloat v[3];
    edge_rows_coef<dfloat>(L, u, ni, L.bcoef + (size_t)w * kEdgeCoef, lane, v);
    if (lane == 0) residual_store_df<NORM>(L, f, nf, lam, c, p, types, v, r, acc);
}

template <int KIND, int A, bool NORM>
__device__ __forceinline__ void residual_face_body_df(const Lv<dfloat>& L, const dfloat* __restrict__ u,
                                                      const dfloat* __restrict__ f, const NullInfo& nf,
                                                      const double* __restrict__ load, float* __restrict__ r, int t,
                                                      DfAcc& acc) {
    int c[3], side;
    if (!face_coords<dfloat, A>(L, t, c, side)) return;
    int types[3];
    face_types<dfloat, A>(L, side, types);
    dfloat v[3], B[3][3];
    face_node<dfloat, KIND, A>(L, u, c, side, types, v, B, false);
    residual_store_df<NORM>(L, f, nf, load, c, lin(L, c[0], c[1], c[2]), types, v, r, acc);
}

template <int KIND, bool NORM, bool HM, int NPT>
__device__ __forceinline__ void residual_int_body_df(const Lv<dfloat>& L, const dfloat* __restrict__ u,
                                                     const dfloat* __restrict__ f, const NullInfo& nf,
                                                     const double* __restrict__ lam, float* __restrict__ r, int b,
                                                     DfAcc& acc) {
    int lo[3], cnt[3];
    interior_box(L, lo, cnt);
    const int total = cnt[0] * cnt[1] * cnt[2];
#pragma unroll 1
    for (int k = 0; k < NPT; ++k) {
        const int t = (b * NPT + k) * kBlock + (int)threadIdx.x;
        if (t >= total) break;
        const int c[3] = {lo[0] + t % cnt[0], lo[1] + (t / cnt[0]) % cnt[1], lo[2] + t / (cnt[0] * cnt[1])};
        dfloat v[3];
        with_interior<dfloat, KIND, kMlDefault>(L, u, c[0], c[1], c[2], [&](const auto& ua, const auto& ca, int p) {
            interior_rows_core<dfloat, KIND, HM>(L, ua, ca, p, v);
        });
        const int types[3] = {ROW_INTERIOR, ROW_INTERIOR, ROW_INTERIOR};
        residual_store_df<NORM>(L, f, nf, lam, c, lin(L, c[0], c[1], c[2]), types, v, r, acc);
    }
}

// Blocks of one launch: edge/corner/x-face warps, y- and z-face threads, interior
// threads of NPT nodes each.
template <int NPT>
__host__ __device__ inline int residual_df_blocks(const Lv<dfloat>& L) {
    const BndSegs sg = bnd_segs(L, kBlock);
    return sg.f2 + (int)((interior_count(L) + (size_t)kBlock * NPT - 1) / ((size_t)kBlock * NPT));
}

template <int KIND, bool NORM, bool HM, int NPT>
__device__ __forceinline__ void residual_df_block(const Lv<dfloat>& L, const dfloat* __restrict__ u,
                                                  const dfloat* __restrict__ f, const NullInfo& nf,
                                                  const double* __restrict__ lam, float* __restrict__ r,
                                                  double* __restrict__ partials, int b) {
    DfAcc acc;
    acc.r2 = 0.f;
    acc.rmax = 0.f;
#pragma unroll
    for (int k = 0; k < 6; ++k) acc.m[k] = dfloat(0.f, 0.f);
    const BndSegs sg = bnd_segs(L, kBlock);
    const int tid = threadIdx.x;
    if (b < sg.e) residual_bnd_body_df<KIND, NORM>(L, u, f, nf, lam, r, (b * kBlock + tid) >> 5, tid & 31, acc);
    else if (b < sg.f0) residual_face_body_df<KIND, 0, NORM>(L, u, f, nf, lam, r, (b - sg.e) * kBlock + tid, acc);
    else if (b < sg.f1) residual_face_body_df<KIND, 1, NORM>(L, u, f, nf, lam, r, (b - sg.f0) * kBlock + tid, acc);
    else if (b < sg.f2) residual_face_body_df<KIND, 2, NORM>(L, u, f, nf, lam, r, (b - sg.f1) * kBlock + tid, acc);
    else residual_int_body_df<KIND, NORM, HM, NPT>(L, u, f, nf, lam, r, b - sg.f2, acc);
    if (NORM) block_reduce_store_df(acc, nf.m > 0 ? 7 : 1, partials, b);
}

template <int KIND, bool NORM, bool HM, int NPT>
__global__ void __launch_bounds__(kBlock, 2) k_residual_df(Lv<dfloat> L, const dfloat* __restrict__ u,
                                                           const dfloat* __restrict__ f, NullInfo nf,
                                                           const double* __restrict__ lam, float* __restrict__ r,
                                                           double* __restrict__ partials) {
    if (L.active && *L.active == 0) return;
    residual_df_block<KIND, NORM, HM, NPT>(L, u, f, nf, lam, r, partials, blockIdx.x);
}

template <typename TE>
__device__ __forceinline__ void add_correction_df_body(const Lv<double>& L, double* __restrict__ u,
                                                       const TE* __restrict__ e, dfloat* __restrict__ u2, int p) {
    if (p >= L.N) return;
    int c[3];
    coords_of(p, L.n, c);
    const NodeInfo ni = node_info(L, c[0], c[1], c[2]);
    for (int i = 0; i < 3; ++i) {
        double x = u[i * L.N + p];
        if (row_type(L, ni, i) != ROW_DIRICHLET) {
            x += f2d_bits(e[i * L.N + p]);   // the FP64 update of the refinement, one DADD
            u[i * L.N + p] = x;
        }
        u2[i * L.N + p] = df_split(x);
    }
}

// r = f - load - A u on every node; block partials of sum r^2 and the rigid moments.
// Resident blocks per SM: two for FP64 (at most 128 registers; the FP64 instance is bound
// by the FP64 pipe and needs the warps to keep it busy, one block at 180 registers ran
// 15% slower), four for FP32 (64 registers with spills: 0.97 ms at one block, 0.79 at
// three, 0.74 at four for 257^3 with colour-split records; the same latency-for-registers
// trade as the smoother's shapes).
template <typename T, typename TR, int KIND, bool NORM, bool HM, int ML>
__global__ void __launch_bounds__(kBlock, sizeof(T) == 4 ? 4 : 2) k_residual(Lv<T> L, const T* __restrict__ u, const T* __restrict__ f,
                                                    NullInfo nf, const double* __restrict__ lam,
                                                    TR* __restrict__ r, double* __restrict__ partials, BndSegs sg) {
    if (L.active && *L.active == 0) return;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int b = blockIdx.x, tid = threadIdx.x;
    if (b < sg.e) residual_bnd_body<T, TR, KIND, NORM>(L, u, f, nf, lam, r, (b * kBlock + tid) >> 5, tid & 31, acc);
    else if (b < sg.f0) residual_face_body<T, TR, KIND, 0, NORM>(L, u, f, nf, lam, r, (b - sg.e) * kBlock + tid, acc);
    else if (b < sg.f1) residual_face_body<T, TR, KIND, 1, NORM>(L, u, f, nf, lam, r, (b - sg.f0) * kBlock + tid, acc);
    else if (b < sg.f2) residual_face_body<T, TR, KIND, 2, NORM>(L, u, f, nf, lam, r, (b - sg.f1) * kBlock + tid, acc);
    else residual_int_body<T, TR, KIND, NORM, HM, ML>(L, u, f, nf, lam, r, (b - sg.f2) * kBlock + tid, acc);
    if (NORM) block_reduce_norms_at(acc, nf.m > 0 ? 7 : 1, partials, blockIdx.x);
}

// ---------------------------------------------------------------------------
// transfers (Section 3.2)
// ---------------------------------------------------------------------------
// weights of fine offsets -1, 0, +1 for coarse index I in one direction
template <typename T>
__device__ __forceinline__ void restrict_weights(const Lv<T>& Lc, int d, int I, T w[3]) {
    if (!Lc.per[d] && I == 0) { w[0] = T(0); w[1] = T(0.5); w[2] = T(0.5); return; }
    if (!Lc.per[d] && I == Lc.n[d] - 1) { w[0] = T(0.5); w[1] = T(0.5); w[2] = T(0); return; }
    w[0] = T(0.25); w[1] = T(0.5); w[2] = T(0.25);
}

template <typename T>
__device__ __forceinline__ void restrict_body(const Lv<T>& Lf, const Lv<T>& Lc, const T* __restrict__ r,
                                              T* __restrict__ fc, const NullInfo& nf, const double* __restrict__ dlam,
                                              int P) {
    if (P >= Lc.N) return;
    int C[3];
    coords_of(P, Lc.n, C);
    const NodeInfo nic = node_info(Lc, C[0], C[1], C[2]);
    T wx[3], wy[3], wz[3];
    restrict_weights(Lc, 0, C[0], wx);
    restrict_weights(Lc, 1, C[1], wy);
    restrict_weights(Lc, 2, C[2], wz);
    T acc[3] = {T(0), T(0), T(0)};
    const bool corr = dlam != nullptr;
    for (int dz = -1; dz <= 1; ++dz) {
        if (wz[dz + 1] == T(0)) continue;
        const int fz = wrapc(Lf, 2, 2 * C[2] + dz);
        for (int dy = -1; dy <= 1; ++dy) {
            if (wy[dy + 1] == T(0)) continue;
            const int fy = wrapc(Lf, 1, 2 * C[1] + dy);
            for (int dx = -1; dx <= 1; ++dx) {
                if (wx[dx + 1] == T(0)) continue;
                const int fx = wrapc(Lf, 0, 2 * C[0] + dx);
                const T w = wx[dx + 1] * wy[dy + 1] * wz[dz + 1];
                const int q = lin(Lf, fx, fy, fz);
                const int cf[3] = {fx, fy, fz};
                NodeInfo nif;
                if (corr) nif = node_info(Lf, fx, fy, fz);
                for (int i = 0; i < 3; ++i) {
                    T v = r[i * Lf.N + q];
                    if (corr && row_type(Lf, nif, i) != ROW_DIRICHLET) v -= rigid_load<T>(nf, dlam, i, cf);
                    acc[i] += w * v;
                }
            }
        }
    }
    for (int i = 0; i < 3; ++i)
        fc[i * Lc.N + P] = (row_type(Lc, nic, i) == ROW_DIRICHLET) ? T(0) : acc[i];
}

template <typename T>
__global__ void k_restrict(Lv<T> Lf, Lv<T> Lc, const T* __restrict__ r, T* __restrict__ fc, NullInfo nf,
                           const double* __restrict__ dlam) {
    if (Lf.active && *Lf.active == 0) return;
    restrict_body<T>(Lf, Lc, r, fc, nf, dlam, blockIdx.x * blockDim.x + threadIdx.x);
}

template <typename T>
__device__ __forceinline__ void prolong_body(const Lv<T>& Lf, const Lv<T>& Lc, const T* __restrict__ ec,
                                             T* __restrict__ u, int p) {
    if (p >= Lf.N) return;
    int c[3];
    coords_of(p, Lf.n, c);
    const NodeInfo ni = node_info(Lf, c[0], c[1], c[2]);
    // per direction: the coarse nodes below and above (the same node at even fine
    // coordinates) and their weights 1 / 0 or 1/2 / 1/2; all eight corners are read and
    // the zero-weight terms add exact zeros, so every thread runs the same instructions
    int lo[3], hi[3];
    T wl[3], wh[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int odd = c[d] & 1;
        lo[d] = c[d] >> 1;
        hi[d] = lo[d] + odd;
        if (Lc.per[d] && hi[d] >= Lc.n[d]) hi[d] -= Lc.n[d];
        wl[d] = odd ? T(0.5) : T(1);
        wh[d] = odd ? T(0.5) : T(0);
    }
    const int nx = Lc.n[0], nxy = Lc.n[0] * Lc.n[1];
    const int cz[2] = {lo[2] * nxy, hi[2] * nxy}, cy[2] = {lo[1] * nx, hi[1] * nx}, cx[2] = {lo[0], hi[0]};
    const T wz[2] = {wl[2], wh[2]}, wy[2] = {wl[1], wh[1]}, wx[2] = {wl[0], wh[0]};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (row_type(Lf, ni, i) == ROW_DIRICHLET) continue;
        const T* e = ec + (size_t)i * Lc.N;
        T v = T(0);
#pragma unroll
        for (int bz = 0; bz < 2; ++bz)
#pragma unroll
            for (int by = 0; by < 2; ++by)
#pragma unroll
                for (int bx = 0; bx < 2; ++bx)   // weights are powers of two: exact products
                    v = xfma(xmul(xmul(wx[bx], wy[by]), wz[bz]), e[cz[bz] + cy[by] + cx[bx]], v);
        u[(size_t)i * Lf.N + p] = xadd(u[(size_t)i * Lf.N + p], v);
    }
}

template <typename T>
__global__ void k_prolong_add(Lv<T> Lf, Lv<T> Lc, const T* __restrict__ ec, T* __restrict__ u) {
    if (Lf.active && *Lf.active == 0) return;
    prolong_body<T>(Lf, Lc, ec, u, blockIdx.x * blockDim.x + threadIdx.x);
}

template <typename T>
__global__ void k_restrict_moduli(Lv<T> Lf, Lv<T> Lc, const T* __restrict__ mf, T* __restrict__ mc) {
    const int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= Lc.N) return;
    int C[3];
    coords_of(P, Lc.n, C);
    T wx[3], wy[3], wz[3];
    restrict_weights(Lc, 0, C[0], wx);
    restrict_weights(Lc, 1, C[1], wy);
    restrict_weights(Lc, 2, C[2], wz);
    for (int k = 0; k < Lf.K; ++k) {
        T acc = T(0);
        for (int dz = -1; dz <= 1; ++dz) {
            if (wz[dz + 1] == T(0)) continue;
            const int fz = wrapc(Lf, 2, 2 * C[2] + dz);
            for (int dy = -1; dy <= 1; ++dy) {
                if (wy[dy + 1] == T(0)) continue;
                const int fy = wrapc(Lf, 1, 2 * C[1] + dy);
                for (int dx = -1; dx <= 1; ++dx) {
                    if (wx[dx + 1] == T(0)) continue;
                    const int fx = wrapc(Lf, 0, 2 * C[0] + dx);
                    acc += wx[dx + 1] * wy[dy + 1] * wz[dz + 1] * mf[k * Lf.N + lin(Lf, fx, fy, fz)];
                }
            }
        }
        mc[k * Lc.N + P] = acc;
    }
}

// M_iV = sum_j (C_(ij)V(p+e_j) - C_(ij)V(p-e_j)) / 2h_j at interior nodes, 0 elsewhere.
template <typename T>
__global__ void k_divc(Lv<T> L, T* __restrict__ M) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= L.N) return;
    int c[3];
    coords_of(p, L.n, c);
    const NodeInfo ni = node_info(L, c[0], c[1], c[2]);
    for (int i = 0; i < 3; ++i)
        for (int V = 0; V < 6; ++V) {
            T acc = T(0);
            if (!ni.boundary) {
                for (int j = 0; j < 3; ++j) {
                    int cp[3] = {c[0], c[1], c[2]}, cm[3] = {c[0], c[1], c[2]};
                    cp[j] = wrapc(L, j, c[j] + 1);
                    cm[j] = wrapc(L, j, c[j] - 1);
                    const T* cc = L.mod + upper(voigt(i, j), V) * L.N;
                    acc += (cc[lin(L, cp[0], cp[1], cp[2])] - cc[lin(L, cm[0], cm[1], cm[2])]) * L.inv2h[j];
                }
            }
            M[(i * 6 + V) * L.N + p] = acc;
        }
}

// FP64 moduli planes -> the FP32 blocked copy (entry c of node q at blocked_index) or
// the FP16 node records (entry c of node q at q * rec + c, padding zero).
template <typename TO>
__global__ void k_to_moduli_copy(const double* __restrict__ in, TO* __restrict__ out, int N, int K) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if constexpr (sizeof(TO) == 2) {
        const int rec = mod_record(K);
        if (i >= (size_t)N * rec) return;
        const int q = (int)(i / rec), c = (int)(i % rec);
        out[i] = __double2half(c < K ? in[(size_t)c * N + q] : 0.0);
    } else {
        const size_t nb = (size_t)((N + 31) / 32) * 32 * K;
        if (i >= nb) return;
        const size_t blk = i / (32 * (size_t)K), r = i % (32 * (size_t)K);
        const int c = (int)(r / 32), q = (int)(blk * 32 + r % 32);
        out[i] = q < N ? (TO)in[(size_t)c * N + q] : TO(0);
    }
}

template <typename TE>
__device__ __forceinline__ void add_correction_body(const Lv<double>& L, double* __restrict__ u,
                                                    const TE* __restrict__ e, int p) {
    if (p >= L.N) return;
    int c[3];
    coords_of(p, L.n, c);
    const NodeInfo ni = node_info(L, c[0], c[1], c[2]);
    for (int i = 0; i < 3; ++i)
        if (row_type(L, ni, i) != ROW_DIRICHLET) u[i * L.N + p] += (double)e[i * L.N + p];
}

template <typename TE>
__global__ void k_add_correction(Lv<double> L, double* __restrict__ u, const TE* __restrict__ e) {
    if (L.active && *L.active == 0) return;
    add_correction_body<TE>(L, u, e, blockIdx.x * blockDim.x + threadIdx.x);
}

// ---------------------------------------------------------------------------
// bottom solve
// ---------------------------------------------------------------------------
template <int KIND>
__global__ void k_bottom_assemble(Lv<double> L, const int* __restrict__ dofs, int nfree, NullInfo nf,
                                  double* __restrict__ A) {
    const int ntot = nfree + nf.m;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)ntot * ntot) return;
    const int row = (int)(t / ntot), col = (int)(t % ntot);
    double v = 0.0;
    if (row < nfree && col < nfree) {
        const int ir = dofs[row] / L.N, pr = dofs[row] % L.N;
        const int ic = dofs[col] / L.N, pc = dofs[col] % L.N;
        int c[3];
        coords_of(pr, L.n, c);
        const NodeInfo ni = node_info(L, c[0], c[1], c[2]);
        const int type = row_type(L, ni, ir);
        UProbe<double> e{ic, {0, 0, 0}};
        coords_of(pc, L.n, e.c0);
        v = boundary_row<double, KIND>(L, e, ni, ir, type == ROW_INTERIOR ? ROW_TRACTION : type);
    } else if (row < nfree && col >= nfree) {
        const int ir = dofs[row] / L.N, pr = dofs[row] % L.N;
        int c[3];
        coords_of(pr, L.n, c);
        v = null_vec(nf, col - nfree, ir, c);
    } else if (row >= nfree && col < nfree) {
        const int ic = dofs[col] / L.N, pc = dofs[col] % L.N;
        int c[3];
        coords_of(pc, L.n, c);
        v = null_vec(nf, row - nfree, ic, c);
    }
    A[t] = v;
}

#ifdef ELAS_KERNELS_TU
// Gauss-Jordan inverse with partial pivoting, X = A^-1 (A is destroyed), one pivot column
// per pair of launches so that the O(n^3) elimination spreads over every SM: the pivot
// launch (one block) picks the first row of largest |A[r][col]|, swaps it up, scales the
// pivot row and saves column col in fcol; the elimination launch updates all other rows.
// A zero pivot sets *singular and every later launch returns at once.
__global__ void k_gj_init(double* __restrict__ X, int n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < (size_t)n * n) X[i] = ((int)(i / n) == (int)(i % n)) ? 1.0 : 0.0;
}

__global__ void k_gj_pivot(double* __restrict__ A, double* __restrict__ X, int n, int col,
                           double* __restrict__ fcol, int* __restrict__ singular) {
    __shared__ int piv;
    __shared__ double pval;
    __shared__ double wv[32];
    __shared__ int wr[32];
    if (*singular) return;
    double bv = -1.0;
    int br = n;
    for (int r = col + threadIdx.x; r < n; r += blockDim.x) {
        const double v = fabs(A[(size_t)r * n + col]);
        if (v > bv) { bv = v; br = r; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, bv, o);
        const int orr = __shfl_down_sync(0xffffffffu, br, o);
        if (ov > bv || (ov == bv && orr < br)) { bv = ov; br = orr; }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { wv[warp] = bv; wr[warp] = br; }
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        bv = lane < nw ? wv[lane] : -1.0;
        br = lane < nw ? wr[lane] : n;
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_down_sync(0xffffffffu, bv, o);
            const int orr = __shfl_down_sync(0xffffffffu, br, o);
            if (ov > bv || (ov == bv && orr < br)) { bv = ov; br = orr; }
        }
        if (lane == 0) {
            piv = br;
            pval = A[(size_t)br * n + col];
            if (bv == 0.0) *singular = 1;
        }
    }
    __syncthreads();
    if (pval == 0.0) return;
    if (piv != col) {
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            double a = A[(size_t)col * n + k]; A[(size_t)col * n + k] = A[(size_t)piv * n + k]; A[(size_t)piv * n + k] = a;
            double x = X[(size_t)col * n + k]; X[(size_t)col * n + k] = X[(size_t)piv * n + k]; X[(size_t)piv * n + k] = x;
        }
    }
    __syncthreads();
    const double inv = 1.0 / pval;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        A[(size_t)col * n + k] *= inv;
        X[(size_t)col * n + k] *= inv;
    }
    for (int r = threadIdx.x; r < n; r += blockDim.x) fcol[r] = A[(size_t)r * n + col];
}

__global__ void k_gj_eliminate(double* __restrict__ A, double* __restrict__ X, int n, int col,
                               const double* __restrict__ fcol, const int* __restrict__ singular) {
    if (*singular) return;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)n * n) return;
    const int r = (int)(idx / n), k = (int)(idx % n);
    if (r == col) return;
    const double fct = fcol[r];
    if (k != col) {
        A[idx] -= fct * A[(size_t)col * n + k];
        X[idx] -= fct * X[(size_t)col * n + k];
    } else {
        X[idx] -= fct * X[(size_t)col * n + col];
        A[idx] = 0.0;
    }
}
#endif

template <typename T>
__global__ void k_bottom_gather(Lv<T> L, const int* __restrict__ dofs, int nfree, int ntot, const T* __restrict__ f,
                                double* __restrict__ b) {
    if (L.active && *L.active == 0) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ntot) return;
    b[i] = i < nfree ? (double)f[dofs[i]] : 0.0;
}

// Row `row` of the bottom solve: u[dofs[row]] = sum_k Ainv[row][k] b[k] (a whole block).
template <typename T>
__device__ __forceinline__ void bottom_matvec_body(const int* __restrict__ dofs, int nfree, int ntot,
                                                   const double* __restrict__ Ainv, const double* __restrict__ b,
                                                   T* __restrict__ u, int row) {
    if (row >= nfree) return;
    double acc = 0.0;
    for (int k = threadIdx.x; k < ntot; k += blockDim.x) acc += Ainv[(size_t)row * ntot + k] * b[k];
    __shared__ double sm[kBlock / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kBlock / 32; ++w) s += sm[w];
        u[dofs[row]] = (T)s;
    }
}

template <typename T>
__global__ void k_bottom_matvec(Lv<T> L, const int* __restrict__ dofs, int nfree, int ntot,
                                const double* __restrict__ Ainv, const double* __restrict__ b, T* __restrict__ u) {
    if (L.active && *L.active == 0) return;
    bottom_matvec_body<T>(dofs, nfree, ntot, Ainv, b, u, blockIdx.x);
}

template <typename T>
__global__ void k_zero(T* __restrict__ a, size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = T(0);
}

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------
// Deterministic sum of the residual partials; with free rigid modes also
//   W^T r = basis^T mom,  dlam = G^-1 W^T r,  lam += dlam,
//   a_lam = basis lam, a_dlam = basis dlam (the loads as t + w x d),
//   ||r - dlam.W||^2 = ||r||^2 - 2 dlam.W^T r + dlam^T G dlam.
__device__ __forceinline__ void finalize_body(const double* __restrict__ partials, int nblocks, const NullInfo& nf,
                                              const double* __restrict__ Ginv, const double* __restrict__ G,
                                              double* __restrict__ lam, double* __restrict__ dlam,
                                              double* __restrict__ alam, double* __restrict__ adlam,
                                              double* __restrict__ out, int update_lam, const BatchFlags& bf) {
    __shared__ double sm[kSumThreads / 32][8];
    sum_partials_block(partials, nblocks, sm);
    if (threadIdx.x == 0) {
        double ss = sm[0][0];
        if (nf.m > 0) {
            double wtr[6], d[6];
            for (int q = 0; q < nf.m; ++q) {
                double v = 0.0;
                for (int mo = 0; mo < 6; ++mo) v += nf.basis[mo][q] * sm[0][1 + mo];
                wtr[q] = v;
            }
            for (int q = 0; q < nf.m; ++q) {
                double v = 0.0;
                for (int k = 0; k < nf.m; ++k) v += Ginv[q * nf.m + k] * wtr[k];
                d[q] = v;
            }
            double c1 = 0.0, c2 = 0.0;
            for (int q = 0; q < nf.m; ++q) {
                c1 += d[q] * wtr[q];
                for (int k = 0; k < nf.m; ++k) c2 += d[q] * G[q * nf.m + k] * d[k];
            }
            ss = ss - 2.0 * c1 + c2;
            if (ss < 0.0) ss = 0.0;
            for (int q = 0; q < nf.m; ++q) {
                dlam[q] = d[q];
                if (update_lam) lam[q] += d[q];
            }
            for (int mo = 0; mo < 6; ++mo) {
                double a = 0.0, b = 0.0;
                for (int q = 0; q < nf.m; ++q) {
                    a += nf.basis[mo][q] * lam[q];
                    b += nf.basis[mo][q] * d[q];
                }
                alam[mo] = a;
                adlam[mo] = b;
                ((float*)(alam + kLoadFloatOffset))[mo] = (float)a;
                ((float*)(adlam + kLoadFloatOffset))[mo] = (float)b;
            }
        }
        out[0] = ss;
        out[1] = sm[0][7];   // max |r| of the residual as evaluated
        if (bf.active) {
            // batched solve: record the relative residual, stop this member when done
            const double rel = bf.r0 > 0.0 ? sqrt(ss) / bf.r0 : 0.0;
            const int k = *bf.count;
            if (k < bf.hist_len) bf.hist[k] = rel;
            *bf.count = k + 1;
            if (!(rel > bf.tol) || k >= bf.max_cycles || !isfinite(rel)) *bf.active = 0;
        }
    }
}

#ifdef ELAS_KERNELS_TU
__global__ void k_finalize(const double* __restrict__ partials, int nblocks, NullInfo nf,
                           const double* __restrict__ Ginv, const double* __restrict__ G,
                           double* __restrict__ lam, double* __restrict__ dlam, double* __restrict__ alam,
                           double* __restrict__ adlam, double* __restrict__ out, int update_lam, BatchFlags bf) {
    if (bf.active && *bf.active == 0) return;
    finalize_body(partials, nblocks, nf, Ginv, G, lam, dlam, alam, adlam, out, update_lam, bf);
}
#endif

#ifdef ELAS_KERNELS_TU
__global__ void k_null_dots(Lv<double> L, NullInfo nf, const double* __restrict__ u, double* __restrict__ partials,
                            int gram) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    if (p < L.N) {
        int c[3];
        coords_of(p, L.n, c);
        const NodeInfo ni = node_info(L, c[0], c[1], c[2]);
        // the six raw rigid-motion moments of u over its non-Dirichlet rows: sum u and
        // sum d x u (d = x - ctr); W_q . u = sum_mode basis[mode][q] * moment[mode]
        double um[3];
        for (int i = 0; i < 3; ++i) um[i] = row_type(L, ni, i) == ROW_DIRICHLET ? 0.0 : u[i * L.N + p];
        const double d0 = nf.off[0] + nf.h[0] * c[0];
        const double d1 = nf.off[1] + nf.h[1] * c[1];
        const double d2 = nf.off[2] + nf.h[2] * c[2];
        acc[0] = um[0];
        acc[1] = um[1];
        acc[2] = um[2];
        acc[3] = d1 * um[2] - d2 * um[1];
        acc[4] = d2 * um[0] - d0 * um[2];
        acc[5] = d0 * um[1] - d1 * um[0];
    }
    (void)gram;
    block_reduce_store<7>(acc, 6, partials);
}
#endif

// W^T W row by row: column q0 of the Gram matrix
#ifdef ELAS_KERNELS_TU
__global__ void k_null_gram_row(Lv<double> L, NullInfo nf, int q0, double* __restrict__ partials) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    if (p < L.N) {
        int c[3];
        coords_of(p, L.n, c);
        const NodeInfo ni = node_info(L, c[0], c[1], c[2]);
        for (int i = 0; i < 3; ++i) {
            if (row_type(L, ni, i) == ROW_DIRICHLET) continue;
            const double w0 = null_vec(nf, q0, i, c);
            for (int q = 0; q < nf.m; ++q) acc[q] += w0 * null_vec(nf, q, i, c);
        }
    }
    block_reduce_store<7>(acc, nf.m, partials);
}
#endif

#ifdef ELAS_KERNELS_TU
__global__ void k_sum_partials(const double* __restrict__ partials, int nblocks, int width, double* __restrict__ out) {
    __shared__ double sm[kSumThreads / 32][8];
    sum_partials_block(partials, nblocks, sm);
    if (threadIdx.x < width) out[threadIdx.x] = sm[0][threadIdx.x];
}
#endif

#ifdef ELAS_KERNELS_TU
// From the raw moments: W^T u = basis^T moment, coef = G^-1 W^T u, and the rigid motion
// (t, w) = basis coef that sum_q coef_q W_q equals (one thread).
__global__ void k_null_motion(NullInfo nf, const double* __restrict__ Ginv, const double* __restrict__ moment,
                              double* __restrict__ motion) {
    if (threadIdx.x != 0) return;
    double wtu[6], coef[6];
    for (int q = 0; q < nf.m; ++q) {
        double v = 0.0;
        for (int mo = 0; mo < 6; ++mo) v += nf.basis[mo][q] * moment[mo];
        wtu[q] = v;
    }
    for (int q = 0; q < nf.m; ++q) {
        double v = 0.0;
        for (int k = 0; k < nf.m; ++k) v += Ginv[q * nf.m + k] * wtu[k];
        coef[q] = v;
    }
    for (int mo = 0; mo < 6; ++mo) {
        double v = 0.0;
        for (int q = 0; q < nf.m; ++q) v += nf.basis[mo][q] * coef[q];
        motion[mo] = v;
    }
}

// u -= t + w x d on the non-Dirichlet rows (the rigid part of u).
__global__ void k_remove_null(Lv<double> L, NullInfo nf, const double* __restrict__ motion, double* __restrict__ u) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= L.N) return;
    int c[3];
    coords_of(p, L.n, c);
    const NodeInfo ni = node_info(L, c[0], c[1], c[2]);
    const double d[3] = {nf.off[0] + nf.h[0] * c[0], nf.off[1] + nf.h[1] * c[1], nf.off[2] + nf.h[2] * c[2]};
    const double w[3] = {motion[3], motion[4], motion[5]};
    const double r[3] = {motion[0] + (w[1] * d[2] - w[2] * d[1]), motion[1] + (w[2] * d[0] - w[0] * d[2]),
                         motion[2] + (w[0] * d[1] - w[1] * d[0])};
    for (int i = 0; i < 3; ++i)
        if (row_type(L, ni, i) != ROW_DIRICHLET) u[i * L.N + p] -= r[i];
}
#endif


// ---------------------------------------------------------------------------
// block-structured AMR transfers (reflux-free coarse/fine treatment)
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool amr_is_ghost(const AmrBox& b, const int n[3], const int c[3]) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (b.ghost[2 * d] && c[d] == 0) return true;
        if (b.ghost[2 * d + 1] && c[d] == n[d] - 1) return true;
    }
    return false;
}

#ifdef ELAS_KERNELS_TU
template <typename T>
__global__ void k_amr_interp(Lv<T> Lf, AmrBox bf, Lv<T> Lc, AmrBox bc, const T* __restrict__ cf,
                             T* __restrict__ ff, int mode) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= Lf.N) return;
    int c[3];
    coords_of(p, Lf.n, c);
    const bool ghost = amr_is_ghost(bf, Lf.n, c);
    if ((mode == 0) != ghost) return;
    int i0[3], i1[3];
    double w1[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int g = bf.grid_lo[d] + c[d];
        i0[d] = g / 2 - bc.grid_lo[d];
        i1[d] = (g + 1) / 2 - bc.grid_lo[d];
        w1[d] = (g & 1) ? 0.5 : 0.0;
    }
    const NodeInfo ni = node_info(Lf, c[0], c[1], c[2]);
    for (int k = 0; k < 3; ++k) {
        if (mode == 1 && row_type(Lf, ni, k) == ROW_DIRICHLET) continue;
        const T* e = cf + (size_t)k * Lc.N;
        double v = 0.0;
        for (int bz = 0; bz < 2; ++bz) {
            const double wz = bz ? w1[2] : 1.0 - w1[2];
            if (wz == 0.0) continue;
            for (int by = 0; by < 2; ++by) {
                const double wy = by ? w1[1] : 1.0 - w1[1];
                if (wy == 0.0) continue;
                for (int bx = 0; bx < 2; ++bx) {
                    const double wx = bx ? w1[0] : 1.0 - w1[0];
                    if (wx == 0.0) continue;
                    v += wx * wy * wz *
                         e[lin(Lc, bx ? i1[0] : i0[0], by ? i1[1] : i0[1], bz ? i1[2] : i0[2])];
                }
            }
        }
        if (mode == 0) ff[(size_t)k * Lf.N + p] = (T)v;
        else ff[(size_t)k * Lf.N + p] += (T)v;
    }
}
#endif

// covered coarse box (in coarse local coordinates): coarse global I with 2I in [valid_lo, valid_hi]
__device__ __forceinline__ void amr_cov_box(const AmrBox& bf, const AmrBox& bc, int lo[3], int cnt[3]) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int a = (bf.valid_lo[d] + 1) / 2, b = bf.valid_hi[d] / 2;
        lo[d] = a - bc.grid_lo[d];
        cnt[d] = b - a + 1;
    }
}

#ifdef ELAS_KERNELS_TU
__global__ void k_amr_inject(Lv<double> Lf, AmrBox bf, Lv<double> Lc, AmrBox bc, const double* __restrict__ ffield,
                             double* __restrict__ cfield) {
    int lo[3], cnt[3];
    amr_cov_box(bf, bc, lo, cnt);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cnt[0] * cnt[1] * cnt[2]) return;
    const int cc[3] = {lo[0] + t % cnt[0], lo[1] + (t / cnt[0]) % cnt[1], lo[2] + t / (cnt[0] * cnt[1])};
    int fc[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) fc[d] = 2 * (bc.grid_lo[d] + cc[d]) - bf.grid_lo[d];
    const int pc = lin(Lc, cc[0], cc[1], cc[2]), pf = lin(Lf, fc[0], fc[1], fc[2]);
    for (int k = 0; k < 3; ++k) cfield[(size_t)k * Lc.N + pc] = ffield[(size_t)k * Lf.N + pf];
}
#endif

#ifdef ELAS_KERNELS_TU
template <typename T>
__global__ void k_amr_restrict(Lv<T> Lf, AmrBox bf, Lv<T> Lc, AmrBox bc, const T* __restrict__ ffield,
                               T* __restrict__ cfield, int K, int zero_dirichlet) {
    int lo[3], cnt[3];
    amr_cov_box(bf, bc, lo, cnt);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cnt[0] * cnt[1] * cnt[2]) return;
    const int cc[3] = {lo[0] + t % cnt[0], lo[1] + (t / cnt[0]) % cnt[1], lo[2] + t / (cnt[0] * cnt[1])};
    double w[3][3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int fcg = 2 * (bc.grid_lo[d] + cc[d]);
        double ww[3];
        if (fcg == 0) { ww[0] = 0.0; ww[1] = 0.5; ww[2] = 0.5; }
        else if (fcg == bf.count[d] - 1) { ww[0] = 0.5; ww[1] = 0.5; ww[2] = 0.0; }
        else { ww[0] = 0.25; ww[1] = 0.5; ww[2] = 0.25; }
        double sum = 0.0;
        for (int o = -1; o <= 1; ++o) {
            const int g = fcg + o;
            if (g < bf.valid_lo[d] || g > bf.valid_hi[d]) ww[o + 1] = 0.0;
            sum += ww[o + 1];
        }
        for (int o = 0; o < 3; ++o) w[d][o] = ww[o] / sum;
    }
    const NodeInfo nic = node_info(Lc, cc[0], cc[1], cc[2]);
    const int pc = lin(Lc, cc[0], cc[1], cc[2]);
    for (int k = 0; k < K; ++k) {
        double acc = 0.0;
        for (int oz = -1; oz <= 1; ++oz) {
            if (w[2][oz + 1] == 0.0) continue;
            for (int oy = -1; oy <= 1; ++oy) {
                if (w[1][oy + 1] == 0.0) continue;
                for (int ox = -1; ox <= 1; ++ox) {
                    if (w[0][ox + 1] == 0.0) continue;
                    const int fx = 2 * (bc.grid_lo[0] + cc[0]) + ox - bf.grid_lo[0];
                    const int fy = 2 * (bc.grid_lo[1] + cc[1]) + oy - bf.grid_lo[1];
                    const int fz = 2 * (bc.grid_lo[2] + cc[2]) + oz - bf.grid_lo[2];
                    acc += w[0][ox + 1] * w[1][oy + 1] * w[2][oz + 1] * (double)ffield[(size_t)k * Lf.N + lin(Lf, fx, fy, fz)];
                }
            }
        }
        if (k < 3 && row_type(Lc, nic, k) == ROW_DIRICHLET) {
            if (zero_dirichlet == 1) acc = 0.0;
            else if (zero_dirichlet == 2) continue;   // keep the coarse boundary value
        }
        cfield[(size_t)k * Lc.N + pc] = (T)acc;
    }
}
#endif

#ifdef ELAS_KERNELS_TU
__global__ void k_amr_norm(Lv<double> L, AmrBox b, AmrBox cov, int has_cov, const double* __restrict__ res,
                           double* __restrict__ partials) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    if (p < L.N) {
        int c[3];
        coords_of(p, L.n, c);
        // valid nodes only (ghost layers, relaxed or not, are not composite equations)
        bool skip = false;
        for (int d = 0; d < 3; ++d) {
            const int g = b.grid_lo[d] + c[d];
            skip |= (g < b.valid_lo[d] || g > b.valid_hi[d]);
        }
        if (!skip && has_cov) {
            bool in = true;
            for (int d = 0; d < 3; ++d) {
                const int g2 = 2 * (b.grid_lo[d] + c[d]);
                in &= (g2 >= cov.valid_lo[d] && g2 <= cov.valid_hi[d]);
            }
            skip = in;
        }
        if (!skip)
            for (int k = 0; k < 3; ++k) {
                const double r = res[(size_t)k * L.N + p];
                acc[0] += r * r;
            }
    }
    block_reduce_store<7>(acc, 1, partials);
}
#endif

#ifdef ELAS_KERNELS_TU
template <typename TU, typename TC>
__global__ void k_amr_add(Lv<TU> L, AmrBox b, TU* __restrict__ u, const TC* __restrict__ cor) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= L.N) return;
    int c[3];
    coords_of(p, L.n, c);
    if (amr_is_ghost(b, L.n, c)) return;
    for (int k = 0; k < 3; ++k) u[(size_t)k * L.N + p] += (TU)cor[(size_t)k * L.N + p];
}

// a := (TO) b, n elements
template <typename TO, typename TI>
__global__ void k_cast(TO* __restrict__ a, const TI* __restrict__ b, size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = (TO)b[i];
}
#endif

}  // namespace

template <typename T, int A>
void launch_faces_apply(const Lv<T>& L, const T* u, T* out, cudaStream_t s) {
    const size_t n = face_count<T, A>(L);
    if (!n) return;
    count_launch();
    if (L.K == 2) k_apply_face<T, 2, A><<<blocks_for(n), kBlock, 0, s>>>(L, u, out);
    else k_apply_face<T, 21, A><<<blocks_for(n), kBlock, 0, s>>>(L, u, out);
}

template <typename T, int A>
void launch_faces_sweep(const Lv<T>& L, const T* u_in, T* u_out, const T* f, int colour, const NullInfo& nfv,
                        const double* load, cudaStream_t s) {
    const size_t n = face_count<T, A>(L);
    if (!n) return;
    count_launch();
    if (L.K == 2) k_half_sweep_face<T, 2, A><<<blocks_for(n), kBlock, 0, s>>>(L, u_in, u_out, f, colour, nfv, load);
    else k_half_sweep_face<T, 21, A><<<blocks_for(n), kBlock, 0, s>>>(L, u_in, u_out, f, colour, nfv, load);
}

}  // namespace elas
