// Device-side definitions shared by the kernels: level geometry, row
// classification, moduli access and the discrete operator.
//
// The operator follows Runnels et al., Section 2.1.1: the product-rule split
//   D(u)_i = C_ijkl,j (u_k,l - eps0_kl) + C_ijkl (u_k,lj - eps0_kl,j)
// with central first differences, compact second differences, four-corner mixed
// differences and central differences of the nodal moduli.  Boundary conditions
// are boundary-operator rows (Section 2.1, Eq. 1b-1d): Dirichlet rows are held
// fixed; a traction row is the balance of the node's half (quarter, eighth)
// control cell, i.e. the product-rule terms of its non-boundary directions plus,
// for each boundary direction a, -(2/h_a) s_a Cbar_iakl Dbar_l u_k (the stress at
// the half-cell face; the prescribed traction goes to the right-hand side);
// Neumann rows are -(2/h_a) C_iaia s_a D_a u_i.  Near a boundary plane of
// direction l the first derivative D_l is one-sided and second order.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "elas_dfloat.cuh"

namespace elas {

enum : int { ROW_INTERIOR = 0, ROW_DIRICHLET = 1, ROW_TRACTION = 2, ROW_NEUMANN = 3 };

// Geometry of one level, passed by value to every kernel.
template <typename T>
struct Lv {
    int n[3];
    int per[3];
    int N;
    int K;                 // moduli components: 2 (lambda, mu) or 21 (Voigt upper triangle)
    // moduli layout: kModPlanes = one plane per component (FP64 levels); kModBlocked =
    // planes per block of 32 consecutive nodes (FP32 copies); kModRecords = node-major
    // records (FP16 copies)
    int mlay;
    signed char bc[6][3];  // boundary type per (face, component); 0 on periodic faces
    T h[3], inv2h[3], invh[3], invh2[3], inv4hh[3];   // inv4hh[d] for the pair != d
    const T* __restrict__ mod;
    const int* __restrict__ bnodes;   // linear indices of the edge and corner nodes
    int nbnd;
    // optional: M_iV = sum_j d_j C_(ij)V (18 planes, interior nodes), precomputed so the
    // modulus-gradient term costs 18 FMAs instead of 54 differences
    const T* __restrict__ divc;
    // optional per-grid flag of a batched solve: kernels of a converged member return at once
    const int* __restrict__ active;
    // optional FP16 copy of the moduli read by FP32 kernels instead of `mod`
    const __half* __restrict__ modh;
    // coefficients of the edge and corner rows: for bnodes[w], kEdgeCoef entries
    // [row i][slot][component k] (see edge_slot_node), so a row is a 27-slot dot product;
    // set up with the moduli, required by the smoother and the residual
    const T* __restrict__ bcoef;
    // colour-split layout (kModSplit): offset, in elements, of the odd-index half
    size_t msplit1;
    // damping of the Jacobi smoother (colour kJacobiColour); the other smoothers ignore it
    T omega;
    // bit A set: the face nodes of direction A are in bnodes (rows from stored
    // coefficients), not in the face kernels
    int xface_list;
};

// Which nodes one smoother pass updates.  Colours 0 and 1: red-black, (i + j + k) mod 2;
// 2..9: the eight colours (i mod 2) + 2 (j mod 2) + 4 (k mod 2), offset by 2;
// kJacobiColour: every node (damped block Jacobi).
constexpr int kJacobiColour = 10;
__host__ __device__ __forceinline__ bool sweep_active(int colour, int x, int y, int z) {
    if (colour < 2) return ((x + y + z) & 1) == colour;
    if (colour < kJacobiColour) return ((x & 1) | ((y & 1) << 1) | ((z & 1) << 2)) == colour - 2;
    return true;
}

// Edge and corner rows reach 3 nodes per direction: c-1, c, c+1 where the node is not on a
// boundary plane of that direction (wrapped when periodic), c, c+s, c+2s (s inward) where
// it is.  Slot t0 + 3 t1 + 9 t2 names one of the 27; the slot of the node itself is
// edge_center_slot.  Coefficients per node: 3 rows x 27 slots x 3 components.
constexpr int kEdgeCoef = 243;

// Moduli layouts.  Planes: component c of node q at c * N + q.  Blocked (FP32 copies):
// the nodes are cut into blocks of 32 consecutive linear indices and each block stores
// its K components as K runs of 32, so c of q sits at (q / 32) * 32 K + 32 c + q % 32: a
// warp's loads of one component stay as contiguous as in planes, while the K components
// of a node are compile-time offsets (multiples of 128 bytes) from one address.
// Records (FP16 copies): node-major, lambda, mu or the 21 components padded to 24, so a
// node costs one address and three 16-byte loads.
// Colour split (FP32 copies of general moduli on levels with odd nx and ny): there the
// parity of the linear index q equals the red-black colour (i + j + k) mod 2, so the even
// and the odd q form the two colours.  Each colour is stored blocked as above, with
// kSplitK components per node: the 21 moduli followed by the 18 entries of the modulus
// divergence M_iV = sum_j d_j C_(ij)V (i * 6 + V).  Component c of node q sits at
// (q & 1) * msplit1 + blocked_index(kSplitK, c, q >> 1).  A half-sweep then reads only its
// colour's records, contiguous for a warp, and no neighbour moduli at all.
enum : int { kModPlanes = 0, kModBlocked = 1, kModRecords = 2, kModSplit = 3 };
constexpr int kSplitK = 39;
__host__ __device__ constexpr int mod_record(int K) { return K == 2 ? 2 : 24; }
__host__ __device__ inline size_t blocked_index(int K, int c, int q) {
    return (size_t)(q >> 5) * (32 * K) + 32 * c + (q & 31);
}
// Elements of one colour half of the split layout (count nodes, blocks of 32).
__host__ __device__ inline size_t split_half_entries(int count) { return (size_t)((count + 31) / 32) * 32 * kSplitK; }

// Moduli component c of node q in the level's layout.
template <typename T>
__device__ __forceinline__ T modc(const Lv<T>& L, int c, int q) {
    if (sizeof(T) == 4) {
        if (L.mlay == kModRecords) return T(__half2float(L.modh[(size_t)q * mod_record(L.K) + c]));
        if (L.mlay == kModBlocked) return L.mod[blocked_index(L.K, c, q)];
        if (L.mlay == kModSplit) return L.mod[(q & 1) * L.msplit1 + blocked_index(kSplitK, c, q >> 1)];
    }
    return L.mod[(size_t)c * L.N + q];
}

// Component c of node q from a blocked FP32 copy (c is a compile-time constant in the
// unrolled stencil: the address of q is computed once, the components are offsets).
template <int KIND>
__device__ __forceinline__ float blk_float(const float* __restrict__ mod, int q, int c) {
    constexpr int K = KIND == 2 ? 2 : 21;
    return __ldg(mod + (size_t)(q >> 5) * (32 * K) + (q & 31) + 32 * c);
}

// Component c of node q's FP16 record, read as aligned 16-byte pieces shared by repeated
// calls (the selects fold away for constant c).
template <int KIND>
__device__ __forceinline__ float rec_half(const __half* __restrict__ mod, int q, int c) {
    unsigned w;
    if (KIND == 2) {
        w = __ldg(reinterpret_cast<const unsigned*>(mod) + q);
    } else {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(mod) + (size_t)q * 3 + (c >> 3));
        const int k = (c & 7) >> 1;
        w = k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
    }
    return __half2float(__ushort_as_half((unsigned short)((c & 1) ? (w >> 16) : (w & 0xffffu))));
}

// ---- rounded arithmetic the compiler never contracts -----------------------------
// The interior stencil, its diagonal block and the 3x3 solve spell out every
// multiply-add with these, so the result does not depend on how the compiler fuses
// operations in a given kernel: every launch shape of the smoother computes
// identical bits.
template <typename T> __device__ __forceinline__ T xadd(T a, T b);
template <typename T> __device__ __forceinline__ T xsub(T a, T b);
template <typename T> __device__ __forceinline__ T xmul(T a, T b);
template <typename T> __device__ __forceinline__ T xfma(T a, T b, T c);   // a * b + c, one rounding
template <> __device__ __forceinline__ float xadd(float a, float b) { return __fadd_rn(a, b); }
template <> __device__ __forceinline__ float xsub(float a, float b) { return __fsub_rn(a, b); }
template <> __device__ __forceinline__ float xmul(float a, float b) { return __fmul_rn(a, b); }
template <> __device__ __forceinline__ float xfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <> __device__ __forceinline__ double xadd(double a, double b) { return __dadd_rn(a, b); }
template <> __device__ __forceinline__ double xsub(double a, double b) { return __dsub_rn(a, b); }
template <> __device__ __forceinline__ double xmul(double a, double b) { return __dmul_rn(a, b); }
template <> __device__ __forceinline__ double xfma(double a, double b, double c) { return __fma_rn(a, b, c); }
template <> __device__ __forceinline__ dfloat xadd(dfloat a, dfloat b) { return df_add(a, b); }
template <> __device__ __forceinline__ dfloat xsub(dfloat a, dfloat b) { return df_sub(a, b); }
template <> __device__ __forceinline__ dfloat xmul(dfloat a, dfloat b) { return df_mul(a, b); }
template <> __device__ __forceinline__ dfloat xfma(dfloat a, dfloat b, dfloat c) { return df_fma(a, b, c); }

// ---- Voigt helpers ----------------------------------------------------------
__host__ __device__ constexpr int voigt(int i, int j) { return i == j ? i : 6 - i - j; }
__host__ __device__ constexpr int upper(int a, int b) {
    return a <= b ? a * (11 - a) / 2 + b : b * (11 - b) / 2 + a;
}
__host__ __device__ constexpr int pair_index(int j, int l) {  // (0,1)->2 (0,2)->1 (1,2)->0
    return 3 - j - l;
}

// C_ijkl at node q.
template <typename T, int KIND>
__device__ __forceinline__ T Cm(const Lv<T>& L, int q, int i, int j, int k, int l) {
    if (KIND == 2) {
        const T lam = modc(L, 0, q);
        const T mu = modc(L, 1, q);
        T v = T(0);
        if (i == j && k == l) v += lam;
        if (i == k && j == l) v += mu;
        if (i == l && j == k) v += mu;
        return v;
    } else {
        return modc(L, upper(voigt(i, j), voigt(k, l)), q);
    }
}

template <typename T, int KIND>
__device__ __forceinline__ bool Cnz(int i, int j, int k, int l) {
    if (KIND == 2) return (i == j && k == l) || (i == k && j == l) || (i == l && j == k);
    return true;
}

// ---- node classification ------------------------------------------------------
struct NodeInfo {
    int c[3];
    signed char side[3];   // -1 low boundary plane, +1 high, 0 none (or periodic)
    bool boundary;
};

template <typename T>
__device__ __forceinline__ NodeInfo node_info(const Lv<T>& L, int x, int y, int z) {
    NodeInfo ni;
    ni.c[0] = x; ni.c[1] = y; ni.c[2] = z;
    ni.boundary = false;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        int s = 0;
        if (!L.per[d]) {
            if (ni.c[d] == 0) s = -1;
            else if (ni.c[d] == L.n[d] - 1) s = 1;
        }
        ni.side[d] = (signed char)s;
        ni.boundary |= (s != 0);
    }
    return ni;
}

// Row type of component c at a node (Dirichlet over Neumann over traction).
template <typename T>
__device__ __forceinline__ int row_type(const Lv<T>& L, const NodeInfo& ni, int c) {
    if (!ni.boundary) return ROW_INTERIOR;
    bool dir = false, neu = false;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (ni.side[d] == 0) continue;
        const int f = 2 * d + (ni.side[d] > 0 ? 1 : 0);
        const int t = L.bc[f][c];
        dir |= (t == ROW_DIRICHLET);
        neu |= (t == ROW_NEUMANN);
    }
    return dir ? ROW_DIRICHLET : (neu ? ROW_NEUMANN : ROW_TRACTION);
}

template <typename T>
__device__ __forceinline__ int lin(const Lv<T>& L, int x, int y, int z) {
    return x + L.n[0] * (y + L.n[1] * z);
}

// Node coordinates of slot `slot` of a boundary node (see kEdgeCoef).
template <typename T>
__device__ __forceinline__ void edge_slot_node(const Lv<T>& L, const NodeInfo& ni, int slot, int a[3]) {
    const int t[3] = {slot % 3, (slot / 3) % 3, slot / 9};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (ni.side[d] == 0) {
            int v = ni.c[d] + t[d] - 1;
            if (L.per[d]) v = v < 0 ? v + L.n[d] : (v >= L.n[d] ? v - L.n[d] : v);
            a[d] = v;
        } else {
            a[d] = ni.c[d] - ni.side[d] * t[d];
        }
    }
}

__device__ __forceinline__ int edge_center_slot(const NodeInfo& ni) {
    return (ni.side[0] == 0 ? 1 : 0) + 3 * (ni.side[1] == 0 ? 1 : 0) + 9 * (ni.side[2] == 0 ? 1 : 0);
}

// Coordinate c + s e_d with periodic wrap.
template <typename T>
__device__ __forceinline__ int wrapc(const Lv<T>& L, int d, int v) {
    if (L.per[d]) {
        if (v < 0) v += L.n[d];
        else if (v >= L.n[d]) v -= L.n[d];
    }
    return v;
}

// ---- field accessors (coordinates already wrapped / in range) ----------------------
template <typename T>
struct UField {
    const T* __restrict__ u;
    int N, n0, n1;
    __device__ __forceinline__ T at(int k, const int a[3]) const { return u[k * N + a[0] + n0 * (a[1] + n1 * a[2])]; }
};

// Unit vector e_(kk, c0): the operator applied to it gives column (kk, c0).
template <typename T>
struct UProbe {
    int kk, c0[3];
    __device__ __forceinline__ T at(int k, const int a[3]) const {
        return (k == kk && a[0] == c0[0] && a[1] == c0[1] && a[2] == c0[2]) ? T(1) : T(0);
    }
};

// ---- generic boundary-node row -----------------------------------------------------
// First derivative in direction l at node c of the field given by g(int[3]): one-sided
// second order where c lies on a boundary plane of l, central otherwise.
template <typename T, class G>
__device__ __forceinline__ T deriv_c(const Lv<T>& L, const G& g, const int c[3], int l) {
    int side = 0;
    if (!L.per[l]) {
        if (c[l] == 0) side = -1;
        else if (c[l] == L.n[l] - 1) side = 1;
    }
    int a[3] = {c[0], c[1], c[2]};
    if (side == 0) {
        a[l] = wrapc(L, l, c[l] + 1);
        const T up = g(a);
        a[l] = wrapc(L, l, c[l] - 1);
        const T um = g(a);
        return (up - um) * L.inv2h[l];
    }
    const int dirn = -side;   // inward
    const T g0 = g(a);
    a[l] = c[l] + dirn;
    const T g1 = g(a);
    a[l] = c[l] + 2 * dirn;
    const T g2 = g(a);
    return T(dirn) * (T(-3) * g0 + T(4) * g1 - g2) * L.inv2h[l];
}

// Row i (interior or traction type) at a node, generic in the field.
template <typename T, int KIND, class U>
__device__ __noinline__ T pde_row_generic(const Lv<T>& L, const U& u, const NodeInfo& ni, int i) {
    const int* c = ni.c;
    const int p = lin(L, c[0], c[1], c[2]);
    T acc = T(0);
    // product-rule terms of the non-boundary directions
    for (int j = 0; j < 3; ++j) {
        if (ni.side[j] != 0) continue;
        int cp[3] = {c[0], c[1], c[2]}, cm[3] = {c[0], c[1], c[2]};
        cp[j] = wrapc(L, j, c[j] + 1);
        cm[j] = wrapc(L, j, c[j] - 1);
        const int qp = lin(L, cp[0], cp[1], cp[2]);
        const int qm = lin(L, cm[0], cm[1], cm[2]);
        for (int k = 0; k < 3; ++k) {
            auto uk = [&](const int a[3]) { return u.at(k, a); };
            // central difference in j of u_k, as a field
            auto gj = [&](const int a[3]) {
                int ap[3] = {a[0], a[1], a[2]}, am[3] = {a[0], a[1], a[2]};
                ap[j] = wrapc(L, j, a[j] + 1);
                am[j] = wrapc(L, j, a[j] - 1);
                return (u.at(k, ap) - u.at(k, am)) * L.inv2h[j];
            };
            for (int l = 0; l < 3; ++l) {
                if (!Cnz<T, KIND>(i, j, k, l)) continue;
                const T C0 = Cm<T, KIND>(L, p, i, j, k, l);
                const T dC = (Cm<T, KIND>(L, qp, i, j, k, l) - Cm<T, KIND>(L, qm, i, j, k, l)) * L.inv2h[j];
                const T Dl = deriv_c(L, uk, c, l);
                T DD;
                if (l == j) DD = (u.at(k, cp) - T(2) * u.at(k, c) + u.at(k, cm)) * L.invh2[j];
                else DD = deriv_c(L, gj, c, l);
                acc += dC * Dl + C0 * DD;
            }
        }
    }
    // half-cell terms of the boundary directions
    for (int a = 0; a < 3; ++a) {
        if (ni.side[a] == 0) continue;
        const T s = T(ni.side[a]);
        const int inward = -ni.side[a];
        int cn[3] = {c[0], c[1], c[2]};
        cn[a] = c[a] + inward;
        const int qn = lin(L, cn[0], cn[1], cn[2]);
        T sacc = T(0);
        for (int k = 0; k < 3; ++k) {
            auto uk = [&](const int b[3]) { return u.at(k, b); };
            for (int l = 0; l < 3; ++l) {
                if (!Cnz<T, KIND>(i, a, k, l)) continue;
                const T Cbar = T(0.5) * (Cm<T, KIND>(L, p, i, a, k, l) + Cm<T, KIND>(L, qn, i, a, k, l));
                T Dbar;
                if (l == a) Dbar = T(inward) * (u.at(k, cn) - u.at(k, c)) * L.invh[a];
                else Dbar = T(0.5) * (deriv_c(L, uk, c, l) + deriv_c(L, uk, cn, l));
                sacc += Cbar * Dbar;
            }
        }
        acc += -(T(2) * L.invh[a]) * s * sacc;
    }
    return acc;
}

// Neumann row i at a boundary node.
template <typename T, int KIND, class U>
__device__ __noinline__ T neumann_row(const Lv<T>& L, const U& u, const NodeInfo& ni, int i) {
    const int p = lin(L, ni.c[0], ni.c[1], ni.c[2]);
    T acc = T(0);
    auto ui = [&](const int a[3]) { return u.at(i, a); };
    for (int a = 0; a < 3; ++a) {
        if (ni.side[a] == 0) continue;
        const int f = 2 * a + (ni.side[a] > 0 ? 1 : 0);
        if (L.bc[f][i] != ROW_NEUMANN) continue;
        const T C = Cm<T, KIND>(L, p, i, a, i, a);
        acc += -(T(2) * L.invh[a]) * C * T(ni.side[a]) * deriv_c(L, ui, ni.c, a);
    }
    return acc;
}

// Row i of A u at any node (Dirichlet rows return u_i).
template <typename T, int KIND, class U>
__device__ __forceinline__ T boundary_row(const Lv<T>& L, const U& u, const NodeInfo& ni, int i, int type) {
    if (type == ROW_DIRICHLET) return u.at(i, ni.c);
    if (type == ROW_NEUMANN) return neumann_row<T, KIND>(L, u, ni, i);
    return pde_row_generic<T, KIND>(L, u, ni, i);
}

// ---- interior fast path ------------------------------------------------------------
// All three rows of D_H u at a node that lies on no boundary plane.
// All three rows of D_H u at a node on no boundary plane, through accessors:
// ua(k, dx, dy, dz) = u_k at the offset node, ca(c, dx, dy, dz) = moduli plane c there
// (offsets are compile-time after unrolling; p = linear index for the optional
// precomputed modulus divergence).
template <typename T, int KIND, bool HAS_M, class UA, class CA>
__device__ __forceinline__ void interior_rows_core(const Lv<T>& L, const UA& ua, const CA& ca, int p, T out[3]) {
    T G[3][3];      // du_k/dx_l
    T Hd[3][3];     // d2u_k/dx_j2
    T Hm[3][3];     // mixed: Hm[k][pair]
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const T u0 = ua(k, 0, 0, 0);
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            const T up = ua(k, l == 0, l == 1, l == 2), um = ua(k, -(l == 0), -(l == 1), -(l == 2));
            G[k][l] = xmul(xsub(up, um), L.inv2h[l]);
            Hd[k][l] = xmul(xadd(xfma(T(-2), u0, up), um), L.invh2[l]);
        }
        auto mixed = [&](T pp, T pm, T mp, T mm, T s) { return xmul(xadd(xsub(xsub(pp, pm), mp), mm), s); };
        Hm[k][0] = mixed(ua(k, 0, 1, 1), ua(k, 0, 1, -1), ua(k, 0, -1, 1), ua(k, 0, -1, -1), L.inv4hh[0]);
        Hm[k][1] = mixed(ua(k, 1, 0, 1), ua(k, 1, 0, -1), ua(k, -1, 0, 1), ua(k, -1, 0, -1), L.inv4hh[1]);
        Hm[k][2] = mixed(ua(k, 1, 1, 0), ua(k, 1, -1, 0), ua(k, -1, 1, 0), ua(k, -1, -1, 0), L.inv4hh[2]);
    }
    // engineering strain of the gradient, Voigt order
    const T e[6] = {G[0][0], G[1][1], G[2][2], xadd(G[1][2], G[2][1]), xadd(G[0][2], G[2][0]),
                    xadd(G[0][1], G[1][0])};
#pragma unroll
    for (int i = 0; i < 3; ++i) out[i] = T(0);
    if (KIND == 2) {
        // isotropic: C_ijkl = lam d_ij d_kl + mu (d_ik d_jl + d_il d_jk)
        const T lam = ca(0, 0, 0, 0), mu = ca(1, 0, 0, 0);
        T dlam[3], dmu[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            dlam[j] = xmul(xsub(ca(0, j == 0, j == 1, j == 2), ca(0, -(j == 0), -(j == 1), -(j == 2))), L.inv2h[j]);
            dmu[j] = xmul(xsub(ca(1, j == 0, j == 1, j == 2), ca(1, -(j == 0), -(j == 1), -(j == 2))), L.inv2h[j]);
        }
        const T div = xadd(xadd(G[0][0], G[1][1]), G[2][2]);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            // (d_j C_ijkl) G_kl = dlam_i div + dmu_j (G_ij + G_ji)
            T t1 = xmul(dlam[i], div);
#pragma unroll
            for (int j = 0; j < 3; ++j) t1 = xfma(dmu[j], xadd(G[i][j], G[j][i]), t1);
            // C_ijkl H_k,jl = lam d_i(div) + mu (lap u_i + d_i div)
            const T lap = xadd(xadd(Hd[i][0], Hd[i][1]), Hd[i][2]);
            T graddiv = (i == 0) ? Hd[0][0] : Hm[0][pair_index(i, 0)];
#pragma unroll
            for (int k = 1; k < 3; ++k) graddiv = xadd(graddiv, (k == i) ? Hd[k][k] : Hm[k][pair_index(i, k)]);
            out[i] = xfma(mu, lap, xfma(xadd(lam, mu), graddiv, t1));
        }
    } else {
        // second derivatives grouped by Voigt pair b = (k,l):
        // S[j][b] = d_j d_b u  (diagonal b) or d_j d_l u_k + d_j d_k u_l (shear b)
        T S[3][6];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
#pragma unroll
            for (int b = 0; b < 3; ++b) S[j][b] = (j == b) ? Hd[b][b] : Hm[b][pair_index(j, b)];
#pragma unroll
            for (int b = 3; b < 6; ++b) {
                const int k = (b == 3) ? 1 : 0;
                const int l = (b == 5) ? 1 : 2;
                const T hkl = (j == l) ? Hd[k][j] : Hm[k][pair_index(j, l)];
                const T hlk = (j == k) ? Hd[l][j] : Hm[l][pair_index(j, k)];
                S[j][b] = xadd(hkl, hlk);
            }
        }
        T acc[3] = {T(0), T(0), T(0)};
        if constexpr (HAS_M) {
            // term 1: M_iV e_V, the divergence as components 21 + i * 6 + V of the accessor
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int V = 0; V < 6; ++V) acc[i] = xfma(ca(21 + i * 6 + V, 0, 0, 0), e[V], acc[i]);
        }
        // term 2: C_(ij)b S_jb, centre moduli
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int b = 0; b < 6; ++b) acc[i] = xfma(ca(upper(voigt(i, j), b), 0, 0, 0), S[j][b], acc[i]);
        if constexpr (!HAS_M) {
            // term 1: (d_j C_(ij)V) e_V, one direction at a time (the two neighbour
            // records of direction j are live only within its iteration)
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const int I = voigt(i, j);
#pragma unroll
                    for (int V = 0; V < 6; ++V) {
                        const int cmp = upper(I, V);
                        const T dC = xmul(xsub(ca(cmp, j == 0, j == 1, j == 2), ca(cmp, -(j == 0), -(j == 1), -(j == 2))),
                                          L.inv2h[j]);
                        acc[i] = xfma(dC, e[V], acc[i]);
                    }
                }
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) out[i] = acc[i];
    }
}


// Moduli layouts of the interior accessor (template argument ML): FP64 planes or FP32
// blocks, FP16 node records, FP32 colour split (centre node only).
enum : int { kMlDefault = 0, kMlHalf = 1, kMlSplit = 2 };

// Calls body(ua, ca, p) with the accessors of the interior node (x, y, z): displacement
// planes, and the moduli in the level's layout (ML, above).  Components from 21 on are
// the modulus divergence: FP64 planes in L.divc, or the split records' tail.  Periodic
// directions wrap.
template <typename T, int KIND, int ML, class F>
__device__ __forceinline__ void with_interior(const Lv<T>& L, const T* __restrict__ u, int x, int y, int z,
                                              F&& body) {
    const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
    const int N = L.N;
    int X[3] = {x - 1, x, x + 1}, Y[3] = {y - 1, y, y + 1}, Z[3] = {z - 1, z, z + 1};
    if (L.per[0]) { if (X[0] < 0) X[0] += nx; if (X[2] >= nx) X[2] -= nx; }
    if (L.per[1]) { if (Y[0] < 0) Y[0] += ny; if (Y[2] >= ny) Y[2] -= ny; }
    if (L.per[2]) { if (Z[0] < 0) Z[0] += nz; if (Z[2] >= nz) Z[2] -= nz; }
    const int Ys[3] = {Y[0] * nx, Y[1] * nx, Y[2] * nx};
    const int Zs[3] = {Z[0] * nx * ny, Z[1] * nx * ny, Z[2] * nx * ny};
    auto ua = [&](int k, int dx, int dy, int dz) { return u[k * N + X[dx + 1] + Ys[dy + 1] + Zs[dz + 1]]; };
    const int p = X[1] + Ys[1] + Zs[1];
    if constexpr (sizeof(T) == 4 && ML == kMlSplit) {
        // centre records only (the divergence replaces the neighbour moduli)
        const float* cb = (const float*)L.mod + (p & 1) * L.msplit1 + (size_t)((p >> 1) >> 5) * (32 * kSplitK) +
                          ((p >> 1) & 31);
        auto ca = [&](int c, int, int, int) -> T { return __ldg(cb + 32 * c); };
        body(ua, ca, p);
    } else if constexpr (sizeof(T) == 4) {
        auto ca = [&](int c, int dx, int dy, int dz) -> T {
            const int q = X[dx + 1] + Ys[dy + 1] + Zs[dz + 1];
            if constexpr (ML == kMlHalf) return rec_half<KIND>(L.modh, q, c);
            else return blk_float<KIND>(L.mod, q, c);
        };
        body(ua, ca, p);
    } else {
        auto ca = [&](int c, int dx, int dy, int dz) -> T {
            const int q = X[dx + 1] + Ys[dy + 1] + Zs[dz + 1];
            if (c >= 21) return L.divc[(size_t)(c - 21) * N + q];
            return L.mod[(size_t)c * N + q];
        };
        body(ua, ca, p);
    }
}

// All three rows of D_H u at an interior node, in any moduli layout.
template <typename T, int KIND, bool HAS_M = false>
__device__ __forceinline__ void interior_rows(const Lv<T>& L, const T* __restrict__ u,
                                              int x, int y, int z, T out[3]) {
    if constexpr (sizeof(T) == 4) {
        if (KIND == 21 && L.mlay == kModSplit) {
            auto body = [&](const auto& ua, const auto& ca, int p) { interior_rows_core<T, KIND, true>(L, ua, ca, p, out); };
            with_interior<T, KIND, kMlSplit>(L, u, x, y, z, body);
            return;
        }
    }
    auto body = [&](const auto& ua, const auto& ca, int p) { interior_rows_core<T, KIND, HAS_M>(L, ua, ca, p, out); };
    if constexpr (sizeof(T) == 4) {
        if (L.modh) with_interior<T, KIND, kMlHalf>(L, u, x, y, z, body);
        else with_interior<T, KIND, kMlDefault>(L, u, x, y, z, body);
    } else {
        with_interior<T, KIND, kMlDefault>(L, u, x, y, z, body);
    }
}

// Diagonal 3x3 block of an interior node, B_ik = -2 sum_j C_ijkj / h_j^2, from the
// centre-moduli accessor ca(c, 0, 0, 0).
template <typename T, int KIND, class CA>
__device__ __forceinline__ void interior_block_acc(const Lv<T>& L, const CA& ca, T B[3][3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            T acc = T(0);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                T c;
                if (KIND == 2) {
                    c = T(0);
                    if (i == j && k == j) c = xadd(c, ca(0, 0, 0, 0));
                    if (i == k) c = xadd(c, ca(1, 0, 0, 0));
                    if (i == j && j == k) c = xadd(c, ca(1, 0, 0, 0));
                    if (!Cnz<T, KIND>(i, j, k, j)) continue;
                } else {
                    c = ca(upper(voigt(i, j), voigt(k, j)), 0, 0, 0);
                }
                acc = xfma(c, T(-2) * L.invh2[j], acc);
            }
            B[i][k] = acc;
        }
}

// ---- face-node fast path ------------------------------------------------------------
// Rows and diagonal block of a node on exactly one boundary plane (direction A, side
// -1|+1): the product-rule terms of the two tangential directions (central, with the
// normal derivative one-sided) plus the half-cell term of direction A.  Tangential
// neighbours exist (face interiors exclude edges; periodic tangents wrap).
template <typename T, int KIND, int A>
__device__ __forceinline__ void face_node(const Lv<T>& L, const T* __restrict__ u, const int c[3], int side,
                                          const int types[3], T out[3], T B[3][3], bool wantB) {
    constexpr int T1 = (A + 1) % 3, T2 = (A + 2) % 3;
    const int N = L.N;
    const int inward = -side;
    // coordinates along A for depths 0,1,2 and tangential neighbours (wrapped)
    const int ca[3] = {c[A], c[A] + inward, c[A] + 2 * inward};
    const int t1m = wrapc(L, T1, c[T1] - 1), t1p = wrapc(L, T1, c[T1] + 1);
    const int t2m = wrapc(L, T2, c[T2] - 1), t2p = wrapc(L, T2, c[T2] + 1);
    auto idx = [&](int xa, int x1, int x2) {
        int q[3];
        q[A] = xa;
        q[T1] = x1;
        q[T2] = x2;
        return q[0] + L.n[0] * (q[1] + L.n[1] * q[2]);
    };
    const int c1 = c[T1], c2 = c[T2];
    const int p = idx(ca[0], c1, c2);
    const int pin = idx(ca[1], c1, c2);
    int q1p[3], q1m[3], q2p[3], q2m[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        q1p[m] = idx(ca[m], t1p, c2);
        q1m[m] = idx(ca[m], t1m, c2);
        q2p[m] = idx(ca[m], c1, t2p);
        q2m[m] = idx(ca[m], c1, t2m);
    }
    const int cpp = idx(ca[0], t1p, t2p), cpm = idx(ca[0], t1p, t2m);
    const int cmp = idx(ca[0], t1m, t2p), cmm = idx(ca[0], t1m, t2m);
    const int q2in = idx(ca[2], c1, c2);
    // derivatives: G[k][l] at the node; Dbar[k][l] at the half-cell face; second
    // derivatives X[k][j][l] for tangential j
    T G[3][3], Db[3][3], Hjj[3][3], H12[3], HjA[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const T* uk = u + k * N;
        const T u0 = uk[p], u1 = uk[pin], u2 = uk[q2in];
        G[k][A] = T(inward) * (T(-3) * u0 + T(4) * u1 - u2) * L.inv2h[A];
        Db[k][A] = T(inward) * (u1 - u0) * L.invh[A];
        T d1[3], d2[3];
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            d1[m] = (uk[q1p[m]] - uk[q1m[m]]) * L.inv2h[T1];
            d2[m] = (uk[q2p[m]] - uk[q2m[m]]) * L.inv2h[T2];
        }
        G[k][T1] = d1[0];
        G[k][T2] = d2[0];
        Db[k][T1] = T(0.5) * (d1[0] + d1[1]);
        Db[k][T2] = T(0.5) * (d2[0] + d2[1]);
        Hjj[k][T1] = (uk[q1p[0]] - T(2) * u0 + uk[q1m[0]]) * L.invh2[T1];
        Hjj[k][T2] = (uk[q2p[0]] - T(2) * u0 + uk[q2m[0]]) * L.invh2[T2];
        Hjj[k][A] = T(0);
        H12[k] = (uk[cpp] - uk[cpm] - uk[cmp] + uk[cmm]) * L.inv4hh[A];
        HjA[k][T1] = T(inward) * (T(-3) * d1[0] + T(4) * d1[1] - d1[2]) * L.inv2h[A];
        HjA[k][T2] = T(inward) * (T(-3) * d2[0] + T(4) * d2[1] - d2[2]) * L.inv2h[A];
        HjA[k][A] = T(0);
    }
    // DD(k; j, l) for j tangential
    auto DD = [&](int k, int j, int l) -> T {
        if (l == j) return Hjj[k][j];
        if (l == A) return HjA[k][j];
        return H12[k];
    };
    const int qt[2][2] = {{q1p[0], q1m[0]}, {q2p[0], q2m[0]}};
    const T cA = T(side) * T(1.5) * L.invh[A];   // node weight in its one-sided A-derivative
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int f = 2 * A + (side > 0 ? 1 : 0);
        if (types[i] == ROW_DIRICHLET) {
            out[i] = u[i * N + p];
            if (wantB) { B[i][0] = B[i][1] = B[i][2] = T(0); B[i][i] = T(1); }
            continue;
        }
        if (types[i] == ROW_NEUMANN) {
            const T C = Cm<T, KIND>(L, p, i, A, i, A);
            out[i] = -(T(2) * L.invh[A]) * C * T(side) * G[i][A];
            if (wantB) {
                B[i][0] = B[i][1] = B[i][2] = T(0);
                B[i][i] = -(T(2) * L.invh[A]) * C * T(side) * cA;
            }
            (void)f;
            continue;
        }
        T acc = T(0);
        T b[3] = {T(0), T(0), T(0)};
#pragma unroll
        for (int jj = 0; jj < 2; ++jj) {
            const int j = jj == 0 ? T1 : T2;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
#pragma unroll
                for (int l = 0; l < 3; ++l) {
                    if (!Cnz<T, KIND>(i, j, k, l)) continue;
                    const T C0 = Cm<T, KIND>(L, p, i, j, k, l);
                    const T dC = (Cm<T, KIND>(L, qt[jj][0], i, j, k, l) - Cm<T, KIND>(L, qt[jj][1], i, j, k, l)) *
                                 L.inv2h[j];
                    acc += dC * G[k][l] + C0 * DD(k, j, l);
                    if (wantB) {
                        if (l == A) b[k] += dC * cA;
                        if (l == j) b[k] += C0 * (T(-2) * L.invh2[j]);
                    }
                }
            }
        }
        T sacc = T(0);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
#pragma unroll
            for (int l = 0; l < 3; ++l) {
                if (!Cnz<T, KIND>(i, A, k, l)) continue;
                const T Cb = T(0.5) * (Cm<T, KIND>(L, p, i, A, k, l) + Cm<T, KIND>(L, pin, i, A, k, l));
                sacc += Cb * Db[k][l];
                if (wantB && l == A) b[k] += -(T(2) * L.invh[A] * L.invh[A]) * Cb;
            }
        }
        out[i] = acc - (T(2) * L.invh[A]) * T(side) * sacc;
        if (wantB) { B[i][0] = b[0]; B[i][1] = b[1]; B[i][2] = b[2]; }
    }
}

// Solve B d = r for a 3x3 block (explicit inverse by cofactors).
template <typename T>
__device__ __forceinline__ void solve3(const T B[3][3], const T r[3], T d[3]) {
    auto cof = [](T a, T b, T c, T e) { return xsub(xmul(a, b), xmul(c, e)); };   // a b - c e
    const T c00 = cof(B[1][1], B[2][2], B[1][2], B[2][1]);
    const T c01 = cof(B[1][2], B[2][0], B[1][0], B[2][2]);
    const T c02 = cof(B[1][0], B[2][1], B[1][1], B[2][0]);
    const T det = xfma(B[0][2], c02, xfma(B[0][1], c01, xmul(B[0][0], c00)));
    const T id = T(1) / det;
    const T i00 = xmul(c00, id), i10 = xmul(c01, id), i20 = xmul(c02, id);
    const T i01 = xmul(cof(B[0][2], B[2][1], B[0][1], B[2][2]), id);
    const T i11 = xmul(cof(B[0][0], B[2][2], B[0][2], B[2][0]), id);
    const T i21 = xmul(cof(B[0][1], B[2][0], B[0][0], B[2][1]), id);
    const T i02 = xmul(cof(B[0][1], B[1][2], B[0][2], B[1][1]), id);
    const T i12 = xmul(cof(B[0][2], B[1][0], B[0][0], B[1][2]), id);
    const T i22 = xmul(cof(B[0][0], B[1][1], B[0][1], B[1][0]), id);
    d[0] = xfma(i02, r[2], xfma(i01, r[1], xmul(i00, r[0])));
    d[1] = xfma(i12, r[2], xfma(i11, r[1], xmul(i10, r[0])));
    d[2] = xfma(i22, r[2], xfma(i21, r[1], xmul(i20, r[0])));
}

// ---- rigid-body modes and the equilibrating load -------------------------------------
// Free rigid modes W_q = sum_m basis[m][q] R_m, R_0..2 translations, R_3..5 rotations
// e_a x (x - ctr); zero on Dirichlet rows.
struct NullInfo {
    int m;
    double basis[6][6];
    double ctr[3];
    double lo[3];
    double h[3];
    double off[3];      // lo - ctr
    float off32[3];     // the same offsets and spacings in FP32 for FP32 kernels
    float h32[3];
};

// A load array holds the rigid motion (t, w) as 6 doubles at [0, 6) and as 6 floats
// starting at double offset 8.
constexpr int kLoadFloatOffset = 8;
constexpr int kLoadDoubles = 12;

__device__ __forceinline__ double rigid_mode(const NullInfo& nf, int mode, int c, const int xyz[3]) {
    if (mode < 3) return mode == c ? 1.0 : 0.0;
    const double d[3] = {nf.lo[0] + nf.h[0] * xyz[0] - nf.ctr[0], nf.lo[1] + nf.h[1] * xyz[1] - nf.ctr[1],
                         nf.lo[2] + nf.h[2] * xyz[2] - nf.ctr[2]};
    const int a = mode - 3;
    const int b = (a + 1) % 3, e = (a + 2) % 3;
    if (c == b) return -d[e];
    if (c == e) return d[b];
    return 0.0;
}

// W_q(c) at a node (caller masks Dirichlet rows).
__device__ __forceinline__ double null_vec(const NullInfo& nf, int q, int c, const int xyz[3]) {
    double v = 0.0;
#pragma unroll 1
    for (int mode = 0; mode < 6; ++mode) {
        const double b = nf.basis[mode][q];
        if (b != 0.0) v += b * rigid_mode(nf, mode, c, xyz);
    }
    return v;
}

// Equilibrating load at a non-Dirichlet row from its rigid-motion form a = (t, w):
// t_c + (w x d)_c, d = x - ctr.  (sum_q lam_q W_q = t + w x d with t, w = basis lam.)
// The load is a small correction (the incompatible part of the right-hand side), so
// it is evaluated in FP32 in every kernel, including the FP64 residual: its FP32
// rounding is ~1e-7 of a term that is itself far below the residual tolerance.
template <typename T>
__device__ __forceinline__ T rigid_load(const NullInfo& nf, const double* __restrict__ a, int comp, const int c[3]) {
    const float* at = (const float*)(a + kLoadFloatOffset);
    const float d0 = xfma(nf.h32[0], float(c[0]), nf.off32[0]);
    const float d1 = xfma(nf.h32[1], float(c[1]), nf.off32[1]);
    const float d2 = xfma(nf.h32[2], float(c[2]), nf.off32[2]);
    const float w0 = at[3], w1 = at[4], w2 = at[5];
    float v;
    if (comp == 0) v = xadd(at[0], xsub(xmul(w1, d2), xmul(w2, d1)));
    else if (comp == 1) v = xadd(at[1], xsub(xmul(w2, d0), xmul(w0, d2)));
    else v = xadd(at[2], xsub(xmul(w0, d1), xmul(w1, d0)));
    return T(v);
}

}  // namespace elas
