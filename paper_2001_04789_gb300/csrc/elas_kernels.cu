// Launchers of the multigrid kernels other than the residual and the smoother
// (right-hand side, operator, transfers, bottom solve, reductions, AMR), the launch
// counter and the smoother's tuning table.
#include <array>
#include <map>
#include <mutex>
#include <string>

#define ELAS_KERNELS_TU
#include "elas_kernels.cuh"

namespace elas {

static unsigned long long g_launches = 0;
unsigned long long launch_count() { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }
void count_launch(int n) { __atomic_fetch_add(&g_launches, (unsigned long long)n, __ATOMIC_RELAXED); }


// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
void launch_rhs(const Lv<double>& L, const RhsInputs& in, const BoundaryData& bd, double* f, cudaStream_t s) {
    if (L.K == 2) { count_launch(); k_rhs<2><<<blocks_for(L.N), kBlock, 0, s>>>(L, in, bd, f); }
    else { count_launch(); k_rhs<21><<<blocks_for(L.N), kBlock, 0, s>>>(L, in, bd, f); }
}

void launch_dirichlet(const Lv<double>& L, const BoundaryData& bd, double* u, int keep_free, cudaStream_t s) {
    count_launch();
    k_dirichlet<<<blocks_for(L.N), kBlock, 0, s>>>(L, bd, u, keep_free);
}

template <typename T>
void launch_apply(const Lv<T>& L, const T* u, T* out, cudaStream_t s) {
    const size_t ni = interior_count(L);
    if (ni) {
        count_launch();
        if (L.K == 2) k_apply_int<T, 2, false><<<blocks_for(ni), kBlock, 0, s>>>(L, u, out);
        else if (L.divc) k_apply_int<T, 21, true><<<blocks_for(ni), kBlock, 0, s>>>(L, u, out);
        else k_apply_int<T, 21, false><<<blocks_for(ni), kBlock, 0, s>>>(L, u, out);
    }
    launch_faces_apply<T, 0>(L, u, out, s);
    launch_faces_apply<T, 1>(L, u, out, s);
    launch_faces_apply<T, 2>(L, u, out, s);
    if (L.nbnd) {
        count_launch();
        if (L.K == 2) k_apply_bnd<T, 2><<<blocks_for((size_t)L.nbnd * 32), kBlock, 0, s>>>(L, u, out);
        else k_apply_bnd<T, 21><<<blocks_for((size_t)L.nbnd * 32), kBlock, 0, s>>>(L, u, out);
    }
}

// ---- tuning table of the interior smoother (shared by all translation units) -----------
static std::mutex g_tune_mu;
static std::map<std::array<int, 6>, int> g_tune;
static unsigned long long g_tune_version = 0;   // bumped by every change of the table

unsigned long long tune_version() {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return g_tune_version;
}

int tune_lookup(const std::array<int, 6>& key, int fallback) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    return it == g_tune.end() ? fallback : it->second;
}

void tune_store(const std::array<int, 6>& key, int v) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = v;
    ++g_tune_version;
}

int tune_table_dump(char* buf, int cap) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    std::string out;
    for (auto& kv : g_tune) {
        char line[128];
        snprintf(line, sizeof(line), "%d %d %d %d %d %d %d\n", kv.first[0], kv.first[1], kv.first[2], kv.first[3],
                 kv.first[4], kv.first[5], kv.second);
        out += line;
    }
    if (buf && cap > 0) {
        const int n = (int)out.size() < cap - 1 ? (int)out.size() : cap - 1;
        memcpy(buf, out.data(), n);
        buf[n] = 0;
    }
    return (int)out.size();
}

int tune_table_load(const char* text) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    int count = 0;
    const char* p = text;
    while (p && *p) {
        std::array<int, 6> k;
        int v, used = 0;
        if (sscanf(p, "%d %d %d %d %d %d %d%n", &k[0], &k[1], &k[2], &k[3], &k[4], &k[5], &v, &used) != 7) break;
        if (v >= 0 && v < kNumSweepVariants) {
            g_tune[k] = v;
            ++count;
            ++g_tune_version;
        }
        p += used;
        while (*p == '\n' || *p == ' ') ++p;
    }
    return count;
}


template <typename T>
void launch_restrict(const Lv<T>& Lf, const Lv<T>& Lc, const T* r, T* fc, const NullInfo* nf, const double* dlam,
                     cudaStream_t s) {
    NullInfo nfv{};
    if (nf) nfv = *nf;
    count_launch();
    k_restrict<T><<<blocks_for(Lc.N), kBlock, 0, s>>>(Lf, Lc, r, fc, nfv, dlam);
}

template <typename T>
void launch_prolong_add(const Lv<T>& Lf, const Lv<T>& Lc, const T* ec, T* u, cudaStream_t s) {
    count_launch();
    k_prolong_add<T><<<blocks_for(Lf.N), kBlock, 0, s>>>(Lf, Lc, ec, u);
}

template <typename T>
void launch_restrict_moduli(const Lv<T>& Lf, const Lv<T>& Lc, const T* mf, T* mc, cudaStream_t s) {
    count_launch();
    k_restrict_moduli<T><<<blocks_for(Lc.N), kBlock, 0, s>>>(Lf, Lc, mf, mc);
}

void launch_divc(const Lv<double>& L, double* M, cudaStream_t s) {
    count_launch();
    k_divc<double><<<blocks_for(L.N), kBlock, 0, s>>>(L, M);
}

template <typename T>
void launch_edge_coef(const Lv<T>& L, T* out, cudaStream_t s) {
    const size_t n = (size_t)L.nbnd * kEdgeCoef;
    if (!n) return;
    count_launch();
    if (L.K == 2) k_edge_coef<T, 2><<<blocks_for(n), kBlock, 0, s>>>(L, out);
    else k_edge_coef<T, 21><<<blocks_for(n), kBlock, 0, s>>>(L, out);
}
template void launch_edge_coef<double>(const Lv<double>&, double*, cudaStream_t);
template void launch_edge_coef<float>(const Lv<float>&, float*, cudaStream_t);

size_t moduli_copy_entries(int N, int K, bool half) {
    return half ? (size_t)N * mod_record(K) : (size_t)((N + 31) / 32) * 32 * K;
}

void launch_moduli_copy(const double* in, float* out, int N, int K, cudaStream_t s) {
    count_launch();
    k_to_moduli_copy<float><<<blocks_for(moduli_copy_entries(N, K, false)), kBlock, 0, s>>>(in, out, N, K);
}

// FP64 moduli (21 planes) and divergence (18 planes) -> the FP32 colour-split records.
__global__ void k_to_moduli_split(const double* __restrict__ mod, const double* __restrict__ divc,
                                  float* __restrict__ out, int N, size_t half1, size_t total) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int h = i >= half1 ? 1 : 0;
    const size_t r = h ? i - half1 : i;
    const size_t blk = r / (32 * (size_t)kSplitK), rr = r % (32 * (size_t)kSplitK);
    const int c = (int)(rr / 32);
    const long long q = 2 * (long long)(blk * 32 + rr % 32) + h;
    double v = 0.0;
    if (q < N) v = c < 21 ? mod[(size_t)c * N + q] : divc[(size_t)(c - 21) * N + q];
    out[i] = (float)v;
}

bool split_layout_applies(const int n[3], int K) { return K == 21 && (n[0] & 1) && (n[1] & 1); }

size_t split_entries(int N) { return split_half_entries((N + 1) / 2) + split_half_entries(N / 2); }

void launch_moduli_split(const double* mod, const double* divc, float* out, int N, cudaStream_t s) {
    const size_t total = split_entries(N);
    count_launch();
    k_to_moduli_split<<<blocks_for(total), kBlock, 0, s>>>(mod, divc, out, N, split_half_entries((N + 1) / 2), total);
}

void launch_moduli_copy(const double* in, __half* out, int N, int K, cudaStream_t s) {
    count_launch();
    k_to_moduli_copy<__half><<<blocks_for(moduli_copy_entries(N, K, true)), kBlock, 0, s>>>(in, out, N, K);
}

void launch_add_correction(const Lv<double>& L, double* u, const float* e, cudaStream_t s) {
    count_launch();
    k_add_correction<float><<<blocks_for(L.N), kBlock, 0, s>>>(L, u, e);
}

void launch_add_correction64(const Lv<double>& L, double* u, const double* e, cudaStream_t s) {
    count_launch();
    k_add_correction<double><<<blocks_for(L.N), kBlock, 0, s>>>(L, u, e);
}

void launch_bottom_assemble(const Lv<double>& L, const int* dofs, int nfree, const NullInfo& nf, double* A,
                            cudaStream_t s) {
    const long long n = (long long)(nfree + nf.m) * (nfree + nf.m);
    if (n == 0) return;
    const int nb = (int)((n + kBlock - 1) / kBlock);
    if (L.K == 2) { count_launch(); k_bottom_assemble<2><<<nb, kBlock, 0, s>>>(L, dofs, nfree, nf, A); }
    else { count_launch(); k_bottom_assemble<21><<<nb, kBlock, 0, s>>>(L, dofs, nfree, nf, A); }
}

void launch_invert(double* A, double* Ainv, int n, double* fcol, int* singular_flag, cudaStream_t s) {
    if (n == 0) return;
    const int nb = blocks_for((size_t)n * n);
    count_launch(1 + 2 * n);
    k_gj_init<<<nb, kBlock, 0, s>>>(Ainv, n);
    for (int col = 0; col < n; ++col) {
        k_gj_pivot<<<1, 1024, 0, s>>>(A, Ainv, n, col, fcol, singular_flag);
        k_gj_eliminate<<<nb, kBlock, 0, s>>>(A, Ainv, n, col, fcol, singular_flag);
    }
}

template <typename T>
void launch_bottom_solve(const Lv<T>& L, const int* dofs, int nfree, int ntot, const double* Ainv, const T* f, T* u,
                         double* work, cudaStream_t s) {
    count_launch();
    k_zero<T><<<blocks_for((size_t)3 * L.N), kBlock, 0, s>>>(u, (size_t)3 * L.N);
    if (ntot == 0) return;
    count_launch();
    k_bottom_gather<T><<<blocks_for(ntot), kBlock, 0, s>>>(L, dofs, nfree, ntot, f, work);
    if (nfree > 0) {
        count_launch();
        k_bottom_matvec<T><<<nfree, kBlock, 0, s>>>(L, dofs, nfree, ntot, Ainv, work, u);
    }
}

void launch_finalize(const double* partials, int nblocks, const NullInfo& nf, const double* Ginv, const double* G,
                     double* lam, double* dlam, double* alam, double* adlam, double* out, int update_lam,
                     cudaStream_t s, BatchFlags bflags) {
    count_launch();
    k_finalize<<<1, kSumThreads, 0, s>>>(partials, nblocks, nf, Ginv, G, lam, dlam, alam, adlam, out, update_lam, bflags);
}

void launch_null_dots(const Lv<double>& L, const NullInfo& nf, const double* u, double* partials, int* nblocks,
                      int gram, cudaStream_t s) {
    const int nb = blocks_for(L.N);
    *nblocks = nb;
    if (gram) {
        // gram row q0 = gram - 1
        count_launch();
        k_null_gram_row<<<nb, kBlock, 0, s>>>(L, nf, gram - 1, partials);
    } else {
        count_launch();
        k_null_dots<<<nb, kBlock, 0, s>>>(L, nf, u, partials, 0);
    }
}

void launch_sum_partials(const double* partials, int nblocks, int width, double* out, cudaStream_t s) {
    count_launch();
    k_sum_partials<<<1, kSumThreads, 0, s>>>(partials, nblocks, width, out);
}

void launch_remove_null(const Lv<double>& L, const NullInfo& nf, const double* Ginv, const double* moment,
                        double* motion, double* u, cudaStream_t s) {
    count_launch(2);
    k_null_motion<<<1, 32, 0, s>>>(nf, Ginv, moment, motion);
    k_remove_null<<<blocks_for(L.N), kBlock, 0, s>>>(L, nf, motion, u);
}

template <typename T>
void launch_amr_interp(const Lv<T>& Lf, const AmrBox& bf, const Lv<T>& Lc, const AmrBox& bc, const T* cfield,
                       T* ffield, int mode, cudaStream_t s) {
    count_launch();
    k_amr_interp<T><<<blocks_for(Lf.N), kBlock, 0, s>>>(Lf, bf, Lc, bc, cfield, ffield, mode);
}

static size_t amr_cov_count(const AmrBox& bf) {
    size_t n = 1;
    for (int d = 0; d < 3; ++d) n *= (size_t)(bf.valid_hi[d] / 2 - (bf.valid_lo[d] + 1) / 2 + 1);
    return n;
}

void launch_amr_inject(const Lv<double>& Lf, const AmrBox& bf, const Lv<double>& Lc, const AmrBox& bc,
                       const double* ffield, double* cfield, cudaStream_t s) {
    count_launch();
    k_amr_inject<<<blocks_for(amr_cov_count(bf)), kBlock, 0, s>>>(Lf, bf, Lc, bc, ffield, cfield);
}

template <typename T>
void launch_amr_restrict(const Lv<T>& Lf, const AmrBox& bf, const Lv<T>& Lc, const AmrBox& bc, const T* ffield,
                         T* cfield, int K, int zero_dirichlet, cudaStream_t s) {
    count_launch();
    k_amr_restrict<T><<<blocks_for(amr_cov_count(bf)), kBlock, 0, s>>>(Lf, bf, Lc, bc, ffield, cfield, K,
                                                                       zero_dirichlet);
}

int launch_amr_norm(const Lv<double>& L, const AmrBox& b, const AmrBox* cov, const double* res, double* partials,
                    cudaStream_t s) {
    const int nb = blocks_for(L.N);
    AmrBox cv{};
    if (cov) cv = *cov;
    count_launch();
    k_amr_norm<<<nb, kBlock, 0, s>>>(L, b, cv, cov ? 1 : 0, res, partials);
    return nb;
}

template <typename TU, typename TC>
void launch_amr_add(const Lv<TU>& L, const AmrBox& b, TU* u, const TC* cor, cudaStream_t s) {
    count_launch();
    k_amr_add<TU, TC><<<blocks_for(L.N), kBlock, 0, s>>>(L, b, u, cor);
}

template <typename TO, typename TI>
void launch_cast(TO* a, const TI* b, size_t n, cudaStream_t s) {
    count_launch();
    k_cast<TO, TI><<<blocks_for(n), kBlock, 0, s>>>(a, b, n);
}

template void launch_amr_interp<double>(const Lv<double>&, const AmrBox&, const Lv<double>&, const AmrBox&,
                                        const double*, double*, int, cudaStream_t);
template void launch_amr_interp<float>(const Lv<float>&, const AmrBox&, const Lv<float>&, const AmrBox&,
                                       const float*, float*, int, cudaStream_t);
template void launch_amr_restrict<double>(const Lv<double>&, const AmrBox&, const Lv<double>&, const AmrBox&,
                                          const double*, double*, int, int, cudaStream_t);
template void launch_amr_restrict<float>(const Lv<float>&, const AmrBox&, const Lv<float>&, const AmrBox&,
                                         const float*, float*, int, int, cudaStream_t);
template void launch_amr_add<double, double>(const Lv<double>&, const AmrBox&, double*, const double*, cudaStream_t);
template void launch_amr_add<double, float>(const Lv<double>&, const AmrBox&, double*, const float*, cudaStream_t);
template void launch_amr_add<float, float>(const Lv<float>&, const AmrBox&, float*, const float*, cudaStream_t);
template void launch_cast<float, double>(float*, const double*, size_t, cudaStream_t);

// ---- stress output ------------------------------------------------------------------
// sigma = C : (grad u + ebar - eps0) at every node (Eq. 1c's stress), six tensor
// components 11 22 33 23 31 12; first derivatives central, one-sided second order on the
// boundary planes of a non-periodic direction (the operator's own differences).
template <int KIND>
__global__ void k_stress(Lv<double> L, const double* __restrict__ u, const double* __restrict__ eps0, MeanStrain mean,
                         double* __restrict__ out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= L.N) return;
    int c[3];
    coords_of(p, L.n, c);
    UField<double> uf{u, L.N, L.n[0], L.n[1]};
    double G[3][3];
    for (int k = 0; k < 3; ++k) {
        auto uk = [&](const int a[3]) { return uf.at(k, a); };
        for (int l = 0; l < 3; ++l) G[k][l] = deriv_c(L, uk, c, l);
    }
    double e[3][3];
    for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) {
            const int v = voigt(k, l);
            e[k][l] = 0.5 * (G[k][l] + G[l][k]) + mean.e[v] - (eps0 ? eps0[(size_t)v * L.N + p] : 0.0);
        }
    const int I[6] = {0, 1, 2, 1, 2, 0}, J[6] = {0, 1, 2, 2, 0, 1};
    for (int a = 0; a < 6; ++a) {
        double s = 0.0;
        for (int k = 0; k < 3; ++k)
            for (int l = 0; l < 3; ++l)
                if (Cnz<double, KIND>(I[a], J[a], k, l)) s += Cm<double, KIND>(L, p, I[a], J[a], k, l) * e[k][l];
        out[(size_t)a * L.N + p] = s;
    }
}

void launch_stress(const Lv<double>& L, const double* u, const double* eps0, const MeanStrain& mean, double* out,
                   cudaStream_t s) {
    count_launch();
    if (L.K == 2) k_stress<2><<<blocks_for(L.N), kBlock, 0, s>>>(L, u, eps0, mean, out);
    else k_stress<21><<<blocks_for(L.N), kBlock, 0, s>>>(L, u, eps0, mean, out);
}

// ---- ALU peak: independent FMA chains ------------------------------------------------
// Each thread runs kFmaChains independent chains x <- x b + a (b < 1, so the values stay
// bounded) for iters rounds, unrolled by four; nothing else is issued in the loop but
// its counter.  The sum is stored only under a condition the inputs never meet, so the
// chains cannot be removed.  FLOPs per launch: 2 kFmaChains iters x threads.
constexpr int kFmaChains = 16;
template <typename T>
__global__ void __launch_bounds__(256) k_fma_chain(T a, T b, int iters, T* __restrict__ out) {
    T x[kFmaChains];
#pragma unroll
    for (int j = 0; j < kFmaChains; ++j) x[j] = a + T(j) * T(1e-3) + T(threadIdx.x) * T(1e-6);
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kFmaChains; ++j) x[j] = fma(x[j], b, a);
    }
    T sum = T(0);
#pragma unroll
    for (int j = 0; j < kFmaChains; ++j) sum += x[j];
    if (sum == T(-12345)) out[threadIdx.x] = sum;
}

double measure_fma_flops(int precision, int iters, float* ms, void* out, cudaStream_t s) {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * 8, threads = 256;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    count_launch();
    cudaEventRecord(e0, s);
    if (precision == 0) k_fma_chain<double><<<blocks, threads, 0, s>>>(0.5, 0.999, iters, (double*)out);
    else k_fma_chain<float><<<blocks, threads, 0, s>>>(0.5f, 0.999f, iters, (float*)out);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    *ms = 0.f;
    cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return 2.0 * kFmaChains * (double)iters * blocks * threads;
}

// explicit instantiations
template void launch_apply<double>(const Lv<double>&, const double*, double*, cudaStream_t);
template void launch_apply<float>(const Lv<float>&, const float*, float*, cudaStream_t);
template void launch_restrict<double>(const Lv<double>&, const Lv<double>&, const double*, double*, const NullInfo*,
                                      const double*, cudaStream_t);
template void launch_restrict<float>(const Lv<float>&, const Lv<float>&, const float*, float*, const NullInfo*,
                                     const double*, cudaStream_t);
template void launch_prolong_add<double>(const Lv<double>&, const Lv<double>&, const double*, double*, cudaStream_t);
template void launch_prolong_add<float>(const Lv<float>&, const Lv<float>&, const float*, float*, cudaStream_t);
template void launch_restrict_moduli<double>(const Lv<double>&, const Lv<double>&, const double*, double*,
                                             cudaStream_t);
template void launch_bottom_solve<double>(const Lv<double>&, const int*, int, int, const double*, const double*,
                                          double*, double*, cudaStream_t);
template void launch_bottom_solve<float>(const Lv<float>&, const int*, int, int, const double*, const float*, float*,
                                         double*, cudaStream_t);

}  // namespace elas
