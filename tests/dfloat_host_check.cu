// Host driver for tests/test_dfloat_host.py: applies one double-float operation of the
// solver's csrc/elas_dfloat.cuh (the same source the kernels use, compiled for the host
// with round-to-nearest binary32/binary64 and no contraction) to n records read from a
// raw file, and writes the results as raw FP32 / FP64 values.  All checking is done by
// the Python test, with exact rational arithmetic.
//
//   dfloat_host_check <op> <n> <in> <out>
//   op        record in                        record out
//   two_sum   a, b                     (f32)   s, e        (f32)
//   fast_sum  a, b                     (f32)   s, e        (f32)
//   add       x.hi, x.lo, y.hi, y.lo   (f32)   hi, lo      (f32)
//   mul       x.hi, x.lo, y.hi, y.lo   (f32)   hi, lo      (f32)
//   mulf      x.hi, x.lo, y            (f32)   hi, lo      (f32)
//   fma       a.hi, a.lo, b.hi, b.lo, c.hi, c.lo (f32)   hi, lo (f32)
//   dot27     27 pairs a_i, 27 pairs b_i (f32) hi, lo of sum a_i b_i by df_fma (f32)
//   to_float  hi, lo                   (f32)   f           (f32)
//   split     v                        (f64)   hi, lo      (f32)
//   ctor      v                        (f64)   hi, lo      (f32)   (the constant constructor)
//   f2d       x                        (f32)   v           (f64)
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../paper_2001_04789_gb300/csrc/elas_dfloat.cuh"

using elas::dfloat;

template <typename T>
static std::vector<T> read_all(const char* path, size_t count) {
    std::vector<T> v(count);
    FILE* f = std::fopen(path, "rb");
    if (!f || std::fread(v.data(), sizeof(T), count, f) != count) {
        std::fprintf(stderr, "cannot read %zu values from %s\n", count, path);
        std::exit(2);
    }
    std::fclose(f);
    return v;
}

template <typename T>
static void write_all(const char* path, const std::vector<T>& v) {
    FILE* f = std::fopen(path, "wb");
    if (!f || std::fwrite(v.data(), sizeof(T), v.size(), f) != v.size()) {
        std::fprintf(stderr, "cannot write %s\n", path);
        std::exit(2);
    }
    std::fclose(f);
}

static void put(std::vector<float>& out, size_t i, dfloat x) {
    out[2 * i] = x.hi;
    out[2 * i + 1] = x.lo;
}

int main(int argc, char** argv) {
    if (argc != 5) {
        std::fprintf(stderr, "usage: %s op n in out\n", argv[0]);
        return 2;
    }
    const std::string op = argv[1];
    const size_t n = std::strtoull(argv[2], nullptr, 10);
    const char* in = argv[3];
    const char* outp = argv[4];
    std::vector<float> out(2 * n);
    if (op == "two_sum" || op == "fast_sum") {
        auto a = read_all<float>(in, 2 * n);
        for (size_t i = 0; i < n; ++i)
            put(out, i, op == "two_sum" ? elas::df_two_sum(a[2 * i], a[2 * i + 1])
                                        : elas::df_fast_two_sum(a[2 * i], a[2 * i + 1]));
    } else if (op == "add" || op == "mul") {
        auto a = read_all<float>(in, 4 * n);
        for (size_t i = 0; i < n; ++i) {
            const dfloat x(a[4 * i], a[4 * i + 1]), y(a[4 * i + 2], a[4 * i + 3]);
            put(out, i, op == "add" ? elas::df_add(x, y) : elas::df_mul(x, y));
        }
    } else if (op == "mulf") {
        auto a = read_all<float>(in, 3 * n);
        for (size_t i = 0; i < n; ++i) put(out, i, elas::df_mul(dfloat(a[3 * i], a[3 * i + 1]), a[3 * i + 2]));
    } else if (op == "fma") {
        auto a = read_all<float>(in, 6 * n);
        for (size_t i = 0; i < n; ++i) {
            const float* r = &a[6 * i];
            put(out, i, elas::df_fma(dfloat(r[0], r[1]), dfloat(r[2], r[3]), dfloat(r[4], r[5])));
        }
    } else if (op == "dot27") {
        auto a = read_all<float>(in, 108 * n);
        for (size_t i = 0; i < n; ++i) {
            const float* r = &a[108 * i];
            dfloat acc(0.f, 0.f);
            for (int k = 0; k < 27; ++k)
                acc = elas::df_fma(dfloat(r[2 * k], r[2 * k + 1]), dfloat(r[54 + 2 * k], r[55 + 2 * k]), acc);
            put(out, i, acc);
        }
    } else if (op == "to_float") {
        auto a = read_all<float>(in, 2 * n);
        out.resize(n);
        for (size_t i = 0; i < n; ++i) out[i] = elas::df_to_float(dfloat(a[2 * i], a[2 * i + 1]));
    } else if (op == "split" || op == "ctor") {
        auto a = read_all<double>(in, n);
        for (size_t i = 0; i < n; ++i) put(out, i, op == "split" ? elas::df_split(a[i]) : dfloat(a[i]));
    } else if (op == "f2d") {
        auto a = read_all<float>(in, n);
        std::vector<double> o(n);
        for (size_t i = 0; i < n; ++i) o[i] = elas::f2d_bits(a[i]);
        write_all(outp, o);
        return 0;
    } else {
        std::fprintf(stderr, "unknown op %s\n", op.c_str());
        return 2;
    }
    write_all(outp, out);
    return 0;
}
