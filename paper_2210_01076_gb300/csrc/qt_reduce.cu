// qt_reduce.cu -- FP64-class reductions over device states: the fidelity
// |<a|b>|^2 of two states and the probabilities of the values of a few qubits
// (squared amplitudes are the probabilities of the basis states, qTask
// Section II-A).  Any dtype on either side: each amplitude is read as a
// float-float pair (binary32 exactly; float-float as stored; binary64 split
// into hi + lo), products are split exactly with an FMA and accumulated with
// two-sum per thread, and the per-thread results are reduced in binary64.
#include <cuda_runtime.h>

#include <cstdint>

#include "qt_arith.cuh"
#include "qt_internal.h"
#include "qt_launch.cuh"

namespace qt {

namespace {

constexpr int kRedThreads = 256;

template <int DT>
__device__ __forceinline__ void load_df(const void* s, uint64_t i, df& re, df& im) {
    if constexpr (DT == QT_C64) {
        const float2 a = static_cast<const float2*>(s)[i];
        re = {a.x, 0.0f};
        im = {a.y, 0.0f};
    } else if constexpr (DT == QT_C128_DF) {
        const float4 a = static_cast<const float4*>(s)[i];
        re = {a.x, a.y};
        im = {a.z, a.w};
    } else {
        const double2 a = static_cast<const double2*>(s)[i];
        const float rh = __double2float_rn(a.x), ih = __double2float_rn(a.y);
        re = {rh, __double2float_rn(a.x - double(rh))};
        im = {ih, __double2float_rn(a.y - double(ih))};
    }
}

// acc += sign * a * b, with the leading product split exactly
__device__ __forceinline__ void acc_prod(df& acc, df a, df b, float sign) {
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    p = __fmul_rn(sign, p);
    e = __fmul_rn(sign, e);
    const df t = two_sum(acc.hi, p);
    acc = fast_two_sum(t.hi, __fadd_rn(acc.lo, __fadd_rn(t.lo, e)));
}

__device__ __forceinline__ double to_double(df a) { return double(a.hi) + double(a.lo); }

__device__ __forceinline__ double block_sum_d(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kRedThreads / 32; ++w) s += red[w];
    return s;
}

template <int DA, int DB>
__global__ void __launch_bounds__(kRedThreads) k_fid_partial(const void* __restrict__ a, const void* __restrict__ b,
                                                             uint64_t n, double* __restrict__ partials) {
    __shared__ double red[kRedThreads / 32];
    df sre = {0.0f, 0.0f}, sim = {0.0f, 0.0f}, na = {0.0f, 0.0f}, nb = {0.0f, 0.0f};
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n; i += stride) {
        df ar, ai, br, bi;
        load_df<DA>(a, i, ar, ai);
        load_df<DB>(b, i, br, bi);
        // conj(a) b = (ar br + ai bi) + i (ar bi - ai br)
        acc_prod(sre, ar, br, 1.0f);
        acc_prod(sre, ai, bi, 1.0f);
        acc_prod(sim, ar, bi, 1.0f);
        acc_prod(sim, ai, br, -1.0f);
        acc_prod(na, ar, ar, 1.0f);
        acc_prod(na, ai, ai, 1.0f);
        acc_prod(nb, br, br, 1.0f);
        acc_prod(nb, bi, bi, 1.0f);
    }
    const double v[4] = {to_double(sre), to_double(sim), to_double(na), to_double(nb)};
    for (int k = 0; k < 4; ++k) {
        const double s = block_sum_d(v[k], red);
        if (threadIdx.x == 0) partials[4 * blockIdx.x + k] = s;
    }
}

// |a_i - b_i|^2 in binary64: every dtype converts exactly enough (binary32
// exactly, float-float as hi + lo rounded once, binary64 as is) that the
// difference of two states within 1e-12 of each other is resolved.
template <int DT>
__device__ __forceinline__ void load_f64(const void* s, uint64_t i, double& re, double& im) {
    if constexpr (DT == QT_C64) {
        const float2 a = static_cast<const float2*>(s)[i];
        re = double(a.x);
        im = double(a.y);
    } else if constexpr (DT == QT_C128_DF) {
        const float4 a = static_cast<const float4*>(s)[i];
        re = double(a.x) + double(a.y);
        im = double(a.z) + double(a.w);
    } else {
        const double2 a = static_cast<const double2*>(s)[i];
        re = a.x;
        im = a.y;
    }
}

__device__ __forceinline__ double block_max_d(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kRedThreads / 32; ++w) s = fmax(s, red[w]);
    return s;
}

// per block: max over its amplitudes of |a_i - b_i|^2
template <int DA, int DB>
__global__ void __launch_bounds__(kRedThreads) k_maxdiff_partial(const void* __restrict__ a,
                                                                 const void* __restrict__ b, uint64_t n,
                                                                 double* __restrict__ partials) {
    __shared__ double red[kRedThreads / 32];
    double m = 0.0;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n; i += stride) {
        double ar, ai, br, bi;
        load_f64<DA>(a, i, ar, ai);
        load_f64<DB>(b, i, br, bi);
        const double dr = ar - br, di = ai - bi;
        m = fmax(m, dr * dr + di * di);
    }
    const double s = block_max_d(m, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kRedThreads) k_max_final(const double* __restrict__ partials, int nrows,
                                                          double* __restrict__ out) {
    __shared__ double red[kRedThreads / 32];
    double m = 0.0;
    for (int r = threadIdx.x; r < nrows; r += blockDim.x) m = fmax(m, partials[r]);
    const double s = block_max_d(m, red);
    if (threadIdx.x == 0) *out = s;
}

__global__ void k_sum_columns(const double* __restrict__ partials, int nrows, int ncols, double* __restrict__ out) {
    for (int col = blockIdx.x * blockDim.x + threadIdx.x; col < ncols; col += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int r = 0; r < nrows; ++r) s += partials[size_t(r) * ncols + col];
        out[col] = s;
    }
}

template <int DT>
__global__ void __launch_bounds__(kRedThreads) k_prob_partial(const void* __restrict__ s, uint64_t n,
                                                              QubitList ql, double* __restrict__ partials) {
    extern __shared__ double bins[];
    const int nb = 1 << ql.k;
    for (int j = threadIdx.x; j < nb; j += blockDim.x) bins[j] = 0.0;
    __syncthreads();
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n; i += stride) {
        df re, im, p = {0.0f, 0.0f};
        load_df<DT>(s, i, re, im);
        acc_prod(p, re, re, 1.0f);
        acc_prod(p, im, im, 1.0f);
        uint32_t bin = 0;
        for (int j = 0; j < ql.k; ++j) bin |= uint32_t((i >> ql.q[j]) & 1u) << j;
        atomicAdd(&bins[bin], to_double(p));
    }
    __syncthreads();
    for (int j = threadIdx.x; j < nb; j += blockDim.x) partials[size_t(blockIdx.x) * nb + j] = bins[j];
}

template <int DA>
int launch_fid_a(int db, const void* a, const void* b, uint64_t n, double* partials, int nblocks, cudaStream_t st) {
    void (*k)(const void*, const void*, uint64_t, double*) = db == QT_C128  ? k_fid_partial<DA, QT_C128>
                                                            : db == QT_C64 ? k_fid_partial<DA, QT_C64>
                                                                           : k_fid_partial<DA, QT_C128_DF>;
    return launch_k(k, dim3(nblocks), dim3(kRedThreads), 0, st, a, b, n, partials);
}

template <int DA>
int launch_maxdiff_a(int db, const void* a, const void* b, uint64_t n, double* partials, int nblocks,
                     cudaStream_t st) {
    void (*k)(const void*, const void*, uint64_t, double*) = db == QT_C128  ? k_maxdiff_partial<DA, QT_C128>
                                                            : db == QT_C64 ? k_maxdiff_partial<DA, QT_C64>
                                                                           : k_maxdiff_partial<DA, QT_C128_DF>;
    return launch_k(k, dim3(nblocks), dim3(kRedThreads), 0, st, a, b, n, partials);
}

}  // namespace

int launch_max_sq_diff(int da, const void* a, int db, const void* b, uint64_t n, double* partials, int nblocks,
                       double* out, void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc;
    switch (da) {
        case QT_C128: rc = launch_maxdiff_a<QT_C128>(db, a, b, n, partials, nblocks, st); break;
        case QT_C64: rc = launch_maxdiff_a<QT_C64>(db, a, b, n, partials, nblocks, st); break;
        default: rc = launch_maxdiff_a<QT_C128_DF>(db, a, b, n, partials, nblocks, st); break;
    }
    if (rc) return rc;
    return launch_k(k_max_final, dim3(1), dim3(kRedThreads), 0, st, static_cast<const double*>(partials), nblocks,
                    out);
}

int reduce_blocks(uint64_t n) {
    const uint64_t blocks = (n + kRedThreads - 1) / kRedThreads;
    return int(std::min<uint64_t>(std::max<uint64_t>(blocks, 1), uint64_t(device_sm_count()) * 4));
}

int launch_fidelity(int da, const void* a, int db, const void* b, uint64_t n, double* partials, int nblocks,
                    double* out4, void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc;
    switch (da) {
        case QT_C128: rc = launch_fid_a<QT_C128>(db, a, b, n, partials, nblocks, st); break;
        case QT_C64: rc = launch_fid_a<QT_C64>(db, a, b, n, partials, nblocks, st); break;
        default: rc = launch_fid_a<QT_C128_DF>(db, a, b, n, partials, nblocks, st); break;
    }
    if (rc) return rc;
    return launch_k(k_sum_columns, dim3(1), dim3(32), 0, st, static_cast<const double*>(partials), nblocks, 4, out4);
}

int launch_probabilities(int dtype, const void* s, uint64_t n, const QubitList& ql, double* partials, int nblocks,
                         double* out, void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int nb = 1 << ql.k;
    const size_t smem = sizeof(double) * nb;
    void (*k)(const void*, uint64_t, QubitList, double*) = dtype == QT_C128  ? k_prob_partial<QT_C128>
                                                           : dtype == QT_C64 ? k_prob_partial<QT_C64>
                                                                             : k_prob_partial<QT_C128_DF>;
    const int rc = launch_k(k, dim3(nblocks), dim3(kRedThreads), smem, st, s, n, ql, partials);
    if (rc) return rc;
    return launch_k(k_sum_columns, dim3((nb + 255) / 256), dim3(256), 0, st, static_cast<const double*>(partials),
                    nblocks, nb, out);
}

}  // namespace qt
