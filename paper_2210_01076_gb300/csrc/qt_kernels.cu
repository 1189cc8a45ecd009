// qt_kernels.cu -- sm_103a kernels of the qTask hot path.
//
// The state vector (qTask Section II-A) is 2^n amplitudes in HBM, split into
// partitions of 2^p consecutive amplitudes (the paper's blocks, Section
// III-C).  A fused pass applies a sequence of gate ops to every amplitude of
// the partitions on its worklist:
//
//   * one CTA owns one tile: the 2^(lt+nh) amplitudes that share all index
//     bits outside {0..lt-1} u {h_0..h_{nh-1}}.  It loads the tile as 2^nh
//     contiguous runs of 2^lt amplitudes (coalesced), applies every op of the
//     pass in shared memory, and stores it back -- one HBM read and one write
//     per amplitude per pass, however many gates the pass holds;
//   * an op whose controls or diagonal qubit lie outside the tile is uniform
//     over the tile and is skipped or applied as a scalar;
//   * tiles whose high qubits reach into the partition index couple the
//     partitions {q ^ m : m in span(M)} (a "group"); the worklist lists
//     group bases, so full and incremental runs execute identical code per
//     amplitude and give identical bits.
//
// The paper's swap/scale tasks (non-superposition gates) map to the X, ANTI,
// SWAP, DIAG and PHASE ops (no arithmetic or one multiply); its matrix-vector
// tasks (superposition gates) to the DENSE and REAL ops (Section III-C).
//
// Arithmetic policies:
//   ArF64  -- IEEE binary64 (QT_C128)
//   ArF32  -- binary32 (QT_C64)
//   ArDF   -- float-float (QT_C128_DF): each real is hi + lo, two binary32
//             values; products use the exact FMA residual, sums the
//             error-free two-sum (Dekker / Knuth), so every op runs on the
//             FP32 pipes, ~60x the FP64 rate of GB300.
#include <cuda_runtime.h>

#include <cstdint>

#include "qt_arith.cuh"
#include "qt_internal.h"
#include "qt_launch.cuh"

namespace qt {

// ---------------------------------------------------------------- helpers --
// Expand a counter into a tile index by inserting the op's fixed bits.
__device__ __forceinline__ uint32_t expand_fixed(uint32_t k, const DevOp& op) {
    uint32_t i = k;
    for (int f = 0; f < op.nfix; ++f) {
        const uint32_t b = uint32_t(op.fixpos[f]);
        const uint32_t lowm = (1u << b) - 1u;
        i = ((i & ~lowm) << 1) | (i & lowm) | (uint32_t((op.fixval >> f) & 1u) << b);
    }
    return i;
}

template <class A>
__device__ __forceinline__ void apply_op(typename A::amp_t* tile, uint32_t tb, const DevOp& op, uint64_t base) {
    using cx = typename A::cx;
    const uint32_t iters = 1u << (tb - op.nfix);
    switch (op.kind) {
        case OP_DENSE: {
            const cx u00 = A::mat(op, 0), u01 = A::mat(op, 1), u10 = A::mat(op, 2), u11 = A::mat(op, 3);
            const uint32_t tbit = 1u << op.b0;
            for (uint32_t k = threadIdx.x; k < iters; k += blockDim.x) {
                const uint32_t i0 = expand_fixed(k, op), i1 = i0 | tbit;
                const cx x0 = A::ld(tile[i0]), x1 = A::ld(tile[i1]);
                tile[i0] = A::st(A::lin2(u00, x0, u01, x1));
                tile[i1] = A::st(A::lin2(u10, x0, u11, x1));
            }
            break;
        }
        case OP_REAL: {
            const cx u00 = A::mat(op, 0), u01 = A::mat(op, 1), u10 = A::mat(op, 2), u11 = A::mat(op, 3);
            const uint32_t tbit = 1u << op.b0;
            for (uint32_t k = threadIdx.x; k < iters; k += blockDim.x) {
                const uint32_t i0 = expand_fixed(k, op), i1 = i0 | tbit;
                const cx x0 = A::ld(tile[i0]), x1 = A::ld(tile[i1]);
                tile[i0] = A::st(A::lin2r(u00, x0, u01, x1));
                tile[i1] = A::st(A::lin2r(u10, x0, u11, x1));
            }
            break;
        }
        case OP_IREAL: {
            const cx u00 = A::mat(op, 0), u01 = A::mat(op, 1), u10 = A::mat(op, 2), u11 = A::mat(op, 3);
            const uint32_t tbit = 1u << op.b0;
            for (uint32_t k = threadIdx.x; k < iters; k += blockDim.x) {
                const uint32_t i0 = expand_fixed(k, op), i1 = i0 | tbit;
                const cx x0 = A::ld(tile[i0]), x1 = A::ld(tile[i1]);
                tile[i0] = A::st(A::lin2i(u00, x0, u01, x1));
                tile[i1] = A::st(A::lin2i(u11, x1, u10, x0));
            }
            break;
        }
        case OP_X: {
            const uint32_t tbit = 1u << op.b0;
            for (uint32_t k = threadIdx.x; k < iters; k += blockDim.x) {
                const uint32_t i0 = expand_fixed(k, op), i1 = i0 | tbit;
                const typename A::amp_t t0 = tile[i0];
                tile[i0] = tile[i1];
                tile[i1] = t0;
            }
            break;
        }
        case OP_ANTI: {
            const cx m01 = A::mat(op, 0), m10 = A::mat(op, 1);
            const uint32_t tbit = 1u << op.b0;
            for (uint32_t k = threadIdx.x; k < iters; k += blockDim.x) {
                const uint32_t i0 = expand_fixed(k, op), i1 = i0 | tbit;
                const cx x0 = A::ld(tile[i0]), x1 = A::ld(tile[i1]);
                tile[i0] = A::st(A::mul(m01, x1));
                tile[i1] = A::st(A::mul(m10, x0));
            }
            break;
        }
        case OP_SWAP: {
            // fixed bits: q0 = 1, q1 = 0 -> i is the (1,0) index; partner (0,1)
            const uint32_t flip = (1u << op.b0) | (1u << op.b1);
            for (uint32_t k = threadIdx.x; k < iters; k += blockDim.x) {
                const uint32_t ia = expand_fixed(k, op), ib = ia ^ flip;
                const typename A::amp_t t0 = tile[ia];
                tile[ia] = tile[ib];
                tile[ib] = t0;
            }
            break;
        }
        case OP_DIAG: {
            const cx d0 = A::mat(op, 0), d1 = A::mat(op, 1);
            if (op.b0 < 0) {
                const cx d = ((base >> op.gq) & 1) ? d1 : d0;
                for (uint32_t k = threadIdx.x; k < iters; k += blockDim.x) {
                    const uint32_t i = expand_fixed(k, op);
                    tile[i] = A::st(A::mul(d, A::ld(tile[i])));
                }
            } else {
                for (uint32_t k = threadIdx.x; k < iters; k += blockDim.x) {
                    const uint32_t i = expand_fixed(k, op);
                    const cx d = ((i >> op.b0) & 1) ? d1 : d0;
                    tile[i] = A::st(A::mul(d, A::ld(tile[i])));
                }
            }
            break;
        }
        case OP_PHASE: {
            const cx f = A::mat(op, 0);
            const int sub = op.sub;
            for (uint32_t k = threadIdx.x; k < iters; k += blockDim.x) {
                const uint32_t i = expand_fixed(k, op);
                const cx x = A::ld(tile[i]);
                cx y;
                if (sub == PH_NEG) y = A::neg(x);
                else if (sub == PH_POS_I) y = A::mul_i(x);
                else if (sub == PH_NEG_I) y = A::mul_negi(x);
                else y = A::mul(f, x);
                tile[i] = A::st(y);
            }
            break;
        }
        default:
            break;
    }
}

// One CTA per tile.  blockIdx.x = group index * 2^tpg_log2 + tile index.
template <class A>
__global__ void __launch_bounds__(kThreads) k_pass(typename A::amp_t* dst,
                                                    const typename A::amp_t* src, const DevPass dp,
                                                    const DevOp* __restrict__ ops,
                                                    const uint32_t* __restrict__ worklist) {
    using amp_t = typename A::amp_t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    amp_t* tile = reinterpret_cast<amp_t*>(smem_raw);
    __shared__ uint64_t choff[1 << kMaxTileHigh];

    const uint32_t tb = uint32_t(dp.lt + dp.nh);
    const uint32_t T = 1u << tb;
    const uint32_t gi = blockIdx.x >> dp.tpg_log2;
    const uint32_t tau = blockIdx.x & ((1u << dp.tpg_log2) - 1u);
    uint32_t g;
    if (worklist != nullptr) {
        g = worklist[gi];
    } else {
        // gi-th partition index with the coupling bits M cleared
        g = gi;
        uint32_t M = dp.M;
        while (M) {
            const uint32_t b = uint32_t(__ffs(M) - 1);
            M &= M - 1;
            const uint32_t lowm = (1u << b) - 1u;
            g = ((g & ~lowm) << 1) | (g & lowm);
        }
    }
    uint64_t x = uint64_t(tau) << dp.lt;
    for (int k = 0; k < dp.nins; ++k) {
        const uint32_t b = uint32_t(dp.ins[k]);
        const uint64_t lowm = (uint64_t(1) << b) - 1u;
        x = ((x & ~lowm) << 1) | (x & lowm);
    }
    const uint64_t base = (uint64_t(g) << dp.p) | x;
    if (threadIdx.x < (1u << dp.nh)) {
        uint64_t off = 0;
        for (int k = 0; k < dp.nh; ++k)
            if ((threadIdx.x >> k) & 1u) off |= uint64_t(1) << dp.h[k];
        choff[threadIdx.x] = off;
    }
    __syncthreads();
    const uint32_t lowmask = (1u << dp.lt) - 1u;
    for (uint32_t j = threadIdx.x; j < T; j += blockDim.x) tile[j] = src[base | choff[j >> dp.lt] | (j & lowmask)];
    __syncthreads();
    const DevOp* pops = ops + dp.op_offset;
    for (int oi = 0; oi < dp.nops; ++oi) {
        const DevOp op = pops[oi];
        if ((base & op.cm_glob) != op.cm_glob) continue;  // uniform over the CTA
        apply_op<A>(tile, tb, op, base);
        __syncthreads();
    }
    for (uint32_t j = threadIdx.x; j < T; j += blockDim.x) dst[base | choff[j >> dp.lt] | (j & lowmask)] = tile[j];
}

template <class A>
int launch_pass_t(void* dst, const void* src, const DevPass& dp, const DevOp* ops, const uint32_t* worklist,
                  uint32_t ngroups, cudaStream_t st) {
    using amp_t = typename A::amp_t;
    const size_t smem = sizeof(amp_t) << (dp.lt + dp.nh);
    static DeviceOnce attr;
    const int rc = attr.run([](int) {
        return int(cudaFuncSetAttribute(k_pass<A>, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 1024));
    });
    if (rc) return rc;
    const uint64_t nblocks = uint64_t(ngroups) << dp.tpg_log2;
    if (nblocks == 0) return 0;
    if (nblocks > 0x7fffffffull || smem > 128 * 1024) return int(cudaErrorInvalidConfiguration);
    return launch_k(k_pass<A>, dim3(unsigned(nblocks)), dim3(kThreads), smem, st, static_cast<amp_t*>(dst),
                    static_cast<const amp_t*>(src), dp, ops, worklist);
}

int launch_pass(int dtype, void* dst, const void* src, const DevPass& dp, const DevOp* ops, const uint32_t* worklist,
                uint32_t ngroups, int* err, void* stream) {
    if (dp.reg_kernel) return launch_pass_reg(dtype, dst, src, dp, ops, worklist, ngroups, err, stream);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (dtype) {
        case QT_C128: return launch_pass_t<ArF64>(dst, src, dp, ops, worklist, ngroups, st);
        case QT_C64: return launch_pass_t<ArF32>(dst, src, dp, ops, worklist, ngroups, st);
        case QT_C128_DF: return launch_pass_t<ArDF>(dst, src, dp, ops, worklist, ngroups, st);
        default: return int(cudaErrorInvalidValue);
    }
}

size_t bytes_per_amp(int dtype) { return dtype == QT_C64 ? 8 : 16; }

// Host-side encoding of a matrix entry for each arithmetic.
void encode_matrix(int dtype, const HostOp& op, DevOp* out) {
    for (int k = 0; k < 8; ++k) out->m.d[k] = 0.0;
    if (dtype == QT_C128) {
        for (int k = 0; k < 8; ++k) out->m.d[k] = op.m[k];
    } else if (dtype == QT_C64) {
        float f[16] = {0};
        for (int k = 0; k < 8; ++k) f[k] = float(op.m[k]);
        for (int k = 0; k < 16; ++k) out->m.f[k] = f[k];
    } else {
        float f[16];
        for (int k = 0; k < 8; ++k) {
            const float hi = float(op.m[k]);
            const float lo = float(op.m[k] - double(hi));
            f[2 * k] = hi;
            f[2 * k + 1] = lo;
        }
        for (int k = 0; k < 16; ++k) out->m.f[k] = f[k];
    }
}

// ---------------------------------------------------- device properties --
int device_sm_count() {
    static DeviceOnce once;
    static int nsm[DeviceOnce::kMaxDevices];
    const int rc = once.run(
        [](int d) { return int(cudaDeviceGetAttribute(&nsm[d], cudaDevAttrMultiProcessorCount, d)); });
    int dev = 0;
    if (rc || cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= DeviceOnce::kMaxDevices || nsm[dev] < 1)
        return 1;  // only sizes grid-stride loops; the launch itself reports the error
    return nsm[dev];
}

// ------------------------------------------------------- state utilities --
__global__ void k_copy_parts(uint4* __restrict__ dst, const uint4* __restrict__ src, const uint32_t* __restrict__ parts,
                             uint32_t nparts, uint32_t vec_per_part_log2) {
    const uint64_t total = uint64_t(nparts) << vec_per_part_log2;
    for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < total;
         i += uint64_t(gridDim.x) * blockDim.x) {
        const uint64_t pi = i >> vec_per_part_log2;
        const uint64_t off = i & ((uint64_t(1) << vec_per_part_log2) - 1);
        const uint64_t v = (uint64_t(parts[pi]) << vec_per_part_log2) | off;
        dst[v] = src[v];
    }
}

__global__ void k_copy_bytes(unsigned char* __restrict__ dst, const unsigned char* __restrict__ src,
                             const uint32_t* __restrict__ parts, uint32_t nparts, uint32_t bytes_per_part) {
    const uint64_t total = uint64_t(nparts) * bytes_per_part;
    for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < total;
         i += uint64_t(gridDim.x) * blockDim.x) {
        const uint64_t pi = i / bytes_per_part, off = i % bytes_per_part;
        const uint64_t v = uint64_t(parts[pi]) * bytes_per_part + off;
        dst[v] = src[v];
    }
}

int launch_copy_parts(int dtype, void* dst, const void* src, int p, const uint32_t* parts, uint32_t nparts,
                      void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (nparts == 0) return 0;
    const uint64_t bytes = uint64_t(bytes_per_amp(dtype)) << p;
    if (bytes >= 16) {
        const uint32_t vlog2 = uint32_t(p + (dtype == QT_C64 ? 3 : 4) - 4);
        const uint64_t total = uint64_t(nparts) << vlog2;
        const unsigned grid = unsigned(std::min<uint64_t>((total + 255) / 256, uint64_t(device_sm_count()) * 16));
        return launch_k(k_copy_parts, dim3(grid), dim3(256), 0, st, static_cast<uint4*>(dst),
                        static_cast<const uint4*>(src), parts, nparts, vlog2);
    }
    const uint64_t total = uint64_t(nparts) * bytes;
    const unsigned grid = unsigned(std::min<uint64_t>((total + 255) / 256, uint64_t(device_sm_count()) * 16));
    return launch_k(k_copy_bytes, dim3(grid), dim3(256), 0, st, static_cast<unsigned char*>(dst),
                    static_cast<const unsigned char*>(src), parts, nparts, uint32_t(bytes));
}

__global__ void k_set_first_one(void* state, int dtype) {
    if (dtype == QT_C128) {
        static_cast<double2*>(state)[0] = make_double2(1.0, 0.0);
    } else if (dtype == QT_C64) {
        static_cast<float2*>(state)[0] = make_float2(1.0f, 0.0f);
    } else {
        static_cast<float4*>(state)[0] = make_float4(1.0f, 0.0f, 0.0f, 0.0f);
    }
}

int launch_init_zero_state(int dtype, void* state, uint64_t namps, void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(state, 0, namps * bytes_per_amp(dtype), st);
    if (e != cudaSuccess) return int(e);
    return launch_k(k_set_first_one, dim3(1), dim3(1), 0, st, state, dtype);
}

// Float-float to binary64 for reading out QT_C128_DF states (not on the hot path).
__global__ void k_df_to_f64(double2* __restrict__ dst, const float4* __restrict__ src, uint64_t first, uint64_t count) {
    for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < count;
         i += uint64_t(gridDim.x) * blockDim.x) {
        const float4 a = src[first + i];
        dst[i] = make_double2(double(a.x) + double(a.y), double(a.z) + double(a.w));
    }
}

int launch_read_convert(int dtype, void* dst, const void* state, uint64_t first, uint64_t count, void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (count == 0) return 0;
    if (dtype == QT_C128_DF) {
        const unsigned grid = unsigned(std::min<uint64_t>((count + 255) / 256, uint64_t(device_sm_count()) * 16));
        return launch_k(k_df_to_f64, dim3(grid), dim3(256), 0, st, static_cast<double2*>(dst),
                        static_cast<const float4*>(state), first, count);
    }
    const size_t b = bytes_per_amp(dtype);
    return int(cudaMemcpyAsync(dst, static_cast<const char*>(state) + first * b, count * b, cudaMemcpyDeviceToDevice,
                               st));
}

// --------------------------------------------------------------- norm -----
// sum |a|^2 with float-float per-thread accumulation (exact squares by FMA),
// binary64 block tree, one partial per block, then a binary64 final sum.
constexpr int kNormThreads = 256;

__device__ __forceinline__ void df_acc_sq(df& acc, float h, float l) {
    // (h + l)^2 ~= h*h + 2*h*l, with h*h split exactly
    const float p = __fmul_rn(h, h);
    float e = __fmaf_rn(h, h, -p);
    e = __fmaf_rn(__fmul_rn(2.0f, h), l, e);
    const df t = two_sum(acc.hi, p);
    acc = fast_two_sum(t.hi, __fadd_rn(acc.lo, __fadd_rn(t.lo, e)));
}

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[kNormThreads / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kNormThreads / 32; ++w) s += red[w];
    return s;
}

template <int DT>
__global__ void __launch_bounds__(kNormThreads) k_norm_partial(const void* __restrict__ state, uint64_t namps,
                                                                double* __restrict__ partials) {
    double v = 0.0;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    if (DT == QT_C128) {
        const double2* s = static_cast<const double2*>(state);
        for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < namps; i += stride) {
            const double2 a = s[i];
            v = __fma_rn(a.x, a.x, __fma_rn(a.y, a.y, v));
        }
    } else {
        df acc = {0.0f, 0.0f};
        if (DT == QT_C64) {
            const float2* s = static_cast<const float2*>(state);
            for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < namps; i += stride) {
                const float2 a = s[i];
                df_acc_sq(acc, a.x, 0.0f);
                df_acc_sq(acc, a.y, 0.0f);
            }
        } else {
            const float4* s = static_cast<const float4*>(state);
            for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < namps; i += stride) {
                const float4 a = s[i];
                df_acc_sq(acc, a.x, a.y);
                df_acc_sq(acc, a.z, a.w);
            }
        }
        v = double(acc.hi) + double(acc.lo);
    }
    const double s = block_sum(v);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kNormThreads) k_norm_final(const double* __restrict__ partials, int n,
                                                              double* __restrict__ out) {
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v += partials[i];
    const double s = block_sum(v);
    if (threadIdx.x == 0) *out = s;
}

int norm_partials_needed(uint64_t namps) {
    const uint64_t blocks = (namps + kNormThreads - 1) / kNormThreads;
    const uint64_t cap = std::min<uint64_t>(uint64_t(device_sm_count()) * 8, kMaxNormPartials);
    return int(std::min<uint64_t>(std::max<uint64_t>(blocks, 1), cap));
}

int launch_norm(int dtype, const void* state, uint64_t namps, double* partials, int npartials, double* out_dev,
                void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (npartials < 1 || npartials > kMaxNormPartials) return int(cudaErrorInvalidConfiguration);
    void (*kp)(const void*, uint64_t, double*) = dtype == QT_C128 ? k_norm_partial<QT_C128>
                                                 : dtype == QT_C64 ? k_norm_partial<QT_C64>
                                                                   : k_norm_partial<QT_C128_DF>;
    const int rc = launch_k(kp, dim3(npartials), dim3(kNormThreads), 0, st, state, namps, partials);
    if (rc) return rc;
    return launch_k(k_norm_final, dim3(1), dim3(kNormThreads), 0, st, static_cast<const double*>(partials),
                    npartials, out_dev);
}

}  // namespace qt
