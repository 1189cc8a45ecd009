// qt_pass_reg.cu -- register-resident fused pass (tiles of 2^7..2^13 amplitudes).
//
// Same contract as the shared-memory pass of qt_kernels.cu (one CTA per tile
// of the worklist's partition groups, one HBM read and one write per
// amplitude per pass), but every thread keeps its 2^RB amplitudes of the tile
// in registers for the whole pass:
//
//   tile index j = lane bits (j bits 0..4, the lane id) | register bits
//                  (register index r) | warp bits (warp id)
//
// so a warp always holds 32 consecutive amplitudes (coalesced loads and
// stores, conflict-free shared memory).  An op whose target is a lane bit
// exchanges the partner amplitude with a warp shuffle (the low-stride
// qubits).  An op whose target is register bit k first exchanges register
// bits 0 and k (register moves, resolved at compile time) so that one copy of
// each op's code serves every register bit, which keeps the kernel small
// enough for the instruction cache.  Before an op whose target is a warp bit
// the host inserts an OP_PERM, which rewrites the layout through shared
// memory (one read and one write of the tile).  Diagonal ops, phases and
// controls need no particular layout: each thread knows the index of every
// amplitude it holds.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "qt_arith.cuh"
#include "qt_internal.h"
#include "qt_launch.cuh"
#include "qt_tc.cuh"

// This file is compiled twice: as itself, with the kernels that have no
// merged phase groups (RC_PH_GROUP) and the library's entry points, and from
// qt_pass_grp.cu with QT_PASS_PHASE_GROUPS = 1, the same kernels with group
// support (a separate instantiation, so that passes without groups run code
// that has none).
#ifndef QT_PASS_PHASE_GROUPS
#define QT_PASS_PHASE_GROUPS 0
#endif

namespace qt {

template <int V>
struct IC {
    static constexpr int value = V;
};

// Call f(IC<k>) for a runtime k in [0, RB).
template <int RB, class F>
__device__ __forceinline__ void dispatch_k(int k, F&& f) {
    if (k == 0) {
        f(IC<0>{});
    } else if (k == 1) {
        f(IC<1>{});
    } else if constexpr (RB > 2) {
        if (k == 2) {
            f(IC<2>{});
        } else if constexpr (RB > 3) {
            if (k == 3) {
                f(IC<3>{});
            } else if constexpr (RB > 4) {
                if (k == 4) f(IC<4>{});
            }
        }
    }
}

template <class A, int RB>
struct RegOps {
    using cx = typename A::cx;
    static constexpr int R = 1 << RB;

    // exchange register-index bits 0 and K (K > 0).  Moved values go through
    // A::mv, a copy that issues on the FMA pipe (see qt_arith.cuh).
    template <int K>
    static __device__ __forceinline__ void swap_bits(cx (&x)[R]) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if ((r & 1) && !((r >> K) & 1)) {
                const int r2 = r ^ (1 | (1 << K));
                const cx t = x[r];
                x[r] = A::mv(x[r2]);
                x[r2] = A::mv(t);
            }
        }
    }

    // one-target ops on register bit 0: pairs (x[2i], x[2i+1]).  DENSE, REAL,
    // IREAL and ANTI ops never carry conditions (only X, SWAP and PHASE do; the
    // host checks it), so their loops need no per-amplitude predicate.
    template <int KIND>
    static __device__ __forceinline__ void pair_reg0(cx (&x)[R], const DevOp* op) {
        if constexpr (KIND == OP_DENSE) {
            const cx u00 = A::matp(op, 0), u01 = A::matp(op, 1), u10 = A::matp(op, 2), u11 = A::matp(op, 3);
#pragma unroll
            for (int r = 0; r < R; r += 2) {
                const cx a = x[r], b = x[r + 1];
                x[r] = A::lin2(u00, a, u01, b);
                x[r + 1] = A::lin2(u10, a, u11, b);
            }
        } else if constexpr (KIND == OP_REAL) {
            const cx u00 = A::matp(op, 0), u01 = A::matp(op, 1), u10 = A::matp(op, 2), u11 = A::matp(op, 3);
#pragma unroll
            for (int r = 0; r < R; r += 2) {
                const cx a = x[r], b = x[r + 1];
                x[r] = A::lin2r(u00, a, u01, b);
                x[r + 1] = A::lin2r(u10, a, u11, b);
            }
        } else if constexpr (KIND == OP_IREAL) {
            const cx u00 = A::matp(op, 0), u01 = A::matp(op, 1), u10 = A::matp(op, 2), u11 = A::matp(op, 3);
#pragma unroll
            for (int r = 0; r < R; r += 2) {
                const cx a = x[r], b = x[r + 1];
                x[r] = A::lin2i(u00, a, u01, b);
                x[r + 1] = A::lin2i(u11, b, u10, a);
            }
        } else {  // OP_ANTI
            const cx m01 = A::matp(op, 0), m10 = A::matp(op, 1);
#pragma unroll
            for (int r = 0; r < R; r += 2) {
                const cx a = x[r], b = x[r + 1];
                x[r] = A::mul(m01, b);
                x[r + 1] = A::mul(m10, a);
            }
        }
    }

    // a dense 2x2 on register bit K > 0: pairs (x[r], x[r | 2^K]) in place
    template <int K>
    static __device__ __forceinline__ void dense_regk(cx (&x)[R], const DevOp* op) {
        const cx u00 = A::matp(op, 0), u01 = A::matp(op, 1), u10 = A::matp(op, 2), u11 = A::matp(op, 3);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if ((r >> K) & 1) continue;
            const int r1 = r | (1 << K);
            const cx a = x[r], b = x[r1];
            x[r] = A::lin2(u00, a, u01, b);
            x[r1] = A::lin2(u10, a, u11, b);
        }
    }

    static __device__ __forceinline__ void x_reg0(cx (&x)[R], bool thr_ok, uint32_t cmr, uint32_t cvr) {
#pragma unroll
        for (int r = 0; r < R; r += 2) {
            if (!(thr_ok && ((uint32_t(r) ^ cvr) & cmr) == cmr)) continue;
            const cx a = x[r];
            x[r] = A::mv(x[r + 1]);
            x[r + 1] = A::mv(a);
        }
    }

    // one-target ops on lane bit b: the partner amplitude p comes from lane ^
    // 2^b.  A lane whose bit is 0 computes u00 x + u01 p, a lane whose bit is
    // 1 computes u11 x + u10 p: the coefficients are chosen once per op.
    template <int KIND>
    static __device__ __forceinline__ void pair_lane(cx (&x)[R], const DevOp* op, int b, uint32_t lane) {
        const int mask = 1 << b;
        const int hi = int((lane >> b) & 1u);
        if constexpr (KIND == OP_DENSE || KIND == OP_REAL || KIND == OP_IREAL) {
            const cx cs = A::sel(hi, A::matp(op, 3), A::matp(op, 0));
            const cx cp = A::sel(hi, A::matp(op, 2), A::matp(op, 1));
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const cx p = A::shfl(x[r], mask);
                if constexpr (KIND == OP_DENSE) x[r] = A::lin2(cs, x[r], cp, p);
                else if constexpr (KIND == OP_REAL) x[r] = A::lin2r(cs, x[r], cp, p);
                else x[r] = A::lin2i(cs, x[r], cp, p);
            }
        } else {  // OP_ANTI: bit-0 output m01 a1, bit-1 output m10 a0
            const cx c = A::sel(hi, A::matp(op, 1), A::matp(op, 0));
#pragma unroll
            for (int r = 0; r < R; ++r) x[r] = A::mul(c, A::shfl(x[r], mask));
        }
    }

    static __device__ __forceinline__ void x_lane(cx (&x)[R], int b, bool thr_ok, uint32_t cmr, uint32_t cvr) {
        const int mask = 1 << b;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const cx p = A::shfl(x[r], mask);
            if (thr_ok && ((uint32_t(r) ^ cvr) & cmr) == cmr) x[r] = p;
        }
    }

    // SWAP on register bits K0 < K1: exchange (bit K0, bit K1) = (1,0) and (0,1)
    template <int K0, int K1>
    static __device__ __forceinline__ void swap_rr(cx (&x)[R], bool thr_ok, uint32_t cmr, uint32_t cvr) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (!((r >> K0) & 1) || ((r >> K1) & 1)) continue;
            const int r2 = r ^ ((1 << K0) | (1 << K1));
            if (!(thr_ok && ((uint32_t(r) ^ cvr) & cmr) == cmr)) continue;
            const cx a = x[r];
            x[r] = A::mv(x[r2]);
            x[r2] = A::mv(a);
        }
    }

    // SWAP of lane bit b with register bit K
    template <int K>
    static __device__ __forceinline__ void swap_lr(cx (&x)[R], int b, uint32_t lane, bool thr_ok, uint32_t cmr,
                                                   uint32_t cvr) {
        const int mask = 1 << b;
        const bool lb = (lane >> b) & 1u;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (r & (1 << K)) continue;
            const int r1 = r | (1 << K);
            // (lane bit, reg bit) of x[r] is (lb, 0), of x[r1] (lb, 1); the
            // partner of (1,0) is (0,1) at lane ^ b, register r1, and back
            const cx from_r1 = A::shfl(x[r1], mask);
            const cx from_r = A::shfl(x[r], mask);
            if (!(thr_ok && ((uint32_t(r) ^ cvr) & cmr) == cmr)) continue;
            if (lb) x[r] = from_r1;
            else x[r1] = from_r;
        }
    }

    // SWAP of two lane bits
    static __device__ __forceinline__ void swap_ll(cx (&x)[R], int b0, int b1, uint32_t lane, bool thr_ok,
                                                   uint32_t cmr, uint32_t cvr) {
        const int mask = (1 << b0) | (1 << b1);
        const bool differ = ((lane >> b0) ^ (lane >> b1)) & 1u;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const cx p = A::shfl(x[r], mask);
            if (differ && thr_ok && ((uint32_t(r) ^ cvr) & cmr) == cmr) x[r] = p;
        }
    }

    // diag(d0, d1) on a qubit whose value is the same for all of the
    // thread's amplitudes (tbit), or is bit k of the register index
    static __device__ __forceinline__ void diag_u(cx (&x)[R], const DevOp* op, int tbit) {
        const cx d = A::sel(tbit, A::matp(op, 1), A::matp(op, 0));
#pragma unroll
        for (int r = 0; r < R; ++r) x[r] = A::mul(d, x[r]);
    }

    static __device__ __forceinline__ void diag_r(cx (&x)[R], const DevOp* op, int k) {
#pragma unroll
        for (int r = 0; r < R; ++r) x[r] = A::mul(A::matp(op, (r >> k) & 1), x[r]);
    }

    // multiply all the thread's amplitudes (mcls 0) or those whose register
    // index has bit k set (mcls 1) by f
    template <class F>
    static __device__ __forceinline__ void apply01(cx (&x)[R], int mcls, int k, F&& f) {
        if (mcls == 0) {
#pragma unroll
            for (int r = 0; r < R; ++r) x[r] = f(x[r]);
        } else {
            dispatch_k<RB>(k, [&](auto kc) {
                constexpr int K = decltype(kc)::value;
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if ((r >> K) & 1) x[r] = f(x[r]);
            });
        }
    }

    // multiply the amplitudes whose conditions hold by the phase; with one
    // unflipped register condition bit (mcls 1, bit k) the registers that
    // cannot qualify are skipped at compile time
    template <class F>
    static __device__ __forceinline__ void masked(cx (&x)[R], int mcls, int k, uint32_t cmr, uint32_t cvr, F&& f) {
        if (mcls == 0) {
#pragma unroll
            for (int r = 0; r < R; ++r) x[r] = f(x[r]);
        } else if (mcls == 1) {
            dispatch_k<RB>(k, [&](auto kc) {
                constexpr int K = decltype(kc)::value;
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if ((r >> K) & 1) x[r] = f(x[r]);
            });
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (((uint32_t(r) ^ cvr) & cmr) == cmr) x[r] = f(x[r]);
        }
    }
};

// Index of the first amplitude of tile t: the partition group base (from the
// worklist, or the t-th group when the worklist is null) and the tile
// counter deposited into the partition bits that are not tile bits.
__device__ __forceinline__ uint64_t tile_base(const DevPass& dp, const uint32_t* __restrict__ worklist, uint32_t t) {
    const uint32_t gi = t >> dp.tpg_log2;
    const uint32_t tau = t & ((1u << dp.tpg_log2) - 1u);
    uint32_t g;
    if (worklist != nullptr) {
        g = worklist[gi];
    } else {
        g = gi;  // gi-th partition index with the coupling bits M cleared
        uint32_t M = dp.M;
        while (M) {
            const uint32_t b = uint32_t(__ffs(M) - 1);
            M &= M - 1;
            const uint32_t lowm = (1u << b) - 1u;
            g = ((g & ~lowm) << 1) | (g & lowm);
        }
    }
    uint64_t xb = uint64_t(tau) << dp.lt;
#pragma unroll
    for (int k = 0; k < kMaxTileHigh; ++k) {
        if (k < dp.nins) {
            const uint32_t b = uint32_t(dp.ins[k]);
            const uint64_t lowm = (uint64_t(1) << b) - 1u;
            xb = ((xb & ~lowm) << 1) | (xb & lowm);
        }
    }
    return (uint64_t(g) << dp.p) | xb;
}

// Offsets of the tile's 2^nh contiguous runs (chunks) of 2^lt amplitudes.
__device__ __forceinline__ void chunk_offsets(const DevPass& dp, uint64_t* choff) {
    for (uint32_t c = threadIdx.x; c < (1u << dp.nh); c += blockDim.x) {
        uint64_t off = 0;
#pragma unroll
        for (int k = 0; k < kMaxTileHigh; ++k)
            if (k < dp.nh && ((c >> k) & 1u)) off |= uint64_t(1) << dp.h[k];
        choff[c] = off;
    }
}

// Tile index of each of a thread's amplitudes in one layout: the bits held
// by the lane and warp ids (with the flip applied) and one tile bit per
// register-index bit.  The lane, register and warp bits hold disjoint tile
// bits, so the index of register r is thr xor the bits of r's set register
// bits.
template <int RB>
struct TileMap {
    uint32_t thr;
    uint32_t rb[RB];
    __device__ __forceinline__ uint32_t idx(int r) const {
        uint32_t j = thr;
#pragma unroll
        for (int k = 0; k < RB; ++k)
            if ((r >> k) & 1) j ^= rb[k];
        return j;
    }
};

// XOR of the amplitude-index offsets of the register-index bits of r
template <int RB>
__device__ __forceinline__ uint64_t reg_offset(const uint64_t (&off)[kMaxRegBits], int r) {
    uint64_t o = 0;
#pragma unroll
    for (int k = 0; k < RB; ++k)
        if ((r >> k) & 1) o ^= off[k];
    return o;
}

// lanes == nullptr: lane bit i holds tile bit i.
template <int RB, class T>
__device__ __forceinline__ TileMap<RB> tile_map(const int8_t* lanes, const T* regs, const T* warps, int nwarp,
                                                uint32_t flip, uint32_t lane, uint32_t wid) {
    TileMap<RB> m;
    uint32_t t = 0;
    if (lanes == nullptr) {
        t = lane;
    } else {
#pragma unroll
        for (int i = 0; i < 5; ++i) t |= ((lane >> i) & 1u) << lanes[i];
    }
#pragma unroll
    for (int w = 0; w < 3; ++w)
        if (w < nwarp) t |= ((wid >> w) & 1u) << warps[w];
    m.thr = t ^ flip;
#pragma unroll
    for (int k = 0; k < RB; ++k) m.rb[k] = 1u << regs[k];
    return m;
}

template <int RB>
__device__ __forceinline__ TileMap<RB> initial_map(const DevPass& dp, uint32_t lane, uint32_t wid) {
    return tile_map<RB>(nullptr, dp.layout, dp.layout + RB, dp.nwarp, 0u, lane, wid);
}

template <int RB>
__device__ __forceinline__ TileMap<RB> layout_map(const TileLayout& L, int nwarp, uint32_t lane, uint32_t wid) {
    return tile_map<RB>(L.lane, L.reg, L.warp, nwarp, L.flip, lane, wid);
}

// ------------------------------------------- mbarriers and bulk copies --
// (the TMA-staged variant below and the tensor-core block op)
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > 1000000000ull) return false;
    return true;
}

__device__ __forceinline__ void bulk_g2s(void* dst_smem, const void* src_gmem, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Apply the pass's ops to the thread's registers x.  The host resolved
// every op against the layout it runs in; the kernel needs a layout only at
// OP_PERM, which carries the old one.  `tile` is the shared-memory buffer
// for layout changes.  Every thread of the CTA must call this.
// State of the tensor-core block op (complex64 kernel with MMA support):
// shared-memory operands (A: the tile split into tf32 hi and lo, 2 x 32 KB;
// B: the block's operand, 32 KB, both 1024-byte aligned), the two mbarriers
// (operand B landed; the MMAs completed) with this thread's phase bits, the
// accumulator's tensor-memory address and the error flag.
struct MmaCtx {
    unsigned char* a_sm;
    unsigned char* b_sm;
    uint64_t* bar_b;
    uint64_t* bar_m;
    uint32_t* s_ok;
    const unsigned char* blk;
    int* err;
    uint32_t tmem;
    uint32_t ph_b, ph_m;
    bool pending;    // MMAs issued whose completion has not been seen
    bool abort;
    bool tile_read;  // a layout change read the A region since the last barrier
};

// The tensor-core block op: the tile (in registers, any layout) is written
// to shared memory as operand A -- row = the seven tile bits outside the
// block, columns = the block's 32 amplitudes (re, im), each value split into
// tf32 hi and lo -- while one thread brings the block's operand B in with
// bulk copies; one thread then issues the 3 x 8 MMAs (Ah Bh + Ah Bl + Al Bh
// over K = 64 in steps of 8) and commits them to an mbarrier; every thread
// waits and reads its row's 32 accumulator columns back from tensor memory:
// warps 0-3 (TMEM lanes 32 w ..) columns 0-31 (block bit 4 = 0), warps 4-7
// columns 32-63.  That fixes the layout after the op (BlockStage).  Every
// wait is bounded; on expiry the op raises the error flag and the kernel
// stops applying ops.  Returns false when aborted.
template <class A, int RB>
__device__ __forceinline__ bool mma_block(typename A::cx (&x)[1 << RB], const DevOp* op, uint32_t lane, uint32_t wid,
                                          MmaCtx* mc) {
    static_assert(RB == 4 && sizeof(typename A::amp_t) == 8, "tensor-core blocks: complex64 tiles of 4096");
    constexpr int R = 1 << RB;
    const BlockStage& bs = *reinterpret_cast<const BlockStage*>(&op->m);
    // A layout change since the last barrier may still be reading the A
    // region (its buffer); the previous block's accumulator reads are
    // ordered by the barrier before the MMAs are issued.
    if (mc->tile_read) __syncthreads();
    mc->tile_read = false;
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(mc->bar_b, uint32_t(kBlockBytes));
        const unsigned char* src = mc->blk + bs.boff;
#pragma unroll
        for (int q = 0; q < 4; ++q) bulk_g2s(mc->b_sm + q * 8192, src + q * 8192, 8192u, mc->bar_b);
    }
    // byte offset of each register's amplitude in operand A: XOR of the
    // contributions of the thread's set lane and warp bits, the flip and the
    // register's set bits
    uint32_t at = bs.a_flip;
#pragma unroll
    for (int i = 0; i < 5; ++i)
        if ((lane >> i) & 1u) at ^= bs.a_lane[i];
#pragma unroll
    for (int w = 0; w < 3; ++w)
        if ((wid >> w) & 1u) at ^= bs.a_warp[w];
    uint32_t ar[RB];
#pragma unroll
    for (int k = 0; k < RB; ++k) ar[k] = bs.a_reg[k];
    unsigned char* a_hi = mc->a_sm;
    unsigned char* a_lo = mc->a_sm + 32768;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        uint32_t off = at;
#pragma unroll
        for (int k = 0; k < RB; ++k)
            if ((r >> k) & 1) off ^= ar[k];
        const float rh = tc::to_tf32(x[r].re), ih = tc::to_tf32(x[r].im);
        *reinterpret_cast<float2*>(a_hi + off) = make_float2(rh, ih);
        *reinterpret_cast<float2*>(a_lo + off) =
            make_float2(tc::to_tf32(__fsub_rn(x[r].re, rh)), tc::to_tf32(__fsub_rn(x[r].im, ih)));
    }
    tc::fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
        const bool landed = mbar_wait_bounded(mc->bar_b, mc->ph_b);
        if (landed) {
            tc::fence_after_sync();
            constexpr uint32_t idesc = tc::idesc_tf32(128, 64);
            const uint32_t ah = tc::saddr(a_hi), al = tc::saddr(a_lo);
            const uint32_t bh = tc::saddr(mc->b_sm), bl = bh + 16384u;
#pragma unroll
            for (int s = 0; s < 8; ++s) {
                const uint32_t ka = uint32_t(s >> 2) * 16384u + uint32_t(s & 3) * 32u;
                const uint32_t kb = uint32_t(s >> 2) * 8192u + uint32_t(s & 3) * 32u;
                tc::mma_tf32(mc->tmem, tc::sdesc_sw128(ah + ka), tc::sdesc_sw128(bh + kb), idesc, s > 0 ? 1u : 0u);
                tc::mma_tf32(mc->tmem, tc::sdesc_sw128(ah + ka), tc::sdesc_sw128(bl + kb), idesc, 1u);
                tc::mma_tf32(mc->tmem, tc::sdesc_sw128(al + ka), tc::sdesc_sw128(bh + kb), idesc, 1u);
            }
            tc::mma_commit(mc->bar_m);
        }
        *mc->s_ok = landed ? 1u : 0u;
    }
    mc->ph_b ^= 1u;
    __syncthreads();
    const bool issued = *mc->s_ok != 0;
    const bool done = issued && mbar_wait_bounded(mc->bar_m, mc->ph_m);
    if (issued) mc->ph_m ^= 1u;
    mc->pending = issued && !done;
    if (__syncthreads_or(!done)) {
        if (threadIdx.x == 0) atomicExch(mc->err, 1);
        mc->abort = true;
        return false;
    }
    tc::fence_after_sync();
    uint32_t v[32];
    tc::tmem_ld32(mc->tmem + ((32u * (wid & 3u)) << 16) + (wid >> 2) * 32u, v);
    tc::tmem_ld_wait();
#pragma unroll
    for (int r = 0; r < R; ++r) {
        x[r].re = __uint_as_float(v[2 * r]);
        x[r].im = __uint_as_float(v[2 * r + 1]);
    }
    tc::fence_before_sync();
    return true;
}

// Copy ops [c0, c0 + cn) of a pass into shared memory (all threads).
__device__ __forceinline__ void stage_ops(DevOp* s_ops, const DevOp* __restrict__ pops, int c0, int cn) {
    const uint4* srcv = reinterpret_cast<const uint4*>(pops + c0);
    uint4* dstv = reinterpret_cast<uint4*>(s_ops);
    constexpr int kVec = int(sizeof(DevOp) / sizeof(uint4));
    for (int i = threadIdx.x; i < cn * kVec; i += blockDim.x) dstv[i] = srcv[i];
}

// s_ops: the caller's shared-memory staging area of kOpChunk ops.
template <class A, int RB, bool PG, bool MG = false>
__device__ __forceinline__ void run_ops(typename A::cx (&x)[1 << RB], const DevOp* __restrict__ pops, int nops,
                                        uint64_t base, uint32_t lane, uint32_t wid, typename A::amp_t* tile,
                                        DevOp* s_ops, MmaCtx* mc = nullptr) {
    using RO = RegOps<A, RB>;
    using cx = typename A::cx;
    constexpr int R = 1 << RB;
    // The ops are staged in shared memory, a chunk at a time: every thread
    // reads every op, and a shared-memory broadcast keeps that off the
    // critical path that a global load would be on.  Each op's header (its
    // dispatch code, bits and conditions, resolved on the host) is read field
    // by field where it is used; the dispatch is a short tree of comparisons over ranges
    // of codes (measured faster than a jump table, and than loading the next
    // header early), and only the classes that can carry conditions (X,
    // SWAP, phases) test them.
    for (int c0 = 0; c0 < nops; c0 += kOpChunk) {
    const int cn = nops - c0 < kOpChunk ? nops - c0 : kOpChunk;
    // the previous chunk has been read by all.  (Before the first chunk no
    // barrier is needed: every caller reaches run_ops after a barrier that
    // follows all reads of its previous tile's ops, or with none.)
    if (c0 > 0) __syncthreads();
    stage_ops(s_ops, pops, c0, cn);
    __syncthreads();
    for (int oi = 0; oi < cn; ++oi) {
        const DevOp* op = s_ops + oi;
        // header fields are read from shared memory where they are used
        const RegHdr& h = op->rh;
        const int code = h.code;
        if (code <= RC_X_L) {  // layout change, pair ops, X
            if (code == RC_PERM) {
                const TileMap<RB> from =
                    layout_map<RB>(*reinterpret_cast<const TileLayout*>(&op->m), op->nwarp, lane, wid);
                __syncthreads();  // the previous layout change has been read by all
#pragma unroll
                for (int r = 0; r < R; ++r) tile[from.idx(r)] = A::st(x[r]);
                __syncthreads();
                const TileMap<RB> to = tile_map<RB>(nullptr, op->perm, op->perm + RB, op->nwarp, 0u, lane, wid);
#pragma unroll
                for (int r = 0; r < R; ++r) x[r] = A::ld(tile[to.idx(r)]);
                if constexpr (MG) mc->tile_read = true;
                continue;
            }
            const int ren = h.ren;
            if (ren > 0) {
                // target on register bit ren: bring it to register bit 0 (the
                // host tracks the same exchange; it happens even when the op is
                // skipped below, so the layout stays in step)
                dispatch_k<RB>(ren, [&](auto kc) {
                    if constexpr (decltype(kc)::value > 0) RO::template swap_bits<decltype(kc)::value>(x);
                });
            }
            if (code <= RC_IREAL_L) {
                // DENSE, REAL, ANTI and IREAL ops carry no conditions (only
                // X, SWAP and phases do; the planner's emulator checks it):
                // no condition tests.  Odd codes are the register-bit
                // variants.
                if (code & 1) {
                    if (code < RC_ANTI_R) {
                        if (code == RC_DENSE_R) {
                            // complex64 plans DENSE ops on register bit b in place
                            if constexpr (std::is_same<A, ArF32>::value) {
                                if (h.b > 0) {
                                    dispatch_k<RB>(h.b, [&](auto kc) {
                                        constexpr int K = decltype(kc)::value;
                                        if constexpr (K > 0) RO::template dense_regk<K>(x, op);
                                    });
                                } else {
                                    RO::template pair_reg0<OP_DENSE>(x, op);
                                }
                            } else {
                                RO::template pair_reg0<OP_DENSE>(x, op);
                            }
                        }
                        else RO::template pair_reg0<OP_REAL>(x, op);
                    } else {
                        if (code == RC_ANTI_R) RO::template pair_reg0<OP_ANTI>(x, op);
                        else RO::template pair_reg0<OP_IREAL>(x, op);
                    }
                } else {
                    if (code < RC_ANTI_L) {
                        if (code == RC_DENSE_L) RO::template pair_lane<OP_DENSE>(x, op, h.a, lane);
                        else RO::template pair_lane<OP_REAL>(x, op, h.a, lane);
                    } else {
                        if (code == RC_ANTI_L) RO::template pair_lane<OP_ANTI>(x, op, h.a, lane);
                        else RO::template pair_lane<OP_IREAL>(x, op, h.a, lane);
                    }
                }
                continue;
            }
            const uint64_t cmg = op->cm_glob;
            if ((base & cmg) != cmg) continue;  // a control outside the tile is 0: uniform skip
            const uint32_t cmt = h.cm_thr, cmr = h.cm_reg, cvr = h.cv_reg;
            if ((cmt | cmr) == 0) {
                // no condition inside the tile (at most a control outside it)
                if (code == RC_X_R) RO::x_reg0(x, true, 0u, 0u);
                else RO::x_lane(x, h.a, true, 0u, 0u);
                continue;
            }
            const bool thr_ok = ((threadIdx.x ^ h.cv_thr) & cmt) == cmt;
            if (code == RC_X_R) RO::x_reg0(x, thr_ok, cmr, cvr);
            else RO::x_lane(x, h.a, thr_ok, cmr, cvr);
            continue;
        }
        if (code <= RC_SWAP_LL) {
            const uint64_t cmg = op->cm_glob;
            if ((base & cmg) != cmg) continue;
            const bool thr_ok = ((threadIdx.x ^ h.cv_thr) & h.cm_thr) == h.cm_thr;
            const uint32_t cmr = h.cm_reg, cvr = h.cv_reg;
            if (code == RC_SWAP_LL) RO::swap_ll(x, h.a, h.b, lane, thr_ok, cmr, cvr);
            else if (code == RC_SWAP_LR)
                dispatch_k<RB>(h.b, [&](auto kc) {
                    RO::template swap_lr<decltype(kc)::value>(x, h.a, lane, thr_ok, cmr, cvr);
                });
            else
                dispatch_k<RB>(h.a, [&](auto a) {
                    dispatch_k<RB>(h.b, [&](auto b) {
                        constexpr int K0 = decltype(a)::value, K1 = decltype(b)::value;
                        if constexpr (K0 < K1) RO::template swap_rr<K0, K1>(x, thr_ok, cmr, cvr);
                    });
                });
            continue;
        }
        if (code <= RC_DIAG_R) {  // diagonals carry no conditions
            if (code == RC_DIAG_R) RO::diag_r(x, op, h.a);
            else RO::diag_u(x, op, code == RC_DIAG_G ? int((base >> h.a) & 1u) : int((threadIdx.x >> h.a) & 1u));
            continue;
        }
        if constexpr (MG) {
            if (code == RC_MMA) {
                if (!mma_block<A, RB>(x, op, lane, wid, mc)) return;
                continue;
            }
        }
        {
            const uint64_t cmg = op->cm_glob;
            if ((base & cmg) != cmg) continue;
        }
        const bool thr_ok = ((threadIdx.x ^ h.cv_thr) & h.cm_thr) == h.cm_thr;
        const uint32_t cmr = h.cm_reg, cvr = h.cv_reg;
        const int mcls = h.mcls;
        if (PG && code == RC_PH_GROUP) {
            if constexpr (PG) {
                // Merged phases, step by step: a thread multiplies the factors of
                // the step's terms whose conditions hold for it, then applies the
                // product to the step's registers.  The conditions outside the
                // tile are the same for every thread of the CTA: each warp tests
                // them for 32 terms at once (a ballot) and then walks only the
                // terms that hold, in order.
                const int nt = op->b1;
                const PhTerm* terms = reinterpret_cast<const PhTerm*>(op + 1);
                uint64_t live = 0;
                for (int i0 = 0; i0 < nt; i0 += 32) {
                    const int i = i0 + int(lane);
                    const bool ok = i < nt && (base & terms[i].cm_glob) == terms[i].cm_glob;
                    live |= uint64_t(__ballot_sync(0xffffffffu, ok)) << i0;
                }
                uint64_t ends;
                memcpy(&ends, op->perm, sizeof ends);  // bit i: term i ends its step
                uint64_t rest = nt >= 64 ? ~uint64_t(0) : (uint64_t(1) << nt) - 1;
                ends |= uint64_t(1) << (nt - 1);  // the group's last term always ends a step
                // every step clears at least its last term from `rest`: at most nt steps
                for (int guard = 0; rest && guard < 64; ++guard) {
                    const int e = __ffsll(static_cast<long long>(ends & rest)) - 1;
                    const uint64_t step = rest & (e >= 63 ? ~uint64_t(0) : (uint64_t(2) << e) - 1);
                    uint64_t m = live & step;
                    cx f = A::matp(op, 0);
                    bool go = false;
                    while (m) {
                        const int i = __ffsll(static_cast<long long>(m)) - 1;
                        m &= m - 1;
                        const PhTerm& t = terms[i];
                        if (((threadIdx.x ^ t.cv_thr) & t.cm_thr) == t.cm_thr) {
                            f = go ? A::mul(A::coef(t), f) : A::coef(t);
                            go = true;
                        }
                    }
                    if (go) RO::apply01(x, terms[e].mcls, terms[e].k, [&](cx v) { return A::mul(f, v); });
                    rest &= ~step;
                }
                oi += (nt + kTermsPerSlot - 1) / kTermsPerSlot;  // the term slots
            }
        } else if (thr_ok) {
            if (code == RC_PH_NEG) RO::masked(x, mcls, h.a, cmr, cvr, [](cx v) { return A::neg(v); });
            else if (code == RC_PH_POS_I) RO::masked(x, mcls, h.a, cmr, cvr, [](cx v) { return A::mul_i(v); });
            else if (code == RC_PH_NEG_I) RO::masked(x, mcls, h.a, cmr, cvr, [](cx v) { return A::mul_negi(v); });
            else if (code == RC_PH_GEN) {
                const cx f = A::matp(op, 0);
                RO::masked(x, mcls, h.a, cmr, cvr, [&](cx v) { return A::mul(f, v); });
            }
        }
    }
    }
}

// One CTA per tile: load from HBM into registers, run the ops, store.  When
// a thread's binary32 amplitudes take at most 32 registers the kernel is held
// to 64 registers so that 4 CTAs (32 warps) share an SM: measured 6% faster
// than the 80-register, 3-CTA schedule on float-float complex128 (2^11
// tiles) and 4% on complex64 (2^12 tiles), the extra warps hiding the
// latency of the per-op decode and of the layout changes.  (Binary64 keeps
// its registers: it would spill, and its FP64 rate bounds it anyway.)
template <class A, int RB>
constexpr int reg_min_blocks() {
    return (!std::is_same<typename A::amp_t, double2>::value &&
            (1 << RB) * int(sizeof(typename A::amp_t)) / 4 <= 32) ? 4 : 1;
}

// Dynamic shared memory of the kernel with tensor-core blocks: operand A
// (64 KB, also the layout-change buffer), operand B (32 KB), and slack to
// align both to 1024 bytes (the 128-byte swizzle's repeat).
constexpr size_t kMmaSmemBytes = 1024 + 65536 + size_t(kBlockBytes);

template <class A, int RB, bool PG, bool MG = false>
__global__ void __launch_bounds__(256, MG ? 2 : reg_min_blocks<A, RB>()) k_pass_reg(typename A::amp_t* dst,
                                                   const typename A::amp_t* src, const DevPass dp,
                                                   const DevOp* __restrict__ ops,
                                                   const uint32_t* __restrict__ worklist, int* err) {
    using amp_t = typename A::amp_t;
    using cx = typename A::cx;
    constexpr int R = 1 << RB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    amp_t* tile = reinterpret_cast<amp_t*>(smem_raw);
    __shared__ uint64_t choff[1 << kMaxTileHigh];
    const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    MmaCtx mc;
    if constexpr (MG) {
        // operands at 1024-byte boundaries; the accumulator in tensor memory
        __shared__ __align__(8) uint64_t bars[2];
        __shared__ uint32_t s_tmem, s_ok;
        const uint32_t pad = (1024u - (tc::saddr(smem_raw) & 1023u)) & 1023u;
        mc.a_sm = smem_raw + pad;
        mc.b_sm = mc.a_sm + 65536;
        mc.bar_b = &bars[0];
        mc.bar_m = &bars[1];
        mc.s_ok = &s_ok;
        mc.blk = dp.blk;
        mc.err = err;
        mc.ph_b = mc.ph_m = 0;
        mc.pending = mc.abort = mc.tile_read = false;
        tile = reinterpret_cast<amp_t*>(mc.a_sm);
        if (threadIdx.x == 0) {
            mbar_init(mc.bar_b, 1);
            mbar_init(mc.bar_m, 1);
            mbar_fence_init();
        }
        if (wid == 0) {
            tc::tmem_alloc(&s_tmem, tc::kTmemCols);
            tc::tmem_relinquish();
        }
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        mc.tmem = s_tmem;
    }
    // the tile's first amplitude: one thread computes it for the CTA.  (The
    // ops are staged after the tile's loads are issued, so that the two
    // latencies overlap: staging them before this barrier measured slower.)
    __shared__ uint64_t s_base;
    __shared__ __align__(16) DevOp s_ops[kOpChunk];
    if (threadIdx.x == 0) s_base = tile_base(dp, worklist, blockIdx.x);
    chunk_offsets(dp, choff);
    __syncthreads();
    const uint64_t base = s_base;
    const uint32_t lowmask = (1u << dp.lt) - 1u;
    // The amplitude index of tile index j is base | (j & lowmask) |
    // choff[j >> lt]: XOR-linear in j, with the base's bits disjoint from the
    // image.  A thread's register r holds tile index thr ^ (register bits of
    // r), so its amplitude index is the index of thr XOR the offsets of r's
    // register bits (dp.rin / dp.rout, from the host).
    cx x[R];
    {
        const TileMap<RB> m = initial_map<RB>(dp, lane, wid);
        const uint64_t g = base | choff[m.thr >> dp.lt] | (m.thr & lowmask);
#pragma unroll
        for (int r = 0; r < R; ++r) x[r] = A::ld(src[g ^ reg_offset<RB>(dp.rin, r)]);
    }
    run_ops<A, RB, PG, MG>(x, ops + dp.op_offset, dp.nops, base, lane, wid, tile, s_ops, &mc);
    // A pass whose gates were all relabels has no ops, so no barrier has
    // separated the loads from the stores; its final layout sends amplitudes
    // to positions that other warps of the CTA load (in place: dst == src).
    if (dp.nops == 0) __syncthreads();
    if (!MG || !mc.abort) {
        const TileMap<RB> m = layout_map<RB>(dp.fin, dp.nwarp, lane, wid);
        const uint64_t g = base | choff[m.thr >> dp.lt] | (m.thr & lowmask);
#pragma unroll
        for (int r = 0; r < R; ++r) dst[g ^ reg_offset<RB>(dp.rout, r)] = A::st(x[r]);
    }
    if constexpr (MG) {
        // an aborted block may still have MMAs in flight: wait for them
        // (bounded) before the accumulator's memory is given back
        if (threadIdx.x == 0 && mc.pending) mbar_wait_bounded(mc.bar_m, mc.ph_m);
        tc::fence_before_sync();
        __syncthreads();
        if (wid == 0) {
            tc::fence_after_sync();
            tc::tmem_dealloc(mc.tmem, tc::kTmemCols);
        }
    }
}

// ----------------------------------------------------- TMA-staged variant --
// A persistent CTA walks the launch's tiles with a stride of gridDim.x.  While
// it computes tile i, the bulk-copy engine (cp.async.bulk, one copy per
// contiguous chunk, completion counted on an mbarrier) brings tile i+1 into a
// second shared-memory buffer, so HBM reads overlap the arithmetic.  Every
// wait on the mbarrier is bounded (1 s of %globaltimer); on expiry the CTA
// raises the error flag and returns, and the host reports QT_ERR_TIMEOUT.
template <class A, int RB, bool PG>
__global__ void __launch_bounds__(256, (RB <= 3 ? 3 : 1)) k_pass_tma(typename A::amp_t* dst,
                                                   const typename A::amp_t* src, const DevPass dp,
                                                   const DevOp* __restrict__ ops,
                                                   const uint32_t* __restrict__ worklist, uint32_t ntiles,
                                                   int* __restrict__ err) {
    using amp_t = typename A::amp_t;
    using cx = typename A::cx;
    constexpr int R = 1 << RB;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const uint32_t tb = uint32_t(dp.lt + dp.nh);
    amp_t* inbuf = reinterpret_cast<amp_t*>(smem_raw);  // staged tile, indexed by tile index
    amp_t* tile = inbuf + (1u << tb);                   // layout changes
    __shared__ uint64_t choff[1 << kMaxTileHigh];
    __shared__ __align__(8) uint64_t bar;
    __shared__ __align__(16) DevOp s_ops[kOpChunk];
    const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    chunk_offsets(dp, choff);
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    const uint32_t nchunks = 1u << dp.nh;
    const uint32_t chunk_bytes = uint32_t(sizeof(amp_t)) << dp.lt;
    auto issue = [&](uint32_t t) {  // warp 0 stages tile t into inbuf
        if (wid == 0 && !dp.test_stall) {
            const uint64_t b = tile_base(dp, worklist, t);
            if (lane == 0) mbar_arrive_expect_tx(&bar, chunk_bytes * nchunks);
            __syncwarp();
            for (uint32_t c = lane; c < nchunks; c += 32)
                bulk_g2s(inbuf + (c << dp.lt), src + (b | choff[c]), chunk_bytes, &bar);
        }
    };
    uint32_t t = blockIdx.x;
    if (t < ntiles) issue(t);
    uint32_t parity = 0;
    const uint32_t lowmask = (1u << dp.lt) - 1u;
    for (; t < ntiles; t += gridDim.x) {
        const uint64_t base = tile_base(dp, worklist, t);
        const bool ok = mbar_wait_bounded(&bar, parity);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) atomicExch(err, 1);
            return;
        }
        parity ^= 1u;
        cx x[R];
        {
            const TileMap<RB> m = initial_map<RB>(dp, lane, wid);
#pragma unroll
            for (int r = 0; r < R; ++r) x[r] = A::ld(inbuf[m.idx(r)]);
        }
        __syncthreads();  // inbuf is free: stage the next tile while computing this one
        if (t + gridDim.x < ntiles) issue(t + gridDim.x);
        run_ops<A, RB, PG>(x, ops + dp.op_offset, dp.nops, base, lane, wid, tile, s_ops);
        const TileMap<RB> m = layout_map<RB>(dp.fin, dp.nwarp, lane, wid);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint32_t j = m.idx(r);
            dst[base | choff[j >> dp.lt] | (j & lowmask)] = A::st(x[r]);
        }
    }
}

template <class A, int RB, bool PG>
int launch_reg_t(void* dst, const void* src, const DevPass& dp, const DevOp* ops, const uint32_t* worklist,
                 uint32_t ngroups, int* err, cudaStream_t st) {
    using amp_t = typename A::amp_t;
    const size_t tile_bytes = sizeof(amp_t) << (dp.lt + dp.nh);
    const uint64_t nblocks = uint64_t(ngroups) << dp.tpg_log2;
    if (nblocks == 0) return 0;
    const unsigned threads = 32u << dp.nwarp;
    if (nblocks > 0x7fffffffull || tile_bytes > 64 * 1024 || dp.nreg != RB) return int(cudaErrorInvalidConfiguration);
    const bool tma = dp.tma && err != nullptr && (uint32_t(sizeof(amp_t)) << dp.lt) % 16 == 0;
    if (dp.mma) {
        // tensor-core blocks: complex64 tiles of 4096 amplitudes only
        if constexpr (std::is_same<A, ArF32>::value && RB == 4) {
            if (dp.blk == nullptr || err == nullptr || threads != 256) return int(cudaErrorInvalidConfiguration);
            static DeviceOnce mattr;
            const int rc = mattr.run([](int) {
                return int(cudaFuncSetAttribute(k_pass_reg<A, RB, PG, true>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize, int(kMmaSmemBytes)));
            });
            if (rc) return rc;
            return launch_k(k_pass_reg<A, RB, PG, true>, dim3(unsigned(nblocks)), dim3(threads), kMmaSmemBytes, st,
                            static_cast<amp_t*>(dst), static_cast<const amp_t*>(src), dp, ops, worklist, err);
        } else {
            return int(cudaErrorInvalidConfiguration);
        }
    }
    if (!tma) {
        static DeviceOnce attr;
        const int rc = attr.run([](int) {
            return int(cudaFuncSetAttribute(k_pass_reg<A, RB, PG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            128 * 1024));
        });
        if (rc) return rc;
        return launch_k(k_pass_reg<A, RB, PG>, dim3(unsigned(nblocks)), dim3(threads), tile_bytes, st,
                        static_cast<amp_t*>(dst), static_cast<const amp_t*>(src), dp, ops, worklist, err);
    }
    static DeviceOnce tattr;
    int rc = tattr.run([](int) {
        return int(
            cudaFuncSetAttribute(k_pass_tma<A, RB, PG>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024));
    });
    if (rc) return rc;
    const size_t smem = 2 * tile_bytes;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pass_tma<A, RB, PG>, int(threads), smem);
    if (e != cudaSuccess) return int(e);
    if (per_sm < 1) per_sm = 1;
    const uint64_t grid = std::min<uint64_t>(nblocks, uint64_t(device_sm_count()) * uint64_t(per_sm));
    return launch_k(k_pass_tma<A, RB, PG>, dim3(unsigned(grid)), dim3(threads), smem, st, static_cast<amp_t*>(dst),
                    static_cast<const amp_t*>(src), dp, ops, worklist, uint32_t(nblocks), err);
}

template <class A, bool PG>
int launch_reg_a(void* dst, const void* src, const DevPass& dp, const DevOp* ops, const uint32_t* worklist,
                 uint32_t ngroups, int* err, cudaStream_t st) {
    switch (dp.nreg) {
        case 2: return launch_reg_t<A, 2, PG>(dst, src, dp, ops, worklist, ngroups, err, st);
        case 3: return launch_reg_t<A, 3, PG>(dst, src, dp, ops, worklist, ngroups, err, st);
        case 4: return launch_reg_t<A, 4, PG>(dst, src, dp, ops, worklist, ngroups, err, st);
        case 5: return launch_reg_t<A, 5, PG>(dst, src, dp, ops, worklist, ngroups, err, st);
        default: return int(cudaErrorInvalidConfiguration);
    }
}

// The register kernels of this translation unit for every dtype.
template <bool PG>
int launch_pass_reg_t(int dtype, void* dst, const void* src, const DevPass& dp, const DevOp* ops,
                      const uint32_t* worklist, uint32_t ngroups, int* err, void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (dtype) {
        case QT_C128: return launch_reg_a<ArF64, PG>(dst, src, dp, ops, worklist, ngroups, err, st);
        case QT_C64: return launch_reg_a<ArF32, PG>(dst, src, dp, ops, worklist, ngroups, err, st);
        case QT_C128_DF: return launch_reg_a<ArDF, PG>(dst, src, dp, ops, worklist, ngroups, err, st);
        default: return int(cudaErrorInvalidValue);
    }
}

#if QT_PASS_PHASE_GROUPS
int launch_pass_reg_groups(int dtype, void* dst, const void* src, const DevPass& dp, const DevOp* ops,
                           const uint32_t* worklist, uint32_t ngroups, int* err, void* stream) {
    return launch_pass_reg_t<true>(dtype, dst, src, dp, ops, worklist, ngroups, err, stream);
}
#else

// ------------------------------------------------------------ batched runs --
// Many independent circuits in one persistent launch.  Tiles are dequeued
// from one global counter in wavefront order (all tiles of pass i of every
// circuit before pass i+1), so every tile a CTA waits for was dequeued
// earlier by a running CTA whose own dependencies are earlier still: the
// launch always makes progress, and every wait is bounded anyway.
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ bool wait_counter(const uint32_t* c, uint32_t need) {
    if (ld_acquire(c) >= need) return true;
    const uint64_t t0 = global_ns();
    while (ld_acquire(c) < need) {
        if (global_ns() - t0 > 1000000000ull) return false;
        __nanosleep(100);
    }
    return true;
}

template <class A, int RB>
__device__ __forceinline__ void batch_tile(typename A::amp_t* __restrict__ state, const DevPass& dp, uint32_t t,
                                           const DevOp* __restrict__ ops, typename A::amp_t* tile,
                                           uint64_t* choff) {
    using cx = typename A::cx;
    constexpr int R = 1 << RB;
    const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    __shared__ uint64_t s_base;  // the tile's first amplitude, computed by one thread
    __shared__ __align__(16) DevOp s_ops[kOpChunk];
    if (threadIdx.x == 0) s_base = tile_base(dp, nullptr, t);
    chunk_offsets(dp, choff);
    __syncthreads();
    const uint64_t base = s_base;
    const uint32_t lowmask = (1u << dp.lt) - 1u;
    cx x[R];
    {
        // amplitude indices as in k_pass_reg: the thread's index XOR the
        // offsets of the register bits
        const TileMap<RB> m = initial_map<RB>(dp, lane, wid);
        const uint64_t g = base | choff[m.thr >> dp.lt] | (m.thr & lowmask);
#pragma unroll
        for (int r = 0; r < R; ++r)
            x[r] = A::ld(__ldcg(&state[g ^ reg_offset<RB>(dp.rin, r)]));  // L2: written by other SMs
    }
    run_ops<A, RB, false>(x, ops + dp.op_offset, dp.nops, base, lane, wid, tile, s_ops);
    if (dp.nops == 0) __syncthreads();  // relabels only: the loads of every warp come before any store
    const TileMap<RB> m = layout_map<RB>(dp.fin, dp.nwarp, lane, wid);
    const uint64_t g = base | choff[m.thr >> dp.lt] | (m.thr & lowmask);
#pragma unroll
    for (int r = 0; r < R; ++r) state[g ^ reg_offset<RB>(dp.rout, r)] = A::st(x[r]);
    __threadfence();  // every thread's stores are visible device-wide before the tile is counted done
    __syncthreads();  // choff and tile are reused by the next item
}

template <class A>
__global__ void __launch_bounds__(256) k_batch(typename A::amp_t* __restrict__ arena,
                                               const BatchPass* __restrict__ passes, int npasses,
                                               const DevOp* __restrict__ ops, uint32_t total_items,
                                               uint32_t* __restrict__ head, uint32_t* __restrict__ counters,
                                               int* __restrict__ err) {
    using amp_t = typename A::amp_t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    amp_t* tile = reinterpret_cast<amp_t*>(smem_raw);
    __shared__ uint64_t choff[1 << kMaxTileHigh];
    __shared__ uint32_t s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(head, 1u);
        __syncthreads();
        const uint32_t item = s_item;
        __syncthreads();
        if (item >= total_items) return;
        int lo = 0, hi = npasses - 1;  // last pass whose first item <= item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (passes[mid].first_item <= item) lo = mid;
            else hi = mid - 1;
        }
        const BatchPass* bp = passes + lo;
        bool ok = true;
        if (threadIdx.x == 0 && bp->dep >= 0) ok = wait_counter(counters + bp->dep, bp->dep_need);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) atomicExch(err, 1);
            return;
        }
        __threadfence();
        const DevPass dp = bp->dp;
        amp_t* state = arena + bp->state_off;
        const uint32_t t = item - bp->first_item;
        // Tiles of 2^12 exist for 8-byte amplitudes only (the host rejects
        // them for 16-byte ones); any other shape raises the error flag
        // (2: unsupported tile) instead of leaving the tile undone.
        bool done = true;
        switch (dp.nreg) {
            case 2: batch_tile<A, 2>(state, dp, t, ops, tile, choff); break;
            case 3: batch_tile<A, 3>(state, dp, t, ops, tile, choff); break;
            case 4:
                if constexpr (sizeof(amp_t) == 8) batch_tile<A, 4>(state, dp, t, ops, tile, choff);
                else done = false;
                break;
            default: done = false; break;
        }
        if (!done && threadIdx.x == 0) atomicExch(err, 2);
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(counters + bp->counter, 1u);
        }
    }
}

template <class A>
__global__ void k_batch_init(typename A::amp_t* arena, const uint64_t* __restrict__ firsts, int count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) {
        typename A::cx one;
        if constexpr (sizeof(typename A::amp_t) == 8) one = A::ld(make_float2(1.0f, 0.0f));
        else if constexpr (std::is_same<A, ArDF>::value) one = A::ld(make_float4(1.0f, 0.0f, 0.0f, 0.0f));
        else one = A::ld(make_double2(1.0, 0.0));
        arena[firsts[i]] = A::st(one);
    }
}

int launch_batch_init(int dtype, void* arena, uint64_t arena_amps, const uint64_t* firsts, int count, void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t bpa = bytes_per_amp(dtype);
    cudaError_t e = cudaMemsetAsync(arena, 0, arena_amps * bpa, st);
    if (e != cudaSuccess) return int(e);
    const int grid = (count + 255) / 256;
    if (grid == 0) return 0;
    switch (dtype) {
        case QT_C128:
            return launch_k(k_batch_init<ArF64>, dim3(grid), dim3(256), 0, st, static_cast<double2*>(arena), firsts,
                            count);
        case QT_C64:
            return launch_k(k_batch_init<ArF32>, dim3(grid), dim3(256), 0, st, static_cast<float2*>(arena), firsts,
                            count);
        default:
            return launch_k(k_batch_init<ArDF>, dim3(grid), dim3(256), 0, st, static_cast<float4*>(arena), firsts,
                            count);
    }
}

template <class A>
int launch_batch_t(void* arena, const BatchPass* passes, int npasses, const DevOp* ops, uint32_t total_items,
                   uint32_t* head, uint32_t* counters, int* err, size_t smem, cudaStream_t st) {
    static DeviceOnce attr;
    const int rc = attr.run([](int) {
        return int(cudaFuncSetAttribute(k_batch<A>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024));
    });
    if (rc) return rc;
    if (smem > 64 * 1024) return int(cudaErrorInvalidConfiguration);
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<A>, 256, smem);
    if (e != cudaSuccess) return int(e);
    if (per_sm < 1) per_sm = 1;
    const uint64_t grid = std::min<uint64_t>(total_items, uint64_t(device_sm_count()) * uint64_t(per_sm));
    if (grid == 0) return 0;
    return launch_k(k_batch<A>, dim3(unsigned(grid)), dim3(256), smem, st, static_cast<typename A::amp_t*>(arena),
                    passes, npasses, ops, total_items, head, counters, err);
}

int launch_batch(int dtype, void* arena, const BatchPass* passes, int npasses, const DevOp* ops,
                 uint32_t total_items, uint32_t* head, uint32_t* counters, int* err, size_t smem_bytes,
                 void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (dtype) {
        case QT_C128: return launch_batch_t<ArF64>(arena, passes, npasses, ops, total_items, head, counters, err,
                                                   smem_bytes, st);
        case QT_C64: return launch_batch_t<ArF32>(arena, passes, npasses, ops, total_items, head, counters, err,
                                                  smem_bytes, st);
        default: return launch_batch_t<ArDF>(arena, passes, npasses, ops, total_items, head, counters, err,
                                             smem_bytes, st);
    }
}

int launch_pass_reg(int dtype, void* dst, const void* src, const DevPass& dp, const DevOp* ops,
                    const uint32_t* worklist, uint32_t ngroups, int* err, void* stream) {
    if (dp.groups) return launch_pass_reg_groups(dtype, dst, src, dp, ops, worklist, ngroups, err, stream);
    return launch_pass_reg_t<false>(dtype, dst, src, dp, ops, worklist, ngroups, err, stream);
}
#endif  // QT_PASS_PHASE_GROUPS

}  // namespace qt
