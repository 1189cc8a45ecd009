// qt_arith.cuh -- complex arithmetic policies of the gate kernels.
//   ArF64  IEEE binary64 (QT_C128)
//   ArF32  binary32 (QT_C64)
//   ArDF   float-float (QT_C128_DF): each real is hi + lo, two binary32 values;
//          products are split exactly with an FMA and sums with the error-free
//          two-sum (Knuth; Dekker), so all arithmetic runs on the FP32 pipes.
// Every formula is written with explicit _rn intrinsics so the compiler can
// neither contract nor reorder it: the same op gives the same bits wherever
// it runs, which incremental-versus-full bit identity relies on.
#pragma once
#include <cuda_runtime.h>

#include "qt_internal.h"

namespace qt {

// ------------------------------------------------------------ float-float --
struct df {
    float hi, lo;
};

__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }

__device__ __forceinline__ df two_sum(float a, float b) {
    float s = fadd(a, b);
    float bb = fsub(s, a);
    float e = fadd(fsub(a, fsub(s, bb)), fsub(b, bb));
    return {s, e};
}

__device__ __forceinline__ df fast_two_sum(float a, float b) {
    float s = fadd(a, b);
    float e = fsub(b, fsub(s, a));
    return {s, e};
}

__device__ __forceinline__ df dneg(df a) { return {-a.hi, -a.lo}; }
// Negation and copy as FP32 multiplies by -1 and 1 (exact).  In the register
// kernel the exchanges of X/SWAP ops, register renames and the ±1/±i phases
// otherwise become register moves and sign flips on the half-rate ALU pipe,
// which the op mix saturates while the FMA pipe has room; as multiplies they
// issue on the FMA pipe (measured 16% less time on the benchmark circuit).
// Written as PTX so that the compiler keeps the multiply.
__device__ __forceinline__ float fmul_c(float a, float c) {
    float d;
    asm("mul.rn.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(c));
    return d;
}
__device__ __forceinline__ df dneg_f(df a) { return {fmul_c(a.hi, -1.0f), fmul_c(a.lo, -1.0f)}; }
__device__ __forceinline__ df dcopy_f(df a) { return {fmul_c(a.hi, 1.0f), fmul_c(a.lo, 1.0f)}; }

// sum_k a_k * b_k for K float-float pairs.  Each product's leading term is
// split exactly by an FMA; the leading terms are summed with two_sum and all
// residuals gathered in one float before a final renormalisation.
template <int K>
__device__ __forceinline__ df df_dot(const df (&a)[K], const df (&b)[K]) {
    float p = __fmul_rn(a[0].hi, b[0].hi);
    float err = __fmaf_rn(a[0].hi, b[0].hi, -p);
    err = __fmaf_rn(a[0].hi, b[0].lo, err);
    err = __fmaf_rn(a[0].lo, b[0].hi, err);
    float s = p;
#pragma unroll
    for (int k = 1; k < K; ++k) {
        float pk = __fmul_rn(a[k].hi, b[k].hi);
        float ek = __fmaf_rn(a[k].hi, b[k].hi, -pk);
        ek = __fmaf_rn(a[k].hi, b[k].lo, ek);
        ek = __fmaf_rn(a[k].lo, b[k].hi, ek);
        df t = two_sum(s, pk);
        s = t.hi;
        err = fadd(err, fadd(t.lo, ek));
    }
    return fast_two_sum(s, err);
}

// ----------------------------------------------------------------- policies
struct ArF64 {
    using amp_t = double2;
    struct cx {
        double re, im;
    };
    static __device__ __forceinline__ cx ld(amp_t a) { return {a.x, a.y}; }
    static __device__ __forceinline__ amp_t st(cx v) { return make_double2(v.re, v.im); }
    static __device__ __forceinline__ cx mat(const DevOp& op, int k) { return {op.m.d[2 * k], op.m.d[2 * k + 1]}; }
    // u0 * x0 + u1 * x1
    static __device__ __forceinline__ cx lin2(cx u0, cx x0, cx u1, cx x1) {
        cx r;
        r.re = __fma_rn(u0.re, x0.re, __fma_rn(-u0.im, x0.im, __fma_rn(u1.re, x1.re, __dmul_rn(-u1.im, x1.im))));
        r.im = __fma_rn(u0.re, x0.im, __fma_rn(u0.im, x0.re, __fma_rn(u1.re, x1.im, __dmul_rn(u1.im, x1.re))));
        return r;
    }
    static __device__ __forceinline__ cx lin2r(cx u0, cx x0, cx u1, cx x1) {  // real u
        cx r;
        r.re = __fma_rn(u0.re, x0.re, __dmul_rn(u1.re, x1.re));
        r.im = __fma_rn(u0.re, x0.im, __dmul_rn(u1.re, x1.im));
        return r;
    }
    // u0 x0 + u1 x1 with u0 real and u1 imaginary (OP_IREAL)
    static __device__ __forceinline__ cx lin2i(cx u0, cx x0, cx u1, cx x1) {
        cx r;
        r.re = __fma_rn(u0.re, x0.re, __dmul_rn(-u1.im, x1.im));
        r.im = __fma_rn(u0.re, x0.im, __dmul_rn(u1.im, x1.re));
        return r;
    }
    static __device__ __forceinline__ cx mul(cx a, cx b) {
        return {__fma_rn(a.re, b.re, __dmul_rn(-a.im, b.im)), __fma_rn(a.re, b.im, __dmul_rn(a.im, b.re))};
    }
    static __device__ __forceinline__ cx neg(cx a) { return {-a.re, -a.im}; }
    static __device__ __forceinline__ cx mul_i(cx a) { return {-a.im, a.re}; }
    static __device__ __forceinline__ cx mul_negi(cx a) { return {a.im, -a.re}; }
    static __device__ __forceinline__ cx shfl(cx a, int mask) {
        return {__shfl_xor_sync(0xffffffffu, a.re, mask), __shfl_xor_sync(0xffffffffu, a.im, mask)};
    }
    static __device__ __forceinline__ cx matp(const DevOp* op, int k) { return {op->m.d[2 * k], op->m.d[2 * k + 1]}; }
    static __device__ __forceinline__ cx coef(const PhTerm& t) { return {t.f.d[0], t.f.d[1]}; }
    static __device__ __forceinline__ cx sel(bool c, cx a, cx b) { return c ? a : b; }
    static __device__ __forceinline__ cx mv(cx a) { return a; }
};

struct ArF32 {
    using amp_t = float2;
    struct cx {
        float re, im;
    };
    static __device__ __forceinline__ cx ld(amp_t a) { return {a.x, a.y}; }
    static __device__ __forceinline__ amp_t st(cx v) { return make_float2(v.re, v.im); }
    static __device__ __forceinline__ cx mat(const DevOp& op, int k) { return {op.m.f[2 * k], op.m.f[2 * k + 1]}; }
    static __device__ __forceinline__ cx lin2(cx u0, cx x0, cx u1, cx x1) {
        cx r;
        r.re = __fmaf_rn(u0.re, x0.re, __fmaf_rn(-u0.im, x0.im, __fmaf_rn(u1.re, x1.re, __fmul_rn(-u1.im, x1.im))));
        r.im = __fmaf_rn(u0.re, x0.im, __fmaf_rn(u0.im, x0.re, __fmaf_rn(u1.re, x1.im, __fmul_rn(u1.im, x1.re))));
        return r;
    }
    static __device__ __forceinline__ cx lin2r(cx u0, cx x0, cx u1, cx x1) {
        cx r;
        r.re = __fmaf_rn(u0.re, x0.re, __fmul_rn(u1.re, x1.re));
        r.im = __fmaf_rn(u0.re, x0.im, __fmul_rn(u1.re, x1.im));
        return r;
    }
    static __device__ __forceinline__ cx lin2i(cx u0, cx x0, cx u1, cx x1) {
        cx r;
        r.re = __fmaf_rn(u0.re, x0.re, __fmul_rn(-u1.im, x1.im));
        r.im = __fmaf_rn(u0.re, x0.im, __fmul_rn(u1.im, x1.re));
        return r;
    }
    static __device__ __forceinline__ cx mul(cx a, cx b) {
        return {__fmaf_rn(a.re, b.re, __fmul_rn(-a.im, b.im)), __fmaf_rn(a.re, b.im, __fmul_rn(a.im, b.re))};
    }
    static __device__ __forceinline__ cx neg(cx a) { return {fmul_c(a.re, -1.0f), fmul_c(a.im, -1.0f)}; }
    static __device__ __forceinline__ cx mul_i(cx a) { return {fmul_c(a.im, -1.0f), fmul_c(a.re, 1.0f)}; }
    static __device__ __forceinline__ cx mul_negi(cx a) { return {fmul_c(a.im, 1.0f), fmul_c(a.re, -1.0f)}; }
    static __device__ __forceinline__ cx shfl(cx a, int mask) {
        return {__shfl_xor_sync(0xffffffffu, a.re, mask), __shfl_xor_sync(0xffffffffu, a.im, mask)};
    }
    static __device__ __forceinline__ cx matp(const DevOp* op, int k) { return {op->m.f[2 * k], op->m.f[2 * k + 1]}; }
    static __device__ __forceinline__ cx coef(const PhTerm& t) { return {t.f.f[0], t.f.f[1]}; }
    static __device__ __forceinline__ cx sel(bool c, cx a, cx b) { return c ? a : b; }
    static __device__ __forceinline__ cx mv(cx a) { return {fmul_c(a.re, 1.0f), fmul_c(a.im, 1.0f)}; }
};

struct ArDF {
    using amp_t = float4;  // (re.hi, re.lo, im.hi, im.lo)
    struct cx {
        df re, im;
    };
    static __device__ __forceinline__ cx ld(amp_t a) { return {{a.x, a.y}, {a.z, a.w}}; }
    static __device__ __forceinline__ amp_t st(cx v) { return make_float4(v.re.hi, v.re.lo, v.im.hi, v.im.lo); }
    static __device__ __forceinline__ cx mat(const DevOp& op, int k) {
        return {{op.m.f[4 * k], op.m.f[4 * k + 1]}, {op.m.f[4 * k + 2], op.m.f[4 * k + 3]}};
    }
    static __device__ __forceinline__ cx lin2(cx u0, cx x0, cx u1, cx x1) {
        const df ar[4] = {u0.re, dneg(u0.im), u1.re, dneg(u1.im)};
        const df br[4] = {x0.re, x0.im, x1.re, x1.im};
        const df ai[4] = {u0.re, u0.im, u1.re, u1.im};
        const df bi[4] = {x0.im, x0.re, x1.im, x1.re};
        return {df_dot<4>(ar, br), df_dot<4>(ai, bi)};
    }
    static __device__ __forceinline__ cx lin2r(cx u0, cx x0, cx u1, cx x1) {
        const df a[2] = {u0.re, u1.re};
        const df br[2] = {x0.re, x1.re};
        const df bi[2] = {x0.im, x1.im};
        return {df_dot<2>(a, br), df_dot<2>(a, bi)};
    }
    static __device__ __forceinline__ cx lin2i(cx u0, cx x0, cx u1, cx x1) {
        const df ar[2] = {u0.re, dneg(u1.im)};
        const df br[2] = {x0.re, x1.im};
        const df ai[2] = {u0.re, u1.im};
        const df bi[2] = {x0.im, x1.re};
        return {df_dot<2>(ar, br), df_dot<2>(ai, bi)};
    }
    static __device__ __forceinline__ cx mul(cx a, cx b) {
        const df ar[2] = {a.re, dneg(a.im)};
        const df br[2] = {b.re, b.im};
        const df ai[2] = {a.re, a.im};
        const df bi[2] = {b.im, b.re};
        return {df_dot<2>(ar, br), df_dot<2>(ai, bi)};
    }
    static __device__ __forceinline__ cx neg(cx a) { return {dneg_f(a.re), dneg_f(a.im)}; }
    static __device__ __forceinline__ cx mul_i(cx a) { return {dneg_f(a.im), dcopy_f(a.re)}; }
    static __device__ __forceinline__ cx mul_negi(cx a) { return {dcopy_f(a.im), dneg_f(a.re)}; }
    static __device__ __forceinline__ cx mv(cx a) { return {dcopy_f(a.re), dcopy_f(a.im)}; }
    static __device__ __forceinline__ cx shfl(cx a, int mask) {
        return {{__shfl_xor_sync(0xffffffffu, a.re.hi, mask), __shfl_xor_sync(0xffffffffu, a.re.lo, mask)},
                {__shfl_xor_sync(0xffffffffu, a.im.hi, mask), __shfl_xor_sync(0xffffffffu, a.im.lo, mask)}};
    }
    static __device__ __forceinline__ cx matp(const DevOp* op, int k) {
        return {{op->m.f[4 * k], op->m.f[4 * k + 1]}, {op->m.f[4 * k + 2], op->m.f[4 * k + 3]}};
    }
    static __device__ __forceinline__ cx coef(const PhTerm& t) { return {{t.f.f[0], t.f.f[1]}, {t.f.f[2], t.f.f[3]}}; }
    static __device__ __forceinline__ cx sel(bool c, cx a, cx b) { return c ? a : b; }
};


}  // namespace qt
