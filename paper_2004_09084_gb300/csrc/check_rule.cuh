// The check-node arithmetic shared by the decode kernels: clipping constants,
// hardware transcendentals, message storage formats, the shared-memory view of
// a code's layer table and the exclusive-product evaluation of the
// sum-product rule (arXiv 2004.09084, Methods, step 2).  Every kernel that
// applies the rule includes this file, so that they evaluate it with the same
// instructions in the same order and give bit-identical results.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "qcmet_internal.h"

namespace qcmet {

constexpr float kClipMax = 30.0f;
// Phi(30) = 2 atanh(exp(-30)), the lower end of the clipping interval.
constexpr float kClipMin = 1.8715246e-13f;
constexpr float kLn2 = 0.693147180559945309f;
constexpr float kLog2e = 1.442695040888963407f;

// ---- transcendentals --------------------------------------------------------
//
// The check rule takes exp2 of arguments in [-30 log2(e), 0] and log2 of
// alpha >= 1 and beta >= exp(-30) (beta = 0 only for a check of degree 1,
// whose log is -inf and whose magnitude clips to 30).  No argument or result
// is subnormal, so the flush-to-zero forms of the hardware approximations
// return what the non-flushing ones do, without the subnormal handling.
__device__ __forceinline__ float ex2_ftz(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float lg2_ftz(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ---- message storage formats ---------------------------------------------

template <typename M>
struct Msg;

template <>
struct Msg<float> {
    static __device__ __forceinline__ float load(const float *p) { return *p; }
    static __device__ __forceinline__ float quantize(float x) { return x; }
    static __device__ __forceinline__ void store(float *p, float x) { *p = x; }
};

template <>
struct Msg<__half> {
    static __device__ __forceinline__ float load(const __half *p) { return __half2float(*p); }
    static __device__ __forceinline__ float quantize(float x) {
        return __half2float(__float2half_rn(x));
    }
    static __device__ __forceinline__ void store(__half *p, float x) { *p = __float2half_rn(x); }
};

template <>
struct Msg<__nv_bfloat16> {
    static __device__ __forceinline__ float load(const __nv_bfloat16 *p) {
        return __bfloat162float(*p);
    }
    static __device__ __forceinline__ float quantize(float x) {
        return __bfloat162float(__float2bfloat16_rn(x));
    }
    static __device__ __forceinline__ void store(__nv_bfloat16 *p, float x) {
        *p = __float2bfloat16_rn(x);
    }
};

// ---- shared-memory view of the schedule ------------------------------------

struct Sched {
    const int32_t *w;
    int32_t n_rows, n_layers, nb, Z, mb, n_zero_rows, core_cols, msg_slots;
    const int32_t *layer_first;
    const int4 *rows;     // DevRow
    const int4 *entries;  // DevEntry
    const int32_t *col_kind;
    const int32_t *zero_rows;
    const int32_t *col_core;  // [nb]: index among the core columns, or -1
};

__device__ __forceinline__ Sched make_sched(const int32_t *w) {
    Sched s;
    s.w = w;
    s.n_rows = w[kHdrRows];
    s.n_layers = w[kHdrLayers];
    s.nb = w[kHdrNb];
    s.Z = w[kHdrZ];
    s.mb = w[kHdrMb];
    s.n_zero_rows = w[kHdrZeroRows];
    s.core_cols = w[kHdrCoreCols];
    s.msg_slots = w[kHdrMsgSlots];
    s.layer_first = w + w[kHdrOffLayerFirst];
    s.rows = reinterpret_cast<const int4 *>(w + w[kHdrOffRows]);
    s.entries = reinterpret_cast<const int4 *>(w + w[kHdrOffEntries]);
    s.col_kind = w + w[kHdrOffColKind];
    s.zero_rows = w + w[kHdrOffZeroRows];
    s.col_core = w + w[kHdrOffColCore];
    return s;
}

// ---- index checks of the debug build ------------------------------------------
//
// Built with QCMET_DEBUG_CHECKS=1 (paper_2004_09084_gb300.build.build(debug=True),
// libqcmet_debug.so), the kernels test every index they gather or scatter
// against its array's extent and skip an access that would leave it,
// recording the kind of index in a device word of the translation unit that
// qcmet_debug_checks() reads and clears.  In the release build in_range() is
// the constant true and the tests compile away.
#ifndef QCMET_DEBUG_CHECKS
#define QCMET_DEBUG_CHECKS 0
#endif
enum : uint32_t {
    kBadVariable = 1u,  // a posterior / channel index outside its array
    kBadSlot = 2u,      // a message slot or check index outside the message array
    kBadCheck = 4u,     // a syndrome index outside the frame's checks
};
#if QCMET_DEBUG_CHECKS
static __device__ uint32_t g_qcmet_violations;
#endif

__device__ __forceinline__ bool in_range(long long idx, long long extent, uint32_t kind) {
#if QCMET_DEBUG_CHECKS
    const bool ok = idx >= 0 && idx < extent;
    if (!ok) atomicOr(&g_qcmet_violations, kind);
    return ok;
#else
    (void)idx;
    (void)extent;
    (void)kind;
    return true;
#endif
}

// Extents the checks test against, in elements of the frame's (or group's)
// arrays: core posteriors, channel / all variables, message slots x Z, checks.
struct Bounds {
    long long core, vars, msgs, checks;
};
__device__ __forceinline__ Bounds bounds_of(const Sched &s) {
    Bounds b;
    b.core = (long long)s.core_cols * s.Z;
    b.vars = (long long)s.nb * s.Z;
    b.msgs = (long long)s.msg_slots * s.Z;
    b.checks = (long long)s.mb * s.Z;
    return b;
}

// ---- one check node ----------------------------------------------------------

// (a, b) (x) (c, d): product of two elements a I + b J and c I + d J.
__device__ __forceinline__ void cmul(float a, float b, float c, float d, float &x, float &y) {
    x = fmaf(a, c, b * d);
    y = fmaf(a, d, b * c);
}

// For local edges e = 0..E-1 with u[e] = exp(-|q_e|), call
// emit(e, alpha_e, beta_e) where alpha_e I + beta_e J is
// (oa I + ob J) * prod_{k != e} (I + u_k J).
template <int E, typename Emit>
__device__ __forceinline__ void exclusive_products(const float (&u)[E], float oa, float ob,
                                                   Emit &&emit) {
    if constexpr (E <= 6) {
        float pa[E], pb[E];
        pa[0] = oa;
        pb[0] = ob;
#pragma unroll
        for (int e = 1; e < E; ++e) {
            pa[e] = fmaf(u[e - 1], pb[e - 1], pa[e - 1]);
            pb[e] = fmaf(u[e - 1], pa[e - 1], pb[e - 1]);
        }
        float sa = 1.0f, sb = 0.0f;
#pragma unroll
        for (int e = E - 1; e >= 0; --e) {
            float a, b;
            cmul(pa[e], pb[e], sa, sb, a, b);
            const float nsa = fmaf(u[e], sb, sa);
            const float nsb = fmaf(u[e], sa, sb);
            sa = nsa;
            sb = nsb;
            emit(e, a, b);
        }
    } else {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            float a = oa, b = ob;
#pragma unroll
            for (int k = 0; k < E; ++k) {
                if (k == e) continue;
                const float na = fmaf(u[k], b, a);
                const float nb = fmaf(u[k], a, b);
                a = na;
                b = nb;
            }
            emit(e, a, b);
        }
    }
}

__device__ __forceinline__ float u_of(float q) {
    return ex2_ftz(-kLog2e * fminf(fabsf(q), kClipMax));
}

// ---- two frames at once ---------------------------------------------------------
//
// Two FP32 values in one 64-bit register pair.  The .f32x2 forms of add, sub,
// mul and fma (sm_100 and later) apply the IEEE operation to each lane, so a
// packed evaluation rounds exactly as two scalar ones: kernels that keep
// several frames per thread run the rule on pairs of frames and still give
// the results of the scalar code bit for bit.
struct f2 {
    unsigned long long v;
};
__device__ __forceinline__ f2 f2_make(float lo, float hi) {
    f2 r;
    r.v = ((unsigned long long)__float_as_uint(hi) << 32) | __float_as_uint(lo);
    return r;
}
__device__ __forceinline__ f2 f2_splat(float x) { return f2_make(x, x); }
__device__ __forceinline__ float f2_lo(f2 a) { return __uint_as_float((unsigned)a.v); }
__device__ __forceinline__ float f2_hi(f2 a) { return __uint_as_float((unsigned)(a.v >> 32)); }
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b) {
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
// a * b + c, rounded once per lane (fmaf)
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}

// exclusive_products on two frames at once: the same operations in the same
// order, lane by lane (keep the two in step).
template <int E, typename Emit>
__device__ __forceinline__ void exclusive_products2(const f2 (&u)[E], f2 oa, f2 ob, Emit &&emit) {
    if constexpr (E <= 6) {
        f2 pa[E], pb[E];
        pa[0] = oa;
        pb[0] = ob;
#pragma unroll
        for (int e = 1; e < E; ++e) {
            pa[e] = f2_fma(u[e - 1], pb[e - 1], pa[e - 1]);
            pb[e] = f2_fma(u[e - 1], pa[e - 1], pb[e - 1]);
        }
        f2 sa = f2_splat(1.0f), sb = f2_splat(0.0f);
#pragma unroll
        for (int e = E - 1; e >= 0; --e) {
            // cmul(pa, pb, sa, sb)
            const f2 a = f2_fma(pa[e], sa, f2_mul(pb[e], sb));
            const f2 b = f2_fma(pa[e], sb, f2_mul(pb[e], sa));
            const f2 nsa = f2_fma(u[e], sb, sa);
            const f2 nsb = f2_fma(u[e], sa, sb);
            sa = nsa;
            sb = nsb;
            emit(e, a, b);
        }
    } else {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            f2 a = oa, b = ob;
#pragma unroll
            for (int k = 0; k < E; ++k) {
                if (k == e) continue;
                const f2 na = f2_fma(u[k], b, a);
                const f2 nb = f2_fma(u[k], a, b);
                a = na;
                b = nb;
            }
            emit(e, a, b);
        }
    }
}

// u_of on two frames: |q| clipped per lane, the scaling packed, exp2 per lane.
__device__ __forceinline__ f2 u_of2(float q0, float q1) {
    const f2 t = f2_mul(f2_splat(-kLog2e),
                        f2_make(fminf(fabsf(q0), kClipMax), fminf(fabsf(q1), kClipMax)));
    return f2_make(ex2_ftz(f2_lo(t)), ex2_ftz(f2_hi(t)));
}

}  // namespace qcmet
