// Frame-interleaved, clustered layered BP decoder (arXiv 2004.09084, Methods,
// steps 1-4) for GB300 (sm_103a).
//
// The per-frame kernel of decode.cu gives one CTA a whole frame; every access
// there is a 4- or 8-byte request, and the SM's rate of such requests, not
// DRAM, bounds it.  This kernel stores the frames of a group of four side by
// side -- the four frames' values of one variable (or message, or syndrome
// bit) form one 16-byte word -- so that every posterior, message and channel
// access is a single aligned 16-byte request whatever the circulant shift,
// and one thread computes one check for four frames.
//
//  * Mapping: a thread-block cluster of C CTAs (1 .. 16) owns one or two
//    groups of four frames.  The groups' checks form one range [0, NG Zp)
//    (group 1's start at Zp, Z rounded up to 32), and CTA r of the cluster
//    owns [r Zc, (r + 1) Zc) of it in every row (Zc = ceil(NG Zp / C)
//    rounded up to 32), so that a CTA may hold checks of both groups; two
//    groups per cluster let cluster sizes that do not divide the SM count
//    evenly keep more SMs busy.  Rows of one layer share no column, so a
//    layer needs no synchronisation inside; between layers the posteriors
//    written by one CTA are read by others, so a layer ends with one cluster
//    barrier (barrier.cluster arrive.release / wait.acquire).  Cross-CTA data
//    are read through L2 only (cp.async.cg, ld.global.cg).  The host picks C
//    and the groups per cluster from the device's cluster occupancy, to
//    minimise the checks per SM (times the waves of clusters).
//  * Layouts in library scratch, per group g: channel LLRs [nb][Zp] float4,
//    syndrome bits [mb][Zp] as four bytes, core posteriors [core_cols][Zp]
//    float4, messages [slots][Zp] as four FP32 (16 B) or four 16-bit values
//    (8 B); every row starts on a 128-byte line.  The kernel builds the
//    interleaved channel and syndrome from the caller's frame-major arrays
//    in its prologue and writes the caller's frame-major outputs in its
//    epilogue.  Degree-1 columns keep no state (their
//    q = L_qn - L_rmn(old) is the channel LLR exactly); in the last iteration
//    their posterior replaces the interleaved channel value, which only their
//    own check reads.
//  * Rows of degree <= 4: one thread per check, operands of the next rounds
//    copied into the thread's own shared-memory slots by cp.async while it
//    computes the current round (no block barrier: each thread reads only the
//    slots it filled).  Rows of degree 5..16: two lanes per check; up to
//    degree 12 each lane stages the next 16 checks' operands the same way.
//  * The check rule is check_rule.cuh's exclusive-product form, evaluated per
//    frame in the same operation order as the per-frame kernel, so the two
//    kernels give bit-identical results.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <type_traits>

#include "check_rule.cuh"
#include "qcmet_internal.h"

namespace qcmet {

namespace {

constexpr int kGF = 4;                  // frames per group
constexpr int kGroupStages = 3;         // rounds staged by the rows of degree <= 4 (every variant)
constexpr int kPairStagedMax = 12;      // rows of degree 5 .. 12 stage their operands too

extern __shared__ float4 qcmet_group_smem[];

// ---- cluster primitives -------------------------------------------------------
__device__ __forceinline__ unsigned cluster_ctarank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_nctarank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_idx() {
    unsigned r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
// Every thread of every CTA of the cluster arrives; writes before the arrive
// (release) are visible to reads after the wait (acquire) in any CTA of it.
__device__ __forceinline__ void cluster_sync() {
    asm volatile(
        "barrier.cluster.arrive.release.aligned;\n\t"
        "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// ---- memory accesses with an L2 eviction policy ---------------------------------
//
// Every access of the grouped kernel names an L2 policy (createpolicy).  Per
// iteration the messages (2.9 GB at 128 frames of the rate-0.1 Z = 12500
// code, FP32), channel LLRs and syndrome bits stream through L2 once, while
// the core posteriors (64 MB) are read and written again by about a third of
// the rows.  Marking the stream evict-first keeps most of the posteriors in
// L2: measured at 128 frames x 20 iterations, DRAM bytes per launch fell from
// 110 to 80 GB with FP32 messages (and from 73 to 53 GB with FP16 messages
// when the posteriors are also marked evict-last) and the decode took 7 %
// (17 %) less time.  Level 1 marks the messages, 2 also the channel and
// syndrome, 3 also the posteriors evict-last.  (An access-policy window on
// top of these policies slowed the decode, so the grouped kernel takes none.)
#ifndef QCMET_GROUP_HINT_FP32
#define QCMET_GROUP_HINT_FP32 2
#endif
#ifndef QCMET_GROUP_HINT_16BIT
#define QCMET_GROUP_HINT_16BIT 3
#endif
struct Policies {
    uint64_t msg;   // messages (read once and written once per iteration)
    uint64_t in;    // interleaved channel and syndrome (read once per iteration)
    uint64_t post;  // core posteriors (read and written by about a third of the rows)
};
__device__ __forceinline__ uint64_t policy_normal() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
template <int Level>
__device__ __forceinline__ Policies make_policies() {
    Policies p;
    p.msg = Level >= 1 ? policy_first() : policy_normal();
    p.in = Level >= 2 ? policy_first() : policy_normal();
    p.post = Level >= 3 ? policy_last() : policy_normal();
    return p;
}

// global -> shared copies, through L2 only (16 B) or L1 (8 B)
__device__ __forceinline__ void cp_async16_cg(uint32_t dst, const void *src, uint64_t pol) {
    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;\n" ::"r"(dst),
                 "l"(src), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void cp_async8_ca(uint32_t dst, const void *src, uint64_t pol) {
    asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 8, %2;\n" ::"r"(dst),
                 "l"(src), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ float4 ld16(const float4 *p, uint64_t pol) {
    float4 v;
    asm volatile("ld.global.cg.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ uint2 ld8(const uint2 *p, uint64_t pol) {
    uint2 v;
    asm volatile("ld.global.cg.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;"
                 : "=r"(v.x), "=r"(v.y)
                 : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ uint32_t ld4(const uint32_t *p, uint64_t pol) {
    uint32_t v;
    asm volatile("ld.global.cg.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ void st16(float4 *p, const float4 &v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(v.x),
                 "f"(v.y), "f"(v.z), "f"(v.w), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void st8(uint2 *p, const uint2 &v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v2.u32 [%0], {%1, %2}, %3;" ::"l"(p), "r"(v.x),
                 "r"(v.y), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void g_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void g_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ---- four frames' values -------------------------------------------------------
__device__ __forceinline__ float comp(const float4 &v, int f) {
    return f == 0 ? v.x : f == 1 ? v.y : f == 2 ? v.z : v.w;
}

__device__ __forceinline__ void set_comp(float4 &v, int f, float x) {
    if (f == 0) v.x = x;
    else if (f == 1) v.y = x;
    else if (f == 2) v.z = x;
    else v.w = x;
}

// Check rules: the paper's sum-product rule, or offset/scaled min-sum (the
// learned variant) with weights wt = (scale of an edge to a core variable,
// scale of an edge to a degree-1 variable, offset core, offset degree-1) of
// the row and iteration.
enum : int { kGroupSumProduct = 0, kGroupMinSum = 1 };
constexpr float kGroupNoOtherEdge = 30.0f;  // min over the empty set (a degree-1 check)

// Frames (0, 1) and (2, 3) of a float4 as packed pairs.
__device__ __forceinline__ f2 half_of(const float4 &v, int h) {
    return h == 0 ? f2_make(v.x, v.y) : f2_make(v.z, v.w);
}
__device__ __forceinline__ void set_half(float4 &v, int h, f2 x) {
    if (h == 0) {
        v.x = f2_lo(x);
        v.y = f2_hi(x);
    } else {
        v.z = f2_lo(x);
        v.w = f2_hi(x);
    }
}

// The new message and posterior of edge e for a pair of frames, from the
// exclusive products (a, b) (check_rule.cuh): |r| = ln(a / b) clipped to
// [Phi(30), 30], the sign from the parities p0, p1 (syndrome and the other
// edges' signs); a message that is stored (an edge to a core variable) is
// rounded to the storage format.  Returns r and writes q + r.
template <typename M, bool Stored>
__device__ __forceinline__ f2 emit_pair(f2 a, f2 b, f2 q, unsigned p0, unsigned p1, f2 &post) {
    const f2 d = f2_sub(f2_make(lg2_ftz(f2_lo(a)), lg2_ftz(f2_hi(a))),
                        f2_make(lg2_ftz(f2_lo(b)), lg2_ftz(f2_hi(b))));
    const f2 mag = f2_mul(f2_splat(kLn2), d);
    const float m0 = fminf(fmaxf(f2_lo(mag), kClipMin), kClipMax);
    const float m1 = fminf(fmaxf(f2_hi(mag), kClipMin), kClipMax);
    const float q0 = f2_lo(q), q1 = f2_hi(q);
    const bool n0 = ((p0 ^ (q0 < 0.0f ? 1u : 0u)) & 1u) != 0u;
    const bool n1 = ((p1 ^ (q1 < 0.0f ? 1u : 0u)) & 1u) != 0u;
    float r0 = n0 ? -m0 : m0, r1 = n1 ? -m1 : m1;
    if (Stored) {
        r0 = Msg<M>::quantize(r0);
        r1 = Msg<M>::quantize(r1);
    }
    const f2 r = f2_make(r0, r1);
    post = f2_add(q, r);
    return r;
}

// Messages of four frames: FP32 as one float4 (16 B), 16-bit formats as four
// packed values (8 B).
template <typename M>
struct MsgVec;

template <>
struct MsgVec<float> {
    using V = float4;
    static __device__ __forceinline__ void copy_async(uint32_t dst, const V *src, uint64_t pol) {
        cp_async16_cg(dst, src, pol);
    }
    static __device__ __forceinline__ float4 from_stage(const float4 *p) { return *p; }
    static __device__ __forceinline__ float4 load(const V *p, uint64_t pol) { return ld16(p, pol); }
    static __device__ __forceinline__ void store(V *p, const float4 &v, uint64_t pol) {
        st16(p, v, pol);
    }
};

template <>
struct MsgVec<__half> {
    using V = uint2;
    static __device__ __forceinline__ void copy_async(uint32_t dst, const V *src, uint64_t pol) {
        cp_async8_ca(dst, src, pol);
    }
    static __device__ __forceinline__ float4 unpack(uint2 u) {
        const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&u.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&u.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
    static __device__ __forceinline__ float4 from_stage(const float4 *p) {
        return unpack(*reinterpret_cast<const uint2 *>(p));
    }
    static __device__ __forceinline__ float4 load(const V *p, uint64_t pol) {
        return unpack(ld8(p, pol));
    }
    // v holds values already rounded to half, so the conversion is exact
    static __device__ __forceinline__ void store(V *p, const float4 &v, uint64_t pol) {
        const __half2 a = __floats2half2_rn(v.x, v.y);
        const __half2 b = __floats2half2_rn(v.z, v.w);
        uint2 u;
        u.x = *reinterpret_cast<const uint32_t *>(&a);
        u.y = *reinterpret_cast<const uint32_t *>(&b);
        st8(p, u, pol);
    }
};

template <>
struct MsgVec<__nv_bfloat16> {
    using V = uint2;
    static __device__ __forceinline__ void copy_async(uint32_t dst, const V *src, uint64_t pol) {
        cp_async8_ca(dst, src, pol);
    }
    static __device__ __forceinline__ float4 unpack(uint2 u) {
        const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.x));
        const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
    static __device__ __forceinline__ float4 from_stage(const float4 *p) {
        return unpack(*reinterpret_cast<const uint2 *>(p));
    }
    static __device__ __forceinline__ float4 load(const V *p, uint64_t pol) {
        return unpack(ld8(p, pol));
    }
    static __device__ __forceinline__ void store(V *p, const float4 &v, uint64_t pol) {
        const __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y);
        const __nv_bfloat162 b = __floats2bfloat162_rn(v.z, v.w);
        uint2 u;
        u.x = *reinterpret_cast<const uint32_t *>(&a);
        u.y = *reinterpret_cast<const uint32_t *>(&b);
        st8(p, u, pol);
    }
};

// Sign bits of four frames' values, one per byte (the layout of a syndrome word).
__device__ __forceinline__ uint32_t sign_bytes(const float4 &v) {
    return (v.x < 0.0f ? 1u : 0u) | (v.y < 0.0f ? 0x100u : 0u) | (v.z < 0.0f ? 0x10000u : 0u) |
           (v.w < 0.0f ? 0x1000000u : 0u);
}

// Views of one group's arrays.
template <typename M>
struct GFrame {
    float4 *ch4;                     // [nb][Zp] channel (degree-1 posteriors after the last iteration)
    const uint32_t *syn4;            // [mb][Zp] syndrome bit of frame f in byte f
    float4 *core4;                   // [core_cols][Zp] posteriors of the core columns
    typename MsgVec<M>::V *msg4;     // [slots][Zp] messages
    Policies pol;
    Bounds bd;                       // extents for the debug build's index checks
    int zp;                          // row stride of the arrays (Z rounded up to 32)
    GroupScratch gstride;            // bytes from each array to the next group's
};

// A cluster that owns two groups numbers their checks (and variables) in one
// virtual range: group 0's index v at v, group 1's at Zp + v.  Indices Z ..
// Zp - 1 of a group are padding and stand for no check.
struct VIndex {
    int g;    // group within the cluster (0 or 1)
    int l;    // index within the group; a check or variable when l < Z
};
// With one group per cluster (NG = 1) the virtual range is the group's own
// [0, Z) and both helpers reduce to the identity.
template <int NG>
__device__ __forceinline__ VIndex vsplit(int v, int zp) {
    if constexpr (NG == 1) {
        return VIndex{0, v};
    } else {
        const int g = v >= zp ? 1 : 0;
        return VIndex{g, v - g * zp};
    }
}
// whether a virtual index stands for a check or variable (not padding)
template <int NG>
__device__ __forceinline__ bool real(const VIndex &x, int Z) {
    return NG == 1 || x.l < Z;
}
// p moved from group 0's arrays to group g's (gstride: bytes between the
// groups' copies of p's array)
template <int NG, typename T>
__device__ __forceinline__ T *in_group(T *p, int g, size_t gstride) {
    if constexpr (NG == 1) {
        return p;
    } else {
        using B = typename std::conditional<std::is_const<T>::value, const char, char>::type;
        return reinterpret_cast<T *>(reinterpret_cast<B *>(p) + (g ? gstride : 0));
    }
}

// The check rule on one check of a row of degree DC + D1 <= 4 (core edges
// first) for four frames: lv holds the edges' posteriors (channel LLRs for
// degree-1 columns), ro the old messages of the core edges (zero in the first
// iteration), sy the syndrome bits (frame f in byte f).  The new messages
// replace ro and the new posteriors lv (a degree-1 edge's only in the last
// iteration).
template <int DC, int D1, typename M, int R>
__device__ __forceinline__ void small_rule(float4 (&lv)[DC + D1], float4 (&ro)[DC > 0 ? DC : 1],
                                           uint32_t sy, bool last, float4 wt) {
    constexpr int D = DC + D1;
    if constexpr (R == kGroupMinSum) {
        // min-sum, frame by frame (comparisons, no transcendentals); the
        // operations of the frame kernel's min-sum rows
#pragma unroll
        for (int f = 0; f < kGF; ++f) {
            float q[D];
            unsigned p = (sy >> (8 * f)) & 1u;
            float m1 = INFINITY, m2 = INFINITY;
            int i1 = -1;
#pragma unroll
            for (int e = 0; e < D; ++e) {
                q[e] = e < DC ? comp(lv[e], f) - comp(ro[e < DC ? e : 0], f) : comp(lv[e], f);
                p ^= q[e] < 0.0f ? 1u : 0u;
                const float v = fabsf(q[e]);
                if (v < m1) {
                    m2 = m1;
                    m1 = v;
                    i1 = e;
                } else if (v < m2) {
                    m2 = v;
                }
            }
#pragma unroll
            for (int e = 0; e < D; ++e) {
                if (e >= DC && !last) continue;
                const float mn = D == 1 ? kGroupNoOtherEdge : (e == i1 ? m2 : m1);
                const float a_e = (e >= DC ? wt.y : wt.x) * mn - (e >= DC ? wt.w : wt.z);
                const float mag = fminf(fmaxf(a_e, 0.0f), kClipMax);
                const bool neg = ((p ^ (q[e] < 0.0f ? 1u : 0u)) & 1u) != 0u;
                float rn = neg ? -mag : mag;
                if (e < DC) {
                    rn = Msg<M>::quantize(rn);
                    set_comp(ro[e < DC ? e : 0], f, rn);
                }
                set_comp(lv[e], f, q[e] + rn);
            }
        }
    } else {
        // two frames at a time (packed); their results replace their lanes of
        // the operands (the new message in ro, the posterior q + r in lv)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            f2 q[D], u[D];
            unsigned p0 = (sy >> (16 * h)) & 1u;
            unsigned p1 = (sy >> (16 * h + 8)) & 1u;
#pragma unroll
            for (int e = 0; e < D; ++e) {
                const f2 l = half_of(lv[e], h);
                q[e] = e < DC ? f2_sub(l, half_of(ro[e < DC ? e : 0], h)) : l;
                const float q0 = f2_lo(q[e]), q1 = f2_hi(q[e]);
                p0 ^= q0 < 0.0f ? 1u : 0u;
                p1 ^= q1 < 0.0f ? 1u : 0u;
                u[e] = u_of2(q0, q1);
            }
            exclusive_products2<D>(u, f2_splat(1.0f), f2_splat(0.0f), [&](int e, f2 a, f2 b) {
                if (e >= DC && !last) return;
                f2 post;
                if (e < DC) {
                    const f2 r = emit_pair<M, true>(a, b, q[e], p0, p1, post);
                    set_half(ro[e < DC ? e : 0], h, r);
                } else {
                    emit_pair<M, false>(a, b, q[e], p0, p1, post);
                }
                set_half(lv[e], h, post);
            });
        }
    }
}

// Rows of degree DC + D1 <= 4 (core edges first), one thread per check and
// four frames, software-pipelined through shared memory: while a thread
// computes round k, the operands of rounds k + 1 .. k + S - 1 are being
// copied into its own staging slots.  Rounds of a row touch disjoint
// variables and message slots (a circulant is a permutation), so copying later
// rounds before round k's stores reads nothing those stores change.
// Staging: [S rounds][D + DC operands][blockDim] 16-byte slots.
// (Each row routine is its own function: it runs once per row and layer, and
// a separate register allocation keeps the rows that a code rarely has from
// costing the others spills.)
template <int DC, int D1, typename M, int S, int R, int NG>
__device__ __noinline__ void grow_small(const int4 *__restrict__ ent, int check_base,
                                        const GFrame<M> fr, int lo, int hi, int Z, bool first,
                                        bool last, float4 wt) {
    constexpr int D = DC + D1;
    constexpr int NC = DC > 0 ? DC : 1;
    constexpr int NOP = D + DC;
    using MV = MsgVec<M>;
    using V = typename MV::V;
    const int nt = blockDim.x;
    const int tid = threadIdx.x;
    const uint32_t opb = (uint32_t)nt * 16u;  // bytes between operands
    const uint32_t rb = NOP * opb;            // bytes between rounds
    const float4 *src[D];
    int sh[D];
    V *slot[NC];
    int xo[D], zo[NC];  // variable and slot offsets (index checks of the debug build)
    size_t vs[D];       // bytes to the next group's copy of the edge's variables
#pragma unroll
    for (int e = 0; e < D; ++e) {
        const int4 en = ent[e];
        src[e] = (e < DC ? fr.core4 : fr.ch4) + en.x;
        vs[e] = e < DC ? fr.gstride.core : fr.gstride.ch;
        sh[e] = en.y;
        xo[e] = en.x;
        if (e < DC) {
            slot[e] = fr.msg4 + (size_t)en.z * (size_t)fr.zp;
            zo[e] = en.z;
        }
    }
    const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(qcmet_group_smem + tid);
    const int zp = fr.zp;
    auto issue = [&](int i, int b) {
        const VIndex c = vsplit<NG>(i, zp);
        if (i < hi && real<NG>(c, Z)) {
            const uint32_t sb = s0 + (uint32_t)b * rb;
#pragma unroll
            for (int e = 0; e < D; ++e) {
                int j = c.l + sh[e];
                j = j >= Z ? j - Z : j;
                if (in_range((long long)xo[e] + j, e < DC ? fr.bd.core : fr.bd.vars, kBadVariable))
                    cp_async16_cg(sb + e * opb, in_group<NG>(src[e] + j, c.g, vs[e]),
                                  e < DC ? fr.pol.post : fr.pol.in);
            }
            if (!first) {
#pragma unroll
                for (int e = 0; e < DC; ++e)
                    if (in_range((long long)zo[e] * zp + c.l, fr.bd.msgs, kBadSlot))
                        MV::copy_async(sb + (D + e) * opb,
                                       in_group<NG>(slot[e] + c.l, c.g, fr.gstride.msg), fr.pol.msg);
            }
        }
        g_commit();
    };
    auto syndrome = [&](int i) {
        const VIndex c = vsplit<NG>(i, zp);
        return (i < hi && real<NG>(c, Z) &&
                in_range((long long)check_base + c.l, fr.bd.checks, kBadCheck))
                   ? ld4(in_group<NG>(fr.syn4 + check_base + c.l, c.g, fr.gstride.syn), fr.pol.in)
                   : 0u;
    };
    uint32_t sy[S];
#pragma unroll
    for (int k = 0; k < S - 1; ++k) {
        const int i = lo + tid + k * nt;
        sy[k] = syndrome(i);
        issue(i, k);
    }
    int buf = 0;
    for (int i = lo + tid; i < hi; i += nt) {
        {
            const int nx = i + (S - 1) * nt;
            int nb = buf + (S - 1);
            nb = nb >= S ? nb - S : nb;
            sy[S - 1] = syndrome(nx);
            issue(nx, nb);
        }
        g_wait<S - 1>();
        const VIndex c = vsplit<NG>(i, zp);
        if (real<NG>(c, Z)) {
            const float4 *sv = qcmet_group_smem + tid + (size_t)buf * (rb / 16);
            float4 lv[D], ro[NC];
#pragma unroll
            for (int e = 0; e < D; ++e) lv[e] = sv[(size_t)e * nt];
#pragma unroll
            for (int e = 0; e < DC; ++e)
                ro[e] = first ? make_float4(0.f, 0.f, 0.f, 0.f)
                              : MV::from_stage(sv + (size_t)(D + e) * nt);
            small_rule<DC, D1, M, R>(lv, ro, sy[0], last, wt);
#pragma unroll
            for (int e = 0; e < D; ++e) {
                if (e >= DC && !last) continue;
                int j = c.l + sh[e];
                j = j >= Z ? j - Z : j;
                if (e < DC && in_range((long long)zo[e < DC ? e : 0] * zp + c.l, fr.bd.msgs, kBadSlot))
                    MV::store(in_group<NG>(slot[e < DC ? e : 0] + c.l, c.g, fr.gstride.msg),
                              ro[e < DC ? e : 0], fr.pol.msg);
                if (in_range((long long)xo[e] + j, e < DC ? fr.bd.core : fr.bd.vars, kBadVariable))
                    st16(in_group<NG>(const_cast<float4 *>(src[e]) + j, c.g, vs[e]), lv[e],
                         e < DC ? fr.pol.post : fr.pol.in);
            }
        }
#pragma unroll
        for (int k = 0; k < S - 1; ++k) sy[k] = sy[k + 1];
        buf = buf + 1 == S ? 0 : buf + 1;
    }
}

// Rows of degree 5..16: lanes l and l ^ 16 of a warp share a check, each lane
// owning E = ceil(D/2) edges; the lanes swap their partial products and sign
// parities with shuffles.  Results overwrite the operands in registers and
// are stored as whole 16-byte words.  STAGED: a lane copies the operands of
// the warp's next 16 checks into its own shared-memory slots (cp.async, two
// rounds of 2 E slots) while it computes the current ones; otherwise it loads
// all its edges' operands, then computes.  Both give the same operands.
template <int D, typename M, int R, bool STAGED, int NG>
__device__ __noinline__ void grow_pair(const int4 *__restrict__ ent, int check_base,
                                       const GFrame<M> fr, int lo, int hi, int Z, bool first,
                                       bool last, float4 wt) {
    constexpr int E = (D + 1) / 2;
    using MV = MsgVec<M>;
    const int tid = threadIdx.x;
    const int nt = blockDim.x;
    const int lane = tid & 31;
    const int part = lane >> 4;
    const int warp = tid >> 5;
    const int nwarps = nt >> 5;
    // staging: [2 rounds][2 E slots][nt] 16-byte words, slot el the posterior
    // of the lane's edge el, slot E + el its old message
    const uint32_t opb = (uint32_t)nt * 16u;
    const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(qcmet_group_smem + tid);
    // an edge's variable j (posterior, or channel LLR of a degree-1 column) and
    // its message of check l, in group g's arrays
    auto var_of = [&](const int4 &en, int j, int g) {
        return in_group<NG>((en.z < 0 ? fr.ch4 : fr.core4) + en.x + j, g,
                            en.z < 0 ? fr.gstride.ch : fr.gstride.core);
    };
    auto msg_of = [&](const int4 &en, int l, int g) {
        return in_group<NG>(fr.msg4 + (size_t)en.z * (size_t)fr.zp + l, g, fr.gstride.msg);
    };
    auto issue = [&](int i0, int b) {
        const int i = i0 + (lane & 15);
        const VIndex c = vsplit<NG>(i, fr.zp);
        if (i0 < hi && i < hi && real<NG>(c, Z)) {
#pragma unroll
            for (int el = 0; el < E; ++el) {
                const int e = part * E + el;
                if (e >= D) continue;
                const int4 en = ent[e];
                int j = c.l + en.y;
                j = j >= Z ? j - Z : j;
                const uint32_t sb = s0 + (uint32_t)(b * 2 * E + el) * opb;
                if (in_range((long long)en.x + j, en.z < 0 ? fr.bd.vars : fr.bd.core, kBadVariable))
                    cp_async16_cg(sb, var_of(en, j, c.g), en.z < 0 ? fr.pol.in : fr.pol.post);
                if (!first && en.z >= 0 &&
                    in_range((long long)en.z * fr.zp + c.l, fr.bd.msgs, kBadSlot))
                    MV::copy_async(sb + (uint32_t)E * opb, msg_of(en, c.l, c.g), fr.pol.msg);
            }
        }
        g_commit();
    };
    if constexpr (STAGED) issue(lo + warp * 16, 0);
    int b = 0;
    for (int i0 = lo + warp * 16; i0 < hi; i0 += nwarps * 16) {
        const int i = i0 + (lane & 15);
        const VIndex c = vsplit<NG>(i, fr.zp);
        const bool valid = i < hi && real<NG>(c, Z);
        if constexpr (STAGED) issue(i0 + nwarps * 16, b ^ 1);
        const uint32_t par4 =
            (valid && part == 0 && in_range((long long)check_base + c.l, fr.bd.checks, kBadCheck))
                ? ld4(in_group<NG>(fr.syn4 + check_base + c.l, c.g, fr.gstride.syn), fr.pol.in)
                : 0u;
        float4 lv[E], ro[E];
        if constexpr (STAGED) {
            g_wait<1>();
            const float4 *sv = qcmet_group_smem + tid + (size_t)b * 2 * E * nt;
#pragma unroll
            for (int el = 0; el < E; ++el) {
                const int e = min(part * E + el, D - 1);
                lv[el] = sv[(size_t)el * nt];
                ro[el] = (!first && ent[e].z >= 0) ? MV::from_stage(sv + (size_t)(E + el) * nt)
                                                   : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            b ^= 1;
        } else {
#pragma unroll
            for (int el = 0; el < E; ++el) {
                const int e = min(part * E + el, D - 1);
                const int4 en = ent[e];
                int j = c.l + en.y;
                j = j >= Z ? j - Z : j;
                lv[el] = (valid && in_range((long long)en.x + j, en.z < 0 ? fr.bd.vars : fr.bd.core,
                                            kBadVariable))
                             ? ld16(var_of(en, j, c.g), en.z < 0 ? fr.pol.in : fr.pol.post)
                             : make_float4(0.f, 0.f, 0.f, 0.f);
                ro[el] = (valid && !first && en.z >= 0 &&
                          in_range((long long)en.z * fr.zp + c.l, fr.bd.msgs, kBadSlot))
                             ? MV::load(msg_of(en, c.l, c.g), fr.pol.msg)
                             : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        if constexpr (R == kGroupMinSum) {
            // min-sum, frame by frame: each lane finds the two smallest |q| of
            // its edges and takes the partner lane's smallest by one shuffle
            // (the frame kernel's min-sum pair rows)
#pragma unroll
            for (int f = 0; f < kGF; ++f) {
                float q[E];
                unsigned par = (par4 >> (8 * f)) & 1u;
                float m1 = INFINITY, m2 = INFINITY;
                int i1 = -1;
#pragma unroll
                for (int el = 0; el < E; ++el) {
                    const int e = part * E + el;
                    q[el] = 0.0f;
                    if (valid && e < D) {
                        q[el] = comp(lv[el], f) - comp(ro[el], f);
                        par ^= q[el] < 0.0f ? 1u : 0u;
                        const float v = fabsf(q[el]);
                        if (v < m1) {
                            m2 = m1;
                            m1 = v;
                            i1 = el;
                        } else if (v < m2) {
                            m2 = v;
                        }
                    }
                }
                const float om1 = __shfl_xor_sync(0xffffffffu, m1, 16);
                par ^= __shfl_xor_sync(0xffffffffu, par, 16);
                const float ex1 = fminf(m2, om1);
                const float exo = fminf(m1, om1);
#pragma unroll
                for (int el = 0; el < E; ++el) {
                    const int e = part * E + el;
                    if (e >= D) continue;
                    const bool deg1 = ent[e].z < 0;
                    if (deg1 && !last) continue;
                    const float mn = el == i1 ? ex1 : exo;
                    const float a_e = (deg1 ? wt.y : wt.x) * mn - (deg1 ? wt.w : wt.z);
                    const float mag = fminf(fmaxf(a_e, 0.0f), kClipMax);
                    const bool neg = ((par ^ (q[el] < 0.0f ? 1u : 0u)) & 1u) != 0u;
                    float rn = neg ? -mag : mag;
                    if (!deg1) {
                        rn = Msg<M>::quantize(rn);
                        set_comp(ro[el], f, rn);
                    }
                    set_comp(lv[el], f, q[el] + rn);
                }
            }
        } else {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            f2 q[E], u[E];
            unsigned p0 = (par4 >> (16 * h)) & 1u;
            unsigned p1 = (par4 >> (16 * h + 8)) & 1u;
#pragma unroll
            for (int el = 0; el < E; ++el) {
                const bool own = part * E + el < D;
                q[el] = own ? f2_sub(half_of(lv[el], h), half_of(ro[el], h)) : f2_splat(0.0f);
                const float q0 = f2_lo(q[el]), q1 = f2_hi(q[el]);
                p0 ^= (own && q0 < 0.0f) ? 1u : 0u;
                p1 ^= (own && q1 < 0.0f) ? 1u : 0u;
                u[el] = own ? u_of2(q0, q1) : f2_splat(0.0f);  // 0: the identity factor I + 0 J
            }
            f2 ta = f2_splat(1.0f), tb = f2_splat(0.0f);
#pragma unroll
            for (int el = 0; el < E; ++el) {
                const f2 na = f2_fma(u[el], tb, ta);
                const f2 nb = f2_fma(u[el], ta, tb);
                ta = na;
                tb = nb;
            }
            f2 oa, ob;
            oa.v = __shfl_xor_sync(0xffffffffu, ta.v, 16);
            ob.v = __shfl_xor_sync(0xffffffffu, tb.v, 16);
            const unsigned pp = __shfl_xor_sync(0xffffffffu, p0 | (p1 << 1), 16);
            p0 ^= pp & 1u;
            p1 ^= pp >> 1;
            exclusive_products2<E>(u, oa, ob, [&](int el, f2 a, f2 b) {
                const int e = part * E + el;
                if (e >= D) return;
                const bool deg1 = ent[e].z < 0;
                if (deg1 && !last) return;
                f2 post;
                if (!deg1) {
                    const f2 r = emit_pair<M, true>(a, b, q[el], p0, p1, post);
                    set_half(ro[el], h, r);
                } else {
                    emit_pair<M, false>(a, b, q[el], p0, p1, post);
                }
                set_half(lv[el], h, post);
            });
        }
        }
        if (!valid) continue;
#pragma unroll
        for (int el = 0; el < E; ++el) {
            const int e = part * E + el;
            if (e >= D) continue;
            const int4 en = ent[e];
            if (en.z < 0 && !last) continue;
            int j = c.l + en.y;
            j = j >= Z ? j - Z : j;
            if (en.z >= 0) {
                if (in_range((long long)en.z * fr.zp + c.l, fr.bd.msgs, kBadSlot))
                    MV::store(msg_of(en, c.l, c.g), ro[el], fr.pol.msg);
                if (in_range((long long)en.x + j, fr.bd.core, kBadVariable))
                    st16(var_of(en, j, c.g), lv[el], fr.pol.post);
            } else if (in_range((long long)en.x + j, fr.bd.vars, kBadVariable)) {
                st16(var_of(en, j, c.g), lv[el], fr.pol.in);
            }
        }
    }
}

template <typename M, int S, int R, int NG>
__device__ __forceinline__ void gdispatch(int degree, const int4 *ent, int check_base,
                                          const GFrame<M> &fr, int lo, int hi, int Z, bool first,
                                          bool last, float4 wt) {
    if (degree <= 4) {
        int dc = 0;
        for (int e = 0; e < degree; ++e) dc += ent[e].z >= 0 ? 1 : 0;
        switch (degree * 8 + dc) {
#define QCMET_GSMALL_CASE(DD, CC)                                                            \
    case DD * 8 + CC:                                                                        \
        grow_small<CC, DD - CC, M, S, R, NG>(ent, check_base, fr, lo, hi, Z, first, last, wt); \
        break;
            QCMET_GSMALL_CASE(1, 0)
            QCMET_GSMALL_CASE(1, 1)
            QCMET_GSMALL_CASE(2, 0)
            QCMET_GSMALL_CASE(2, 1)
            QCMET_GSMALL_CASE(2, 2)
            QCMET_GSMALL_CASE(3, 0)
            QCMET_GSMALL_CASE(3, 1)
            QCMET_GSMALL_CASE(3, 2)
            QCMET_GSMALL_CASE(3, 3)
            QCMET_GSMALL_CASE(4, 0)
            QCMET_GSMALL_CASE(4, 1)
            QCMET_GSMALL_CASE(4, 2)
            QCMET_GSMALL_CASE(4, 3)
            QCMET_GSMALL_CASE(4, 4)
#undef QCMET_GSMALL_CASE
            default: break;
        }
        return;
    }
    switch (degree) {
// rows of degree <= kPairStagedMax are staged (the staging area holds their
// two rounds: group_stage_ops), higher ones load directly
#define QCMET_GPAIR_CASE(DD)                                                                         \
    case DD:                                                                                         \
        grow_pair<DD, M, R, (DD <= kPairStagedMax), NG>(ent, check_base, fr, lo, hi, Z, first, last, \
                                                        wt);                                        \
        break;
        QCMET_GPAIR_CASE(5)
        QCMET_GPAIR_CASE(6)
        QCMET_GPAIR_CASE(7)
        QCMET_GPAIR_CASE(8)
        QCMET_GPAIR_CASE(9)
        QCMET_GPAIR_CASE(10)
        QCMET_GPAIR_CASE(11)
        QCMET_GPAIR_CASE(12)
        QCMET_GPAIR_CASE(13)
        QCMET_GPAIR_CASE(14)
        QCMET_GPAIR_CASE(15)
        QCMET_GPAIR_CASE(16)
#undef QCMET_GPAIR_CASE
        default: break;
    }
}

// The frames of the cluster's groups (at most two): frame f < nf[g] of group g
// reads ch[g][f] [n] and syn[g][f] [m] and writes post[g][f] [n] (when not
// null), hard[g][f] [n] and ok[g][f] [1].
constexpr int kMaxGroupsPerCluster = 2;
template <int NG>
struct GroupIO {
    const float *ch[NG][kGF];
    const uint8_t *syn[NG][kGF];
    float *post[NG][kGF];
    uint8_t *hard[NG][kGF];
    uint8_t *ok[NG][kGF];
    int nf[NG];
    int ng;  // groups of the cluster (1 .. NG)
    __device__ int groups() const { return ng; }
    __device__ int nf_of(int g) const { return nf[g]; }
    __device__ const float *ch_of(int g, int f) const { return ch[g][f]; }
    __device__ const uint8_t *syn_of(int g, int f) const { return syn[g][f]; }
    __device__ float *post_of(int g, int f) const { return post[g][f]; }
    __device__ uint8_t *hard_of(int g, int f) const { return hard[g][f]; }
    __device__ uint8_t *ok_of(int g, int f) const { return ok[g][f]; }
};

// The same accessors over a batch job in global memory: the pointers are read
// where the prologue and epilogue use them, so that the persistent kernel
// keeps none of them in registers through the layer loop.
struct JobIO {
    const GroupJob *jb;
    int ng;
    __device__ int groups() const { return ng; }
    __device__ int nf_of(int g) const { return g < ng ? jb->nf[g] : 0; }
    __device__ const float *ch_of(int g, int f) const { return jb->ch[g][f]; }
    __device__ const uint8_t *syn_of(int g, int f) const { return jb->syn[g][f]; }
    __device__ float *post_of(int g, int f) const { return jb->post[g][f]; }
    __device__ uint8_t *hard_of(int g, int f) const { return jb->hard[g][f]; }
    __device__ uint8_t *ok_of(int g, int f) const { return jb->ok[g][f]; }
};

// One cluster decodes its groups (steps 1-4) with the schedule `s` in shared
// memory.  The cluster's checks (and variables) form the virtual range
// [0, ng Zp) (vsplit); CTA r of the cluster's C owns [lo, hi) of it in every
// row.  Every thread of every CTA of the cluster executes the same sequence
// of cluster barriers: one after the prologue, one per layer of every
// iteration and one before the ok flags are written.  s_fail points to two
// shared words of the calling CTA (rank 0's collect each group's
// syndrome-test failures).
//   w_scale, w_offset: min-sum weights [T][mb][2] (R == kGroupMinSum)
template <typename M, int S, int R, int NG, typename IO>
__device__ __forceinline__ void decode_group_body(const Sched &s, const IO &io, GFrame<M> fr,
                                                  int T, int r, int C, unsigned *s_fail,
                                                  const float *w_scale = nullptr,
                                                  const float *w_offset = nullptr) {
    const int nt = blockDim.x;
    const int tid = threadIdx.x;
    const int Z = s.Z;
    const int zp = fr.zp;
    // indices per CTA, a multiple of 32: every warp's 32 checks then start on
    // a 128-byte line of the message and syndrome rows
    const int span = NG == 1 ? Z : io.groups() * zp;
    const int Zc = ((span + C - 1) / C + 31) / 32 * 32;
    const int lo = min(span, r * Zc);
    const int hi = min(span, lo + Zc);
    if (r == 0 && tid < kMaxGroupsPerCluster) s_fail[tid] = 0u;

    // Step 1 and the interleaved copies of this CTA's share: variables
    // [lo, hi) of every column, checks [lo, hi) of every row.  Lanes past nf
    // (a partial group) decode a channel of +1 with a zero syndrome.
    for (int c = 0; c < s.nb; ++c) {
        const bool core = s.col_kind[c] == kColCore;
        const int cc = s.col_core[c];
        const size_t cb = (size_t)c * Z;  // caller's frame-major arrays
        const size_t gb = (size_t)c * zp;
        for (int v = lo + tid; v < hi; v += nt) {
            const VIndex x = vsplit<NG>(v, zp);
            if (!real<NG>(x, Z)) continue;
            float y[kGF];
#pragma unroll
            for (int f = 0; f < kGF; ++f)
                y[f] = f < io.nf_of(x.g) ? __ldcs(io.ch_of(x.g, f) + cb + x.l) : 1.0f;
            const float4 y4 = make_float4(y[0], y[1], y[2], y[3]);
            if (in_range((long long)gb + x.l, fr.bd.vars, kBadVariable))
                *in_group<NG>(fr.ch4 + gb + x.l, x.g, fr.gstride.ch) = y4;
            if (core && in_range((long long)cc * zp + x.l, fr.bd.core, kBadVariable))
                *in_group<NG>(fr.core4 + (size_t)cc * zp + x.l, x.g, fr.gstride.core) = y4;
        }
    }
    for (int l = 0; l < s.mb; ++l) {
        const size_t lb = (size_t)l * Z;
        const size_t gl = (size_t)l * zp;
        for (int i = lo + tid; i < hi; i += nt) {
            const VIndex x = vsplit<NG>(i, zp);
            if (!real<NG>(x, Z)) continue;
            uint32_t w = 0u;
#pragma unroll
            for (int f = 0; f < kGF; ++f)
                if (f < io.nf_of(x.g)) w |= (uint32_t)(__ldcs(io.syn_of(x.g, f) + lb + x.l) & 1u) << (8 * f);
            if (in_range((long long)gl + x.l, fr.bd.checks, kBadCheck))
                *in_group<NG>(const_cast<uint32_t *>(fr.syn4) + gl + x.l, x.g, fr.gstride.syn) = w;
        }
    }
    cluster_sync();

    // Steps 2-3: T iterations x layers; one cluster barrier per layer.
    for (int t = 0; t < T; ++t) {
        const bool first = t == 0;
        const bool last = t == T - 1;
        for (int layer = 0; layer < s.n_layers; ++layer) {
            for (int j = s.layer_first[layer]; j < s.layer_first[layer + 1]; ++j) {
                const int4 row = s.rows[j];
                float4 wt = make_float4(0.f, 0.f, 0.f, 0.f);
                if constexpr (R == kGroupMinSum) {
                    const size_t w = ((size_t)t * s.mb + (size_t)row.w) * 2;
                    wt = make_float4(__ldg(w_scale + w), __ldg(w_scale + w + 1), __ldg(w_offset + w),
                                     __ldg(w_offset + w + 1));
                }
                gdispatch<M, S, R, NG>(row.y, s.entries + row.x, row.z, fr, lo, hi, Z, first, last, wt);
            }
            cluster_sync();
        }
    }

    // Step 4: frame-major posteriors and hard decisions of variables [lo, hi)
    // of every column, then the syndrome test H c = s on checks [lo, hi).
    for (int c = 0; c < s.nb; ++c) {
        const bool core = s.col_kind[c] == kColCore;
        const int cc = s.col_core[c];
        const size_t cb = (size_t)c * Z;
        const size_t gb = (size_t)c * zp;
        for (int v = lo + tid; v < hi; v += nt) {
            const VIndex x = vsplit<NG>(v, zp);
            if (!real<NG>(x, Z)) continue;
            const bool ok = core ? in_range((long long)cc * zp + x.l, fr.bd.core, kBadVariable)
                                 : in_range((long long)gb + x.l, fr.bd.vars, kBadVariable);
            const float4 L4 = !ok  ? make_float4(0.f, 0.f, 0.f, 0.f)
                              : core ? __ldcg(in_group<NG>(fr.core4 + (size_t)cc * zp + x.l, x.g,
                                                           fr.gstride.core))
                                     : __ldcg(in_group<NG>(fr.ch4 + gb + x.l, x.g, fr.gstride.ch));
#pragma unroll
            for (int f = 0; f < kGF; ++f) {
                if (f >= io.nf_of(x.g)) break;
                const float L = comp(L4, f);
                if (io.post_of(x.g, f)) io.post_of(x.g, f)[cb + x.l] = L;
                io.hard_of(x.g, f)[cb + x.l] = L < 0.0f ? 1 : 0;
            }
        }
    }
    uint32_t bad[NG] = {};
    // the syndrome word of check x of the row whose first check is row_first
    auto syn_word = [&](const VIndex &x, size_t row_first) {
        return in_range((long long)row_first + x.l, fr.bd.checks, kBadCheck)
                   ? *in_group<NG>(fr.syn4 + row_first + x.l, x.g, fr.gstride.syn)
                   : 0u;
    };
    for (int zr = 0; zr < s.n_zero_rows; ++zr) {
        const size_t lb = (size_t)s.zero_rows[zr] * zp;
        for (int i = lo + tid; i < hi; i += nt) {
            const VIndex x = vsplit<NG>(i, zp);
            if (real<NG>(x, Z)) bad[x.g] |= syn_word(x, lb);
        }
    }
    for (int j = 0; j < s.n_rows; ++j) {
        const int4 row = s.rows[j];
        const int4 *ent = s.entries + row.x;
        for (int i = lo + tid; i < hi; i += nt) {
            const VIndex x = vsplit<NG>(i, zp);
            if (!real<NG>(x, Z)) continue;
            uint32_t p = syn_word(x, (size_t)row.z);
            for (int e = 0; e < row.y; ++e) {
                const int4 en = ent[e];
                int jj = x.l + en.y;
                jj = jj >= Z ? jj - Z : jj;
                if (in_range((long long)en.x + jj, en.z < 0 ? fr.bd.vars : fr.bd.core, kBadVariable))
                    p ^= sign_bytes(__ldcg(in_group<NG>((en.z < 0 ? fr.ch4 : fr.core4) + en.x + jj, x.g,
                                                        en.z < 0 ? fr.gstride.ch : fr.gstride.core)));
            }
            bad[x.g] |= p;
        }
    }
#pragma unroll
    for (int g = 0; g < NG; ++g) {
        const uint32_t b = __reduce_or_sync(0xffffffffu, bad[g] & 0x01010101u);
        if ((tid & 31) == 0 && b) {
            uint32_t local = (uint32_t)__cvta_generic_to_shared(s_fail + g);
            uint32_t remote;
            asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(0));
            asm volatile("red.relaxed.cluster.shared::cluster.or.b32 [%0], %1;" ::"r"(remote), "r"(b)
                         : "memory");
        }
    }
    cluster_sync();
    if (r == 0 && tid < io.groups() * kGF) {
        const int g = tid / kGF, f = tid % kGF;
        if (f < io.nf_of(g)) io.ok_of(g, f)[0] = ((s_fail[g] >> (8 * f)) & 1u) ? 0 : 1;
    }
}

// Views of one group's scratch for the code of schedule s.
template <typename M>
__device__ __forceinline__ GFrame<M> group_scratch(const Sched &s, void *ch4, uint32_t *syn4,
                                                   void *core4, void *msgs4, GroupScratch gstride) {
    GFrame<M> fr;
    fr.ch4 = static_cast<float4 *>(ch4);
    fr.syn4 = syn4;
    fr.core4 = static_cast<float4 *>(core4);
    fr.msg4 = static_cast<typename MsgVec<M>::V *>(msgs4);
    fr.pol = make_policies<std::is_same<M, float>::value ? QCMET_GROUP_HINT_FP32
                                                          : QCMET_GROUP_HINT_16BIT>();
    fr.zp = (s.Z + 31) & ~31;
    fr.gstride = gstride;
    fr.bd.core = (long long)s.core_cols * fr.zp;
    fr.bd.vars = (long long)s.nb * fr.zp;
    fr.bd.msgs = (long long)s.msg_slots * fr.zp;
    fr.bd.checks = (long long)s.mb * fr.zp;
    return fr;
}

// Copy a code's layer table into shared memory (every thread of the block)
// and rewrite its offsets for the grouped scratch: an entry's variable offset
// becomes (its index among the core columns, or its base column for a
// degree-1 column) x Zp, a row's first check l x Zp.
__device__ __forceinline__ void load_group_image(int32_t *sw, const int32_t *image, int words) {
    const int4 *src = reinterpret_cast<const int4 *>(image);
    int4 *dst = reinterpret_cast<int4 *>(sw);
    for (int k = threadIdx.x; k < words / 4; k += blockDim.x) dst[k] = src[k];
    __syncthreads();
    const int zp = (sw[kHdrZ] + 31) & ~31;
    const int32_t *col_core = sw + sw[kHdrOffColCore];
    int4 *ent = reinterpret_cast<int4 *>(sw + sw[kHdrOffEntries]);
    for (int k = threadIdx.x; k < sw[kHdrEntries]; k += blockDim.x) {
        int4 e = ent[k];
        e.x = (e.z >= 0 ? col_core[e.w] : e.w) * zp;
        ent[k] = e;
    }
    int4 *rows = reinterpret_cast<int4 *>(sw + sw[kHdrOffRows]);
    for (int k = threadIdx.x; k < sw[kHdrRows]; k += blockDim.x) {
        int4 rw = rows[k];
        rw.z = rw.w * zp;
        rows[k] = rw;
    }
    __syncthreads();
}

// K frames of one code: cluster k owns groups NG k .. NG k + NG - 1 (NG = 1 or
// 2 groups per cluster); group g holds frames 4g .. 4g + 3.
//   S    : rounds staged per thread (S - 1 in flight while one is computed)
//   NT   : largest block (launch bound); MINB: blocks per SM the bound asks for
// Shared memory: the staging area, S * stage_ops * blockDim 16-byte slots
// (group_stage_ops), then the layer table.
template <typename M, int S, int NT, int MINB, int R, int NG>
__global__ void __launch_bounds__(NT, MINB) decode_group_kernel(const GroupArgs a) {
    const int C = (int)cluster_nctarank();
    const int r = (int)cluster_ctarank();
    const int k = (int)cluster_idx();
    __shared__ unsigned s_fail[kMaxGroupsPerCluster];
    int32_t *sw = reinterpret_cast<int32_t *>(qcmet_group_smem + (size_t)S * a.stage_ops * blockDim.x);
    load_group_image(sw, a.image, a.image_words);
    const Sched s = make_sched(sw);
    const size_t n = (size_t)a.n, m = (size_t)a.m;
    const int groups = (a.K + kGF - 1) / kGF;
    const int g0 = k * NG;
    GroupIO<NG> io;
    io.ng = min(NG, groups - g0);
#pragma unroll
    for (int g = 0; g < NG; ++g) {
        const int f0 = (g0 + g) * kGF;
        io.nf[g] = g < io.ng ? min(kGF, a.K - f0) : 0;
#pragma unroll
        for (int f = 0; f < kGF; ++f) {
            const bool have = f < io.nf[g];
            io.ch[g][f] = have ? a.ch + (size_t)(f0 + f) * n : nullptr;
            io.syn[g][f] = have ? a.syn + (size_t)(f0 + f) * m : nullptr;
            io.post[g][f] = (have && a.post) ? a.post + (size_t)(f0 + f) * n : nullptr;
            io.hard[g][f] = have ? a.hard + (size_t)(f0 + f) * n : nullptr;
            io.ok[g][f] = have ? a.ok + f0 + f : nullptr;
        }
    }
    GFrame<M> fr = group_scratch<M>(
        s, static_cast<char *>(a.ch4) + (size_t)g0 * a.g_bytes.ch,
        reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(a.syn4) + (size_t)g0 * a.g_bytes.syn),
        static_cast<char *>(a.core4) + (size_t)g0 * a.g_bytes.core,
        static_cast<char *>(a.msgs4) + (size_t)g0 * a.g_bytes.msg, a.g_bytes);
    decode_group_body<M, S, R, NG>(s, io, fr, a.T, r, C, s_fail, a.w_scale, a.w_offset);
}

// Mixed batches: persistent clusters take jobs (one or two groups of up to
// four frames of one code; NG = the most groups a job holds) from an atomic
// counter in the order given -- a work queue, nothing waits on another
// cluster -- reload the layer table when the code changes, and decode the
// job.  Rank 0 takes the next job and the others read it from rank 0's
// shared memory.
// One job with the layer table of its code in shared memory (sw).  A function
// of its own: the persistent loop's state is saved once around it instead of
// staying live through the layer loop.
template <typename M, int S, int NG>
__device__ __noinline__ void decode_job(const GroupJob &jb, const int32_t *sw, int T, int r, int C,
                                        unsigned *s_fail) {
    const Sched s = make_sched(sw);
    const JobIO io{&jb, min(NG, jb.ng)};
    GFrame<M> fr = group_scratch<M>(s, jb.ch4, jb.syn4, jb.core4, jb.msgs4, jb.gstride);
    decode_group_body<M, S, kGroupSumProduct, NG>(s, io, fr, T, r, C, s_fail);
}

// PERSIST = false: one job per cluster (cluster k decodes the k-th job of the
// order, the grid holding a cluster per job).
template <typename M, int S, int NT, int MINB, int NG, bool PERSIST>
__global__ void __launch_bounds__(NT, MINB) decode_group_batch_kernel(const GroupBatchArgs b) {
    const int C = (int)cluster_nctarank();
    const int r = (int)cluster_ctarank();
    __shared__ unsigned s_fail[kMaxGroupsPerCluster];
    __shared__ int s_job;
    int32_t *sw = reinterpret_cast<int32_t *>(qcmet_group_smem + (size_t)S * b.stage_ops * blockDim.x);
    if constexpr (!PERSIST) {
        const int k = (int)cluster_idx();
        if (k >= b.J) return;   // every block of the cluster leaves together
        const GroupJob &jb = b.jobs[b.order[k]];
        load_group_image(sw, jb.image, jb.image_words);
        decode_job<M, S, NG>(jb, sw, b.T, r, C, s_fail);
        return;
    }
    int cur_code = -1;
    for (;;) {
        if (r == 0 && threadIdx.x == 0) s_job = atomicAdd(b.counter, 1);
        cluster_sync();
        int k;
        {
            const uint32_t local = (uint32_t)__cvta_generic_to_shared(&s_job);
            uint32_t remote;
            asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(0));
            asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(k) : "r"(remote) : "memory");
        }
        cluster_sync();  // every CTA has read the job: rank 0 may overwrite it or exit
        if (k >= b.J) break;
        const GroupJob &jb = b.jobs[b.order[k]];
        if (jb.code_id != cur_code) {
            load_group_image(sw, jb.image, jb.image_words);
            cur_code = jb.code_id;
        }
        decode_job<M, S, NG>(jb, sw, b.T, r, C, s_fail);
    }
}

// Launch variants of the kernel: (rounds staged, block bound, blocks per SM).
struct Variant {
    int S, NT, MINB;
    // [message format (sum-product); 3: min-sum, FP32 messages][groups per cluster - 1]
    const void *kern[4][kMaxGroupsPerCluster];
};

template <int S, int NT, int MINB, int NG>
void fill_variant(Variant &v) {
    v.kern[0][NG - 1] =
        reinterpret_cast<const void *>(&decode_group_kernel<float, S, NT, MINB, kGroupSumProduct, NG>);
    v.kern[1][NG - 1] =
        reinterpret_cast<const void *>(&decode_group_kernel<__half, S, NT, MINB, kGroupSumProduct, NG>);
    v.kern[2][NG - 1] = reinterpret_cast<const void *>(
        &decode_group_kernel<__nv_bfloat16, S, NT, MINB, kGroupSumProduct, NG>);
    v.kern[3][NG - 1] =
        reinterpret_cast<const void *>(&decode_group_kernel<float, S, NT, MINB, kGroupMinSum, NG>);
}

template <int S, int NT, int MINB>
Variant make_variant() {
    Variant v{S, NT, MINB, {}};
    fill_variant<S, NT, MINB, 1>(v);
    fill_variant<S, NT, MINB, 2>(v);
    return v;
}

const Variant *variants(int *count) {
    // (four staged rounds measured no faster than three)
    static const Variant v[] = {
        make_variant<kGroupStages, 512, 1>(),
        make_variant<kGroupStages, 256, 2>(),
    };
    *count = (int)(sizeof(v) / sizeof(v[0]));
    return v;
}

// Threads of a CTA owning `zc` checks of each row: the fewest rounds of at
// most `nt_max` checks, spread evenly (a multiple of 32).
int group_threads(int zc, int nt_max) {
    const int rounds = (zc + nt_max - 1) / nt_max;
    int t = (zc + rounds - 1) / rounds;
    t = (t + 31) / 32 * 32;
    return t < 32 ? 32 : (t > nt_max ? nt_max : t);
}

size_t group_smem(int S, int threads, int32_t stage_ops, int32_t image_words) {
    return (size_t)S * stage_ops * threads * 16 + (size_t)image_words * sizeof(int32_t);
}

}  // namespace

size_t group_msg_bytes(int32_t fmt) { return fmt == QCMET_MSG_FP32 ? 16 : 8; }

#ifndef QCMET_GROUP_VARIANT
#define QCMET_GROUP_VARIANT (-1)
#endif

namespace {
// Launch shapes chosen so far, by (device, format, K, Z, table size, stage_ops,
// requested cluster size and groups per cluster, rule): the choice queries the occupancy of up to 64
// shapes, which a repeated decode of the same shape should not pay again.
struct LaunchKey {
    int dev, fmt, K, Z, image_words, stage_ops, want, want_ng, minsum;
    bool operator<(const LaunchKey &o) const {
        return std::tie(dev, fmt, K, Z, image_words, stage_ops, want, want_ng, minsum) <
               std::tie(o.dev, o.fmt, o.K, o.Z, o.image_words, o.stage_ops, o.want, o.want_ng,
                        o.minsum);
    }
};
std::mutex g_launch_mu;
std::map<LaunchKey, GroupLaunch> g_launch_cache;
}  // namespace

int choose_group_launch(int32_t fmt, int32_t K, int32_t Z, int32_t image_words,
                        int32_t stage_ops, int32_t want_cluster, GroupLaunch *out,
                        std::string &err, bool minsum, int32_t want_per_cluster) {
    if (fmt != QCMET_MSG_FP32 && fmt != QCMET_MSG_FP16 && fmt != QCMET_MSG_BF16) {
        err = "unknown message format";
        return QCMET_ERR_INVALID_ARG;
    }
    if (minsum && fmt != QCMET_MSG_FP32) {
        err = "the min-sum rule keeps FP32 messages";
        return QCMET_ERR_INVALID_ARG;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        err = "no CUDA device";
        return QCMET_ERR_CUDA;
    }
    const LaunchKey key{dev,       fmt,          K, Z, image_words, stage_ops, want_cluster,
                        want_per_cluster, minsum ? 1 : 0};
    {
        std::lock_guard<std::mutex> lock(g_launch_mu);
        auto it = g_launch_cache.find(key);
        if (it != g_launch_cache.end()) {
            *out = it->second;
            return QCMET_OK;
        }
    }
    const int kidx = minsum ? 3 : fmt;
    const int G = (K + kGF - 1) / kGF;
    const int zp = (int)group_zp(Z);
    int nv = 0;
    const Variant *var = variants(&nv);
    double best = 0.0;
    bool have = false;
    for (int vi = 0; vi < nv; ++vi) {
        if (QCMET_GROUP_VARIANT >= 0 && vi != QCMET_GROUP_VARIANT) continue;
        for (int ng = 1; ng <= kMaxGroupsPerCluster && ng <= G; ++ng) {
            if (want_per_cluster > 0 && ng != want_per_cluster) continue;
            const void *kern = var[vi].kern[kidx][ng - 1];
            const int clusters = (G + ng - 1) / ng;
            // cluster sizes: the requested one, else 1 .. 16 with at least 128
            // checks per CTA (sizes above 8 are non-portable)
            for (int C = 1; C <= 16; ++C) {
                if (want_cluster > 0 ? C != want_cluster : (C > 1 && ng * Z / C < 128)) continue;
                const int zc = ((ng * zp + C - 1) / C + 31) / 32 * 32;
                const int threads = group_threads(zc, var[vi].NT);
                const size_t smem = group_smem(var[vi].S, threads, stage_ops, image_words);
                cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)smem);
                if (e == cudaSuccess && C > 8)
                    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
                if (e != cudaSuccess) {
                    cudaGetLastError();
                    continue;
                }
                cudaLaunchConfig_t cfg = {};
                cfg.gridDim = dim3((unsigned)(clusters * C));
                cfg.blockDim = dim3((unsigned)threads);
                cfg.dynamicSmemBytes = smem;
                cudaLaunchAttribute attr[1];
                attr[0].id = cudaLaunchAttributeClusterDimension;
                attr[0].val.clusterDim.x = (unsigned)C;
                attr[0].val.clusterDim.y = 1;
                attr[0].val.clusterDim.z = 1;
                cfg.attrs = attr;
                cfg.numAttrs = 1;
                int active = 0;
                e = cudaOccupancyMaxActiveClusters(&active, kern, &cfg);
                if (e != cudaSuccess || active <= 0) {
                    cudaGetLastError();
                    continue;
                }
                // An SM moves the operands of a fixed number of checks per unit
                // of time, so the decode takes ~ waves of clusters x checks per
                // SM: zc per block, twice that when two blocks share an SM.  Ties
                // go to one group per cluster, smaller clusters, the first variant.
                const int waves = (clusters + active - 1) / active;
                const double cost = (double)waves * zc * var[vi].MINB *
                                        (1.0 + 1e-4 * (ng - 1) + 1e-5 * C) +
                                    1e-3 * vi;
                if (!have || cost < best) {
                    best = cost;
                    have = true;
                    out->cluster = C;
                    out->per_cluster = ng;
                    out->threads = threads;
                    out->groups = G;
                    out->active_clusters = active;
                    out->smem = smem;
                    out->variant = vi;
                    out->kidx = kidx;
                    out->stage_ops = stage_ops;
                }
            }
        }
    }
    if (have) {
        std::lock_guard<std::mutex> lock(g_launch_mu);
        g_launch_cache[key] = *out;
    }
    if (!have) {
        err = want_cluster > 0 ? "cluster size " + std::to_string(want_cluster) +
                                     " cannot be scheduled on this device"
                               : "no cluster size can be scheduled on this device";
        return QCMET_ERR_UNSUPPORTED;
    }
    return QCMET_OK;
}

int take_violations_group(uint32_t *bits, std::string &err) {
    *bits = 0;
#if QCMET_DEBUG_CHECKS
    uint32_t v = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_qcmet_violations, sizeof v);
    const uint32_t zero = 0;
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_qcmet_violations, &zero, sizeof zero);
    if (e != cudaSuccess) {
        err = std::string("reading the index-check word: ") + cudaGetErrorString(e);
        return QCMET_ERR_CUDA;
    }
    *bits = v;
#else
    (void)err;
#endif
    return QCMET_OK;
}

int32_t group_stage_ops(const Code &c) {
    int32_t ops = 1;
    for (int32_t l = 0; l < c.mb; ++l) {
        int32_t d = 0, dc = 0;
        for (int32_t col = 0; col < c.nb; ++col) {
            if (!c.base[(size_t)l * c.nb + col]) continue;
            ++d;
            dc += c.col_degree[col] > 1 ? 1 : 0;
        }
        int32_t need = 0;
        if (d >= 1 && d <= 4) need = d + dc;
        // a staged pair row: two rounds of 2 E slots, E = ceil(d / 2)
        if (d > 4 && d <= kPairStagedMax) need = (4 * ((d + 1) / 2) + kGroupStages - 1) / kGroupStages;
        ops = need > ops ? need : ops;
    }
    return ops;
}

GroupScratch group_scratch_bytes(const Code &c, int32_t fmt) {
    auto r256 = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t zp = (size_t)group_zp(c.Z);
    GroupScratch g;
    g.ch = r256((size_t)c.nb * zp * 16);
    g.syn = r256((size_t)c.mb * zp * 4);
    g.core = r256((size_t)c.core_cols * zp * 16);
    g.msg = r256((size_t)c.msg_slots * zp * group_msg_bytes(fmt));
    return g;
}

namespace {
// persistent clusters over jobs of one group; or one cluster per job of one
// or two groups
template <typename M>
const void *group_batch_kernel_ptr(int ng, bool persistent) {
    using K = const void *;
    if (persistent)
        return reinterpret_cast<K>(&decode_group_batch_kernel<M, kGroupStages, 512, 1, 1, true>);
    return ng == 2
               ? reinterpret_cast<K>(&decode_group_batch_kernel<M, kGroupStages, 512, 1, 2, false>)
               : reinterpret_cast<K>(&decode_group_batch_kernel<M, kGroupStages, 512, 1, 1, false>);
}
}  // namespace

int launch_decode_group_batch(const GroupBatchArgs &b, int32_t fmt, int32_t cluster, int32_t max_Z,
                              int32_t max_image_words, void *stream, std::string &err,
                              int32_t groups_per_job, bool cluster_per_job) {
    const int ng = groups_per_job == 2 ? 2 : 1;
    const bool persistent = !cluster_per_job;
    if (persistent && ng != 1) {
        err = "persistent grouped batch clusters take jobs of one group";
        return QCMET_ERR_INVALID_ARG;
    }
    const void *kern = fmt == QCMET_MSG_FP32   ? group_batch_kernel_ptr<float>(ng, persistent)
                       : fmt == QCMET_MSG_FP16 ? group_batch_kernel_ptr<__half>(ng, persistent)
                       : fmt == QCMET_MSG_BF16 ? group_batch_kernel_ptr<__nv_bfloat16>(ng, persistent)
                                               : nullptr;
    if (!kern || cluster < 1 || cluster > 16 || max_Z < 1 ||
        (groups_per_job != 1 && groups_per_job != 2)) {
        err = "invalid grouped batch launch";
        return QCMET_ERR_INVALID_ARG;
    }
    if (b.J <= 0) return QCMET_OK;
    const int C = cluster;
    // a job's checks: ng groups of Zp (Z rounded up to 32) each
    const int span = ng == 1 ? max_Z : ng * (int)group_zp(max_Z);
    const int threads = group_threads((span + C - 1) / C, 512);
    const size_t smem = group_smem(kGroupStages, threads, b.stage_ops, max_image_words);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess && C > 8)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) {
        cudaGetLastError();
        err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e);
        return QCMET_ERR_UNSUPPORTED;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = static_cast<cudaStream_t>(stream);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3((unsigned)(b.J * C));
    int active = 0;
    e = cudaOccupancyMaxActiveClusters(&active, kern, &cfg);
    if (e != cudaSuccess || active <= 0) {
        cudaGetLastError();
        err = "cluster size " + std::to_string(C) + " cannot be scheduled for this batch";
        return QCMET_ERR_UNSUPPORTED;
    }
    // persistent clusters: as many as the device holds at once, at most one
    // per job; else one cluster per job
    const int clusters = persistent && active < b.J ? active : b.J;
    cfg.gridDim = dim3((unsigned)(clusters * C));
    void *args[] = {const_cast<GroupBatchArgs *>(&b)};
    e = cudaLaunchKernelExC(&cfg, kern, args);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        err = std::string("grouped batch launch: ") + cudaGetErrorString(e);
        return QCMET_ERR_CUDA;
    }
    return QCMET_OK;
}

int launch_decode_group(const GroupArgs &a, int32_t fmt, const GroupLaunch &L, void *stream,
                        std::string &err, size_t window_bytes, float hit_ratio) {
    int nv = 0;
    const Variant *var = variants(&nv);
    if (fmt < 0 || fmt > 2 || L.variant < 0 || L.variant >= nv || a.stage_ops != L.stage_ops ||
        L.kidx < 0 || L.kidx > 3 || (L.kidx == 3) != (a.w_scale != nullptr) ||
        L.per_cluster < 1 || L.per_cluster > kMaxGroupsPerCluster) {
        err = "invalid grouped launch";
        return QCMET_ERR_INVALID_ARG;
    }
    const void *kern = var[L.variant].kern[L.kidx][L.per_cluster - 1];
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
    if (e != cudaSuccess) {
        err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e);
        return QCMET_ERR_UNSUPPORTED;
    }
    if (L.cluster > 8) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) {
            err = std::string("cudaFuncSetAttribute(non-portable cluster): ") + cudaGetErrorString(e);
            return QCMET_ERR_UNSUPPORTED;
        }
    }
    const int clusters = (L.groups + L.per_cluster - 1) / L.per_cluster;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(clusters * L.cluster));
    cfg.blockDim = dim3((unsigned)L.threads);
    cfg.dynamicSmemBytes = L.smem;
    cfg.stream = static_cast<cudaStream_t>(stream);
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)L.cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    int na = 1;
    (void)window_bytes;   // the kernel's own eviction policies replace a window
    (void)hit_ratio;
    cfg.attrs = attr;
    cfg.numAttrs = na;
    void *args[] = {const_cast<GroupArgs *>(&a)};
    e = cudaLaunchKernelExC(&cfg, kern, args);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        err = std::string("grouped decode launch: ") + cudaGetErrorString(e);
        return QCMET_ERR_CUDA;
    }
    return QCMET_OK;
}

}  // namespace qcmet
