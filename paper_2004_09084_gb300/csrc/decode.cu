// Fused layered belief-propagation decoder for QC-MET-LDPC syndrome decoding
// on GB300 (sm_103a).
//
// Method (arXiv 2004.09084, Methods, steps 1-4): for every iteration and every
// layer (base row) l, each check m of the layer forms the variable-to-check
// messages q = L_qn - L_rmn(old) (step 3, first equation), computes the new
// check-to-variable messages with the sum-product rule and the syndrome sign
// (step 2), and writes L_qn = q + L_rmn(new) (step 3, second equation).  The
// hard decision c_n = [L_qn < 0] closes the decode (step 4).
//
// GB300 design (ours, not the paper's):
//  * Frames are independent, so one CTA owns one frame for the whole decode
//    and a layer boundary costs one block barrier.  The whole decode -- init,
//    T x layers, hard decision, syndrome test -- is a single launch.  The
//    FP32 sum-product kernel runs 896-thread blocks by default (built with
//    that launch bound, for more registers per thread).
//  * Frame-major state: the posteriors L_qn of the core columns (degree > 1)
//    live in a compact array [K][core_cols][Z] (FP32), messages [K][slot][Z]
//    in FP32 / FP16 / BF16.  The compact array is the state every row
//    re-reads, so it is one contiguous range that an L2 persisting window can
//    cover; the caller's llr_post [K][n] receives the posteriors at the end.
//    Within a circulant, consecutive checks touch consecutive variables, so a
//    warp's gathers are contiguous runs of 128 B (one wrap at most).
//  * Degree-1 variables (a base column with a single circulant) keep no state:
//    for them L_qn - L_rmn(old) equals the channel LLR exactly, so q is read
//    from the channel array and L_qn is written only in tested iterations
//    (the last one, or each early-termination test).
//  * Row paths: degree <= 4, one thread per check, specialised at compile
//    time on the row's (core, degree-1) edge counts (the layout lists core
//    edges first).  With FP32 messages and the sum-product rule these rows
//    are software-pipelined through shared memory: each thread copies the
//    next round's operands with cp.async while it computes the current one,
//    two adjacent checks per thread (8-byte accesses) when Z is even.
//    Other formats and the min-sum rule issue the loads of two checks
//    together instead.  Degree 5..16: two lanes per check, each lane's loads
//    issued together for up to five edges per lane.  The same paths carry
//    the learned min-sum rule.
//  * No software prefetch: bulk L2 prefetches of the next row's operands
//    were evicted before use often enough to add about a third to the DRAM
//    reads, and per-thread prefetches of the next row's first round add
//    requests to the per-SM path that limits the rows; the decode ran faster
//    without either.
//  * The check rule is evaluated in the tanh-product form
//    |r_e| = 2 atanh(prod_{k != e} tanh(|q_k|/2)), which equals
//    Phi(sum_{k != e} Phi(|q_k|)) (Methods, step 2).  With u_k = exp(-|q_k|),
//    prod (1 + u_k J) over the other edges (J the 2x2 swap) is alpha I + beta J
//    with alpha, beta the even and odd elementary symmetric sums of the u_k,
//    and |r_e| = ln(alpha / beta).  Every term is positive, so there is no
//    cancellation at either end of the LLR range; the exclusive products come
//    from prefix and suffix products (no division).
//  * Clipping: |q| is clipped to 30 before the rule and |r| to
//    [Phi(30), 30] after it -- the same function as clipping both Phi
//    arguments to [Phi(30), 30].
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdio>
#include <type_traits>
#include <mutex>

#include "check_rule.cuh"
#include "qcmet_internal.h"

namespace qcmet {

namespace {
#ifndef QCMET_THREADS
#define QCMET_THREADS 1024
#endif
constexpr int kDefaultThreads = QCMET_THREADS;
// Default block of the FP32 sum-product decode.  Its kernel is also built with
// this launch bound, which gives a thread 73 registers instead of 64: the
// paired rows then spill less (rate-0.1 bench workload, Z = 12500: 98.7 ms
// against 102.0 ms for the same 896-thread launch of the 1024-bounded kernel,
// and 103.1 ms at 1024 threads).  Requests for larger blocks take the
// 1024-bounded kernel.
#ifndef QCMET_FP32_THREADS
#define QCMET_FP32_THREADS 896
#endif
constexpr int kFp32Threads = QCMET_FP32_THREADS;
static_assert(kFp32Threads % 32 == 0 && kFp32Threads <= kDefaultThreads, "FP32 block size");

// Per-frame views of the global arrays.
template <typename M>
struct Frame {
    const float *ch;     // [n]
    const uint8_t *syn;  // [m]
    float *post;         // [n] output posteriors (degree-1 columns written in place)
    float *post_core;    // [core_cols][Z] posteriors of the core columns
    M *msg;              // [slots][stride]
    Bounds bd;           // extents for the debug build's index checks
};

// Gather the V2C message q = L_qn - L_rmn(old) of edge `en` at check i.
template <typename M>
__device__ __forceinline__ float gather_q(const int4 &en, int i, const Frame<M> &fr, int Z,
                                          size_t stride, bool first) {
    int j = i + en.y;
    j = j >= Z ? j - Z : j;
    const int v = en.x + j;
    if (en.z < 0)  // degree-1 variable: L_qn - L_rmn(old) = channel LLR
        return in_range(v, fr.bd.vars, kBadVariable) ? __ldcs(fr.ch + v) : 0.0f;
    const float lv = in_range(v, fr.bd.core, kBadVariable) ? fr.post_core[v] : 0.0f;
    const float ro = (first || !in_range((long long)en.z * (long long)stride + i, fr.bd.msgs, kBadSlot))
                         ? 0.0f
                         : Msg<M>::load(fr.msg + (size_t)en.z * stride + i);
    return lv - ro;
}

// Write the new C2V message of edge `en` and the posterior L_qn = q + r.
template <typename M>
__device__ __forceinline__ void scatter_r(const int4 &en, int i, float q, float a, float b,
                                          unsigned par, const Frame<M> &fr, int Z, size_t stride,
                                          bool last) {
    if (en.z < 0 && !last) return;
    float mag = kLn2 * (lg2_ftz(a) - lg2_ftz(b));
    mag = fminf(fmaxf(mag, kClipMin), kClipMax);
    const bool neg = ((par ^ (q < 0.0f ? 1u : 0u)) & 1u) != 0u;
    float rn = neg ? -mag : mag;
    int j = i + en.y;
    j = j >= Z ? j - Z : j;
    const int v = en.x + j;
    if (en.z >= 0) {
        rn = Msg<M>::quantize(rn);
        if (in_range((long long)en.z * (long long)stride + i, fr.bd.msgs, kBadSlot))
            Msg<M>::store(fr.msg + (size_t)en.z * stride + i, rn);
        if (in_range(v, fr.bd.core, kBadVariable)) fr.post_core[v] = q + rn;
    } else if (in_range(v, fr.bd.vars, kBadVariable)) {
        fr.post[v] = q + rn;
    }
}

// Rows of degree D <= 4 use one thread per check.  Each thread first gathers
// the inputs of U checks (i, i + NT, ..., i + (U-1) NT) in straight-line code
// -- checks past Z load from a clamped (valid) index -- so that all of the
// batch's loads are in flight together; then it computes and writes the U
// checks.  (Issuing the next batch's loads before computing the current one
// measured slower at every block size: at 1024 threads it spills, and fewer
// threads leave too few warps to hide the arithmetic's own latency.)
//   first: iteration 0 (old messages are zero and are not read)
//   last : final or tested iteration (degree-1 variables get their posterior)
#ifndef QCMET_BATCH_LOW
#define QCMET_BATCH_LOW 2
#endif
template <int D>
__host__ __device__ constexpr int batch_of() { return QCMET_BATCH_LOW; }

// Rows of degree DC + D1 <= 4 whose DC core edges come first and D1 degree-1
// edges last (the layout's order).  As run_row, one thread per check and U
// checks gathered together, but the edge kinds are known at compile time: the
// core edges read the core posteriors and their message slot, the degree-1
// edges the channel LLR, and the per-row column and slot bases are computed
// once per row.
template <int DC, int D1, typename M>
__device__ __forceinline__ void run_row_split(const int4 *__restrict__ ent, int check_base,
                                              const Frame<M> &fr, int Z, size_t stride, bool first,
                                              bool last) {
    constexpr int D = DC + D1;
    constexpr int NC = DC > 0 ? DC : 1;
    constexpr int U = batch_of<D>();
    const int step = blockDim.x;
    const float *src[D];
    int sh[D];
    int xo[D], zo[DC > 0 ? DC : 1];  // variable and slot offsets (index checks of the debug build)
    M *slot[NC];
#pragma unroll
    for (int e = 0; e < D; ++e) {
        const int4 en = ent[e];
        src[e] = (e < DC ? fr.post_core : fr.ch) + en.x;
        sh[e] = en.y;
        xo[e] = en.x;
        if (e < DC) {
            slot[e] = fr.msg + (size_t)en.z * stride;
            zo[e] = en.z;
        }
    }
    for (int i0 = threadIdx.x; i0 < Z; i0 += step * U) {
        float lv[U][D], ro[U][NC];
        unsigned par[U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const int i = min(i0 + k * step, Z - 1);
            par[k] = in_range((long long)check_base + i, fr.bd.checks, kBadCheck)
                         ? (fr.syn[check_base + i] & 1u)
                         : 0u;
#pragma unroll
            for (int e = 0; e < D; ++e) {
                int j = i + sh[e];
                j = j >= Z ? j - Z : j;
                lv[k][e] = in_range((long long)xo[e] + j, e < DC ? fr.bd.core : fr.bd.vars, kBadVariable)
                                ? src[e][j]
                                : 0.0f;
            }
#pragma unroll
            for (int e = 0; e < DC; ++e)
                ro[k][e] = (first || !in_range((long long)zo[e] * (long long)stride + i, fr.bd.msgs, kBadSlot))
                               ? 0.0f
                               : Msg<M>::load(slot[e] + i);
        }
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const int i = i0 + k * step;
            if (i >= Z) break;
            float q[D], u[D];
            unsigned p = par[k];
#pragma unroll
            for (int e = 0; e < D; ++e) {
                q[e] = e < DC ? lv[k][e] - ro[k][e < DC ? e : 0] : lv[k][e];
                p ^= q[e] < 0.0f ? 1u : 0u;
                u[e] = u_of(q[e]);
            }
            exclusive_products<D>(u, 1.0f, 0.0f, [&](int e, float a, float b) {
                if (e >= DC && !last) return;
                float mag = kLn2 * (lg2_ftz(a) - lg2_ftz(b));
                mag = fminf(fmaxf(mag, kClipMin), kClipMax);
                const bool neg = ((p ^ (q[e] < 0.0f ? 1u : 0u)) & 1u) != 0u;
                float rn = neg ? -mag : mag;
                int j = i + sh[e];
                j = j >= Z ? j - Z : j;
                if (e < DC) {
                    rn = Msg<M>::quantize(rn);
                    if (in_range((long long)zo[e < DC ? e : 0] * (long long)stride + i, fr.bd.msgs, kBadSlot))
                        Msg<M>::store(slot[e < DC ? e : 0] + i, rn);
                    if (in_range((long long)xo[e] + j, fr.bd.core, kBadVariable))
                        const_cast<float *>(src[e])[j] = q[e] + rn;
                } else {
                    if (in_range((long long)xo[e] + j, fr.bd.vars, kBadVariable))
                        fr.post[(src[e] - fr.ch) + j] = q[e] + rn;
                }
            });
        }
    }
}

// Dynamic shared memory of the decode kernels.  The FP32 sum-product kernel
// keeps its staging area at offset 0 (so staging offsets are immediates) and
// the schedule image after it; the other kernels hold only the image.
extern __shared__ int4 qcmet_dyn_smem[];

// ---- asynchronous copies, global -> shared (4 bytes, per thread) ----------
__device__ __forceinline__ void cp_async4(uint32_t dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Two rounds: one computed, one in flight.  Three and four measured no faster
// (the rows are then limited by the SM's own issue and memory throughput).
#ifndef QCMET_ASYNC_STAGES
#define QCMET_ASYNC_STAGES 2
#endif
constexpr int kAsyncStages = QCMET_ASYNC_STAGES;  // rounds in flight + 1
constexpr int kAsyncMaxOps = 8;  // operands per check: D posteriors/LLRs + DC old messages, D <= 4
// staging floats per thread
constexpr int kAsyncStageFloats = kAsyncStages * kAsyncMaxOps * 2;  // room for the paired form

// run_row_split with FP32 messages, software-pipelined through shared memory:
// a thread handles one check per round, and while it computes round r the
// operands of rounds r + 1 .. r + S - 1 are being copied into its own staging
// slots by cp.async, so the loads' latency overlaps the arithmetic without
// holding registers.  Each thread reads only the slots it filled, so a
// per-thread wait_group orders them; no block barrier is needed.  Rounds of
// one row touch disjoint variables and message slots (a circulant is a
// permutation), so copying later rounds before round r's stores reads no
// value that those stores change.  The syndrome bytes of later rounds wait in
// registers.  Staging: [S rounds][D + DC operands][kDefaultThreads] floats.
template <int DC, int D1>
__device__ __forceinline__ void run_row_split_async(const int4 *__restrict__ ent, int check_base,
                                                    const Frame<float> &fr, int Z, size_t stride,
                                                    bool first, bool last) {
    constexpr int D = DC + D1;
    constexpr int NC = DC > 0 ? DC : 1;
    constexpr int S = kAsyncStages;
    constexpr int NOP = D + DC;
    constexpr int SS = kDefaultThreads;       // staging stride, fixed so offsets are immediates
    constexpr uint32_t kOp = SS * 4;          // bytes between operands
    constexpr uint32_t kRound = NOP * kOp;    // bytes between rounds
    const int step = blockDim.x;
    const int tid = threadIdx.x;
    if (tid >= Z) return;
    float *stage = reinterpret_cast<float *>(qcmet_dyn_smem);
    const float *src[D];
    int sh[D];
    int xo[D], zo[DC > 0 ? DC : 1];  // variable and slot offsets (index checks of the debug build)
    float *slot[NC];
#pragma unroll
    for (int e = 0; e < D; ++e) {
        const int4 en = ent[e];
        src[e] = (e < DC ? fr.post_core : fr.ch) + en.x;
        sh[e] = en.y;
        xo[e] = en.x;
        if (e < DC) {
            slot[e] = fr.msg + (size_t)en.z * stride;
            zo[e] = en.z;
        }
    }
    const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(stage + tid);
    // copy the operands of check i into round buffer b (or nothing past Z); one group per round
    auto issue = [&](int i, int b) {
        if (i < Z) {
            const uint32_t sb = s0 + (uint32_t)b * kRound;
#pragma unroll
            for (int e = 0; e < D; ++e) {
                int j = i + sh[e];
                j = j >= Z ? j - Z : j;
                if (in_range((long long)xo[e] + j, e < DC ? fr.bd.core : fr.bd.vars, kBadVariable))
                    cp_async4(sb + e * kOp, src[e] + j);
            }
            if (!first) {
#pragma unroll
                for (int e = 0; e < DC; ++e)
                    if (in_range((long long)zo[e] * (long long)stride + i, fr.bd.msgs, kBadSlot))
                        cp_async4(sb + (D + e) * kOp, slot[e] + i);
            }
        }
        cp_async_commit();
    };
    unsigned sy[S];
#pragma unroll
    for (int r = 0; r < S - 1; ++r) {
        const int i = tid + r * step;
        sy[r] = (i < Z && in_range((long long)check_base + i, fr.bd.checks, kBadCheck))
                    ? fr.syn[check_base + i]
                    : 0u;
        issue(i, r);
    }
    int buf = 0;
    for (int i = tid; i < Z; i += step) {
        {
            const int nx = i + (S - 1) * step;
            int nb = buf + (S - 1);
            nb = nb >= S ? nb - S : nb;
            sy[S - 1] = (nx < Z && in_range((long long)check_base + nx, fr.bd.checks, kBadCheck))
                            ? fr.syn[check_base + nx]
                            : 0u;
            issue(nx, nb);
        }
        cp_async_wait<S - 1>();
        const float *sv = stage + tid + buf * (kRound / 4);
        float q[D], u[D];
        unsigned p = sy[0] & 1u;
#pragma unroll
        for (int e = 0; e < D; ++e) {
            const float lv = sv[e * SS];
            q[e] = (e < DC && !first) ? lv - sv[(D + (e < DC ? e : 0)) * SS] : lv;
            p ^= q[e] < 0.0f ? 1u : 0u;
            u[e] = u_of(q[e]);
        }
        exclusive_products<D>(u, 1.0f, 0.0f, [&](int e, float a, float b) {
            if (e >= DC && !last) return;
            float mag = kLn2 * (lg2_ftz(a) - lg2_ftz(b));
            mag = fminf(fmaxf(mag, kClipMin), kClipMax);
            const bool neg = ((p ^ (q[e] < 0.0f ? 1u : 0u)) & 1u) != 0u;
            const float rn = neg ? -mag : mag;
            int j = i + sh[e];
            j = j >= Z ? j - Z : j;
            if (e < DC) {
                if (in_range((long long)zo[e < DC ? e : 0] * (long long)stride + i, fr.bd.msgs, kBadSlot))
                    slot[e < DC ? e : 0][i] = rn;
                if (in_range((long long)xo[e] + j, fr.bd.core, kBadVariable))
                    const_cast<float *>(src[e])[j] = q[e] + rn;
            } else {
                if (in_range((long long)xo[e] + j, fr.bd.vars, kBadVariable))
                    fr.post[(src[e] - fr.ch) + j] = q[e] + rn;
            }
        });
#pragma unroll
        for (int r = 0; r < S - 1; ++r) sy[r] = sy[r + 1];
        buf = buf + 1 == S ? 0 : buf + 1;
    }
}

__device__ __forceinline__ void cp_async8(uint32_t dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src) : "memory");
}

// run_row_split_async with two adjacent checks (i, i + 1), i even, per thread
// and round, for even Z: the message slots of both checks form one aligned
// 8-byte word, and so do a circulant's two variables when its shift is even
// (then j is even and j + 1 < Z), for loads and stores alike; odd shifts take
// two 4-byte accesses (j + 1 may wrap to 0), and the two syndrome bytes are
// one 16-bit load.  On GB300 a thread's 4-byte accesses are limited per SM by
// the number of requests rather than by bytes (about 48 GB/s per SM for
// 4-byte copies against 81 for 8-byte ones), so fewer, wider requests move the
// same bytes faster.  Staging: [2 rounds][D + DC operands][kDefaultThreads]
// float2.  (Both checks' results are held until the paired stores; at 1024
// threads that costs about 110 bytes of spills, which measured cheaper than
// unpaired posterior stores.)
template <int DC, int D1>
__device__ __forceinline__ void run_row_split_async2(const int4 *__restrict__ ent, int check_base,
                                                     const Frame<float> &fr, int Z, size_t stride,
                                                     bool first, bool last) {
    constexpr int D = DC + D1;
    constexpr int NC = DC > 0 ? DC : 1;
    constexpr int NOP = D + DC;
    constexpr int SS = kDefaultThreads;
    constexpr uint32_t kOp = SS * 8;        // bytes between operands
    constexpr uint32_t kRound = NOP * kOp;  // bytes between rounds
    const int step = 2 * (int)blockDim.x;
    const int tid = threadIdx.x;
    if (2 * tid >= Z) return;
    float2 *stage = reinterpret_cast<float2 *>(qcmet_dyn_smem);
    const float *src[D];
    int sh[D];
    int xo[D], zo[DC > 0 ? DC : 1];  // variable and slot offsets (index checks of the debug build)
    float *slot[NC];
#pragma unroll
    for (int e = 0; e < D; ++e) {
        const int4 en = ent[e];
        src[e] = (e < DC ? fr.post_core : fr.ch) + en.x;
        sh[e] = en.y;
        xo[e] = en.x;
        if (e < DC) {
            slot[e] = fr.msg + (size_t)en.z * stride;
            zo[e] = en.z;
        }
    }
    const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(stage + tid);
    auto issue = [&](int i, int b) {
        if (i < Z) {
            const uint32_t sb = s0 + (uint32_t)b * kRound;
#pragma unroll
            for (int e = 0; e < D; ++e) {
                int j = i + sh[e];
                j = j >= Z ? j - Z : j;
                const long long ext = e < DC ? fr.bd.core : fr.bd.vars;
                if (sh[e] & 1) {
                    const int j1 = j + 1 == Z ? 0 : j + 1;
                    if (in_range((long long)xo[e] + j, ext, kBadVariable))
                        cp_async4(sb + e * kOp, src[e] + j);
                    if (in_range((long long)xo[e] + j1, ext, kBadVariable))
                        cp_async4(sb + e * kOp + 4, src[e] + j1);
                } else if (in_range((long long)xo[e] + j + 1, ext, kBadVariable)) {
                    cp_async8(sb + e * kOp, src[e] + j);
                }
            }
            if (!first) {
#pragma unroll
                for (int e = 0; e < DC; ++e)
                    if (in_range((long long)zo[e] * (long long)stride + i + 1, fr.bd.msgs, kBadSlot))
                        cp_async8(sb + (D + e) * kOp, slot[e] + i);
            }
        }
        cp_async_commit();
    };
    unsigned sy = in_range((long long)check_base + 2 * tid + 1, fr.bd.checks, kBadCheck)
                      ? reinterpret_cast<const uint16_t *>(fr.syn + check_base)[tid]
                      : 0u;
    issue(2 * tid, 0);
    int buf = 0;
    for (int i = 2 * tid; i < Z; i += step) {
        const int nx = i + step;
        const unsigned sy_next =
            (nx < Z && in_range((long long)check_base + nx + 1, fr.bd.checks, kBadCheck))
                ? reinterpret_cast<const uint16_t *>(fr.syn + check_base)[nx >> 1]
                : 0u;
        issue(nx, buf ^ 1);
        cp_async_wait<1>();
        const float2 *sv = stage + tid + buf * (kRound / 8);
        float2 rn2[NC], pc2[NC];
        float pd[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            float q[D], u[D];
            unsigned p = (sy >> (8 * c)) & 1u;
#pragma unroll
            for (int e = 0; e < D; ++e) {
                const float2 l2 = sv[e * SS];
                const float lv = c ? l2.y : l2.x;
                float ro = 0.0f;
                if (e < DC && !first) {
                    const float2 r2 = sv[(D + (e < DC ? e : 0)) * SS];
                    ro = c ? r2.y : r2.x;
                }
                q[e] = e < DC ? lv - ro : lv;
                p ^= q[e] < 0.0f ? 1u : 0u;
                u[e] = u_of(q[e]);
            }
            exclusive_products<D>(u, 1.0f, 0.0f, [&](int e, float a, float b) {
                if (e >= DC && !last) return;
                float mag = kLn2 * (lg2_ftz(a) - lg2_ftz(b));
                mag = fminf(fmaxf(mag, kClipMin), kClipMax);
                const bool neg = ((p ^ (q[e] < 0.0f ? 1u : 0u)) & 1u) != 0u;
                const float rn = neg ? -mag : mag;
                if (e < DC) {
                    if (c) {
                        rn2[e < DC ? e : 0].y = rn;
                        pc2[e < DC ? e : 0].y = q[e] + rn;
                    } else {
                        rn2[e < DC ? e : 0].x = rn;
                        pc2[e < DC ? e : 0].x = q[e] + rn;
                    }
                } else {
                    pd[c] = q[e] + rn;
                }
            });
        }
        // stores: messages as aligned pairs, posteriors as pairs where the shift is even
#pragma unroll
        for (int e = 0; e < D; ++e) {
            if (e >= DC && !last) continue;
            int j = i + sh[e];
            j = j >= Z ? j - Z : j;
            float *dst = e < DC ? const_cast<float *>(src[e]) : fr.post + (src[e] - fr.ch);
            const float v0 = e < DC ? pc2[e < DC ? e : 0].x : pd[0];
            const float v1 = e < DC ? pc2[e < DC ? e : 0].y : pd[1];
            const long long ext = e < DC ? fr.bd.core : fr.bd.vars;
            if (e < DC && in_range((long long)zo[e < DC ? e : 0] * (long long)stride + i + 1, fr.bd.msgs, kBadSlot))
                *reinterpret_cast<float2 *>(slot[e < DC ? e : 0] + i) = rn2[e < DC ? e : 0];
            if (sh[e] & 1) {
                const int j1 = j + 1 == Z ? 0 : j + 1;
                if (in_range((long long)xo[e] + j, ext, kBadVariable)) dst[j] = v0;
                if (in_range((long long)xo[e] + j1, ext, kBadVariable)) dst[j1] = v1;
            } else if (in_range((long long)xo[e] + j + 1, ext, kBadVariable)) {
                *reinterpret_cast<float2 *>(dst + j) = make_float2(v0, v1);
            }
        }
        sy = sy_next;
        buf ^= 1;
    }
}

// Rows of degree 5..16: two lanes per check (lanes l and l ^ 16 of a warp).
// Each lane owns E = ceil(D/2) edges; the lanes swap their partial products
// and sign parities with one shuffle each.  As in the rows of degree <= 4, a
// lane first issues the loads of all its edges (for UP rounds of checks) in
// straight-line code -- source selected, not branched on; indices clamped to
// a valid check and edge -- and then computes: gathering edge by edge waited
// for each load in turn (the two degree-10 rows of the rate-0.1 code took a
// third of the decode that way).
#ifndef QCMET_BATCH_PAIR
#define QCMET_BATCH_PAIR 1
#endif
template <int D, typename M>
__device__ __forceinline__ void run_row_pair(const int4 *__restrict__ ent, int check_base,
                                             const Frame<M> &fr, int Z, size_t stride, bool first,
                                             bool last) {
    constexpr int E = (D + 1) / 2;
    constexpr int UP = QCMET_BATCH_PAIR;
    const int lane = threadIdx.x & 31;
    const int part = lane >> 4;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    for (int i0 = warp * 16 * UP; i0 < Z; i0 += nwarps * 16 * UP) {
        // (more than five edges per lane: too many operands to hold, gather as used)
        constexpr bool kBatch = E <= 5;
        float lv[UP][E], ro[UP][E];
        unsigned par[UP];
#pragma unroll
        for (int k = 0; k < UP; ++k) {
            const int ic = min(i0 + k * 16 + (lane & 15), Z - 1);
            par[k] = (part == 0 && in_range((long long)check_base + ic, fr.bd.checks, kBadCheck))
                         ? (fr.syn[check_base + ic] & 1u)
                         : 0u;
#pragma unroll
            for (int el = 0; el < E && kBatch; ++el) {
                const int e = min(part * E + el, D - 1);
                const int4 en = ent[e];
                int j = ic + en.y;
                j = j >= Z ? j - Z : j;
                const float *src = en.z < 0 ? fr.ch : fr.post_core;
                lv[k][el] = in_range((long long)en.x + j, en.z < 0 ? fr.bd.vars : fr.bd.core, kBadVariable)
                                ? src[en.x + j]
                                : 0.0f;
                const bool has_old = !first && en.z >= 0 &&
                                     in_range((long long)en.z * (long long)stride + ic, fr.bd.msgs, kBadSlot);
                ro[k][el] = has_old ? Msg<M>::load(fr.msg + (size_t)en.z * stride + ic) : 0.0f;
            }
        }
#pragma unroll
        for (int k = 0; k < UP; ++k) {
            const int i = i0 + k * 16 + (lane & 15);
            const bool valid = i < Z;
            float q[E], u[E];
            unsigned p = par[k];
#pragma unroll
            for (int el = 0; el < E; ++el) {
                const bool own = part * E + el < D;
                if constexpr (kBatch) {
                    q[el] = own ? lv[k][el] - ro[k][el] : 0.0f;
                } else {
                    q[el] = (own && valid) ? gather_q<M>(ent[part * E + el], i, fr, Z, stride, first)
                                           : 0.0f;
                }
                p ^= (own && q[el] < 0.0f) ? 1u : 0u;
                u[el] = own ? u_of(q[el]) : 0.0f;  // 0: the identity factor I + 0 J
            }
            // product over this lane's edges
            float ta = 1.0f, tb = 0.0f;
#pragma unroll
            for (int el = 0; el < E; ++el) {
                const float na = fmaf(u[el], tb, ta);
                const float nb = fmaf(u[el], ta, tb);
                ta = na;
                tb = nb;
            }
            const float oa = __shfl_xor_sync(0xffffffffu, ta, 16);
            const float ob = __shfl_xor_sync(0xffffffffu, tb, 16);
            p ^= __shfl_xor_sync(0xffffffffu, p, 16);
            if (!valid) continue;
            exclusive_products<E>(u, oa, ob, [&](int el, float a, float b) {
                const int e = part * E + el;
                if (e < D) scatter_r<M>(ent[e], i, q[el], a, b, p, fr, Z, stride, last);
            });
        }
    }
}

template <typename M, bool A = false>
__device__ __forceinline__ void dispatch_row(int degree, const int4 *ent, int check_base,
                                             const Frame<M> &fr, int Z, size_t stride, bool first,
                                             bool last) {
    if constexpr (A) {
        if (degree <= 4) {
            int dc = 0;
            for (int e = 0; e < degree; ++e) dc += ent[e].z >= 0 ? 1 : 0;
            switch (degree * 8 + dc) {
#define QCMET_ASYNC_CASE(DD, CC)                                                               \
    case DD * 8 + CC:                                                                          \
        if ((Z & 1) == 0)                                                                      \
            run_row_split_async2<CC, DD - CC>(ent, check_base, fr, Z, stride, first, last);   \
        else                                                                                   \
            run_row_split_async<CC, DD - CC>(ent, check_base, fr, Z, stride, first, last);    \
        break;
                QCMET_ASYNC_CASE(1, 0)
                QCMET_ASYNC_CASE(1, 1)
                QCMET_ASYNC_CASE(2, 0)
                QCMET_ASYNC_CASE(2, 1)
                QCMET_ASYNC_CASE(2, 2)
                QCMET_ASYNC_CASE(3, 0)
                QCMET_ASYNC_CASE(3, 1)
                QCMET_ASYNC_CASE(3, 2)
                QCMET_ASYNC_CASE(3, 3)
                QCMET_ASYNC_CASE(4, 0)
                QCMET_ASYNC_CASE(4, 1)
                QCMET_ASYNC_CASE(4, 2)
                QCMET_ASYNC_CASE(4, 3)
                QCMET_ASYNC_CASE(4, 4)
#undef QCMET_ASYNC_CASE
                default: break;
            }
            return;
        }
    }
    if (degree <= 4) {
        // core edges first: their count picks the specialisation
        int dc = 0;
        for (int e = 0; e < degree; ++e) dc += ent[e].z >= 0 ? 1 : 0;
        switch (degree * 8 + dc) {
#define QCMET_SPLIT_CASE(DD, CC) \
    case DD * 8 + CC: run_row_split<CC, DD - CC, M>(ent, check_base, fr, Z, stride, first, last); break;
            QCMET_SPLIT_CASE(1, 0)
            QCMET_SPLIT_CASE(1, 1)
            QCMET_SPLIT_CASE(2, 0)
            QCMET_SPLIT_CASE(2, 1)
            QCMET_SPLIT_CASE(2, 2)
            QCMET_SPLIT_CASE(3, 0)
            QCMET_SPLIT_CASE(3, 1)
            QCMET_SPLIT_CASE(3, 2)
            QCMET_SPLIT_CASE(3, 3)
            QCMET_SPLIT_CASE(4, 0)
            QCMET_SPLIT_CASE(4, 1)
            QCMET_SPLIT_CASE(4, 2)
            QCMET_SPLIT_CASE(4, 3)
            QCMET_SPLIT_CASE(4, 4)
#undef QCMET_SPLIT_CASE
            default: break;
        }
        return;
    }
    switch (degree) {
#define QCMET_PAIR_CASE(DD) \
    case DD: run_row_pair<DD, M>(ent, check_base, fr, Z, stride, first, last); break;
        QCMET_PAIR_CASE(5)
        QCMET_PAIR_CASE(6)
        QCMET_PAIR_CASE(7)
        QCMET_PAIR_CASE(8)
        QCMET_PAIR_CASE(9)
        QCMET_PAIR_CASE(10)
        QCMET_PAIR_CASE(11)
        QCMET_PAIR_CASE(12)
        QCMET_PAIR_CASE(13)
        QCMET_PAIR_CASE(14)
        QCMET_PAIR_CASE(15)
        QCMET_PAIR_CASE(16)
#undef QCMET_PAIR_CASE
        default: break;
    }
}

// ---- offset/scaled min-sum rows (the learned variant; not the paper's rule) ----
//
// |r_e| = min(max(scale * min_{k != e} |q_k| - offset, 0), 30) with the sign of
// step 2 (the upper clip is the sum-product rule's);
// wt = (scale for an edge to a core variable, scale for a degree-1 variable,
// offset core, offset degree-1) of this row and iteration.  The gathers and
// writes are those of the sum-product rows.
constexpr float kNoOtherEdge = 30.0f;  // min over the empty set (a degree-1 check)
#ifndef QCMET_BATCH_MINSUM
#define QCMET_BATCH_MINSUM 1
#endif

template <typename M>
__device__ __forceinline__ void scatter_minsum(const int4 &en, int i, float q, float mn,
                                               unsigned par, const float4 &wt, const Frame<M> &fr,
                                               int Z, size_t stride, bool last) {
    const bool deg1 = en.z < 0;
    if (deg1 && !last) return;
    const float a_e = (deg1 ? wt.y : wt.x) * mn - (deg1 ? wt.w : wt.z);
    const float mag = fminf(fmaxf(a_e, 0.0f), kClipMax);
    const bool neg = ((par ^ (q < 0.0f ? 1u : 0u)) & 1u) != 0u;
    float rn = neg ? -mag : mag;
    int j = i + en.y;
    j = j >= Z ? j - Z : j;
    const int v = en.x + j;
    if (!deg1) {
        rn = Msg<M>::quantize(rn);
        if (in_range((long long)en.z * (long long)stride + i, fr.bd.msgs, kBadSlot))
            Msg<M>::store(fr.msg + (size_t)en.z * stride + i, rn);
        if (in_range(v, fr.bd.core, kBadVariable)) fr.post_core[v] = q + rn;
    } else if (in_range(v, fr.bd.vars, kBadVariable)) {
        fr.post[v] = q + rn;
    }
}

// Rows of degree DC + D1 <= 4, core edges first (the gather of run_row_split).
template <int DC, int D1, typename M>
__device__ __forceinline__ void run_row_minsum(const int4 *__restrict__ ent, int check_base,
                                               const Frame<M> &fr, int Z, size_t stride, bool first,
                                               bool last, const float4 &wt) {
    constexpr int D = DC + D1;
    constexpr int NC = DC > 0 ? DC : 1;
    constexpr int U = QCMET_BATCH_MINSUM;
    const int step = blockDim.x;
    const float *src[D];
    int sh[D];
    int xo[D], zo[DC > 0 ? DC : 1];  // variable and slot offsets (index checks of the debug build)
    M *slot[NC];
#pragma unroll
    for (int e = 0; e < D; ++e) {
        const int4 en = ent[e];
        src[e] = (e < DC ? fr.post_core : fr.ch) + en.x;
        sh[e] = en.y;
        xo[e] = en.x;
        if (e < DC) {
            slot[e] = fr.msg + (size_t)en.z * stride;
            zo[e] = en.z;
        }
    }
    for (int i0 = threadIdx.x; i0 < Z; i0 += step * U) {
        float lv[U][D], ro[U][NC];
        unsigned par[U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const int i = min(i0 + k * step, Z - 1);
            par[k] = in_range((long long)check_base + i, fr.bd.checks, kBadCheck)
                         ? (fr.syn[check_base + i] & 1u)
                         : 0u;
#pragma unroll
            for (int e = 0; e < D; ++e) {
                int j = i + sh[e];
                j = j >= Z ? j - Z : j;
                lv[k][e] = in_range((long long)xo[e] + j, e < DC ? fr.bd.core : fr.bd.vars, kBadVariable)
                                ? src[e][j]
                                : 0.0f;
            }
#pragma unroll
            for (int e = 0; e < DC; ++e)
                ro[k][e] = (first || !in_range((long long)zo[e] * (long long)stride + i, fr.bd.msgs, kBadSlot))
                               ? 0.0f
                               : Msg<M>::load(slot[e] + i);
        }
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const int i = i0 + k * step;
            if (i >= Z) break;
            float q[D];
            unsigned p = par[k];
            float m1 = INFINITY, m2 = INFINITY;
            int i1 = -1;
#pragma unroll
            for (int e = 0; e < D; ++e) {
                q[e] = e < DC ? lv[k][e] - ro[k][e < DC ? e : 0] : lv[k][e];
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
                const float mn = D == 1 ? kNoOtherEdge : (e == i1 ? m2 : m1);
                const float a_e = (e >= DC ? wt.y : wt.x) * mn - (e >= DC ? wt.w : wt.z);
                const float mag = fminf(fmaxf(a_e, 0.0f), kClipMax);
                const bool neg = ((p ^ (q[e] < 0.0f ? 1u : 0u)) & 1u) != 0u;
                float rn = neg ? -mag : mag;
                int j = i + sh[e];
                j = j >= Z ? j - Z : j;
                if (e < DC) {
                    rn = Msg<M>::quantize(rn);
                    if (in_range((long long)zo[e < DC ? e : 0] * (long long)stride + i, fr.bd.msgs, kBadSlot))
                        Msg<M>::store(slot[e < DC ? e : 0] + i, rn);
                    if (in_range((long long)xo[e] + j, fr.bd.core, kBadVariable))
                        const_cast<float *>(src[e])[j] = q[e] + rn;
                } else {
                    if (in_range((long long)xo[e] + j, fr.bd.vars, kBadVariable))
                        fr.post[(src[e] - fr.ch) + j] = q[e] + rn;
                }
            }
        }
    }
}

// Rows of degree 5..16: lanes l and l ^ 16 share a check (as run_row_pair);
// each lane finds the two smallest |q| of its edges and takes the partner's
// smallest by one shuffle.
template <int D, typename M>
__device__ __forceinline__ void run_row_pair_minsum(const int4 *__restrict__ ent, int check_base,
                                                    const Frame<M> &fr, int Z, size_t stride,
                                                    bool first, bool last, const float4 &wt) {
    constexpr int E = (D + 1) / 2;
    const int lane = threadIdx.x & 31;
    const int part = lane >> 4;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    for (int i0 = warp * 16; i0 < Z; i0 += nwarps * 16) {
        const int i = i0 + (lane & 15);
        const bool valid = i < Z;
        const int ic = min(i, Z - 1);
        float q[E];
        unsigned par = (part == 0 && in_range((long long)check_base + ic, fr.bd.checks, kBadCheck))
                           ? (fr.syn[check_base + ic] & 1u)
                           : 0u;
        // all of this lane's loads first (source selected; indices clamped), for
        // at most five edges per lane; more are gathered as used
        constexpr bool kBatch = E <= 5;
        float lv[E], ro[E];
#pragma unroll
        for (int el = 0; el < E && kBatch; ++el) {
            const int4 en = ent[min(part * E + el, D - 1)];
            int j = ic + en.y;
            j = j >= Z ? j - Z : j;
            const float *src = en.z < 0 ? fr.ch : fr.post_core;
            lv[el] = in_range((long long)en.x + j, en.z < 0 ? fr.bd.vars : fr.bd.core, kBadVariable)
                         ? src[en.x + j]
                         : 0.0f;
            ro[el] = (!first && en.z >= 0 &&
                      in_range((long long)en.z * (long long)stride + ic, fr.bd.msgs, kBadSlot))
                         ? Msg<M>::load(fr.msg + (size_t)en.z * stride + ic)
                         : 0.0f;
        }
        float m1 = INFINITY, m2 = INFINITY;
        int i1 = -1;
#pragma unroll
        for (int el = 0; el < E; ++el) {
            const int e = part * E + el;
            q[el] = 0.0f;
            if (valid && e < D) {
                if constexpr (kBatch) {
                    q[el] = lv[el] - ro[el];
                } else {
                    q[el] = gather_q<M>(ent[e], i, fr, Z, stride, first);
                }
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
        if (!valid) continue;
        // excluding this lane's argmin: its next smallest or the partner's
        // smallest; excluding any other edge of this lane: the overall smallest
        const float ex1 = fminf(m2, om1);
        const float exo = fminf(m1, om1);
#pragma unroll
        for (int el = 0; el < E; ++el) {
            const int e = part * E + el;
            if (e < D)
                scatter_minsum<M>(ent[e], i, q[el], el == i1 ? ex1 : exo, par, wt, fr, Z, stride,
                                  last);
        }
    }
}

template <typename M>
__device__ __forceinline__ void dispatch_row_minsum(int degree, const int4 *ent, int check_base,
                                                    const Frame<M> &fr, int Z, size_t stride,
                                                    bool first, bool last, const float4 &wt) {
    if (degree <= 4) {
        int dc = 0;
        for (int e = 0; e < degree; ++e) dc += ent[e].z >= 0 ? 1 : 0;
        switch (degree * 8 + dc) {
#define QCMET_SPLIT_CASE(DD, CC) \
    case DD * 8 + CC:                                                                        \
        run_row_minsum<CC, DD - CC, M>(ent, check_base, fr, Z, stride, first, last, wt); break;
            QCMET_SPLIT_CASE(1, 0)
            QCMET_SPLIT_CASE(1, 1)
            QCMET_SPLIT_CASE(2, 0)
            QCMET_SPLIT_CASE(2, 1)
            QCMET_SPLIT_CASE(2, 2)
            QCMET_SPLIT_CASE(3, 0)
            QCMET_SPLIT_CASE(3, 1)
            QCMET_SPLIT_CASE(3, 2)
            QCMET_SPLIT_CASE(3, 3)
            QCMET_SPLIT_CASE(4, 0)
            QCMET_SPLIT_CASE(4, 1)
            QCMET_SPLIT_CASE(4, 2)
            QCMET_SPLIT_CASE(4, 3)
            QCMET_SPLIT_CASE(4, 4)
#undef QCMET_SPLIT_CASE
            default: break;
        }
        return;
    }
    switch (degree) {
#define QCMET_PAIR_CASE(DD) \
    case DD: run_row_pair_minsum<DD, M>(ent, check_base, fr, Z, stride, first, last, wt); break;
        QCMET_PAIR_CASE(5)
        QCMET_PAIR_CASE(6)
        QCMET_PAIR_CASE(7)
        QCMET_PAIR_CASE(8)
        QCMET_PAIR_CASE(9)
        QCMET_PAIR_CASE(10)
        QCMET_PAIR_CASE(11)
        QCMET_PAIR_CASE(12)
        QCMET_PAIR_CASE(13)
        QCMET_PAIR_CASE(14)
        QCMET_PAIR_CASE(15)
        QCMET_PAIR_CASE(16)
#undef QCMET_PAIR_CASE
        default: break;
    }
}

// Step 4 outputs for frame f: the posterior of every column (core columns
// copied from the compact state) and the hard decisions c_n = [L_qn < 0].
//   deg1_from_channel: no iteration ran, so degree-1 columns still hold the channel
template <typename M>
__device__ __noinline__ void write_outputs(const Sched &s, const DecodeArgs &a, const Frame<M> &fr,
                                           int f, bool deg1_from_channel) {
    const int Z = s.Z;
    const size_t n = (size_t)a.n;
    for (int c = 0; c < s.nb; ++c) {
        const int kind = s.col_kind[c];
        const bool from_channel = kind == kColUnconnected || (kind == kColDegree1 && deg1_from_channel);
        const size_t base = (size_t)c * Z;
        const float *core = kind == kColCore ? fr.post_core + (size_t)s.col_core[c] * Z : nullptr;
        for (int i = threadIdx.x; i < Z; i += blockDim.x) {
            if (!in_range((long long)base + i, fr.bd.vars, kBadVariable)) continue;
            if (core && !in_range((long long)s.col_core[c] * Z + i, fr.bd.core, kBadVariable)) continue;
            float L;
            if (core) {
                L = core[i];
                fr.post[base + i] = L;
            } else if (from_channel) {
                L = fr.ch[base + i];
                fr.post[base + i] = L;
            } else {
                L = fr.post[base + i];
            }
            a.hard[(size_t)f * n + base + i] = L < 0.0f ? 1 : 0;
        }
    }
}

// Nonzero when some check of the row (rows of degree D <= 4, one thread per
// check) has s_m XOR (XOR of its variables' hard decisions) = 1.  The hard
// decision [L < 0] is taken from the posteriors directly: the compact core
// state, and llr_post for degree-1 columns (written in every tested
// iteration).  Loads of U checks are issued together, as in run_row.
template <int D, typename M>
__device__ __forceinline__ int row_fails(const int4 *__restrict__ ent, int check_base,
                                         const Frame<M> &fr, int Z) {
    constexpr int U = 2;
    const int step = blockDim.x;
    for (int i0 = threadIdx.x; i0 < Z; i0 += step * U) {
        float lv[U][D];
        unsigned par[U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const int i = min(i0 + k * step, Z - 1);
            par[k] = in_range((long long)check_base + i, fr.bd.checks, kBadCheck)
                         ? (fr.syn[check_base + i] & 1u)
                         : 0u;
#pragma unroll
            for (int e = 0; e < D; ++e) {
                const int4 en = ent[e];
                int j = i + en.y;
                j = j >= Z ? j - Z : j;
                const float *src = en.z < 0 ? fr.post : fr.post_core;
                lv[k][e] = in_range((long long)en.x + j, en.z < 0 ? fr.bd.vars : fr.bd.core, kBadVariable)
                               ? src[en.x + j]
                               : 0.0f;
            }
        }
        unsigned bad = 0u;
#pragma unroll
        for (int k = 0; k < U; ++k) {
            unsigned p = par[k];
#pragma unroll
            for (int e = 0; e < D; ++e) p ^= lv[k][e] < 0.0f ? 1u : 0u;
            bad |= (i0 + k * step < Z) ? p : 0u;
        }
        if (bad) return 1;
    }
    return 0;
}

template <typename M>
__device__ __forceinline__ int row_fails_any(const int4 *__restrict__ ent, int degree,
                                             int check_base, const Frame<M> &fr, int Z) {
    for (int i = threadIdx.x; i < Z; i += blockDim.x) {
        unsigned p = in_range((long long)check_base + i, fr.bd.checks, kBadCheck)
                         ? (fr.syn[check_base + i] & 1u)
                         : 0u;
        for (int e = 0; e < degree; ++e) {
            const int4 en = ent[e];
            int j = i + en.y;
            j = j >= Z ? j - Z : j;
            const float *src = en.z < 0 ? fr.post : fr.post_core;
            if (in_range((long long)en.x + j, en.z < 0 ? fr.bd.vars : fr.bd.core, kBadVariable))
                p ^= src[en.x + j] < 0.0f ? 1u : 0u;
        }
        if (p) return 1;
    }
    return 0;
}

// The syndrome test H c = s on the current posteriors.  Returns, identically
// in every thread of the block, nonzero when it fails.  A frame that has not
// converged fails in its first rows, so the block stops at the first row with
// a failing check (one barrier-with-OR per row): a failed test costs about one
// row, a passed one a read of every edge's posterior.
template <typename M>
__device__ __noinline__ int syndrome_fails(const Sched s, const Frame<M> fr) {
    const int Z = s.Z;
    int bad = 0;
    for (int zr = 0; zr < s.n_zero_rows; ++zr) {
        const size_t cb = (size_t)s.zero_rows[zr] * Z;
        for (int i = threadIdx.x; i < Z; i += blockDim.x)
            if (in_range((long long)cb + i, fr.bd.checks, kBadCheck)) bad |= fr.syn[cb + i] & 1;
    }
    if (__syncthreads_or(bad)) return 1;
    for (int j = 0; j < s.n_rows; ++j) {
        const int4 row = s.rows[j];
        const int4 *ent = s.entries + row.x;
        switch (row.y) {
            case 1: bad = row_fails<1, M>(ent, row.z, fr, Z); break;
            case 2: bad = row_fails<2, M>(ent, row.z, fr, Z); break;
            case 3: bad = row_fails<3, M>(ent, row.z, fr, Z); break;
            case 4: bad = row_fails<4, M>(ent, row.z, fr, Z); break;
            default: bad = row_fails_any<M>(ent, row.y, row.z, fr, Z); break;
        }
        if (__syncthreads_or(bad)) return 1;
    }
    return 0;
}

// Decode frame f of `a` (steps 1-4) with the schedule `s` already in shared
// memory.  Called by every thread of the block.
enum : int { kRuleSumProduct = 0, kRuleMinSum = 1 };

template <typename M, int R, bool A = false>
__device__ __forceinline__ void decode_one_frame(const Sched &s, const DecodeArgs &a, int f,
                                                 const float *w_scale, const float *w_offset) {
    const int Z = s.Z;
    const size_t n = (size_t)a.n;
    const size_t stride = (size_t)a.slot_stride;
    const int T = a.T;
    Frame<M> fr;
    fr.ch = a.ch + (size_t)f * n;
    fr.syn = a.syn + (size_t)f * (size_t)a.m;
    fr.post = a.post + (size_t)f * n;
    fr.post_core = a.post_core + (size_t)f * (size_t)a.core_cols * Z;
    fr.msg = static_cast<M *>(a.msgs) + (size_t)f * (size_t)a.msg_slots * stride;
    fr.bd.core = (long long)a.core_cols * Z;
    fr.bd.vars = (long long)n;
    fr.bd.msgs = (long long)a.msg_slots * (long long)stride;
    fr.bd.checks = (long long)a.m;

    // Step 1: L_qn = channel LLR for every variable that carries state.
    for (int c = 0; c < s.nb; ++c) {
        if (s.col_kind[c] != kColCore) continue;
        const float *src = fr.ch + (size_t)c * Z;
        float *dst = fr.post_core + (size_t)s.col_core[c] * Z;
        for (int i = threadIdx.x; i < Z; i += blockDim.x)
            if (in_range((long long)c * Z + i, fr.bd.vars, kBadVariable) &&
                in_range((long long)s.col_core[c] * Z + i, fr.bd.core, kBadVariable))
                dst[i] = src[i];
    }
    __syncthreads();

    // Steps 2-3 over T iterations x layers.  With early termination
    // (Discussion, Table tabearly) every check_every-th iteration ends with
    // the hard decision and syndrome test, and a frame that passes stops.
    // Those iterations, like the last one, also write the posteriors of the
    // degree-1 columns, which the test needs.
    int t_stop = T;
    int fail = 1;
    for (int t = 0; t < T; ++t) {
        const bool first = t == 0;
        const bool final_iter = t == T - 1;
        const bool check = final_iter || (a.check_every > 0 && (t + 1) % a.check_every == 0);
        for (int layer = 0; layer < s.n_layers; ++layer) {
            for (int j = s.layer_first[layer]; j < s.layer_first[layer + 1]; ++j) {
                const int4 row = s.rows[j];
                if constexpr (R == kRuleSumProduct) {
                    dispatch_row<M, A>(row.y, s.entries + row.x, row.z, fr, Z, stride, first,
                                       check);
                } else {
                    const size_t w = ((size_t)t * s.mb + (size_t)row.w) * 2;
                    const float4 wt = make_float4(__ldg(w_scale + w), __ldg(w_scale + w + 1),
                                                  __ldg(w_offset + w), __ldg(w_offset + w + 1));
                    dispatch_row_minsum<M>(row.y, s.entries + row.x, row.z, fr, Z, stride, first,
                                           check, wt);
                }
            }
            __syncthreads();
        }
        if (check) {
            fail = syndrome_fails<M>(s, fr);
            if (!fail && a.check_every > 0) {
                t_stop = t + 1;
                break;
            }
        }
    }

    write_outputs<M>(s, a, fr, f, T == 0);
    if (T == 0) {
        __syncthreads();
        fail = syndrome_fails<M>(s, fr);
    }
    if (threadIdx.x == 0) {
        a.ok[f] = fail ? 0 : 1;
        if (a.iters_used) a.iters_used[f] = t_stop;
    }
    __syncthreads();
}

template <typename M, int R, int NT = kDefaultThreads>
__global__ void __launch_bounds__(NT, 1) decode_kernel(const DecodeArgs a, const float *w_scale,
                                                       const float *w_offset) {
    constexpr bool A = std::is_same<M, float>::value && R == kRuleSumProduct;
    int4 *smem_i4 = qcmet_dyn_smem + (A ? kAsyncStageFloats * kDefaultThreads / 4 : 0);
    int32_t *sw = reinterpret_cast<int32_t *>(smem_i4);
    {
        const int4 *src = reinterpret_cast<const int4 *>(a.image);
        for (int k = threadIdx.x; k < a.image_words / 4; k += blockDim.x) smem_i4[k] = src[k];
    }
    __syncthreads();
    const Sched s = make_sched(sw);
    for (int f = blockIdx.x; f < a.K; f += gridDim.x)
        decode_one_frame<M, R, A>(s, a, f, w_scale, w_offset);
}

// Mixed batch: frames of several codes in one launch.  Persistent CTAs take
// frames in the order given (largest first by default) from an atomic
// counter -- a work queue, nothing waits on another CTA -- load the frame's
// layer table into shared memory when the code changes, and decode it.
template <typename M>
__global__ void __launch_bounds__(kDefaultThreads, 1) decode_batch_kernel(const BatchArgs b) {
    constexpr bool A = std::is_same<M, float>::value;
    int4 *smem_i4 = qcmet_dyn_smem + (A ? kAsyncStageFloats * kDefaultThreads / 4 : 0);
    int32_t *sw = reinterpret_cast<int32_t *>(smem_i4);
    __shared__ int s_next;
    int cur_code = -1;
    for (;;) {
        if (threadIdx.x == 0) s_next = atomicAdd(b.counter, 1);
        __syncthreads();
        const int k = s_next;
        __syncthreads();
        if (k >= b.K) break;
        const BatchFrame fd = b.frames[b.order[k]];
        if (fd.code_id != cur_code) {
            const int4 *src = reinterpret_cast<const int4 *>(fd.image);
            for (int w = threadIdx.x; w < fd.image_words / 4; w += blockDim.x) smem_i4[w] = src[w];
            __syncthreads();
            cur_code = fd.code_id;
        }
        const Sched s = make_sched(sw);
        DecodeArgs a;
        a.ch = fd.ch;
        a.syn = fd.syn;
        a.post = fd.post;
        a.post_core = fd.post_core;
        a.msgs = fd.msgs;
        a.hard = fd.hard;
        a.ok = fd.ok;
        a.image = fd.image;
        a.image_words = fd.image_words;
        a.K = 1;
        a.T = b.T;
        a.Z = fd.Z;
        a.n = fd.n;
        a.m = fd.m;
        a.nb = fd.nb;
        a.msg_slots = fd.msg_slots;
        a.core_cols = fd.core_cols;
        a.slot_stride = fd.slot_stride;
        a.check_every = 0;
        a.iters_used = nullptr;
        decode_one_frame<M, kRuleSumProduct, A>(s, a, 0, nullptr, nullptr);
    }
}

}  // namespace

int take_violations_frame(uint32_t *bits, std::string &err) {
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

namespace {

int sm_count_cached() {
    static int count[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (dev < 0 || dev >= 64) return 0;
    if (!count[dev]) cudaDeviceGetAttribute(&count[dev], cudaDevAttrMultiProcessorCount, dev);
    return count[dev];
}

template <typename M, int R = kRuleSumProduct>
int launch_typed(const DecodeArgs &a, int threads, void *stream, std::string &err,
                 size_t window_bytes = 0, float hit_ratio = 0.0f,
                 const CheckRule &rule = CheckRule()) {
    constexpr bool A = std::is_same<M, float>::value && R == kRuleSumProduct;
    const size_t smem = (size_t)a.image_words * sizeof(int32_t) +
                        (A ? (size_t)kAsyncStageFloats * kDefaultThreads * sizeof(float) : 0);
    auto kern = decode_kernel<M, R>;
    if constexpr (A) {
        if (threads <= kFp32Threads) kern = decode_kernel<M, R, kFp32Threads>;
    }
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) {
            err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e);
            return QCMET_ERR_UNSUPPORTED;
        }
    }
    const int sms = sm_count_cached();
    if (sms <= 0) {
        err = "no CUDA device";
        return QCMET_ERR_CUDA;
    }
    const int grid = a.K < sms ? a.K : sms;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = static_cast<cudaStream_t>(stream);
    cudaLaunchAttribute attr[1];
    if (window_bytes > 0) {
        // the core posteriors persist in L2; whatever misses the window streams
        attr[0].id = cudaLaunchAttributeAccessPolicyWindow;
        attr[0].val.accessPolicyWindow.base_ptr = a.post_core;
        attr[0].val.accessPolicyWindow.num_bytes = window_bytes;
        attr[0].val.accessPolicyWindow.hitRatio = hit_ratio;
        attr[0].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
        attr[0].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, a, rule.w_scale, rule.w_offset);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        err = std::string("decode launch: ") + cudaGetErrorString(e);
        return QCMET_ERR_CUDA;
    }
    return QCMET_OK;
}

template <typename M>
int launch_batch_typed(const BatchArgs &b, int threads, int grid, size_t smem, void *stream,
                       std::string &err) {
    auto kern = decode_batch_kernel<M>;
    if (std::is_same<M, float>::value) smem += (size_t)kAsyncStageFloats * kDefaultThreads * sizeof(float);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) {
            err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e);
            return QCMET_ERR_UNSUPPORTED;
        }
    }
    kern<<<grid, threads, smem, static_cast<cudaStream_t>(stream)>>>(b);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        err = std::string("batch decode launch: ") + cudaGetErrorString(e);
        return QCMET_ERR_CUDA;
    }
    return QCMET_OK;
}

}  // namespace

int launch_decode_batch(const BatchArgs &b, int32_t msg_format, int32_t threads,
                        int32_t max_image_words, void *stream, std::string &err) {
    if (threads == 0) threads = kDefaultThreads;
    if (threads < 32 || threads > kDefaultThreads || threads % 32) {
        err = "threads_per_block must be a multiple of 32 in [32, 1024]";
        return QCMET_ERR_INVALID_ARG;
    }
    const int sms = sm_count_cached();
    if (sms <= 0) {
        err = "no CUDA device";
        return QCMET_ERR_CUDA;
    }
    const int grid = b.K < sms ? b.K : sms;
    if (grid <= 0) return QCMET_OK;
    const size_t smem = (size_t)max_image_words * sizeof(int32_t);
    switch (msg_format) {
        case QCMET_MSG_FP32: return launch_batch_typed<float>(b, threads, grid, smem, stream, err);
        case QCMET_MSG_FP16: return launch_batch_typed<__half>(b, threads, grid, smem, stream, err);
        case QCMET_MSG_BF16:
            return launch_batch_typed<__nv_bfloat16>(b, threads, grid, smem, stream, err);
        default: err = "unknown message format"; return QCMET_ERR_INVALID_ARG;
    }
}

int launch_decode(const DecodeArgs &a, int32_t msg_format, int32_t threads, void *stream,
                  std::string &err, size_t window_bytes, float hit_ratio, const CheckRule &rule) {
    if (threads == 0)
        threads = (msg_format == QCMET_MSG_FP32 && !rule.w_scale) ? kFp32Threads : kDefaultThreads;
    if (threads < 32 || threads > kDefaultThreads || threads % 32) {
        err = "threads_per_block must be a multiple of 32 in [32, 1024]";
        return QCMET_ERR_INVALID_ARG;
    }
    if (rule.w_scale) {
        if (msg_format != QCMET_MSG_FP32) {
            err = "the min-sum rule keeps FP32 messages";
            return QCMET_ERR_INVALID_ARG;
        }
        return launch_typed<float, kRuleMinSum>(a, threads, stream, err, window_bytes, hit_ratio,
                                                rule);
    }
    switch (msg_format) {
        case QCMET_MSG_FP32:
            return launch_typed<float>(a, threads, stream, err, window_bytes, hit_ratio);
        case QCMET_MSG_FP16:
            return launch_typed<__half>(a, threads, stream, err, window_bytes, hit_ratio);
        case QCMET_MSG_BF16:
            return launch_typed<__nv_bfloat16>(a, threads, stream, err, window_bytes, hit_ratio);
        default: err = "unknown message format"; return QCMET_ERR_INVALID_ARG;
    }
}

// ---- decoding without device allocations ----------------------------------
//
// Scratch for qcmet_decode_noalloc: one fixed-size array in device memory that
// the library defines at file scope.  Every GPU that loads the library holds
// it until the process exits.  Layout: the code's layer table in the first
// kNoAllocImageBytes, the check-to-variable messages after it.  In host code
// the name g_noalloc_scratch is only a stand-in for the symbol; its device
// address comes from cudaGetSymbolAddress, taken once per device.
namespace {

constexpr size_t kNoAllocBytes = size_t(32) << 20;      // 32 MiB in total
constexpr size_t kNoAllocImageBytes = size_t(64) << 10;  // 64 KiB of it for the layer table

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mutex;
struct NoAllocSlot {
    void *addr = nullptr;             // device address of g_noalloc_scratch
    unsigned long long ctx_id = 0;    // the context it belongs to (cuCtxGetId, never 0)
};
NoAllocSlot g_noalloc_slot[64];

// Unique id (for the life of the process) of the calling thread's current CUDA
// context, 0 when none is current.  The driver calls are reached through the
// runtime's entry-point query, so the library needs no link to libcuda.  The
// address of g_noalloc_scratch belongs to a context: after cudaDeviceReset the
// device's new primary context has a new id and the address is looked up again.
typedef CUresult (*PfnCtxGetCurrent)(CUcontext *);
typedef CUresult (*PfnCtxGetId)(CUcontext, unsigned long long *);

int current_context_id(unsigned long long *id, std::string &err) {
    static std::once_flag once;
    static PfnCtxGetCurrent get_current = nullptr;
    static PfnCtxGetId get_id = nullptr;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult r;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &r) ==
                cudaSuccess && r == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<PfnCtxGetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &r) ==
                cudaSuccess && r == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<PfnCtxGetId>(f);
    });
    *id = 0;
    if (!get_current || !get_id) {
        err = "the CUDA driver does not provide cuCtxGetCurrent / cuCtxGetId";
        return QCMET_ERR_CUDA;
    }
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS) {
        err = "cuCtxGetCurrent failed";
        return QCMET_ERR_CUDA;
    }
    if (!ctx) return QCMET_OK;
    if (get_id(ctx, id) != CUDA_SUCCESS) {
        err = "cuCtxGetId failed";
        return QCMET_ERR_CUDA;
    }
    return QCMET_OK;
}

// Device address of g_noalloc_scratch in the current context: looked up once
// per device and context, then cached.
int noalloc_address(void **out, std::string &err) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return QCMET_ERR_CUDA;
    }
    if (dev < 0 || dev >= 64) {
        err = "device index above 63";
        return QCMET_ERR_UNSUPPORTED;
    }
    unsigned long long id = 0;
    int st = current_context_id(&id, err);
    if (st) return st;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    NoAllocSlot &slot = g_noalloc_slot[dev];
    if (!slot.addr || id == 0 || slot.ctx_id != id) {
        void *p = nullptr;
        // also makes the runtime's context current when none was
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            err = std::string("cudaGetSymbolAddress(g_noalloc_scratch): ") + cudaGetErrorString(e);
            return QCMET_ERR_CUDA;
        }
        st = current_context_id(&id, err);
        if (st) return st;
        slot.addr = p;
        slot.ctx_id = id;
    }
    *out = slot.addr;
    return QCMET_OK;
}

}  // namespace

size_t noalloc_capacity_bytes() { return kNoAllocBytes - kNoAllocImageBytes; }

int launch_decode_noalloc(DecodeArgs a, const int32_t *image_host, size_t image_bytes,
                          void *stream, std::string &err) {
    if (image_bytes > kNoAllocImageBytes) {
        err = "the code's layer table needs " + std::to_string(image_bytes) +
              " bytes; qcmet_decode_noalloc reserves " + std::to_string(kNoAllocImageBytes);
        return QCMET_ERR_INVALID_ARG;
    }
    const size_t msg_bytes =
        ((size_t)a.K * (size_t)a.msg_slots * (size_t)a.slot_stride * sizeof(float) + 255) &
        ~size_t(255);
    const size_t core_bytes = (size_t)a.K * (size_t)a.core_cols * (size_t)a.Z * sizeof(float);
    const size_t need = msg_bytes + core_bytes;
    if (need > noalloc_capacity_bytes()) {
        err = "decoding these frames needs " + std::to_string(need) +
              " bytes of message and state scratch; qcmet_decode_noalloc holds " +
              std::to_string(noalloc_capacity_bytes()) + " (use fewer frames per call or qcmet_decode)";
        return QCMET_ERR_INVALID_ARG;
    }
    void *base = nullptr;
    int st = noalloc_address(&base, err);
    if (st) return st;
    char *p = static_cast<char *>(base);
    // The layer table is copied in every call: the array keeps whatever the
    // previous call left there.  The messages and the core posteriors need no
    // clearing (the first iteration does not read the messages; step 1 writes
    // every core posterior before it is read).
    cudaError_t e = cudaMemcpyAsync(p, image_host, image_bytes, cudaMemcpyHostToDevice,
                                    static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        err = std::string("cudaMemcpyAsync(layer table): ") + cudaGetErrorString(e);
        return QCMET_ERR_CUDA;
    }
    a.image = reinterpret_cast<const int32_t *>(p);
    a.msgs = p + kNoAllocImageBytes;
    a.post_core = reinterpret_cast<float *>(p + kNoAllocImageBytes + msg_bytes);
    return launch_typed<float>(a, kFp32Threads, stream, err);
}

}  // namespace qcmet
