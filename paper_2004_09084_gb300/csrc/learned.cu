// Learned offset/scaled min-sum layered decoder: forward, training forward and
// hand-written backward (sm_103a).
//
// Not part of arXiv 2004.09084's method: a variant of its layered decoder
// (Methods, steps 1-4) in which the check rule of step 2 becomes
//   r_e = (-1)^{s_m} prod_{k != e} sgn(q_k) * min(max(a_e, 0), 30),
//   a_e = w_scale[t][l][type_e] * min_{k != e} |q_k| - w_offset[t][l][type_e],
// with one scale and one offset per (iteration t, base row l, edge type);
// type 0 marks an edge to a variable of degree > 1, type 1 an edge to a
// degree-1 variable.  Steps 1, 3 and 4 are unchanged.
//
// Training loss (per frame): the mean over iterations t and variables n of
// softplus(-(1 - 2 x_n) L_qn^(t)), the cross-entropy of sigma(-L) against the
// transmitted bit x_n, with L^(t) the posterior after iteration t.  The
// backward kernel differentiates the unrolled layered decoder in reverse
// (iterations and layers backwards), carrying the adjoints of the core
// posteriors L_qn and of the stored messages L_rmn.
//
// Layout and mapping follow decode.cu: one CTA per frame for the whole call,
// layer boundary = block barrier, frame-major arrays, degree-1 variables
// without state (for them q = channel LLR exactly, so their message enters the
// loss of its own iteration only and carries no adjoint).
#include <cuda_runtime.h>

#include <cstdio>

#include "qcmet_internal.h"

namespace qcmet {

namespace {

constexpr int kThreads = 512;
constexpr float kNoOther = 30.0f;  // the message clip; also min over an empty set (degree-1 check)

struct LearnedView {
    int32_t n_rows, n_layers, nb, Z, mb, core_cols;
    const int32_t *layer_first;
    const int4 *rows;     // DevRow
    const int4 *entries;  // DevEntry
    const int32_t *col_kind;
    const int32_t *col_core;  // built in shared memory at kernel start
};

// Copy the schedule image to shared memory and build the column -> core index map.
__device__ LearnedView load_view(const LearnedArgs &a, int32_t *sw) {
    const int4 *src = reinterpret_cast<const int4 *>(a.image);
    int4 *dst = reinterpret_cast<int4 *>(sw);
    for (int k = threadIdx.x; k < a.image_words / 4; k += blockDim.x) dst[k] = src[k];
    __syncthreads();
    LearnedView v;
    v.n_rows = sw[kHdrRows];
    v.n_layers = sw[kHdrLayers];
    v.nb = sw[kHdrNb];
    v.Z = sw[kHdrZ];
    v.mb = sw[kHdrMb];
    v.layer_first = sw + sw[kHdrOffLayerFirst];
    v.rows = reinterpret_cast<const int4 *>(sw + sw[kHdrOffRows]);
    v.entries = reinterpret_cast<const int4 *>(sw + sw[kHdrOffEntries]);
    v.col_kind = sw + sw[kHdrOffColKind];
    int32_t *cc = sw + a.image_words;  // nb ints after the image
    if (threadIdx.x == 0) {
        int k = 0;
        for (int c = 0; c < v.nb; ++c) cc[c] = v.col_kind[c] == kColCore ? k++ : -1;
    }
    __syncthreads();
    v.col_core = cc;
    v.core_cols = 0;
    for (int c = 0; c < v.nb; ++c) v.core_cols += v.col_kind[c] == kColCore;
    return v;
}

__device__ __forceinline__ float softplusf(float z) {
    return fmaxf(z, 0.0f) + log1pf(__expf(-fabsf(z)));
}

__device__ __forceinline__ float sigmoidf(float z) {
    const float e = __expf(-fabsf(z));
    return z >= 0.0f ? 1.0f / (1.0f + e) : e / (1.0f + e);
}

// Min-sum parts of one check: smallest |q| (first index i1), second smallest
// (first index i2 != i1), and the product of signs.
template <int D>
__device__ __forceinline__ void two_minima(const float (&q)[D], float &m1, int &i1, float &m2,
                                           int &i2, unsigned &negs) {
    m1 = m2 = INFINITY;
    i1 = i2 = -1;
    negs = 0u;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const float v = fabsf(q[k]);
        negs ^= q[k] < 0.0f ? 1u : 0u;
        if (v < m1) {
            m2 = m1;
            i2 = i1;
            m1 = v;
            i1 = k;
        } else if (v < m2) {
            m2 = v;
            i2 = k;
        }
    }
}

struct FrameView {
    const float *ch;
    const uint8_t *syn;
    const uint8_t *x;
    float *post;
    float *msg;
};

// One check of a row: training forward.  Adds the loss contribution of the
// degree-1 variables to loss_part and records q for the backward pass.
template <int D>
__device__ __forceinline__ void ms_check_forward(const LearnedArgs &a, const LearnedView &v,
                                                 const FrameView &fv, const int4 *ent, int l,
                                                 int check_base, int i, int t, bool last,
                                                 float *qhist_t, float ws0, float ws1, float wo0,
                                                 float wo1, float &loss_part) {
    const int Z = v.Z;
    const size_t stride = (size_t)a.slot_stride;
    float q[D];
    int vv[D];
#pragma unroll
    for (int e = 0; e < D; ++e) {
        const int4 en = ent[e];
        int j = i + en.y;
        j = j >= Z ? j - Z : j;
        vv[e] = en.w * Z + j;  // frame variable (column en.w)
        const float *src = en.z < 0 ? fv.ch : fv.post;
        const float lv = src[vv[e]];
        const float ro = (t > 0 && en.z >= 0) ? fv.msg[(size_t)en.z * stride + i] : 0.0f;
        q[e] = lv - ro;
    }
    float m1, m2;
    int i1, i2;
    unsigned negs;
    two_minima<D>(q, m1, i1, m2, i2, negs);
    negs ^= fv.syn[check_base + i] & 1u;
#pragma unroll
    for (int e = 0; e < D; ++e) {
        const int4 en = ent[e];
        const bool deg1 = en.z < 0;
        float mn = e == i1 ? m2 : m1;
        if (D == 1) mn = kNoOther;
        const float a_e = (deg1 ? ws1 : ws0) * mn - (deg1 ? wo1 : wo0);
        const bool neg = ((negs ^ (q[e] < 0.0f ? 1u : 0u)) & 1u) != 0u;
        const float mag = fminf(fmaxf(a_e, 0.0f), kNoOther);
        const float r = neg ? -mag : mag;
        const float L = q[e] + r;
        if (!deg1) {
            fv.msg[(size_t)en.z * stride + i] = r;
            fv.post[vv[e]] = L;
            qhist_t[(size_t)en.z * stride + i] = q[e];
        } else {
            if (last) fv.post[vv[e]] = L;
            const float sx = fv.x[vv[e]] ? -1.0f : 1.0f;
            loss_part += softplusf(-sx * L);
        }
    }
    (void)l;
}

__device__ void ms_row_forward(const LearnedArgs &a, const LearnedView &v, const FrameView &fv,
                               int j, int t, bool last, float *qhist_t, float &loss_part) {
    const int4 row = v.rows[j];
    const int l = row.w;
    const size_t wi = ((size_t)t * v.mb + l) * 2;
    const float ws0 = a.w_scale[wi], ws1 = a.w_scale[wi + 1];
    const float wo0 = a.w_offset[wi], wo1 = a.w_offset[wi + 1];
    const int4 *ent = v.entries + row.x;
    for (int i = threadIdx.x; i < v.Z; i += blockDim.x) {
        switch (row.y) {
#define QCMET_MS_CASE(DD)                                                                       \
    case DD:                                                                                    \
        ms_check_forward<DD>(a, v, fv, ent, l, row.z, i, t, last, qhist_t, ws0, ws1, wo0, wo1,  \
                             loss_part);                                                        \
        break;
            QCMET_MS_CASE(1)
            QCMET_MS_CASE(2)
            QCMET_MS_CASE(3)
            QCMET_MS_CASE(4)
            QCMET_MS_CASE(5)
            QCMET_MS_CASE(6)
            QCMET_MS_CASE(7)
            QCMET_MS_CASE(8)
            QCMET_MS_CASE(9)
            QCMET_MS_CASE(10)
            QCMET_MS_CASE(11)
            QCMET_MS_CASE(12)
            QCMET_MS_CASE(13)
            QCMET_MS_CASE(14)
            QCMET_MS_CASE(15)
            QCMET_MS_CASE(16)
#undef QCMET_MS_CASE
            default: break;
        }
    }
}

// Training forward: loss per frame, and q and the core posteriors of every
// iteration for the backward pass.  (Decoding with learned weights runs in the
// fused decode kernel of decode.cu.)
__global__ void __launch_bounds__(kThreads, 1) ms_forward_kernel(const LearnedArgs a) {
    extern __shared__ int4 smem_i4[];
    int32_t *sw = reinterpret_cast<int32_t *>(smem_i4);
    const LearnedView v = load_view(a, sw);
    const int Z = v.Z;
    const size_t n = (size_t)a.n;
    const size_t stride = (size_t)a.slot_stride;
    const size_t core_vars = (size_t)v.core_cols * Z;
    for (int f = blockIdx.x; f < a.K; f += gridDim.x) {
        FrameView fv;
        fv.ch = a.ch + (size_t)f * n;
        fv.syn = a.syn + (size_t)f * a.m;
        fv.x = a.x + (size_t)f * n;
        fv.post = a.post + (size_t)f * n;
        fv.msg = a.msgs + (size_t)f * a.msg_slots * stride;
        for (int c = 0; c < v.nb; ++c) {
            if (v.col_kind[c] != kColCore) continue;
            for (int i = threadIdx.x; i < Z; i += blockDim.x)
                fv.post[(size_t)c * Z + i] = fv.ch[(size_t)c * Z + i];
        }
        __syncthreads();
        float loss_part = 0.0f;
        for (int t = 0; t < a.T; ++t) {
            const bool last = t == a.T - 1;
            float *qh = a.qhist + ((size_t)f * a.T + t) * a.msg_slots * stride;
            for (int layer = 0; layer < v.n_layers; ++layer) {
                for (int j = v.layer_first[layer]; j < v.layer_first[layer + 1]; ++j)
                    ms_row_forward(a, v, fv, j, t, last, qh, loss_part);
                __syncthreads();
            }
            {
                // loss of the core posteriors after iteration t, and their snapshot
                float *Lh = a.Lhist + ((size_t)f * a.T + t) * core_vars;
                for (int c = 0; c < v.nb; ++c) {
                    const int cc = v.col_core[c];
                    if (cc < 0) continue;
                    for (int i = threadIdx.x; i < Z; i += blockDim.x) {
                        const float L = fv.post[(size_t)c * Z + i];
                        Lh[(size_t)cc * Z + i] = L;
                        const float sx = fv.x[(size_t)c * Z + i] ? -1.0f : 1.0f;
                        loss_part += softplusf(-sx * L);
                    }
                }
                __syncthreads();
            }
        }
        {
            // loss = sum / (T n); unconnected columns contribute their constant channel term
            for (int c = 0; c < v.nb; ++c) {
                if (v.col_kind[c] != kColUnconnected) continue;
                for (int i = threadIdx.x; i < Z; i += blockDim.x) {
                    const float sx = fv.x[(size_t)c * Z + i] ? -1.0f : 1.0f;
                    loss_part += (float)a.T * softplusf(-sx * fv.ch[(size_t)c * Z + i]);
                }
            }
            for (int o = 16; o > 0; o >>= 1) loss_part += __shfl_xor_sync(0xffffffffu, loss_part, o);
            __shared__ float red[kThreads / 32];
            if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = loss_part;
            __syncthreads();
            if (threadIdx.x == 0) {
                float s = 0.0f;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
                a.loss[f] = a.T > 0 ? s / ((float)a.T * (float)n) : 0.0f;
            }
            __syncthreads();
        }
    }
}

// Backward of one check at iteration t.
template <int D>
__device__ __forceinline__ void ms_check_backward(const LearnedArgs &a, const LearnedView &v,
                                                  const FrameView &fv, const int4 *ent, int i,
                                                  int check_base, const float *qhist_t, float *gL,
                                                  float *gR, float ws0, float ws1, float wo0,
                                                  float wo1, float scale, float (&acc)[4]) {
    const int Z = v.Z;
    const size_t stride = (size_t)a.slot_stride;
    float q[D], gq[D], gr[D];
    int vv[D];
#pragma unroll
    for (int e = 0; e < D; ++e) {
        const int4 en = ent[e];
        int j = i + en.y;
        j = j >= Z ? j - Z : j;
        vv[e] = en.w * Z + j;  // frame variable (column en.w)
        if (en.z < 0) {
            q[e] = fv.ch[vv[e]];
            gq[e] = 0.0f;
            gr[e] = 0.0f;  // set below from the loss of this iteration
        } else {
            q[e] = qhist_t[(size_t)en.z * stride + i];
            const float g = gL[(size_t)v.col_core[en.w] * Z + j];
            gq[e] = g;
            gr[e] = g + gR[(size_t)en.z * stride + i];
        }
    }
    float m1, m2;
    int i1, i2;
    unsigned negs;
    two_minima<D>(q, m1, i1, m2, i2, negs);
    negs ^= fv.syn[check_base + i] & 1u;
#pragma unroll
    for (int e = 0; e < D; ++e) {
        const int4 en = ent[e];
        const bool deg1 = en.z < 0;
        float mn = e == i1 ? m2 : m1;
        const int arg = e == i1 ? i2 : i1;
        if (D == 1) mn = kNoOther;
        const float ws = deg1 ? ws1 : ws0;
        const float a_e = ws * mn - (deg1 ? wo1 : wo0);
        const bool neg = ((negs ^ (q[e] < 0.0f ? 1u : 0u)) & 1u) != 0u;
        const float sg = neg ? -1.0f : 1.0f;
        if (deg1) {
            // L_qn^(t) = channel + r: its loss term is the message's only use
            const float r = sg * fminf(fmaxf(a_e, 0.0f), kNoOther);
            const float sx = fv.x[vv[e]] ? -1.0f : 1.0f;
            gr[e] = scale * (-sx) * sigmoidf(-sx * (q[e] + r));
        }
        if (a_e <= 0.0f || a_e >= kNoOther) continue;  // the clip holds |r| constant
        acc[deg1 ? 1 : 0] += gr[e] * sg * mn;   // d/d w_scale
        acc[deg1 ? 3 : 2] += -gr[e] * sg;       // d/d w_offset
        if (arg >= 0) {
            float contrib = gr[e] * sg * ws * (q[arg] < 0.0f ? -1.0f : 1.0f);
#pragma unroll
            for (int k = 0; k < D; ++k)
                if (k == arg) gq[k] += contrib;
        }
    }
    // q = L_qn(before) - L_rmn(old): hand the adjoints back
#pragma unroll
    for (int e = 0; e < D; ++e) {
        const int4 en = ent[e];
        if (en.z < 0) continue;
        int j = i + en.y;
        j = j >= Z ? j - Z : j;
        gL[(size_t)v.col_core[en.w] * Z + j] = gq[e];
        gR[(size_t)en.z * stride + i] = -gq[e];
    }
}

__global__ void __launch_bounds__(kThreads, 1) ms_backward_kernel(const LearnedArgs a) {
    extern __shared__ int4 smem_i4[];
    int32_t *sw = reinterpret_cast<int32_t *>(smem_i4);
    const LearnedView v = load_view(a, sw);
    // per-CTA gradient accumulators of one iteration: [row][4] (scale0, scale1, offset0, offset1)
    float *gacc = reinterpret_cast<float *>(sw + a.image_words + ((v.nb + 3) & ~3));
    const int Z = v.Z;
    const size_t n = (size_t)a.n;
    const size_t stride = (size_t)a.slot_stride;
    const size_t core_vars = (size_t)v.core_cols * Z;
    const float scale = a.T > 0 ? 1.0f / ((float)a.T * (float)n) : 0.0f;
    for (int f = blockIdx.x; f < a.K; f += gridDim.x) {
        FrameView fv;
        fv.ch = a.ch + (size_t)f * n;
        fv.syn = a.syn + (size_t)f * a.m;
        fv.x = a.x + (size_t)f * n;
        fv.post = nullptr;
        fv.msg = nullptr;
        float *gL = a.gL + (size_t)f * core_vars;
        float *gR = a.gR + (size_t)f * a.msg_slots * stride;
        for (size_t k = threadIdx.x; k < core_vars; k += blockDim.x) gL[k] = 0.0f;
        for (size_t k = threadIdx.x; k < (size_t)a.msg_slots * stride; k += blockDim.x) gR[k] = 0.0f;
        __syncthreads();
        for (int t = a.T - 1; t >= 0; --t) {
            for (int k = threadIdx.x; k < v.mb * 4; k += blockDim.x) gacc[k] = 0.0f;
            // loss of the core posteriors after iteration t
            const float *Lh = a.Lhist + ((size_t)f * a.T + t) * core_vars;
            for (int c = 0; c < v.nb; ++c) {
                const int cc = v.col_core[c];
                if (cc < 0) continue;
                for (int i = threadIdx.x; i < Z; i += blockDim.x) {
                    const float sx = fv.x[(size_t)c * Z + i] ? -1.0f : 1.0f;
                    gL[(size_t)cc * Z + i] += scale * (-sx) * sigmoidf(-sx * Lh[(size_t)cc * Z + i]);
                }
            }
            __syncthreads();
            const float *qh = a.qhist + ((size_t)f * a.T + t) * a.msg_slots * stride;
            for (int layer = v.n_layers - 1; layer >= 0; --layer) {
                for (int j = v.layer_first[layer]; j < v.layer_first[layer + 1]; ++j) {
                    const int4 row = v.rows[j];
                    const int l = row.w;
                    const size_t wi = ((size_t)t * v.mb + l) * 2;
                    const float ws0 = a.w_scale[wi], ws1 = a.w_scale[wi + 1];
                    const float wo0 = a.w_offset[wi], wo1 = a.w_offset[wi + 1];
                    const int4 *ent = v.entries + row.x;
                    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                    for (int i = threadIdx.x; i < Z; i += blockDim.x) {
                        switch (row.y) {
#define QCMET_MSB_CASE(DD)                                                                      \
    case DD:                                                                                    \
        ms_check_backward<DD>(a, v, fv, ent, i, row.z, qh, gL, gR, ws0, ws1, wo0, wo1, scale, \
                              acc);                                                             \
        break;
                            QCMET_MSB_CASE(1)
                            QCMET_MSB_CASE(2)
                            QCMET_MSB_CASE(3)
                            QCMET_MSB_CASE(4)
                            QCMET_MSB_CASE(5)
                            QCMET_MSB_CASE(6)
                            QCMET_MSB_CASE(7)
                            QCMET_MSB_CASE(8)
                            QCMET_MSB_CASE(9)
                            QCMET_MSB_CASE(10)
                            QCMET_MSB_CASE(11)
                            QCMET_MSB_CASE(12)
                            QCMET_MSB_CASE(13)
                            QCMET_MSB_CASE(14)
                            QCMET_MSB_CASE(15)
                            QCMET_MSB_CASE(16)
#undef QCMET_MSB_CASE
                            default: break;
                        }
                    }
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        float s = acc[k];
                        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                        if ((threadIdx.x & 31) == 0 && s != 0.0f) atomicAdd(&gacc[l * 4 + k], s);
                    }
                }
                __syncthreads();
            }
            // flush this iteration's gradients: layout [t][l][type] for scale and offset
            for (int k = threadIdx.x; k < v.mb * 4; k += blockDim.x) {
                const int l = k >> 2, slot = k & 3;
                const float val = gacc[k];
                if (val == 0.0f) continue;
                const size_t wi = ((size_t)t * v.mb + l) * 2 + (slot & 1);
                atomicAdd(slot < 2 ? &a.g_scale[wi] : &a.g_offset[wi], val);
            }
            __syncthreads();
        }
    }
}

int sm_count() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return sms;
}

template <typename Kern>
int launch_learned(Kern kern, const LearnedArgs &a, size_t smem, void *stream, std::string &err) {
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) {
            err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e);
            return QCMET_ERR_UNSUPPORTED;
        }
    }
    const int sms = sm_count();
    if (sms <= 0) {
        err = "no CUDA device";
        return QCMET_ERR_CUDA;
    }
    const int grid = a.K < sms ? a.K : sms;
    kern<<<grid, kThreads, smem, static_cast<cudaStream_t>(stream)>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        err = std::string("learned min-sum launch: ") + cudaGetErrorString(e);
        return QCMET_ERR_CUDA;
    }
    return QCMET_OK;
}

}  // namespace

int launch_learned_forward(const LearnedArgs &a, void *stream, std::string &err) {
    const size_t smem = ((size_t)a.image_words + ((size_t)a.nb + 3) / 4 * 4) * sizeof(int32_t);
    return launch_learned(ms_forward_kernel, a, smem, stream, err);
}

int launch_learned_backward(const LearnedArgs &a, void *stream, std::string &err) {
    const size_t smem = ((size_t)a.image_words + ((size_t)a.nb + 3) / 4 * 4 + (size_t)a.mb * 4) *
                        sizeof(int32_t);
    return launch_learned(ms_backward_kernel, a, smem, stream, err);
}

}  // namespace qcmet
