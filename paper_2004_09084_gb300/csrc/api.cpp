// C ABI of the decoder library: argument checks, per-handle device state and
// the calls declared in include/qcmet.h.  The decode itself is one launch of
// the fused kernel in decode.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "l2_persist.h"
#include "qcmet_internal.h"
#include "trace.h"

namespace {

thread_local std::string g_last_error;

int fail(int status, const std::string &msg) {
    g_last_error = msg;
    return status;
}

int cuda_fail(const char *what, cudaError_t e) {
    return fail(e == cudaErrorMemoryAllocation ? QCMET_ERR_OOM : QCMET_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

size_t round256(size_t x) { return (x + 255) & ~size_t(255); }

// QCMET_KERNEL_AUTO: the grouped kernel for fixed-iteration decodes (measured
// at 128 frames of the rate-0.1 Z = 12500 code: 7 % faster than the per-frame
// kernel with FP32 messages, 15-20 % with FP16).  It spreads even one partial
// group of frames over a cluster of up to 16 SMs, where the per-frame kernel
// gives each frame one SM, so it serves sum-product decodes of any K; the
// learned min-sum decode keeps the per-frame kernel below four frames.  Codes
// whose padded rows overflow the grouped kernel's 32-bit offsets go to the
// per-frame kernel.
bool use_group_by_default(const qcmet::Code &c, int32_t K, bool minsum) {
    if ((int64_t)c.nb * qcmet::group_zp(c.Z) > INT32_MAX) return false;
    return minsum ? K >= 4 : K >= 1;
}

size_t msg_bytes(int32_t fmt) { return fmt == QCMET_MSG_FP32 ? 4 : 2; }

// Upload the schedule image once, on the current device.
int ensure_device(qcmet::Code &c) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail("cudaGetDevice", e);
    if (c.d_image) {
        if (dev != c.device)
            return fail(QCMET_ERR_UNSUPPORTED, "code handle was first used on device " +
                                                   std::to_string(c.device) +
                                                   "; create one handle per device");
        return QCMET_OK;
    }
    const size_t bytes = c.image.words.size() * sizeof(int32_t);
    void *p = nullptr;
    e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) return cuda_fail("cudaMalloc(schedule)", e);
    e = cudaMemcpy(p, c.image.words.data(), bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(p);
        return cuda_fail("cudaMemcpy(schedule)", e);
    }
    c.d_image = static_cast<int32_t *>(p);
    c.image_bytes = bytes;
    c.device = dev;
    return QCMET_OK;
}

// Grow a device buffer to at least `need` bytes (contents are not kept).
int grow(void **buf, size_t *have, size_t need, const char *what) {
    if (*have >= need) return QCMET_OK;
    if (*buf) {
        cudaError_t e = cudaFree(*buf);
        if (e != cudaSuccess) return cuda_fail("cudaFree", e);
        *buf = nullptr;
        *have = 0;
    }
    cudaError_t e = cudaMalloc(buf, need);
    if (e != cudaSuccess) {
        *buf = nullptr;
        return cuda_fail(what, e);
    }
    *have = need;
    return QCMET_OK;
}

struct KernelChoice {
    int32_t kernel = QCMET_KERNEL_AUTO;
    int32_t cluster = 0;
    int32_t per_cluster = 0;
};

int check_options(const qcmet_decode_options *o, int32_t *fmt, int32_t *threads,
                  bool *l2_persist = nullptr, KernelChoice *kc = nullptr) {
    *fmt = QCMET_MSG_FP32;
    *threads = 0;
    if (l2_persist) *l2_persist = false;
    if (kc) *kc = KernelChoice();
    if (!o) return QCMET_OK;
    if (o->kernel != QCMET_KERNEL_AUTO && o->kernel != QCMET_KERNEL_FRAME &&
        o->kernel != QCMET_KERNEL_GROUP)
        return fail(QCMET_ERR_INVALID_ARG, "unknown kernel");
    if (o->cluster_size < 0 || o->cluster_size > 16)
        return fail(QCMET_ERR_INVALID_ARG, "cluster_size must be 0 (automatic) or 1 .. 16");
    if (o->groups_per_cluster < 0 || o->groups_per_cluster > 2)
        return fail(QCMET_ERR_INVALID_ARG, "groups_per_cluster must be 0 (automatic), 1 or 2");
    if (o->msg_format != QCMET_MSG_FP32 && o->msg_format != QCMET_MSG_FP16 &&
        o->msg_format != QCMET_MSG_BF16)
        return fail(QCMET_ERR_INVALID_ARG, "unknown msg_format");
    if (o->threads_per_block != 0 &&
        (o->threads_per_block < 32 || o->threads_per_block > 1024 || o->threads_per_block % 32))
        return fail(QCMET_ERR_INVALID_ARG, "threads_per_block must be 0 or a multiple of 32 in [32, 1024]");
    if (o->l2_persist != 0 && o->l2_persist != 1)
        return fail(QCMET_ERR_INVALID_ARG, "l2_persist must be 0 or 1");
    for (int32_t r : o->reserved)
        if (r != 0) return fail(QCMET_ERR_INVALID_ARG, "reserved option fields must be 0");
    *fmt = o->msg_format;
    *threads = o->threads_per_block;
    if (l2_persist) *l2_persist = o->l2_persist == 1;
    if (kc) {
        kc->kernel = o->kernel;
        kc->cluster = o->cluster_size;
        kc->per_cluster = o->groups_per_cluster;
    }
    return QCMET_OK;
}

// Size an L2 persisting window over `bytes` of decoder state on the current
// device: the persisting part of L2 is raised (for this context) to cover it
// where the device allows, and the hit ratio is the fraction of the window
// that fits in that part.  No window (window = 0) on a device without
// persisting L2, or when one window cannot cover the whole state: measured on
// GB300, a window over a quarter of 512 MB of core posteriors doubled the
// decode time, while states up to the 128 MiB window gained.  *raised tells
// whether the limit was raised, and *prior_limit what it was before.
int l2_window(size_t bytes, size_t *window, float *hit, bool *raised, size_t *prior_limit) {
    *window = 0;
    *hit = 0.0f;
    *raised = false;
    *prior_limit = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail("cudaGetDevice", e);
    int max_persist = 0, max_window = 0;
    e = cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, dev);
    if (e != cudaSuccess) return cuda_fail("cudaDeviceGetAttribute(persisting L2)", e);
    e = cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, dev);
    if (e != cudaSuccess) return cuda_fail("cudaDeviceGetAttribute(access policy window)", e);
    if (max_persist <= 0 || max_window <= 0 || bytes == 0 || bytes > (size_t)max_window)
        return QCMET_OK;
    const size_t w = bytes;
    size_t limit = 0;
    e = cudaDeviceGetLimit(&limit, cudaLimitPersistingL2CacheSize);
    if (e != cudaSuccess) return cuda_fail("cudaDeviceGetLimit(persisting L2)", e);
    const size_t want = std::min(w, (size_t)max_persist);
    if (limit < want) {
        e = cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want);
        if (e != cudaSuccess) return cuda_fail("cudaDeviceSetLimit(persisting L2)", e);
        *raised = true;
        *prior_limit = limit;
        e = cudaDeviceGetLimit(&limit, cudaLimitPersistingL2CacheSize);
        if (e != cudaSuccess) return cuda_fail("cudaDeviceGetLimit(persisting L2)", e);
    }
    *window = w;
    *hit = limit >= w ? 1.0f : (float)((double)limit / (double)w);
    return QCMET_OK;
}

// The grouped kernel (decode_group.cu) for K frames: interleaved scratch of
// ceil(K/4) groups, one or two groups per cluster.
int decode_group(qcmet::Code &c, const float *llr_ch, const uint8_t *syndrome, int32_t K,
                 int32_t T, uint8_t *hard, float *llr_post, uint8_t *ok, int32_t fmt,
                 const KernelChoice &kc, bool l2p, void *stream, const float *w_scale = nullptr,
                 const float *w_offset = nullptr) {
    const int32_t stage_ops = qcmet::group_stage_ops(c);
    qcmet::GroupLaunch L;
    std::string err;
    int st = qcmet::choose_group_launch(fmt, K, c.Z, (int32_t)c.image.words.size(), stage_ops,
                                        kc.cluster, &L, err, w_scale != nullptr, kc.per_cluster);
    if (st) return fail(st, err);
    const size_t G = (size_t)L.groups;
    const size_t n = (size_t)c.nb * c.Z, m = (size_t)c.mb * c.Z;
    if ((int64_t)c.nb * qcmet::group_zp(c.Z) > INT32_MAX)
        return fail(QCMET_ERR_INVALID_ARG, "code too large for the grouped kernel's 32-bit offsets");
    const qcmet::GroupScratch gs = qcmet::group_scratch_bytes(c, fmt);
    const size_t b_ch = G * gs.ch, b_syn = G * gs.syn, b_core = G * gs.core, b_msg = G * gs.msg;
    st = grow(&c.d_group, &c.group_bytes, b_ch + b_syn + b_core + b_msg + 256,
              "cudaMalloc(grouped scratch)");
    if (st) return st;
    char *p = static_cast<char *>(c.d_group);
    // the grouped kernel sets L2 eviction priorities per access; it takes no
    // persisting window (l2_persist is accepted and ignored)
    (void)l2p;
    qcmet::GroupArgs a;
    a.ch = llr_ch;
    a.syn = syndrome;
    a.post = llr_post;
    a.hard = hard;
    a.ok = ok;
    a.ch4 = p;
    a.syn4 = reinterpret_cast<uint32_t *>(p + b_ch);
    a.core4 = p + b_ch + b_syn;
    a.msgs4 = p + b_ch + b_syn + b_core;
    a.g_bytes = gs;
    a.image = c.d_image;
    a.image_words = (int32_t)c.image.words.size();
    a.K = K;
    a.T = T;
    a.n = (int32_t)n;
    a.m = (int32_t)m;
    a.core_cols = c.core_cols;
    a.msg_slots = c.msg_slots;
    a.stage_ops = stage_ops;
    a.w_scale = w_scale;
    a.w_offset = w_offset;
    qcmet::TraceRange range("qcmet decode: grouped kernel, %d frames, %d layer groups x %d iterations, "
                            "%d groups, %d per cluster of %d%s", K, (int)c.layer_first.size() - 1, T,
                            L.groups, L.per_cluster, L.cluster, w_scale ? ", min-sum rule" : "");
    st = qcmet::launch_decode_group(a, fmt, L, stream, err);
    if (st) return fail(st, err);
    return QCMET_OK;
}

int decode_device(qcmet::Code &c, const float *llr_ch, const uint8_t *syndrome, int32_t K,
                  int32_t T, uint8_t *hard, float *llr_post, uint8_t *ok,
                  const qcmet_decode_options *opts, void *stream, int32_t check_every = 0,
                  int32_t *iters_used = nullptr, const float *w_scale = nullptr,
                  const float *w_offset = nullptr) {
    int32_t fmt, threads;
    bool l2p = false;
    KernelChoice kc;
    int st = check_options(opts, &fmt, &threads, &l2p, &kc);
    if (st) return st;
    if (K < 0) return fail(QCMET_ERR_INVALID_ARG, "K must be >= 0");
    if (T < 0) return fail(QCMET_ERR_INVALID_ARG, "iterations must be >= 0");
    if (K == 0) return QCMET_OK;
    if (!llr_ch || !syndrome || !hard || !ok)
        return fail(QCMET_ERR_INVALID_ARG, "llr_ch, syndrome, hard and ok must not be NULL");
    if (!aligned16(llr_ch) || !aligned16(syndrome) || !aligned16(hard) || !aligned16(ok) ||
        (llr_post && !aligned16(llr_post)))
        return fail(QCMET_ERR_ALIGNMENT, "device pointers must be 16-byte aligned");
    st = ensure_device(c);
    if (st) return st;
    const bool group_ok = check_every == 0;
    if (kc.kernel == QCMET_KERNEL_GROUP && !group_ok)
        return fail(QCMET_ERR_UNSUPPORTED,
                    "the grouped kernel serves fixed-iteration decodes only");
    if (kc.kernel == QCMET_KERNEL_GROUP ||
        (kc.kernel == QCMET_KERNEL_AUTO && group_ok && use_group_by_default(c, K, w_scale != nullptr))) {
        qcmet::release_persisting_l2();
        return decode_group(c, llr_ch, syndrome, K, T, hard, llr_post, ok, fmt, kc, l2p, stream,
                            w_scale, w_offset);
    }

    const size_t n = (size_t)c.nb * c.Z;
    const size_t stride = qcmet::slot_stride(c.Z);
    const size_t need_msgs = (size_t)K * (size_t)c.msg_slots * stride * msg_bytes(fmt);
    st = grow(&c.d_msgs, &c.msgs_bytes, need_msgs ? need_msgs : 16, "cudaMalloc(messages)");
    if (st) return st;
    float *post = llr_post;
    if (!post) {
        void *p = c.d_post;
        st = grow(&p, &c.post_bytes, (size_t)K * n * sizeof(float), "cudaMalloc(posteriors)");
        c.d_post = static_cast<float *>(p);
        if (st) return st;
        post = c.d_post;
    }
    const size_t need_core = (size_t)K * (size_t)c.core_cols * (size_t)c.Z * sizeof(float);
    {
        void *p = c.d_core;
        st = grow(&p, &c.core_bytes, need_core ? need_core : 16, "cudaMalloc(core posteriors)");
        c.d_core = static_cast<float *>(p);
        if (st) return st;
    }
    size_t window = 0;
    float hit = 0.0f;
    if (l2p) {
        bool raised = false;
        size_t prior = 0;
        st = l2_window(need_core, &window, &hit, &raised, &prior);
        if (raised || window > 0) qcmet::note_persisting_l2(raised, prior);
        if (st) return st;
    }
    if (window == 0) qcmet::release_persisting_l2();

    qcmet::DecodeArgs a;
    a.ch = llr_ch;
    a.syn = syndrome;
    a.post = post;
    a.post_core = c.d_core;
    a.msgs = c.d_msgs;
    a.hard = hard;
    a.ok = ok;
    a.image = c.d_image;
    a.image_words = (int32_t)c.image.words.size();
    a.K = K;
    a.T = T;
    a.Z = c.Z;
    a.n = (int32_t)n;
    a.m = c.mb * c.Z;
    a.nb = c.nb;
    a.msg_slots = c.msg_slots;
    a.core_cols = c.core_cols;
    a.slot_stride = (int64_t)stride;
    a.check_every = check_every;
    a.iters_used = iters_used;
    qcmet::CheckRule rule;
    rule.w_scale = w_scale;
    rule.w_offset = w_offset;
    std::string err;
    qcmet::TraceRange range("qcmet decode: frame kernel, %d frames, %d layer groups x %d iterations%s",
                            K, (int)c.layer_first.size() - 1, T,
                            w_scale ? ", min-sum rule" : (check_every ? ", early stop" : ""));
    st = qcmet::launch_decode(a, fmt, threads, stream, err, window, hit, rule);
    if (st) return fail(st, err);
    return QCMET_OK;
}

}  // namespace

namespace qcmet {
namespace {
// Per device: whether a windowed launch was issued since the last release,
// and the persisting-L2 size to put back where the library raised it.
struct L2State {
    bool windowed = false;
    bool raised = false;
    size_t prior = 0;
};
std::mutex g_l2_mutex;
L2State g_l2[64];

int current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        (void)cudaGetLastError();
        return -1;
    }
    return dev;
}
}  // namespace

void note_persisting_l2(bool raised, size_t prior_limit) {
    const int dev = current_device();
    if (dev < 0) return;
    std::lock_guard<std::mutex> lock(g_l2_mutex);
    L2State &s = g_l2[dev];
    s.windowed = true;
    if (raised && !s.raised) {
        s.raised = true;
        s.prior = prior_limit;
    }
}

void release_persisting_l2() {
    const int dev = current_device();
    if (dev < 0) return;
    std::lock_guard<std::mutex> lock(g_l2_mutex);
    L2State &s = g_l2[dev];
    if (!s.windowed) return;
    s.windowed = false;
    if (cudaCtxResetPersistingL2Cache() != cudaSuccess) (void)cudaGetLastError();
    if (s.raised) {
        s.raised = false;
        if (cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, s.prior) != cudaSuccess)
            (void)cudaGetLastError();
    }
}

int ensure_device_image(Code &c) { return ensure_device(c); }
int set_error(int status, const std::string &msg) { return fail(status, msg); }
}  // namespace qcmet

extern "C" {

int qcmet_code_create_ex(const int8_t *base, const int32_t *shifts, int32_t mb, int32_t nb,
                         int32_t Z, int32_t merge_mode, qcmet_code **out) {
    if (!out) return fail(QCMET_ERR_INVALID_ARG, "out must not be NULL");
    *out = nullptr;
    qcmet_code *h = new (std::nothrow) qcmet_code;
    if (!h) return fail(QCMET_ERR_OOM, "host allocation failed");
    std::string err;
    int st;
    try {
        st = qcmet::build_code(base, shifts, mb, nb, Z, merge_mode, h->c, err);
    } catch (const std::bad_alloc &) {
        st = QCMET_ERR_OOM;
        err = "host allocation failed";
    }
    if (st) {
        delete h;
        return fail(st, err);
    }
    *out = h;
    return QCMET_OK;
}

int qcmet_code_create(const int8_t *base, const int32_t *shifts, int32_t mb, int32_t nb,
                      int32_t Z, qcmet_code **out) {
    return qcmet_code_create_ex(base, shifts, mb, nb, Z, QCMET_MERGE_EXACT, out);
}

void qcmet_code_destroy(qcmet_code *code) {
    if (!code) return;
    qcmet::Code &c = code->c;
    if (c.d_image) cudaFree(c.d_image);
    if (c.d_msgs) cudaFree(c.d_msgs);
    if (c.d_post) cudaFree(c.d_post);
    if (c.d_core) cudaFree(c.d_core);
    if (c.d_io) cudaFree(c.d_io);
    if (c.d_group) cudaFree(c.d_group);
    if (c.d_learned) cudaFree(c.d_learned);
    delete code;
}

int qcmet_code_get_info(const qcmet_code *code, qcmet_code_info *info) {
    if (!code || !info) return fail(QCMET_ERR_INVALID_ARG, "code and info must not be NULL");
    const qcmet::Code &c = code->c;
    info->mb = c.mb;
    info->nb = c.nb;
    info->Z = c.Z;
    info->n = c.nb * c.Z;
    info->m = c.mb * c.Z;
    info->edges = (int64_t)c.circulants * c.Z;
    info->circulants = c.circulants;
    info->msg_slots = c.msg_slots;
    info->degree1_columns = c.degree1_columns;
    info->layers = (int32_t)c.layer_first.size() - 1;
    info->max_row_degree = c.max_row_degree;
    info->merge_mode = c.merge_mode;
    return QCMET_OK;
}

int qcmet_code_get_schedule(const qcmet_code *code, int32_t *rows, int32_t *layer_first) {
    if (!code) return fail(QCMET_ERR_INVALID_ARG, "code must not be NULL");
    const qcmet::Code &c = code->c;
    if (rows) {
        for (int32_t i = 0; i < c.mb; ++i)
            rows[i] = i < (int32_t)c.sched_rows.size() ? c.sched_rows[i] : -1;
    }
    if (layer_first)
        std::memcpy(layer_first, c.layer_first.data(), c.layer_first.size() * sizeof(int32_t));
    return QCMET_OK;
}

int qcmet_decode_ex(const qcmet_code *code, const float *llr_ch, const uint8_t *syndrome,
                    int32_t K, int32_t iterations, uint8_t *hard, float *llr_post, uint8_t *ok,
                    const qcmet_decode_options *opts, void *stream) {
    if (!code) return fail(QCMET_ERR_INVALID_ARG, "code must not be NULL");
    return decode_device(const_cast<qcmet_code *>(code)->c, llr_ch, syndrome, K, iterations, hard,
                         llr_post, ok, opts, stream);
}

int qcmet_decode(const qcmet_code *code, const float *llr_ch, const uint8_t *syndrome, int32_t K,
                 int32_t iterations, uint8_t *hard, float *llr_post, uint8_t *ok, void *stream) {
    return qcmet_decode_ex(code, llr_ch, syndrome, K, iterations, hard, llr_post, ok, nullptr,
                           stream);
}

int qcmet_decode_early_stop(const qcmet_code *code, const float *llr_ch, const uint8_t *syndrome,
                            int32_t K, int32_t max_iterations, int32_t check_every, uint8_t *hard,
                            float *llr_post, uint8_t *ok, int32_t *iterations_used,
                            const qcmet_decode_options *opts, void *stream) {
    if (!code) return fail(QCMET_ERR_INVALID_ARG, "code must not be NULL");
    if (check_every < 1) return fail(QCMET_ERR_INVALID_ARG, "check_every must be >= 1");
    if (K > 0 && !iterations_used)
        return fail(QCMET_ERR_INVALID_ARG, "iterations_used must not be NULL");
    if (iterations_used && !aligned16(iterations_used))
        return fail(QCMET_ERR_ALIGNMENT, "device pointers must be 16-byte aligned");
    return decode_device(const_cast<qcmet_code *>(code)->c, llr_ch, syndrome, K, max_iterations,
                         hard, llr_post, ok, opts, stream, check_every, iterations_used);
}

int qcmet_decode_host(const qcmet_code *code, const float *llr_ch, const uint8_t *syndrome,
                      int32_t K, int32_t iterations, uint8_t *hard, float *llr_post, uint8_t *ok,
                      const qcmet_decode_options *opts, void *stream) {
    if (!code) return fail(QCMET_ERR_INVALID_ARG, "code must not be NULL");
    if (K < 0) return fail(QCMET_ERR_INVALID_ARG, "K must be >= 0");
    if (iterations < 0) return fail(QCMET_ERR_INVALID_ARG, "iterations must be >= 0");
    if (K == 0) return QCMET_OK;
    if (!llr_ch || !syndrome || !hard || !ok)
        return fail(QCMET_ERR_INVALID_ARG, "llr_ch, syndrome, hard and ok must not be NULL");
    qcmet::Code &c = const_cast<qcmet_code *>(code)->c;
    int st = ensure_device(c);
    if (st) return st;
    const size_t n = (size_t)c.nb * c.Z, m = (size_t)c.mb * c.Z;
    const size_t b_ch = round256((size_t)K * n * sizeof(float));
    const size_t b_syn = round256((size_t)K * m);
    const size_t b_hard = round256((size_t)K * n);
    const size_t b_post = llr_post ? round256((size_t)K * n * sizeof(float)) : 0;
    const size_t b_ok = round256((size_t)K);
    st = grow(&c.d_io, &c.io_bytes, b_ch + b_syn + b_hard + b_post + b_ok, "cudaMalloc(staging)");
    if (st) return st;
    char *base = static_cast<char *>(c.d_io);
    float *d_ch = reinterpret_cast<float *>(base);
    uint8_t *d_syn = reinterpret_cast<uint8_t *>(base + b_ch);
    uint8_t *d_hard = reinterpret_cast<uint8_t *>(base + b_ch + b_syn);
    float *d_post = llr_post ? reinterpret_cast<float *>(base + b_ch + b_syn + b_hard) : nullptr;
    uint8_t *d_ok = reinterpret_cast<uint8_t *>(base + b_ch + b_syn + b_hard + b_post);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    qcmet::TraceRange range("qcmet decode_host: %d frames", K);
    cudaError_t e = cudaMemcpyAsync(d_ch, llr_ch, (size_t)K * n * sizeof(float),
                                    cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail("cudaMemcpyAsync(llr_ch)", e);
    e = cudaMemcpyAsync(d_syn, syndrome, (size_t)K * m, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail("cudaMemcpyAsync(syndrome)", e);
    st = decode_device(c, d_ch, d_syn, K, iterations, d_hard, d_post, d_ok, opts, stream);
    if (st) return st;
    e = cudaMemcpyAsync(hard, d_hard, (size_t)K * n, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail("cudaMemcpyAsync(hard)", e);
    if (llr_post) {
        e = cudaMemcpyAsync(llr_post, d_post, (size_t)K * n * sizeof(float),
                            cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail("cudaMemcpyAsync(llr_post)", e);
    }
    e = cudaMemcpyAsync(ok, d_ok, (size_t)K, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail("cudaMemcpyAsync(ok)", e);
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail("cudaStreamSynchronize", e);
    return QCMET_OK;
}

int qcmet_decode_noalloc(const qcmet_code *code, const float *llr_ch, const uint8_t *syndrome,
                         int32_t K, int32_t iterations, uint8_t *hard, float *llr_post,
                         uint8_t *ok, void *stream) {
    if (!code) return fail(QCMET_ERR_INVALID_ARG, "code must not be NULL");
    if (K < 0) return fail(QCMET_ERR_INVALID_ARG, "K must be >= 0");
    if (iterations < 0) return fail(QCMET_ERR_INVALID_ARG, "iterations must be >= 0");
    if (K == 0) return QCMET_OK;
    if (!llr_ch || !syndrome || !hard || !llr_post || !ok)
        return fail(QCMET_ERR_INVALID_ARG,
                    "llr_ch, syndrome, hard, llr_post and ok must not be NULL "
                    "(qcmet_decode_noalloc keeps the posteriors in llr_post)");
    if (!aligned16(llr_ch) || !aligned16(syndrome) || !aligned16(hard) || !aligned16(ok) ||
        !aligned16(llr_post))
        return fail(QCMET_ERR_ALIGNMENT, "device pointers must be 16-byte aligned");
    const qcmet::Code &c = code->c;
    qcmet::DecodeArgs a;
    a.ch = llr_ch;
    a.syn = syndrome;
    a.post = llr_post;
    a.post_core = nullptr;  // set by the launcher: inside the static scratch
    a.msgs = nullptr;       // set by the launcher: inside the static scratch
    a.hard = hard;
    a.ok = ok;
    a.image = nullptr;  // set by the launcher: a copy inside the static scratch
    a.image_words = (int32_t)c.image.words.size();
    a.K = K;
    a.T = iterations;
    a.Z = c.Z;
    a.n = c.nb * c.Z;
    a.m = c.mb * c.Z;
    a.nb = c.nb;
    a.msg_slots = c.msg_slots;
    a.core_cols = c.core_cols;
    a.slot_stride = (int64_t)qcmet::slot_stride(c.Z);
    a.check_every = 0;
    a.iters_used = nullptr;
    std::string err;
    int st = qcmet::launch_decode_noalloc(a, c.image.words.data(),
                                          c.image.words.size() * sizeof(int32_t), stream, err);
    if (st) return fail(st, err);
    return QCMET_OK;
}

// ---- learned offset/scaled min-sum ----------------------------------------

namespace {

size_t r256(size_t x) { return (x + 255) & ~size_t(255); }

// base columns of degree > 1 (those whose posteriors are decoder state)
size_t core_cols_of(const qcmet::Code &c) {
    size_t k = 0;
    for (int32_t d : c.col_degree) k += d > 1;
    return k;
}

// Fill the code-dependent fields and carve the learned scratch for K frames and
// T iterations (training adds q and posterior histories and the adjoints).
int learned_setup(qcmet::Code &c, int32_t K, int32_t T, bool train, bool need_post,
                  qcmet::LearnedArgs &a) {
    int st = ensure_device(c);
    if (st) return st;
    const size_t n = (size_t)c.nb * c.Z, stride = qcmet::slot_stride(c.Z);
    const size_t msgs = r256((size_t)K * c.msg_slots * stride * sizeof(float));
    const size_t post = need_post ? r256((size_t)K * n * sizeof(float)) : 0;
    const size_t core_vars = core_cols_of(c) * (size_t)c.Z;
    const size_t qhist = train ? r256((size_t)K * T * c.msg_slots * stride * sizeof(float)) : 0;
    const size_t lhist = train ? r256((size_t)K * T * core_vars * sizeof(float)) : 0;
    const size_t gl = train ? r256((size_t)K * core_vars * sizeof(float)) : 0;
    const size_t gr = train ? r256((size_t)K * c.msg_slots * stride * sizeof(float)) : 0;
    const size_t total = msgs + post + qhist + lhist + gl + gr + 256;
    st = grow(&c.d_learned, &c.learned_bytes, total, "cudaMalloc(learned scratch)");
    if (st) return st;
    char *p = static_cast<char *>(c.d_learned);
    a = qcmet::LearnedArgs{};
    a.msgs = reinterpret_cast<float *>(p);
    p += msgs;
    a.post = need_post ? reinterpret_cast<float *>(p) : nullptr;
    p += post;
    a.qhist = train ? reinterpret_cast<float *>(p) : nullptr;
    p += qhist;
    a.Lhist = train ? reinterpret_cast<float *>(p) : nullptr;
    p += lhist;
    a.gL = train ? reinterpret_cast<float *>(p) : nullptr;
    p += gl;
    a.gR = train ? reinterpret_cast<float *>(p) : nullptr;
    a.image = c.d_image;
    a.image_words = (int32_t)c.image.words.size();
    a.K = K;
    a.T = T;
    a.Z = c.Z;
    a.n = (int32_t)n;
    a.m = c.mb * c.Z;
    a.nb = c.nb;
    a.mb = c.mb;
    a.msg_slots = c.msg_slots;
    a.slot_stride = (int64_t)stride;
    return QCMET_OK;
}

}  // namespace

int qcmet_minsum_decode(const qcmet_code *code, const float *llr_ch, const uint8_t *syndrome,
                        int32_t K, int32_t iterations, const float *w_scale, const float *w_offset,
                        uint8_t *hard, float *llr_post, uint8_t *ok, void *stream) {
    if (!code) return fail(QCMET_ERR_INVALID_ARG, "code must not be NULL");
    if (K < 0 || iterations < 0) return fail(QCMET_ERR_INVALID_ARG, "K and iterations must be >= 0");
    if (K == 0) return QCMET_OK;
    if (!llr_ch || !syndrome || !hard || !ok || (iterations > 0 && (!w_scale || !w_offset)))
        return fail(QCMET_ERR_INVALID_ARG, "llr_ch, syndrome, w_scale, w_offset, hard and ok must not be NULL");
    if (!aligned16(llr_ch) || !aligned16(syndrome) || !aligned16(hard) || !aligned16(ok) ||
        (llr_post && !aligned16(llr_post)) || (w_scale && !aligned16(w_scale)) ||
        (w_offset && !aligned16(w_offset)))
        return fail(QCMET_ERR_ALIGNMENT, "device pointers must be 16-byte aligned");
    qcmet::Code &c = const_cast<qcmet_code *>(code)->c;
    // the fused decode kernel with the min-sum rule (FP32 messages)
    static const float kNoWeights[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (iterations == 0) w_scale = w_offset = kNoWeights;  // never read; selects the rule
    return decode_device(c, llr_ch, syndrome, K, iterations, hard, llr_post, ok, nullptr, stream,
                         0, nullptr, w_scale, w_offset);
}

int qcmet_minsum_forward(const qcmet_code *code, const float *llr_ch, const uint8_t *syndrome,
                         const uint8_t *bits, int32_t K, int32_t iterations, const float *w_scale,
                         const float *w_offset, float *loss, void *stream) {
    if (!code) return fail(QCMET_ERR_INVALID_ARG, "code must not be NULL");
    if (K < 0 || iterations < 0) return fail(QCMET_ERR_INVALID_ARG, "K and iterations must be >= 0");
    qcmet::Code &c = const_cast<qcmet_code *>(code)->c;
    c.learned_ready = false;
    if (K == 0) return QCMET_OK;
    if (!llr_ch || !syndrome || !bits || !loss || (iterations > 0 && (!w_scale || !w_offset)))
        return fail(QCMET_ERR_INVALID_ARG, "llr_ch, syndrome, bits, w_scale, w_offset and loss must not be NULL");
    if (!aligned16(llr_ch) || !aligned16(syndrome) || !aligned16(bits) || !aligned16(loss) ||
        (w_scale && !aligned16(w_scale)) || (w_offset && !aligned16(w_offset)))
        return fail(QCMET_ERR_ALIGNMENT, "device pointers must be 16-byte aligned");
    qcmet::LearnedArgs a;
    int st = learned_setup(c, K, iterations, true, true, a);
    if (st) return st;
    a.ch = llr_ch;
    a.syn = syndrome;
    a.x = bits;
    a.w_scale = w_scale;
    a.w_offset = w_offset;
    a.loss = loss;
    std::string err;
    qcmet::TraceRange range("qcmet min-sum forward: %d frames x %d iterations", K, iterations);
    st = qcmet::launch_learned_forward(a, stream, err);
    if (st) return fail(st, err);
    c.learned_last = a;
    c.learned_ready = true;
    return QCMET_OK;
}

int qcmet_minsum_backward(const qcmet_code *code, float *g_scale, float *g_offset, void *stream) {
    if (!code) return fail(QCMET_ERR_INVALID_ARG, "code must not be NULL");
    qcmet::Code &c = const_cast<qcmet_code *>(code)->c;
    if (!c.learned_ready)
        return fail(QCMET_ERR_INVALID_ARG, "qcmet_minsum_backward needs a preceding qcmet_minsum_forward on this handle");
    if (!g_scale || !g_offset) return fail(QCMET_ERR_INVALID_ARG, "g_scale and g_offset must not be NULL");
    if (!aligned16(g_scale) || !aligned16(g_offset))
        return fail(QCMET_ERR_ALIGNMENT, "device pointers must be 16-byte aligned");
    qcmet::LearnedArgs a = c.learned_last;
    const size_t nw = (size_t)a.T * c.mb * 2 * sizeof(float);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(g_scale, 0, nw, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(g_offset, 0, nw, s);
    if (e != cudaSuccess) return cuda_fail("cudaMemsetAsync(gradients)", e);
    if (a.T == 0) return QCMET_OK;
    a.g_scale = g_scale;
    a.g_offset = g_offset;
    std::string err;
    qcmet::TraceRange range("qcmet min-sum backward: %d frames x %d iterations", a.K, a.T);
    int st = qcmet::launch_learned_backward(a, stream, err);
    if (st) return fail(st, err);
    return QCMET_OK;
}

int qcmet_group_plan(const qcmet_code *code, int32_t K, const qcmet_decode_options *opts,
                     qcmet_group_plan_t *plan) {
    if (!code || !plan) return fail(QCMET_ERR_INVALID_ARG, "code and plan must not be NULL");
    if (K < 1) return fail(QCMET_ERR_INVALID_ARG, "need K >= 1");
    int32_t fmt = 0, threads = 0;
    KernelChoice kc;
    int st = check_options(opts, &fmt, &threads, nullptr, &kc);
    if (st) return st;
    const qcmet::Code &c = code->c;
    if ((int64_t)c.nb * qcmet::group_zp(c.Z) > INT32_MAX)
        return fail(QCMET_ERR_INVALID_ARG, "code too large for the grouped kernel's 32-bit offsets");
    qcmet::GroupLaunch L;
    std::string err;
    st = qcmet::choose_group_launch(fmt, K, c.Z, (int32_t)c.image.words.size(),
                                    qcmet::group_stage_ops(c), kc.cluster, &L, err, false,
                                    kc.per_cluster);
    if (st) return fail(st, err);
    plan->cluster_size = L.cluster;
    plan->groups_per_cluster = L.per_cluster;
    plan->threads_per_block = L.threads;
    plan->clusters = (L.groups + L.per_cluster - 1) / L.per_cluster;
    plan->blocks = plan->clusters * L.cluster;
    plan->active_clusters = L.active_clusters;
    plan->shared_bytes = (int32_t)L.smem;
    plan->reserved = 0;
    return QCMET_OK;
}

int qcmet_debug_checks(uint32_t *violations) {
    if (!violations) return fail(QCMET_ERR_INVALID_ARG, "violations must not be NULL");
    *violations = 0;
#ifndef QCMET_DEBUG_CHECKS
#define QCMET_DEBUG_CHECKS 0
#endif
#if QCMET_DEBUG_CHECKS
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail("cudaDeviceSynchronize", e);
    uint32_t a = 0, b = 0;
    std::string err;
    int st = qcmet::take_violations_frame(&a, err);
    if (!st) st = qcmet::take_violations_group(&b, err);
    if (st) return fail(st, err);
    *violations = a | b;
    return QCMET_OK;
#else
    return fail(QCMET_ERR_UNSUPPORTED, "this library was built without index checks "
                                       "(build libqcmet_debug.so for them)");
#endif
}

const char *qcmet_last_error(void) { return g_last_error.c_str(); }

const char *qcmet_status_string(int status) {
    switch (status) {
        case QCMET_OK: return "ok";
        case QCMET_ERR_INVALID_ARG: return "invalid argument";
        case QCMET_ERR_SHIFT_RANGE: return "circulant shift outside [0, Z)";
        case QCMET_ERR_DEGREE_LIMIT: return "row degree above QCMET_MAX_ROW_DEGREE";
        case QCMET_ERR_ALIGNMENT: return "pointer not 16-byte aligned";
        case QCMET_ERR_OOM: return "out of memory";
        case QCMET_ERR_CUDA: return "CUDA error";
        case QCMET_ERR_TIMEOUT: return "device wait timed out";
        case QCMET_ERR_UNSUPPORTED: return "unsupported";
        default: return "unknown status";
    }
}

int qcmet_version(void) { return QCMET_VERSION; }

}  // extern "C"
