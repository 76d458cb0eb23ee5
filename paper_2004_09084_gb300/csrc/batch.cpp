// Mixed batches: frames of several codes decoded by one launch, captured once
// into a CUDA graph and replayed.  Two kernels can serve a batch: the
// per-frame batch kernel (decode.cu; thread blocks take frames from a queue)
// and the grouped batch kernel (decode_group.cu; clusters take groups of up
// to four frames of one code, stored interleaved, from a queue).  The plan
// picks the kernel and its launch configuration by timing candidates on the
// batch itself.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "qcmet_internal.h"
#include "trace.h"

struct qcmet_batch {
    std::vector<qcmet_frame> frames;
    int32_t K = 0, T = 0, fmt = QCMET_MSG_FP32;
    std::vector<const qcmet_code *> codes;          // distinct codes, by first appearance
    std::vector<int32_t> frame_code;                // [K] index into codes
    std::vector<qcmet_code *> alt;                  // same codes with the other exact schedule
    qcmet_batch_config cfg{};
    int32_t max_image_words = 0;
    int32_t max_Z = 0;
    int32_t stage_ops = 1;                          // grouped kernel: most staged operands
    void *d_scratch = nullptr;                      // messages (+ posteriors), descriptors, order, counter
    qcmet::BatchFrame *d_frames = nullptr;
    int32_t *d_order = nullptr;
    int32_t *d_counter = nullptr;
    // grouped kernel: jobs of up to four frames of one code
    std::vector<std::vector<int32_t>> job_frames;   // frames of each job
    void *d_group = nullptr;                        // per-job interleaved scratch, jobs, order
    qcmet::GroupJob *d_jobs = nullptr;
    int32_t *d_jorder = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

size_t r256(size_t x) { return (x + 255) & ~size_t(255); }
size_t msg_size(int32_t fmt) { return fmt == QCMET_MSG_FP32 ? 4 : 2; }

int cuda_err(const char *what, cudaError_t e) {
    return qcmet::set_error(e == cudaErrorMemoryAllocation ? QCMET_ERR_OOM : QCMET_ERR_CUDA,
                            std::string(what) + ": " + cudaGetErrorString(e));
}

// Descriptors for one configuration: which schedule variant and which order.
int write_descriptors(qcmet_batch &b, bool alt, bool largest_first, cudaStream_t s) {
    std::vector<qcmet::BatchFrame> fd(b.K);
    char *p = static_cast<char *>(b.d_scratch);
    size_t off = 0;
    b.max_image_words = 0;
    for (int32_t k = 0; k < b.K; ++k) {
        const qcmet_code *h = alt && b.alt[b.frame_code[k]] ? b.alt[b.frame_code[k]]
                                                            : b.codes[b.frame_code[k]];
        qcmet::Code &c = const_cast<qcmet_code *>(h)->c;
        int st = qcmet::ensure_device_image(c);
        if (st) return st;
        const qcmet_frame &f = b.frames[k];
        qcmet::BatchFrame &d = fd[k];
        d.image = c.d_image;
        d.image_words = (int32_t)c.image.words.size();
        d.code_id = b.frame_code[k];
        d.ch = f.llr_ch;
        d.syn = f.syndrome;
        d.hard = f.hard;
        d.ok = f.ok;
        d.Z = c.Z;
        d.n = c.nb * c.Z;
        d.m = c.mb * c.Z;
        d.nb = c.nb;
        d.msg_slots = c.msg_slots;
        d.core_cols = c.core_cols;
        d.slot_stride = (int64_t)qcmet::slot_stride(c.Z);
        d.msgs = p + off;
        off += r256((size_t)c.msg_slots * (size_t)d.slot_stride * msg_size(b.fmt));
        d.post_core = reinterpret_cast<float *>(p + off);
        off += r256((size_t)c.core_cols * (size_t)c.Z * sizeof(float));
        if (f.llr_post) {
            d.post = f.llr_post;
        } else {
            d.post = reinterpret_cast<float *>(p + off);
            off += r256((size_t)d.n * sizeof(float));
        }
        b.max_image_words = std::max(b.max_image_words, d.image_words);
    }
    std::vector<int32_t> order(b.K);
    for (int32_t k = 0; k < b.K; ++k) order[k] = k;
    if (largest_first) {
        std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
            const qcmet::Code &cx = b.codes[b.frame_code[x]]->c, &cy = b.codes[b.frame_code[y]]->c;
            return (int64_t)cx.circulants * cx.Z > (int64_t)cy.circulants * cy.Z;
        });
    }
    cudaError_t e = cudaMemcpyAsync(b.d_frames, fd.data(), fd.size() * sizeof(qcmet::BatchFrame),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b.d_order, order.data(), order.size() * sizeof(int32_t),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // host vectors go out of scope
    if (e != cudaSuccess) return cuda_err("cudaMemcpyAsync(batch descriptors)", e);
    return QCMET_OK;
}

size_t group_job_bytes(const qcmet::Code &c, int32_t fmt) {
    return qcmet::group_scratch_bytes(c, fmt).total();
}

// Jobs of the grouped kernel for one configuration: schedule variant and order.
int write_jobs(qcmet_batch &b, bool alt, bool largest_first, cudaStream_t s) {
    const int32_t J = (int32_t)b.job_frames.size();
    std::vector<qcmet::GroupJob> jobs(J);
    char *p = static_cast<char *>(b.d_group);
    size_t off = 0;
    b.max_image_words = 0;
    for (int32_t j = 0; j < J; ++j) {
        const std::vector<int32_t> &fr = b.job_frames[j];
        const int32_t cid = b.frame_code[fr[0]];
        const qcmet_code *h = alt && b.alt[cid] ? b.alt[cid] : b.codes[cid];
        qcmet::Code &c = const_cast<qcmet_code *>(h)->c;
        int st = qcmet::ensure_device_image(c);
        if (st) return st;
        qcmet::GroupJob &g = jobs[j];
        std::memset(&g, 0, sizeof(g));
        g.image = c.d_image;
        g.image_words = (int32_t)c.image.words.size();
        g.code_id = cid;
        g.nf = (int32_t)fr.size();
        for (int32_t f = 0; f < g.nf; ++f) {
            const qcmet_frame &q = b.frames[fr[f]];
            g.ch[f] = q.llr_ch;
            g.syn[f] = q.syndrome;
            g.post[f] = q.llr_post;
            g.hard[f] = q.hard;
            g.ok[f] = q.ok;
        }
        if ((int64_t)c.nb * qcmet::group_zp(c.Z) > INT32_MAX) {
            return qcmet::set_error(QCMET_ERR_INVALID_ARG,
                                    "code too large for the grouped kernel's 32-bit offsets");
        }
        const qcmet::GroupScratch gs = qcmet::group_scratch_bytes(c, b.fmt);
        g.ch4 = p + off;
        off += gs.ch;
        g.syn4 = reinterpret_cast<uint32_t *>(p + off);
        off += gs.syn;
        g.core4 = p + off;
        off += gs.core;
        g.msgs4 = p + off;
        off += gs.msg;
        b.max_image_words = std::max(b.max_image_words, g.image_words);
    }
    std::vector<int32_t> order(J);
    for (int32_t j = 0; j < J; ++j) order[j] = j;
    if (largest_first) {
        std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
            const qcmet::Code &cx = b.codes[b.frame_code[b.job_frames[x][0]]]->c;
            const qcmet::Code &cy = b.codes[b.frame_code[b.job_frames[y][0]]]->c;
            return (int64_t)cx.circulants * cx.Z > (int64_t)cy.circulants * cy.Z;
        });
    }
    cudaError_t e = cudaMemcpyAsync(b.d_jobs, jobs.data(), jobs.size() * sizeof(qcmet::GroupJob),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b.d_jorder, order.data(), order.size() * sizeof(int32_t),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // host vectors go out of scope
    if (e != cudaSuccess) return cuda_err("cudaMemcpyAsync(batch jobs)", e);
    return QCMET_OK;
}

// kernel: QCMET_KERNEL_FRAME (size = threads per block) or QCMET_KERNEL_GROUP
// (size = cluster size)
int launch(qcmet_batch &b, int32_t T, int32_t kernel, int32_t size, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(b.d_counter, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return cuda_err("cudaMemsetAsync(batch counter)", e);
    std::string err;
    int st;
    if (kernel == QCMET_KERNEL_GROUP) {
        qcmet::GroupBatchArgs a;
        a.jobs = b.d_jobs;
        a.order = b.d_jorder;
        a.counter = b.d_counter;
        a.J = (int32_t)b.job_frames.size();
        a.T = T;
        a.stage_ops = b.stage_ops;
        st = qcmet::launch_decode_group_batch(a, b.fmt, size, b.max_Z, b.max_image_words, s, err);
    } else {
        qcmet::BatchArgs a;
        a.frames = b.d_frames;
        a.order = b.d_order;
        a.counter = b.d_counter;
        a.K = b.K;
        a.T = T;
        st = qcmet::launch_decode_batch(a, b.fmt, size, b.max_image_words, s, err);
    }
    if (st) return qcmet::set_error(st, err);
    return QCMET_OK;
}

int write_config(qcmet_batch &b, int32_t kernel, bool alt, bool largest, cudaStream_t s) {
    return kernel == QCMET_KERNEL_GROUP ? write_jobs(b, alt, largest, s)
                                        : write_descriptors(b, alt, largest, s);
}

void release(qcmet_batch *b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->d_scratch) cudaFree(b->d_scratch);
    if (b->d_group) cudaFree(b->d_group);
    for (qcmet_code *a : b->alt)
        if (a) qcmet_code_destroy(a);
    delete b;
}

}  // namespace

extern "C" {

int qcmet_batch_create(const qcmet_frame *frames, int32_t K, int32_t iterations,
                       int32_t msg_format, int32_t autotune, void *stream, qcmet_batch **out) {
    if (!out) return qcmet::set_error(QCMET_ERR_INVALID_ARG, "out must not be NULL");
    *out = nullptr;
    if (!frames || K < 1 || iterations < 0)
        return qcmet::set_error(QCMET_ERR_INVALID_ARG, "need frames, K >= 1 and iterations >= 0");
    if (msg_format != QCMET_MSG_FP32 && msg_format != QCMET_MSG_FP16 && msg_format != QCMET_MSG_BF16)
        return qcmet::set_error(QCMET_ERR_INVALID_ARG, "unknown msg_format");
    qcmet_batch *b = new (std::nothrow) qcmet_batch;
    if (!b) return qcmet::set_error(QCMET_ERR_OOM, "host allocation failed");
    b->frames.assign(frames, frames + K);
    b->K = K;
    b->T = iterations;
    b->fmt = msg_format;
    std::map<const qcmet_code *, int32_t> ids;
    size_t bytes = 0;
    for (int32_t k = 0; k < K; ++k) {
        const qcmet_frame &f = frames[k];
        auto bad = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) != 0; };
        if (!f.code || !f.llr_ch || !f.syndrome || !f.hard || !f.ok) {
            release(b);
            return qcmet::set_error(QCMET_ERR_INVALID_ARG, "frame " + std::to_string(k) +
                                                              ": code, llr_ch, syndrome, hard and ok must not be NULL");
        }
        if (bad(f.llr_ch) || bad(f.syndrome) || bad(f.hard) || bad(f.ok) ||
            (f.llr_post && bad(f.llr_post))) {
            release(b);
            return qcmet::set_error(QCMET_ERR_ALIGNMENT, "frame " + std::to_string(k) +
                                                            ": device pointers must be 16-byte aligned");
        }
        auto it = ids.find(f.code);
        if (it == ids.end()) {
            it = ids.emplace(f.code, (int32_t)b->codes.size()).first;
            b->codes.push_back(f.code);
        }
        b->frame_code.push_back(it->second);
        const qcmet::Code &c = f.code->c;
        b->max_Z = std::max(b->max_Z, c.Z);
        b->stage_ops = std::max(b->stage_ops, qcmet::group_stage_ops(c));
        bytes += r256((size_t)c.msg_slots * qcmet::slot_stride(c.Z) * msg_size(msg_format));
        bytes += r256((size_t)c.core_cols * (size_t)c.Z * sizeof(float));
        if (!f.llr_post) bytes += r256((size_t)c.nb * c.Z * sizeof(float));
    }
    // the other exact schedule of each code (base-row order <-> merged), for the autotuner
    for (const qcmet_code *h : b->codes) {
        const qcmet::Code &c = h->c;
        qcmet_code *alt = nullptr;
        if (autotune && c.merge_mode != QCMET_MERGE_GREEDY) {
            const int32_t other = c.merge_mode == QCMET_MERGE_EXACT ? QCMET_MERGE_NONE : QCMET_MERGE_EXACT;
            int st = qcmet_code_create_ex(c.base.data(), c.shifts.data(), c.mb, c.nb, c.Z, other, &alt);
            if (st) {
                release(b);
                return st;
            }
        }
        b->alt.push_back(alt);
    }
    const size_t desc = r256((size_t)K * sizeof(qcmet::BatchFrame));
    const size_t ord = r256((size_t)K * sizeof(int32_t));
    cudaError_t e = cudaMalloc(&b->d_scratch, bytes + desc + ord + 256);
    if (e != cudaSuccess) {
        release(b);
        return cuda_err("cudaMalloc(batch scratch)", e);
    }
    char *base = static_cast<char *>(b->d_scratch);
    b->d_frames = reinterpret_cast<qcmet::BatchFrame *>(base + bytes);
    b->d_order = reinterpret_cast<int32_t *>(base + bytes + desc);
    b->d_counter = reinterpret_cast<int32_t *>(base + bytes + desc + ord);
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    // grouped kernel: the frames of each code, four at a time, in the order given
    {
        std::vector<std::vector<int32_t>> by_code(b->codes.size());
        for (int32_t k = 0; k < K; ++k) by_code[b->frame_code[k]].push_back(k);
        size_t gbytes = 0;
        for (size_t cid = 0; cid < by_code.size(); ++cid) {
            const std::vector<int32_t> &v = by_code[cid];
            for (size_t i = 0; i < v.size(); i += 4) {
                b->job_frames.emplace_back(v.begin() + i, v.begin() + std::min(v.size(), i + 4));
                gbytes += group_job_bytes(b->codes[cid]->c, msg_format);
            }
        }
        const size_t J = b->job_frames.size();
        const size_t jd = r256(J * sizeof(qcmet::GroupJob));
        e = cudaMalloc(&b->d_group, gbytes + jd + r256(J * sizeof(int32_t)));
        if (e != cudaSuccess) {
            release(b);
            return cuda_err("cudaMalloc(grouped batch scratch)", e);
        }
        char *gb = static_cast<char *>(b->d_group);
        b->d_jobs = reinterpret_cast<qcmet::GroupJob *>(gb + gbytes);
        b->d_jorder = reinterpret_cast<int32_t *>(gb + gbytes + jd);
    }

    // candidates (all give the same results): the per-frame kernel with block
    // size 512 or 1024, the grouped kernel with clusters of 2, 4, 5, 8 or 16
    // blocks; each with the codes' own schedule or the other exact one, and
    // the work taken largest first or as given
    struct Cand { int32_t kernel; int32_t size; bool alt; bool largest; };
    std::vector<Cand> cands;
    const bool have_alt =
        std::any_of(b->alt.begin(), b->alt.end(), [](qcmet_code *a) { return a != nullptr; });
    if (autotune) {
        for (int32_t kern : {QCMET_KERNEL_FRAME, QCMET_KERNEL_GROUP})
            for (int32_t size : kern == QCMET_KERNEL_FRAME ? std::vector<int32_t>{512, 1024}
                                                          : std::vector<int32_t>{2, 4, 5, 8, 16})
                for (bool alt : {false, true})
                    for (bool lf : {true, false})
                        if (!alt || have_alt) cands.push_back({kern, size, alt, lf});
    } else {
        cands.push_back({QCMET_KERNEL_GROUP, 4, false, true});
    }
    Cand best = cands[0];
    float best_ms = -1.0f;
    int32_t timed = 0;
    if (cands.size() > 1) {
        // enough iterations that the per-launch work (interleaving, outputs,
        // syndrome test) does not decide the choice
        const int32_t Tt = std::min<int32_t>(iterations, 12);
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        for (const Cand &c : cands) {
            int st = write_config(*b, c.kernel, c.alt, c.largest, s);
            if (!st) st = launch(*b, Tt, c.kernel, c.size, s);   // warm-up
            if (st == QCMET_ERR_UNSUPPORTED) continue;           // a cluster size this device cannot hold
            if (!st) {
                cudaEventRecord(e0, s);
                for (int r = 0; r < 2 && !st; ++r) st = launch(*b, Tt, c.kernel, c.size, s);
                cudaEventRecord(e1, s);
            }
            if (st) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                release(b);
                return st;
            }
            cudaEventSynchronize(e1);
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            ++timed;
            if (best_ms < 0.0f || ms < best_ms) {
                best_ms = ms;
                best = c;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (timed == 0) {
            release(b);
            return qcmet::set_error(QCMET_ERR_UNSUPPORTED, "no batch configuration can be launched");
        }
    }
    int st = write_config(*b, best.kernel, best.alt, best.largest, s);
    if (st) {
        release(b);
        return st;
    }
    b->cfg.threads_per_block = best.kernel == QCMET_KERNEL_FRAME ? best.size : 0;
    b->cfg.alternate_schedule = best.alt ? 1 : 0;
    b->cfg.largest_first = best.largest ? 1 : 0;
    b->cfg.trial_ms = best_ms;
    b->cfg.candidates = (int32_t)cands.size();
    b->cfg.kernel = best.kernel;
    b->cfg.cluster_size = best.kernel == QCMET_KERNEL_GROUP ? best.size : 0;

    // capture counter reset + launch into a graph on a private stream
    cudaStream_t cap;
    e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        release(b);
        return cuda_err("cudaStreamCreateWithFlags", e);
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        st = launch(*b, iterations, best.kernel, best.size, cap);
        cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
        if (!st && e2 != cudaSuccess) st = cuda_err("cudaStreamEndCapture", e2);
    } else {
        st = cuda_err("cudaStreamBeginCapture", e);
    }
    if (!st) {
        e = cudaGraphInstantiate(&b->exec, graph, 0);
        if (e != cudaSuccess) st = cuda_err("cudaGraphInstantiate", e);
    }
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cap);
    if (st) {
        release(b);
        return st;
    }
    *out = b;
    return QCMET_OK;
}

int qcmet_batch_run(qcmet_batch *batch, void *stream) {
    if (!batch || !batch->exec) return qcmet::set_error(QCMET_ERR_INVALID_ARG, "batch must not be NULL");
    qcmet::TraceRange range("qcmet batch: %d frames x %d iterations", batch->K, batch->T);
    cudaError_t e = cudaGraphLaunch(batch->exec, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_err("cudaGraphLaunch", e);
    return QCMET_OK;
}

int qcmet_batch_get_config(const qcmet_batch *batch, qcmet_batch_config *out) {
    if (!batch || !out) return qcmet::set_error(QCMET_ERR_INVALID_ARG, "batch and out must not be NULL");
    *out = batch->cfg;
    return QCMET_OK;
}

void qcmet_batch_destroy(qcmet_batch *batch) { release(batch); }

}  // extern "C"
