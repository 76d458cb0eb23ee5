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

#include "l2_persist.h"
#include "qcmet_internal.h"
#include "trace.h"

// Grouped kernel, one launch per code: the code's groups [g0, g1) (consecutive
// in the batch's group list), its jobs [j0, j1) in the job array, the cluster
// size and the groups per job chosen for them.
struct CodeLaunch {
    int32_t code, g0, g1, j0, j1, cluster, ng, Z;
};

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
    // grouped kernel: groups of up to four frames of one code (the groups of a
    // code consecutive); a job holds one group, or two with per-code launches
    std::vector<std::vector<int32_t>> job_frames;   // frames of each group
    void *d_group = nullptr;                        // per-group interleaved scratch, jobs, order
    qcmet::GroupJob *d_jobs = nullptr;
    int32_t *d_jorder = nullptr;
    // grouped kernel, one concurrent launch per code: shapes, work counters,
    // streams, and the fork event followed by one join event per code
    std::vector<CodeLaunch> per_code;
    int32_t *d_code_counters = nullptr;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
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

// Jobs of the grouped kernel for one configuration: schedule variant and
// order; with per_code, the jobs of each code's launch (b.per_code), two
// consecutive groups per job where its plan says so.  Each group's scratch is
// sized in d_group one group after another; a job spreads its groups' share
// over its arrays.
int write_jobs(qcmet_batch &b, bool alt, bool largest_first, bool per_code, cudaStream_t s) {
    const int32_t G = (int32_t)b.job_frames.size();
    char *p = static_cast<char *>(b.d_group);
    std::vector<size_t> goff(G);
    std::vector<qcmet::GroupScratch> gsz(G);
    std::vector<qcmet::Code *> gcode(G);
    size_t off = 0;
    for (int32_t g = 0; g < G; ++g) {
        const int32_t cid = b.frame_code[b.job_frames[g][0]];
        const qcmet_code *h = alt && b.alt[cid] ? b.alt[cid] : b.codes[cid];
        qcmet::Code &c = const_cast<qcmet_code *>(h)->c;
        int st = qcmet::ensure_device_image(c);
        if (st) return st;
        if ((int64_t)c.nb * qcmet::group_zp(c.Z) > INT32_MAX) {
            return qcmet::set_error(QCMET_ERR_INVALID_ARG,
                                    "code too large for the grouped kernel's 32-bit offsets");
        }
        gcode[g] = &c;
        gsz[g] = qcmet::group_scratch_bytes(c, b.fmt);
        goff[g] = off;
        off += gsz[g].total();
    }
    std::vector<std::pair<int32_t, int32_t>> spec;   // (first group, groups) of each job
    if (per_code) {
        for (CodeLaunch &L : b.per_code) {
            L.j0 = (int32_t)spec.size();
            for (int32_t g = L.g0; g < L.g1; g += L.ng) spec.push_back({g, std::min(L.ng, L.g1 - g)});
            L.j1 = (int32_t)spec.size();
        }
    } else {
        for (int32_t g = 0; g < G; ++g) spec.push_back({g, 1});
    }
    const int32_t J = (int32_t)spec.size();
    std::vector<qcmet::GroupJob> jobs(J);
    b.max_image_words = 0;
    for (int32_t j = 0; j < J; ++j) {
        const int32_t g0 = spec[j].first;
        const qcmet::Code &c = *gcode[g0];
        qcmet::GroupJob &job = jobs[j];
        std::memset(&job, 0, sizeof(job));
        job.image = c.d_image;
        job.image_words = (int32_t)c.image.words.size();
        job.code_id = b.frame_code[b.job_frames[g0][0]];
        job.ng = spec[j].second;
        for (int32_t i = 0; i < job.ng; ++i) {
            const std::vector<int32_t> &fr = b.job_frames[g0 + i];
            job.nf[i] = (int32_t)fr.size();
            for (int32_t f = 0; f < job.nf[i]; ++f) {
                const qcmet_frame &q = b.frames[fr[f]];
                job.ch[i][f] = q.llr_ch;
                job.syn[i][f] = q.syndrome;
                job.post[i][f] = q.llr_post;
                job.hard[i][f] = q.hard;
                job.ok[i][f] = q.ok;
            }
        }
        // a job of ng groups owns ng consecutive groups' scratch (same code, same
        // sizes) and lays it out array by array: both groups' channel words,
        // then both groups' syndrome words, posteriors and messages
        const qcmet::GroupScratch &gs = gsz[g0];
        const size_t ng = (size_t)job.ng;
        char *base = p + goff[g0];
        job.ch4 = base;
        job.syn4 = reinterpret_cast<uint32_t *>(base + ng * gs.ch);
        job.core4 = base + ng * (gs.ch + gs.syn);
        job.msgs4 = base + ng * (gs.ch + gs.syn + gs.core);
        job.gstride = gs;
        b.max_image_words = std::max(b.max_image_words, job.image_words);
    }
    std::vector<int32_t> order(J);
    for (int32_t j = 0; j < J; ++j) order[j] = j;
    if (largest_first && !per_code) {
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

// Candidate kind of the grouped kernel with one concurrent launch per code.
constexpr int32_t kPerCodeLaunches = 3;

// One launch of the grouped batch kernel per code, each on its own stream and
// with its own work counter, all forked from and joined back into s (graph
// branches when s is being captured).
int launch_per_code(qcmet_batch &b, int32_t T, cudaStream_t s) {
    const int32_t n = (int32_t)b.per_code.size();
    cudaError_t e = cudaMemsetAsync(b.d_code_counters, 0, (size_t)n * sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaEventRecord(b.events[0], s);
    if (e != cudaSuccess) return cuda_err("batch fork", e);
    std::string err;
    for (int32_t i = 0; i < n; ++i) {
        const CodeLaunch &L = b.per_code[i];
        e = cudaStreamWaitEvent(b.streams[i], b.events[0], 0);
        if (e != cudaSuccess) return cuda_err("cudaStreamWaitEvent(batch fork)", e);
        qcmet::GroupBatchArgs a;
        a.jobs = b.d_jobs;
        a.order = b.d_jorder + L.j0;
        a.counter = b.d_code_counters + i;
        a.J = L.j1 - L.j0;
        a.T = T;
        a.stage_ops = b.stage_ops;
        int st = qcmet::launch_decode_group_batch(a, b.fmt, L.cluster, L.Z, b.max_image_words,
                                                  b.streams[i], err, L.ng, true);
        if (st) return qcmet::set_error(st, err);
        e = cudaEventRecord(b.events[1 + i], b.streams[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b.events[1 + i], 0);
        if (e != cudaSuccess) return cuda_err("batch join", e);
    }
    return QCMET_OK;
}

// Shapes of the per-code launches (cluster size, one or two groups per job,
// one block per SM): each code's time is modelled as its rows x a fixed cost
// per row (the first rounds' fill), plus its layers x a cluster barrier, plus
// its circulants x the cost of one circulant's check x the checks each block
// owns; starting from the fewest SMs per code, the slowest code takes its
// next faster shape while all codes together fit the device's SMs.  (Constants measured on the grouped kernel: 2.2 us per row,
// 1 us per barrier, 0.82 ns per circulant and check of four frames.)
void plan_per_code(qcmet_batch &b, const std::vector<int32_t> &groups_of_code) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        sms = 0;
    }
    struct Opt { int32_t cluster, ng, sms; double us; };
    const size_t nc = b.codes.size();
    std::vector<std::vector<Opt>> opts(nc);
    std::vector<size_t> cur(nc, 0);
    for (size_t c = 0; c < nc; ++c) {
        const qcmet::Code &k = b.codes[c]->c;
        const int32_t G = groups_of_code[c];
        const double rows = (double)k.sched_rows.size();
        const double layers = (double)k.layer_first.size() - 1.0;
        const int32_t zp = (int32_t)qcmet::group_zp(k.Z);
        for (int32_t ng = 1; ng <= (G > 1 ? 2 : 1); ++ng) {
            const int32_t span = ng == 1 ? k.Z : ng * zp;   // a job's checks
            for (int32_t C : {1, 2, 4, 5, 8}) {
                if (C > 1 && (span + C - 1) / C < 64) break;
                const int32_t zc = ((span + C - 1) / C + 31) / 32 * 32;
                const int32_t need = (G + ng - 1) / ng * C;
                const double us = rows * 2.2 + layers * 1.0 + k.circulants * 0.82e-3 * zc;
                opts[c].push_back({C, ng, need, us});
            }
        }
        // start from the fewest SMs, the faster of equals
        for (size_t o = 1; o < opts[c].size(); ++o) {
            const Opt &a = opts[c][o], &z = opts[c][cur[c]];
            if (a.sms < z.sms || (a.sms == z.sms && a.us < z.us)) cur[c] = o;
        }
    }
    // Clusters must fit inside the device's GPCs, and launches that together
    // ask for every SM end up waiting for one another: the plan keeps 5 % of
    // the SMs free and uses cluster sizes of 1, 2, 4, 5 and 8 only (measured
    // on GB300: clusters of 3 beside clusters of 5 and single blocks left part
    // of the launches to a second wave).
    sms = sms * 95 / 100;
    int32_t used = 0;
    for (size_t c = 0; c < nc; ++c) used += opts[c][cur[c]].sms;
    for (;;) {
        size_t worst = 0;
        for (size_t c = 1; c < nc; ++c)
            if (opts[c][cur[c]].us > opts[worst][cur[worst]].us) worst = c;
        const Opt &w = opts[worst][cur[worst]];
        size_t pick = SIZE_MAX;
        for (size_t o = 0; o < opts[worst].size(); ++o) {
            const Opt &a = opts[worst][o];
            if (a.us >= w.us || used - w.sms + a.sms > sms) continue;
            if (pick == SIZE_MAX || a.sms < opts[worst][pick].sms ||
                (a.sms == opts[worst][pick].sms && a.us < opts[worst][pick].us))
                pick = o;
        }
        if (pick == SIZE_MAX) break;
        used += opts[worst][pick].sms - w.sms;
        cur[worst] = pick;
    }
    b.per_code.clear();
    int32_t g = 0;
    for (size_t c = 0; c < nc; ++c) {
        const Opt &o = opts[c][cur[c]];
        // the job range is set when the jobs are written
        b.per_code.push_back({(int32_t)c, g, g + groups_of_code[c], 0, 0, o.cluster, o.ng,
                              b.codes[c]->c.Z});
        g += groups_of_code[c];
    }
}

// kernel: QCMET_KERNEL_FRAME (size = threads per block), QCMET_KERNEL_GROUP
// (size = cluster size) or kPerCodeLaunches
int launch(qcmet_batch &b, int32_t T, int32_t kernel, int32_t size, cudaStream_t s) {
    if (kernel == kPerCodeLaunches) return launch_per_code(b, T, s);
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
    // per-code launches take each code's jobs in the order given
    if (kernel == kPerCodeLaunches) return write_jobs(b, alt, false, true, s);
    return kernel == QCMET_KERNEL_GROUP ? write_jobs(b, alt, largest, false, s)
                                        : write_descriptors(b, alt, largest, s);
}

void release(qcmet_batch *b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (cudaStream_t st : b->streams) cudaStreamDestroy(st);
    for (cudaEvent_t ev : b->events) cudaEventDestroy(ev);
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
        const size_t jo = r256(J * sizeof(int32_t));
        const size_t nc = b->codes.size();
        e = cudaMalloc(&b->d_group, gbytes + jd + jo + r256(nc * sizeof(int32_t)));
        if (e != cudaSuccess) {
            release(b);
            return cuda_err("cudaMalloc(grouped batch scratch)", e);
        }
        char *gb = static_cast<char *>(b->d_group);
        b->d_jobs = reinterpret_cast<qcmet::GroupJob *>(gb + gbytes);
        b->d_jorder = reinterpret_cast<int32_t *>(gb + gbytes + jd);
        b->d_code_counters = reinterpret_cast<int32_t *>(gb + gbytes + jd + jo);
        // one concurrent launch per code: shapes, streams, fork and join events
        std::vector<int32_t> groups_of_code(nc);
        for (size_t cid = 0; cid < nc; ++cid)
            groups_of_code[cid] = (int32_t)((by_code[cid].size() + 3) / 4);
        plan_per_code(*b, groups_of_code);
        for (size_t i = 0; i < nc; ++i) {
            cudaStream_t st;
            e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
            if (e != cudaSuccess) {
                release(b);
                return cuda_err("cudaStreamCreateWithFlags", e);
            }
            b->streams.push_back(st);
        }
        for (size_t i = 0; i <= nc; ++i) {
            cudaEvent_t ev;
            e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e != cudaSuccess) {
                release(b);
                return cuda_err("cudaEventCreateWithFlags", e);
            }
            b->events.push_back(ev);
        }
    }

    // candidates (all give the same results): the per-frame kernel with block
    // size 512 or 1024, the grouped kernel with clusters of 2, 4, 5, 8 or 16
    // blocks; each with the codes' own schedule or the other exact one, and
    // the work taken largest first or as given; and the grouped kernel with
    // one concurrent launch per code (plan_per_code), with either schedule
    struct Cand { int32_t kernel; int32_t size; bool alt; bool largest; };
    std::vector<Cand> cands;
    const bool have_alt =
        std::any_of(b->alt.begin(), b->alt.end(), [](qcmet_code *a) { return a != nullptr; });
    if (autotune == 2) {
        cands.push_back({kPerCodeLaunches, 0, false, false});
    } else if (autotune) {
        for (int32_t kern : {QCMET_KERNEL_FRAME, QCMET_KERNEL_GROUP})
            for (int32_t size : kern == QCMET_KERNEL_FRAME ? std::vector<int32_t>{512, 1024}
                                                          : std::vector<int32_t>{2, 4, 5, 8, 16})
                for (bool alt : {false, true})
                    for (bool lf : {true, false})
                        if (!alt || have_alt) cands.push_back({kern, size, alt, lf});
        for (bool alt : {false, true})
            if (!alt || have_alt) cands.push_back({kPerCodeLaunches, 0, alt, false});
    } else {
        cands.push_back({QCMET_KERNEL_GROUP, 4, false, true});
    }
    Cand best = cands[0];
    float best_ms = -1.0f;
    int32_t timed = 0;
    std::vector<std::pair<float, Cand>> finalists;   // (trial ms, candidate)
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
            finalists.push_back({ms, c});
            if (best_ms < 0.0f || ms < best_ms) {
                best_ms = ms;
                best = c;
            }
        }
        if (timed == 0) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            release(b);
            return qcmet::set_error(QCMET_ERR_UNSUPPORTED, "no batch configuration can be launched");
        }
        // The short trials carry each launch's fixed costs (interleaving,
        // outputs, syndrome test) at 12 iterations instead of `iterations`, which
        // can reorder close candidates: the four fastest are timed again, once,
        // at the full count (at most 100 iterations).
        const int32_t Tf = std::min<int32_t>(iterations, 100);
        if (Tf > Tt && finalists.size() > 1) {
            std::sort(finalists.begin(), finalists.end(),
                      [](const std::pair<float, Cand> &x, const std::pair<float, Cand> &y) {
                          return x.first < y.first;
                      });
            if (finalists.size() > 4) finalists.resize(4);
            best_ms = -1.0f;
            for (const auto &fc : finalists) {
                const Cand &c = fc.second;
                int st = write_config(*b, c.kernel, c.alt, c.largest, s);
                if (!st) {
                    cudaEventRecord(e0, s);
                    st = launch(*b, Tf, c.kernel, c.size, s);
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
                if (best_ms < 0.0f || ms < best_ms) {
                    best_ms = ms;
                    best = c;
                }
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
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
    b->cfg.kernel = best.kernel == kPerCodeLaunches ? QCMET_KERNEL_GROUP : best.kernel;
    b->cfg.cluster_size = best.kernel == QCMET_KERNEL_GROUP ? best.size : 0;
    b->cfg.per_code_launches = best.kernel == kPerCodeLaunches ? (int32_t)b->per_code.size() : 0;

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
    qcmet::release_persisting_l2();
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
