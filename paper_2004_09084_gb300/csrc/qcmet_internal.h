// Internal declarations shared by the host builder, the C ABI glue and the
// CUDA kernels of the decoder library.  Not installed; not part of the ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/qcmet.h"

namespace qcmet {

// Column classes of the base matrix.
enum ColumnKind : int32_t {
    kColUnconnected = 0,  // no circulant in the column: L_qn stays the channel LLR
    kColDegree1 = 1,      // one circulant: L_qn - L_rmn(old) is the channel LLR exactly
    kColCore = 2,         // two or more circulants: posterior and messages are state
};

// One circulant of a base row as the layer kernel reads it.
struct DevEntry {
    int32_t var_base;  // core column: cc * Z, its offset among the core posteriors
                       // (cc = index among core columns); degree-1 column: c * Z
    int32_t shift;     // circulant shift a
    int32_t slot;      // message slot for core columns, -1 for a degree-1 column
    int32_t col;       // base column c (frame variables c*Z .. c*Z + Z - 1)
};

// One scheduled base row.
struct DevRow {
    int32_t first_entry;  // index of its first DevEntry
    int32_t degree;       // number of circulants (1..QCMET_MAX_ROW_DEGREE)
    int32_t check_base;   // l * Z: first check of the row
    int32_t row;          // base row l
};

// Flat device image of a code's schedule: a header followed by int32 arrays.
// Layout (all int32, offsets in elements from the start):
//   header[kHdrWords]: see the kHdr* indices below
//   layer_first[n_layers + 1]           (padded to a multiple of 4)
//   rows[n_rows]   (DevRow, 4 ints each)
//   entries[n_entries] (DevEntry, 4 ints each)
//   col_kind[nb]                         (padded to a multiple of 4)
//   zero_rows[...]: base rows with no circulant (their checks test s_m = 0)
//   col_core[nb]: index of a core column among the core columns, else -1 (padded)
enum : int32_t {
    kHdrRows = 0, kHdrLayers, kHdrEntries, kHdrNb, kHdrZ, kHdrMb,
    kHdrOffLayerFirst, kHdrOffRows, kHdrOffEntries, kHdrOffColKind, kHdrOffZeroRows,
    kHdrZeroRows, kHdrOffColCore, kHdrCoreCols, kHdrMsgSlots, kHdrPad1, kHdrWords
};

struct ScheduleImage {
    std::vector<int32_t> words;
    int32_t off_layer_first = 0;
    int32_t off_rows = 0;
    int32_t off_entries = 0;
    int32_t off_col_kind = 0;
    int32_t off_zero_rows = 0;
    int32_t n_zero_rows = 0;
};

// Arguments of the learned min-sum kernels (learned.cu).
struct LearnedArgs {
    const float *ch;          // [K][n]
    const uint8_t *syn;       // [K][m]
    const uint8_t *x;         // [K][n] transmitted bits (training)
    float *post;              // [K][n] posteriors
    float *msgs;              // [K][slots][stride] messages (FP32)
    const float *w_scale;     // [T][mb][2]
    const float *w_offset;    // [T][mb][2]
    float *qhist;             // [K][T][slots][stride] q of core edges (training)
    float *Lhist;             // [K][T][core_cols*Z] core posteriors after each iteration (training)
    float *loss;              // [K] (training)
    float *g_scale;           // [T][mb][2] (backward, accumulated)
    float *g_offset;          // [T][mb][2] (backward, accumulated)
    float *gL;                // [K][core_cols*Z] adjoint of the core posteriors (backward)
    float *gR;                // [K][slots][stride] adjoint of the stored messages (backward)
    uint8_t *hard;            // [K][n] (inference)
    uint8_t *ok;              // [K] (inference)
    const int32_t *image;
    int32_t image_words;
    int32_t K, T, Z, n, m, nb, mb, msg_slots;
    int64_t slot_stride;
};

struct Code {
    int32_t mb = 0, nb = 0, Z = 0;
    int32_t merge_mode = QCMET_MERGE_EXACT;
    std::vector<int8_t> base;
    std::vector<int32_t> shifts;
    std::vector<int32_t> col_degree;        // [nb]
    std::vector<int32_t> sched_rows;        // base rows in visiting order
    std::vector<int32_t> layer_first;       // [layers + 1] into sched_rows
    std::vector<int32_t> zero_rows;         // rows with no circulant
    int32_t circulants = 0;
    int32_t msg_slots = 0;
    int32_t core_cols = 0;                  // columns of degree > 1
    int32_t degree1_columns = 0;
    int32_t max_row_degree = 0;
    ScheduleImage image;

    // device state (created at the first decode)
    int device = -1;
    int32_t *d_image = nullptr;
    size_t image_bytes = 0;
    void *d_msgs = nullptr;       // message scratch
    size_t msgs_bytes = 0;
    float *d_post = nullptr;      // posterior scratch when the caller passes no llr_post
    size_t post_bytes = 0;
    float *d_core = nullptr;      // [K][core_cols][Z] posteriors of the core columns
    size_t core_bytes = 0;
    // staging buffers of qcmet_decode_host
    void *d_io = nullptr;
    size_t io_bytes = 0;
    // grouped (frame-interleaved, clustered) decode: interleaved channel,
    // syndrome, core posteriors and messages of ceil(K/4) groups
    void *d_group = nullptr;
    size_t group_bytes = 0;
    // learned min-sum: scratch and the arguments of the last training forward
    void *d_learned = nullptr;
    size_t learned_bytes = 0;
    bool learned_ready = false;
    LearnedArgs learned_last{};
};

// Shared by the C ABI files (api.cpp, batch.cpp): upload a code's layer table
// once per device, and record a failing call's message for qcmet_last_error.
int ensure_device_image(Code &c);
int set_error(int status, const std::string &msg);

// Host builder (layout.cpp).  Returns a QCMET status; fills `err` on failure.
int build_code(const int8_t *base, const int32_t *shifts, int32_t mb, int32_t nb, int32_t Z,
               int32_t merge_mode, Code &code, std::string &err);

// Message slot stride in elements: Z rounded up so that every slot starts on
// a 16-byte boundary for every message format.
inline size_t slot_stride(int32_t Z) { return (static_cast<size_t>(Z) + 15) & ~static_cast<size_t>(15); }

// Kernel launch arguments (decode.cu).
struct DecodeArgs {
    const float *ch;         // [K][n]
    const uint8_t *syn;      // [K][m]
    float *post;             // [K][n] posterior output (the caller's llr_post or scratch)
    float *post_core;        // [K][core_cols*Z] posteriors of the core columns (decoder state)
    void *msgs;              // [K][msg_slots][slot_stride] messages
    uint8_t *hard;           // [K][n]
    uint8_t *ok;             // [K]
    const int32_t *image;    // schedule image (device)
    int32_t image_words;
    int32_t K, T, Z, n, m, nb;
    int32_t msg_slots;
    int32_t core_cols;
    int64_t slot_stride;     // elements
    int32_t check_every;     // > 0: early termination test every check_every iterations
    int32_t *iters_used;     // [K] iterations each frame ran, or nullptr
};

// Check-node rule of the fused decode kernel: the paper's sum-product rule, or
// offset/scaled min-sum with weights [T][mb][2] (FP32, device; the learned
// variant).
struct CheckRule {
    const float *w_scale = nullptr;   // nullptr: sum-product
    const float *w_offset = nullptr;
};

int launch_learned_forward(const LearnedArgs &a, void *stream, std::string &err);
int launch_learned_backward(const LearnedArgs &a, void *stream, std::string &err);

// One frame of a mixed batch (device array; decode.cu's batch kernel).
struct BatchFrame {
    const int32_t *image;    // the frame's code: schedule image (device)
    const float *ch;         // [n]
    const uint8_t *syn;      // [m]
    float *post;             // [n]
    float *post_core;        // [core_cols * Z]
    uint8_t *hard;           // [n]
    uint8_t *ok;             // [1]
    void *msgs;              // [msg_slots][slot_stride] messages
    int64_t slot_stride;
    int32_t image_words;
    int32_t code_id;         // frames with equal code_id share the image
    int32_t Z, n, m, nb;
    int32_t msg_slots;
    int32_t core_cols;
};

struct BatchArgs {
    const BatchFrame *frames;  // [K]
    const int32_t *order;      // [K] frame indices in the order CTAs take them
    int32_t *counter;          // work counter (zero before the launch)
    int32_t K, T;
};

int launch_decode_batch(const BatchArgs &b, int32_t msg_format, int32_t threads,
                        int32_t max_image_words, void *stream, std::string &err);

// Launch the fused decode kernel for one message format (decode.cu).
// window_bytes > 0 attaches an L2 persisting access-policy window of that many
// bytes, starting at a.post_core, with the given hit ratio, to the launch.
int launch_decode(const DecodeArgs &a, int32_t msg_format, int32_t threads, void *stream,
                  std::string &err, size_t window_bytes = 0, float hit_ratio = 0.0f,
                  const CheckRule &rule = CheckRule());

// The grouped kernel's interleaved scratch for one group stores every column,
// message slot and syndrome row with the row stride Zp = Z rounded up to 32,
// so that each starts on a 128-byte line and the 32 checks of a warp whose
// first check is a multiple of 32 read whole lines of messages and syndrome
// words.
inline int64_t group_zp(int64_t Z) { return (Z + 31) / 32 * 32; }

// Bytes of one group's scratch arrays (each a multiple of 256).
struct GroupScratch {
    size_t ch, syn, core, msg;
    size_t total() const { return ch + syn + core + msg; }
};
GroupScratch group_scratch_bytes(const Code &c, int32_t msg_format);

// Arguments of the grouped decode kernel (decode_group.cu): frames 4g .. 4g+3
// form group g and are stored interleaved, one 16-byte word per variable.
struct GroupArgs {
    const float *ch;         // [K][n] caller's channel LLRs (frame-major)
    const uint8_t *syn;      // [K][m] caller's syndromes
    float *post;             // [K][n] output posteriors, or nullptr
    uint8_t *hard;           // [K][n]
    uint8_t *ok;             // [K]
    void *ch4;               // [G][nb][Zp] float4: interleaved channel (scratch)
    uint32_t *syn4;          // [G][mb][Zp]: syndrome bit of frame f in byte f (scratch)
    void *core4;             // [G][core_cols][Zp] float4: core posteriors (scratch)
    void *msgs4;             // [G][msg_slots][Zp] messages, 16 B (FP32) or 8 B (16-bit) (scratch)
    GroupScratch g_bytes;    // bytes between consecutive groups of each array
    const int32_t *image;    // schedule image (device)
    int32_t image_words;
    int32_t K, T, n, m, core_cols, msg_slots;
    int32_t stage_ops;       // most operands staged per check (rows of degree <= 4)
    const float *w_scale;    // min-sum weights [T][mb][2], or nullptr (sum-product rule)
    const float *w_offset;
};

// Launch shape of the grouped kernel: clusters of `cluster` CTAs, each owning
// `per_cluster` of the `groups` groups.
struct GroupLaunch {
    int32_t cluster = 0;
    int32_t per_cluster = 1;
    int32_t threads = 0;
    int32_t groups = 0;
    int32_t active_clusters = 0;  // clusters of this shape the device holds at once
    int32_t variant = 0;          // kernel build (rounds staged, block bound, blocks per SM)
    int32_t kidx = 0;             // message format, or 3 for the min-sum rule (FP32 messages)
    int32_t stage_ops = 0;
    size_t smem = 0;
};

// One job of a mixed batch on the grouped kernel: one or two groups of up to
// four frames of one code, stored interleaved in the jobs' own scratch.  With
// two groups, group 1's arrays follow group 0's at `gstride` bytes per array.
struct GroupJob {
    const int32_t *image;    // the code's schedule image (device)
    int32_t image_words;
    int32_t code_id;         // jobs with equal code_id share the image
    int32_t nf[2];           // frames in each group (1..4; 0 for an absent group 1)
    int32_t ng;              // groups in the job (1 or 2)
    int32_t pad;
    const float *ch[2][4];   // per group and frame [n]
    const uint8_t *syn[2][4];  // per group and frame [m]
    float *post[2][4];       // per group and frame [n], or nullptr
    uint8_t *hard[2][4];     // per group and frame [n]
    uint8_t *ok[2][4];       // per group and frame [1]
    void *ch4;               // group 0's [nb][Zp] float4
    uint32_t *syn4;          // group 0's [mb][Zp]
    void *core4;             // group 0's [core_cols][Zp] float4
    void *msgs4;             // group 0's [msg_slots][Zp] messages
    GroupScratch gstride;    // bytes from group 0's arrays to group 1's
};

struct GroupBatchArgs {
    const GroupJob *jobs;    // [J]
    const int32_t *order;    // [J] job indices in the order clusters take them
    int32_t *counter;        // work counter (zero before the launch)
    int32_t J, T;
    int32_t stage_ops;       // most operands staged per check over the batch's codes
};

// One launch of the grouped batch kernel with clusters of `cluster` blocks
// sized for expansion factors up to max_Z and jobs of up to groups_per_job
// groups (1 or 2): persistent clusters taking jobs from the counter (jobs of
// one group), or with cluster_per_job one cluster per job; -8 (UNSUPPORTED)
// when that cluster size cannot be scheduled.
int launch_decode_group_batch(const GroupBatchArgs &b, int32_t msg_format, int32_t cluster,
                              int32_t max_Z, int32_t max_image_words, void *stream,
                              std::string &err, int32_t groups_per_job = 1,
                              bool cluster_per_job = false);

// Debug build: read and clear the index-check words of the two kernel files.
int take_violations_frame(uint32_t *bits, std::string &err);
int take_violations_group(uint32_t *bits, std::string &err);

// The most operands a check of a row of degree <= 4 stages (its edges'
// posteriors or channel LLRs plus the old messages of its core edges).
int32_t group_stage_ops(const Code &c);

// Bytes of one group's message for one check and slot (four frames).
size_t group_msg_bytes(int32_t msg_format);
// Pick the cluster size (want_cluster > 0 forces it), the groups per cluster
// (want_per_cluster > 0 forces it), kernel build and block size for K frames
// of a code with expansion Z.
int choose_group_launch(int32_t msg_format, int32_t K, int32_t Z, int32_t image_words,
                        int32_t stage_ops, int32_t want_cluster, GroupLaunch *out,
                        std::string &err, bool minsum = false, int32_t want_per_cluster = 0);
int launch_decode_group(const GroupArgs &a, int32_t msg_format, const GroupLaunch &L,
                        void *stream, std::string &err, size_t window_bytes = 0,
                        float hit_ratio = 0.0f);

// Launch the FP32 decode kernel with its messages and layer table in the
// library's static device scratch (decode.cu): no device allocation.
int launch_decode_noalloc(DecodeArgs a, const int32_t *image_host, size_t image_bytes,
                          void *stream, std::string &err);
size_t noalloc_capacity_bytes();

}  // namespace qcmet

// The opaque handle of the C ABI.
struct qcmet_code {
    qcmet::Code c;
};
