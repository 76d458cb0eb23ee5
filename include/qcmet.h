/*
 * qcmet.h -- C ABI of the GB300 layered belief-propagation syndrome decoder for
 * quasi-cyclic multi-edge-type (QC-MET) LDPC codes.
 *
 * Method: arXiv 2004.09084 (Li et al., "High-throughput GPU layered decoder of
 * multi-edge type low density parity check codes in continuous-variable
 * quantum key distribution systems"), Methods section, steps 1-4: layered
 * sum-product decoding with the Phi check rule, where the syndrome bit s_m
 * flips the sign of every message leaving check m.
 *
 * Conventions shared by every call:
 *  - A code is a base matrix of mb x nb blocks and an expansion factor Z.  A
 *    block with base[l*nb + c] = 1 is the Z x Z identity cyclically shifted to
 *    the right by shifts[l*nb + c] (Results, the sentence after Eq. (m)), so
 *    check l*Z + i is connected to variable c*Z + (i + shift) mod Z.  Blocks
 *    with base = 0 are all-zero.  n = nb*Z variables, m = mb*Z checks.
 *  - One decoding iteration visits every base row once ("layer", Methods).
 *  - Frame-major layouts: frame k of an [K][n] array starts at element k*n.
 *  - Status codes: QCMET_OK (0) or a negative QCMET_ERR_*; a failing call
 *    never aborts or traps.  qcmet_last_error() returns a message for the
 *    last failing call of the calling thread.
 *
 * Tracing: with the environment variable QCMET_NVTX=1 (read once, at the
 * library's first call) the host calls push NVTX ranges in the "qcmet"
 * domain: one per decode launch, named with its kernel, frame count and
 * layer-group schedule (a decode runs all layer groups of all iterations in
 * one launch), plus ranges around qcmet_decode_host, batch runs and the
 * min-sum training calls.
 *
 * Thread safety: distinct code handles are independent.  One handle owns
 * device scratch; calls on the same handle must not run concurrently (on two
 * host threads or on two streams that overlap on the GPU).
 */
#ifndef QCMET_H
#define QCMET_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QCMET_VERSION 100

/* status codes */
#define QCMET_OK 0
#define QCMET_ERR_INVALID_ARG (-1)   /* null pointer, size out of range, bad enum     */
#define QCMET_ERR_SHIFT_RANGE (-2)   /* a shift outside [0, Z) on a circulant block   */
#define QCMET_ERR_DEGREE_LIMIT (-3)  /* a base row with more than QCMET_MAX_ROW_DEGREE */
#define QCMET_ERR_ALIGNMENT (-4)     /* a device pointer not 16-byte aligned          */
#define QCMET_ERR_OOM (-5)           /* device or host allocation failed              */
#define QCMET_ERR_CUDA (-6)          /* a CUDA runtime call or a launch failed        */
#define QCMET_ERR_TIMEOUT (-7)       /* a bounded device-side wait gave up            */
#define QCMET_ERR_UNSUPPORTED (-8)   /* valid request this build does not serve       */

/* Largest number of circulants in one base row (check degree in blocks). */
#define QCMET_MAX_ROW_DEGREE 16

/* Layer schedules (Results, Eqs. (m), (m1), (m2): merging unrelated rows).
 *  NONE   -- one layer per base row, base-row order (the Methods schedule).
 *  EXACT  -- rows that share no column with any row between them are merged;
 *            the order of every pair of rows that share a column is kept, so
 *            results are bit-identical to NONE.
 *  GREEDY -- each row joins the first earlier layer it shares no column with
 *            (the grouping of the paper's Eq. (m2) example); this may move a
 *            row ahead of a related row and so changes the decoder's order. */
#define QCMET_MERGE_NONE 0
#define QCMET_MERGE_EXACT 1
#define QCMET_MERGE_GREEDY 2

/* Storage format of the check-to-variable messages L_rmn.  Arithmetic and the
 * posteriors L_qn are FP32 in every format. */
#define QCMET_MSG_FP32 0
#define QCMET_MSG_FP16 1
#define QCMET_MSG_BF16 2

typedef struct qcmet_code qcmet_code; /* opaque, owned by the library */

typedef struct {
    int32_t mb, nb, Z;         /* base matrix shape and expansion factor          */
    int32_t n, m;              /* variables nb*Z and checks mb*Z                   */
    int64_t edges;             /* Tanner-graph edges: circulants * Z               */
    int32_t circulants;        /* non-zero blocks                                  */
    int32_t msg_slots;         /* circulants whose column has degree > 1           */
    int32_t degree1_columns;   /* base columns of degree 1                         */
    int32_t layers;            /* layers of the schedule after merging             */
    int32_t max_row_degree;    /* largest number of circulants in one row          */
    int32_t merge_mode;        /* QCMET_MERGE_*                                     */
} qcmet_code_info;

/*
 * Build a code from its base matrix (Results, Eq. (m) and the H_compact
 * description: which blocks are circulants, their shifts, Z).
 *   base   : host [mb*nb] row-major, 1 = circulant, 0 = all-zero block
 *   shifts : host [mb*nb] row-major, 0 <= shift < Z where base = 1, ignored elsewhere
 *   merge_mode : QCMET_MERGE_* (qcmet_code_create uses QCMET_MERGE_EXACT)
 *   out    : receives a handle; free it with qcmet_code_destroy
 * The inputs are copied; the caller keeps ownership of its arrays.  Host-only:
 * no GPU is touched until the first decode.  Errors: INVALID_ARG (null
 * pointer, mb/nb/Z < 1, base value other than 0/1, n or m >= 2^31),
 * SHIFT_RANGE, DEGREE_LIMIT, OOM.
 */
int qcmet_code_create(const int8_t *base, const int32_t *shifts, int32_t mb, int32_t nb,
                      int32_t Z, qcmet_code **out);
int qcmet_code_create_ex(const int8_t *base, const int32_t *shifts, int32_t mb, int32_t nb,
                         int32_t Z, int32_t merge_mode, qcmet_code **out);

/* Release a handle and every device buffer it owns.  Waits for the device to
 * finish with them.  NULL is a no-op. */
void qcmet_code_destroy(qcmet_code *code);

/* Sizes of a code (host-only). */
int qcmet_code_get_info(const qcmet_code *code, qcmet_code_info *info);

/*
 * The layer schedule (host-only): rows[0..mb) receives the base rows in the
 * order one iteration visits them (rows with no circulant are left out and
 * the remaining entries are -1); layer_first[0..layers] receives the index in
 * rows[] where each layer starts.  Either pointer may be NULL.
 */
int qcmet_code_get_schedule(const qcmet_code *code, int32_t *rows, int32_t *layer_first);

/*
 * l2_persist = 1 asks the decode kernel to keep the posteriors of the core
 * columns (K * core_columns * Z floats, the state every layer re-reads) in L2:
 * the launch carries a persisting access-policy window over them.  Such a
 * call raises the calling context's persisting-L2 limit
 * (cudaLimitPersistingL2CacheSize) to the window size when it is lower.  The
 * part of L2 set aside that way is lost to every other kernel (measured on
 * GB300: grouped decodes of 128 frames ran 26 % slower with 68 MB set aside
 * than with the default), so the library's next decode or batch run on that
 * device without a window first resets the persisting lines and puts the limit
 * back to the value it found.  Both are context-wide host calls, not stream
 * operations: a windowed decode still running then keeps less of its state in
 * L2.  The option is ignored on a device without persisting L2 and when that
 * state is larger than the device's largest window (a partial window measured
 * slower than none).  It changes no result, only speed.
 */
/*
 * Decode kernels.  Both evaluate the same arithmetic per check and frame, so
 * the choice changes no result, only speed and scratch:
 *  QCMET_KERNEL_FRAME -- one thread block owns one frame for the whole decode
 *     (frame-major state); the grid is min(K, SM count) blocks.  Serves every
 *     call, including early termination and the min-sum rule.
 *  QCMET_KERNEL_GROUP -- frames are taken four at a time and stored
 *     interleaved (the four frames' values of a variable, a message or a
 *     syndrome bit form one 16-byte word), and a thread-block cluster of
 *     cluster_size blocks (0 = chosen by the library from the device's
 *     cluster occupancy; else 1 .. 16, sizes above 8 where the device allows
 *     them) shares the checks of each row of one or two groups, with one
 *     cluster barrier per layer.  Sum-product or min-sum rule, fixed
 *     iterations.  Scratch: ceil(K/4) * (16 nb Zp + 4 mb Zp + 16 core_columns
 *     Zp + msg_slots Zp (16 for FP32, 8 for 16-bit messages)) bytes, Zp = Z
 *     rounded up to 32, each term rounded up to 256.
 *     The grouped kernel gives each memory access an L2 eviction priority
 *     (the streamed messages, channel and syndrome evict first, so that the
 *     core posteriors stay in L2) and ignores l2_persist.
 *  QCMET_KERNEL_AUTO (0) -- the grouped kernel for fixed-iteration
 *     sum-product decodes of any number of frames and for min-sum decodes of
 *     at least four frames, else the frame kernel.
 */
#define QCMET_KERNEL_AUTO 0
#define QCMET_KERNEL_FRAME 1
#define QCMET_KERNEL_GROUP 2

typedef struct {
    int32_t msg_format;        /* QCMET_MSG_*; 0 = FP32                               */
    int32_t threads_per_block; /* frame kernel: 0 = library default; else a multiple
                                  of 32, <= 1024 (the grouped kernel sizes its own)  */
    int32_t l2_persist;        /* 0 = off, 1 = persisting L2 window over the state  */
    int32_t kernel;            /* QCMET_KERNEL_*                                    */
    int32_t cluster_size;      /* grouped kernel: 0 = automatic, else 1 .. 16        */
    int32_t groups_per_cluster; /* grouped kernel: 0 = automatic, else 1 or 2       */
    int32_t reserved[2];       /* set to 0                                          */
} qcmet_decode_options;
/* The frame kernel's default block is 896 threads for FP32 messages (a kernel
 * built for that size, with more registers per thread) and 1024 for
 * FP16/BF16.  The block size changes no result. */

/*
 * Decode K frames with a fixed number of layered iterations (Methods, steps
 * 1-4; no early termination).
 *   llr_ch   : device [K][n] FP32 channel LLRs 2R/sigma^2 (step 1)
 *   syndrome : device [K][m] uint8, s_m in {0,1} (step 2); only bit 0 is read
 *   K        : frames, >= 0 (0 is a no-op)
 *   iterations : >= 0; 0 returns the hard decision of the channel LLRs
 *   hard     : device [K][n] uint8 out, c_n = 1 iff L_qn < 0 (step 4)
 *   llr_post : device [K][n] FP32 out, the posteriors L_qn after the last
 *              layer of the last iteration; may be NULL
 *   ok       : device [K] uint8 out, 1 iff H*hard = syndrome for that frame
 *   stream   : cudaStream_t (NULL = legacy default stream); the call only
 *              enqueues work and returns (stream-ordered, asynchronous)
 * Every device pointer must be 16-byte aligned (ALIGNMENT otherwise) and
 * must not overlap another.  The library keeps per-handle device scratch for
 * the messages (K * msg_slots * Z values), grown on demand, and uploads the
 * code's layer table on the first call.  Resources: one launch of min(K, SM
 * count) thread blocks, each owning a frame at a time; with FP32 messages a
 * block also takes 128 KiB of dynamic shared memory (operand staging) besides
 * the layer table.  Errors: INVALID_ARG, ALIGNMENT, OOM, CUDA, UNSUPPORTED.
 */
int qcmet_decode(const qcmet_code *code, const float *llr_ch, const uint8_t *syndrome,
                 int32_t K, int32_t iterations, uint8_t *hard, float *llr_post, uint8_t *ok,
                 void *stream);

/* qcmet_decode with options (NULL = defaults). */
int qcmet_decode_ex(const qcmet_code *code, const float *llr_ch, const uint8_t *syndrome,
                    int32_t K, int32_t iterations, uint8_t *hard, float *llr_post, uint8_t *ok,
                    const qcmet_decode_options *opts, void *stream);

/*
 * qcmet_decode_ex with early termination (Discussion, Table tabearly): after
 * every check_every-th iteration each frame takes its hard decision and tests
 * H c = s; a frame that passes stops there.  Frames are independent, so each
 * stops on its own.  A stopped frame's outputs equal those of a fixed decode
 * of exactly iterations_used[k] iterations.
 *   max_iterations : >= 0, the iteration limit (the last iteration is always tested)
 *   check_every    : >= 1; a failed test stops at the first base row with a
 *                    failing check (about a tenth of an iteration), a passed one
 *                    reads every edge's posterior once
 *   iterations_used: device [K] int32 out, iterations each frame ran
 * Other arguments, errors and scratch as qcmet_decode_ex.
 */
int qcmet_decode_early_stop(const qcmet_code *code, const float *llr_ch, const uint8_t *syndrome,
                            int32_t K, int32_t max_iterations, int32_t check_every, uint8_t *hard,
                            float *llr_post, uint8_t *ok, int32_t *iterations_used,
                            const qcmet_decode_options *opts, void *stream);

/*
 * qcmet_decode_ex for callers whose data live in host memory: every pointer
 * is a host pointer (pinned memory gives the fastest copies).  The call
 * copies the inputs to library-owned device buffers on `stream`, decodes,
 * copies hard / llr_post (if not NULL) / ok back, and synchronises `stream`
 * before it returns.
 */
int qcmet_decode_host(const qcmet_code *code, const float *llr_ch, const uint8_t *syndrome,
                      int32_t K, int32_t iterations, uint8_t *hard, float *llr_post, uint8_t *ok,
                      const qcmet_decode_options *opts, void *stream);

/*
 * qcmet_decode with FP32 messages for callers that cannot allocate device
 * memory.  The paper has no counterpart; this is a service of this library.
 *
 * Who needs it: code that must not call cudaMalloc -- for example a
 * reconciliation pipeline that keeps several streams busy and cannot afford
 * the device-wide synchronisation an allocation implies, or a plug-in whose
 * host application owns all device memory through its own pool.
 * qcmet_decode allocates scratch on a handle's first use (and when K grows);
 * this call allocates nothing: it calls no cudaMalloc, cudaFree or other
 * allocating routine.
 *
 * Its scratch is one fixed array of 32 MiB that the library defines in device
 * memory; every GPU that loads the library holds it until the process exits.
 * 64 KiB of it hold a copy of the code's layer table, the rest the messages
 * and the posteriors of the core columns (degree > 1): the call needs
 * roundup(K * msg_slots * roundup(Z, 16) * 4, 256) + K * core_columns * Z * 4
 * bytes of the remaining 32 MiB - 64 KiB and returns QCMET_ERR_INVALID_ARG,
 * with a message that states both sizes, when that does not fit (e.g. at
 * Z = 12500, 230 slots and 10 core columns it takes at most 2 frames per
 * call; at Z = 64, over 400).
 *
 * Arguments, layouts and results are those of qcmet_decode, except that
 * llr_post must not be NULL (the degree-1 posteriors are written there while
 * decoding) and no options are taken (FP32 messages, default block size).  The results equal
 * qcmet_decode's bit for bit.
 *
 * All calls share the one array and it keeps what the last call left; this
 * call rewrites everything it reads before reading it.  Calls whose work can
 * overlap on the GPU (different streams, or host threads) race on the array:
 * order them on one stream.  Each call copies the code's layer table (a few
 * KiB) from host memory into the array with cudaMemcpyAsync on `stream`.
 *
 * Set-up: the first call on each device (with that device current) looks up
 * the array's device address with cudaGetSymbolAddress, a synchronous runtime
 * call, and keeps it for that device's CUDA context.  A new context on the
 * device (e.g. after cudaDeviceReset) is detected by its context id, and the
 * next call looks the address up again.
 * The array itself is placed in device memory when CUDA loads the library's
 * device code on that device (by default, lazily, at the library's first
 * kernel launch or symbol lookup there), not by this call.
 */
int qcmet_decode_noalloc(const qcmet_code *code, const float *llr_ch, const uint8_t *syndrome,
                         int32_t K, int32_t iterations, uint8_t *hard, float *llr_post,
                         uint8_t *ok, void *stream);

/*
 * Learned offset/scaled min-sum (not part of the paper's method; a variant of
 * its layered decoder, Methods steps 1-4, whose check rule of step 2 becomes)
 *   r_e = (-1)^{s_m} prod_{k != e} sgn(q_k) * min(max(a_e, 0), 30),
 *   a_e = w_scale[t][l][type_e] * min_{k != e} |q_k| - w_offset[t][l][type_e]
 * for iteration t, base row l, and edge type 0 (edge to a variable of degree
 * > 1) or 1 (edge to a degree-1 variable).  The clip at 30 is the one the
 * sum-product rule uses; without it unscaled min-sum can grow posteriors past
 * the FP32 range.  Weights are device FP32 arrays of shape [iterations][mb][2],
 * row-major.
 *
 * qcmet_minsum_decode: decode with given weights; outputs as qcmet_decode
 *   (FP32 messages, llr_post may be NULL); the grouped kernel for four frames
 *   or more, the frame kernel otherwise (identical results).
 * qcmet_minsum_forward: training forward.  bits = device [K][n] uint8
 *   transmitted bits; loss = device [K] FP32 out, per frame the mean over
 *   iterations t and variables n of softplus(-(1 - 2 x_n) L_qn^(t)), the
 *   cross-entropy of sigma(-L) against the bits, L^(t) the posterior after
 *   iteration t.  Keeps what the backward needs in the handle's scratch
 *   (about K * iterations * (msg_slots + core columns) * Z * 4 bytes); the
 *   inputs and weights must stay untouched until the backward has run.
 * qcmet_minsum_backward: gradient of the SUM of the last forward's losses with
 *   respect to the weights, written to g_scale and g_offset ([iterations][mb][2]
 *   device FP32, overwritten).  INVALID_ARG without a preceding forward.
 * All three are stream-ordered; the same handle must not run them concurrently.
 */
int qcmet_minsum_decode(const qcmet_code *code, const float *llr_ch, const uint8_t *syndrome,
                        int32_t K, int32_t iterations, const float *w_scale, const float *w_offset,
                        uint8_t *hard, float *llr_post, uint8_t *ok, void *stream);
int qcmet_minsum_forward(const qcmet_code *code, const float *llr_ch, const uint8_t *syndrome,
                         const uint8_t *bits, int32_t K, int32_t iterations, const float *w_scale,
                         const float *w_offset, float *loss, void *stream);
int qcmet_minsum_backward(const qcmet_code *code, float *g_scale, float *g_offset, void *stream);

/*
 * Mixed batches: frames of different codes (rates, lengths) decoded by ONE
 * launch of the layered decoder, so that short and long codewords share the
 * GPU (the paper decodes many codewords of one code at once, Results,
 * multi-codeword decoding; mixing codes is this library's extension).
 *
 * A batch is a plan over fixed buffers: qcmet_batch_create records the frames,
 * allocates the messages (and posteriors where llr_post is NULL), chooses a
 * launch configuration and captures the launch in a CUDA graph;
 * qcmet_batch_run replays that graph on `stream` (asynchronous).  To decode
 * new data, write it into the same input buffers and run again.
 *
 * Two kernels can serve a batch (the choices of qcmet_decode_options.kernel):
 * the frame kernel, whose persistent thread blocks take frames from a work
 * counter, and the grouped kernel, whose persistent thread-block clusters
 * take groups of up to four frames of one code (consecutive frames of that
 * code in the batch, stored interleaved in the plan's scratch) from a work
 * counter.  Autotuning (autotune = 1) times, on this batch with
 * min(iterations, 12) iterations, every combination of kernel and its size
 * (block of 512 or 1024 threads; cluster of 2, 4, 5, 8 or 16 blocks, sizes the
 * device cannot hold skipped; or the grouped kernel as one concurrent launch
 * per code, each code's groups given a cluster size and one or two blocks per
 * SM so that all codes share the device's SMs and finish together), layer schedule
 * (each code's own, or the other schedule that gives identical results:
 * base-row order <-> merged rows, Results Eqs. (m1), (m2)) and work order
 * (largest first, or as given), times the four fastest again with
 * min(iterations, 100) iterations, and keeps the fastest.  All candidates give
 * the same results, so the choice affects time only.  Autotuning runs trial
 * decodes, so the inputs must be valid and the outputs writable at creation.
 * Without autotuning (autotune = 0) the plan takes the grouped kernel with
 * clusters of 4; autotune = 2 takes the per-code concurrent launches without
 * timing anything.
 */
typedef struct {
    const qcmet_code *code;   /* the frame's code                          */
    const float *llr_ch;      /* device [n] channel LLRs                   */
    const uint8_t *syndrome;  /* device [m] syndrome bits                  */
    uint8_t *hard;            /* device [n] out                            */
    float *llr_post;          /* device [n] out, or NULL                   */
    uint8_t *ok;              /* device [1] out, 1 iff H*hard = syndrome   */
} qcmet_frame;

typedef struct qcmet_batch qcmet_batch;

typedef struct {
    int32_t threads_per_block;   /* frame kernel: chosen block size (0 for the grouped) */
    int32_t alternate_schedule;  /* 1: the codes' other exact schedule was faster       */
    int32_t largest_first;       /* 1: work is taken in decreasing edge count          */
    int32_t candidates;          /* configurations timed (1 without autotuning)        */
    float trial_ms;              /* the winner's trial time: one decode of min(iterations,
                                    100) iterations (two of 12 when iterations <= 12;
                                    -1 if nothing was timed)                          */
    int32_t kernel;              /* QCMET_KERNEL_FRAME or QCMET_KERNEL_GROUP            */
    int32_t cluster_size;        /* grouped kernel, one launch: blocks per cluster (else 0) */
    int32_t per_code_launches;   /* grouped kernel, one concurrent launch per code: the
                                    number of launches (else 0)                        */
} qcmet_batch_config;

/* frames: host array [K] (copied); msg_format: QCMET_MSG_*.  Pointers must be
 * 16-byte aligned.  Errors: INVALID_ARG, ALIGNMENT, OOM, CUDA. */
int qcmet_batch_create(const qcmet_frame *frames, int32_t K, int32_t iterations,
                       int32_t msg_format, int32_t autotune, void *stream, qcmet_batch **out);
int qcmet_batch_run(qcmet_batch *batch, void *stream);
int qcmet_batch_get_config(const qcmet_batch *batch, qcmet_batch_config *out);
/* Frees the plan (not the codes or the caller's buffers).  NULL is a no-op. */
void qcmet_batch_destroy(qcmet_batch *batch);

/*
 * The launch shape a grouped-kernel decode of K frames of `code` with these
 * options (NULL = defaults; msg_format and cluster_size are used) would take on
 * the current device: clusters of cluster_size blocks, each owning
 * groups_per_cluster groups of four frames (1 or 2; with 2 the cluster's blocks
 * split the two groups' checks between them), threads_per_block threads and
 * shared_bytes of dynamic shared memory per block; `clusters` clusters, `blocks`
 * blocks in all, of which the device holds active_clusters clusters at once.
 * The library chooses the shape to minimise the checks each SM owns per row
 * (times the waves of clusters); the choice changes no result.  Nothing runs
 * on the device.  Errors: INVALID_ARG, UNSUPPORTED (no shape schedulable),
 * CUDA.
 */
typedef struct {
    int32_t cluster_size;
    int32_t groups_per_cluster;
    int32_t threads_per_block;
    int32_t clusters;
    int32_t blocks;
    int32_t active_clusters;
    int32_t shared_bytes;
    int32_t reserved;
} qcmet_group_plan_t;
int qcmet_group_plan(const qcmet_code *code, int32_t K, const qcmet_decode_options *opts,
                     qcmet_group_plan_t *plan);

/*
 * Index checks of the debug build.  libqcmet_debug.so (the same sources built
 * with QCMET_DEBUG_CHECKS=1) tests every index its kernels gather or scatter
 * -- posteriors and channel LLRs, message slots, syndrome bits -- against the
 * extent of its array and skips an access that would leave it, recording the
 * kind: bit 0 a variable index, bit 1 a message slot, bit 2 a check index.
 * This call waits for the current device to finish its work, returns the bits
 * recorded since the last call in *violations and clears them.  The release
 * build compiles no checks: it sets *violations = 0 and returns
 * QCMET_ERR_UNSUPPORTED.  Errors: INVALID_ARG (NULL), CUDA.
 */
int qcmet_debug_checks(uint32_t *violations);

/* Message of the last failing call on this thread ("" if none). */
const char *qcmet_last_error(void);

/* Fixed description of a status code. */
const char *qcmet_status_string(int status);

/* QCMET_VERSION of the loaded library. */
int qcmet_version(void);

#ifdef __cplusplus
}
#endif

#endif /* QCMET_H */
