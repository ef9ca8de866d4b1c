/*
 * boa.h -- C-ABI of the B300 BOA Constrictor library (libboa.so).
 *
 * BOA Constrictor (arXiv 2511.11337) compresses bytes losslessly by pairing a
 * small autoregressive Mamba next-byte predictor with a range coder.  The
 * input is split into independent streams; all active streams are stepped
 * together on the GPU, each with its own coder, and the first byte of every
 * stream is stored raw (paper, section "Coders & Parallelisation").
 *
 * Conventions for every call:
 *   - Return value: BOA_OK (0) or an error code; on error the thread-local
 *     message from boa_last_error() says what went wrong.  A failed call
 *     leaves caller buffers in an unspecified state but never writes past
 *     the capacities it was given.
 *   - Ownership: every buffer is owned by the caller; the library keeps no
 *     pointer to it after the call returns.  A boa_model owns its device
 *     weights and its device workspace (grown on demand, freed by
 *     boa_free_model).
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *     global memory on the model's device.
 *   - Calls on one model are re-entrant: any number of host threads may call
 *     into the same model at once.  Each such call holds the model's lock
 *     for its whole duration (its workspace, tuning, profiling counters and
 *     tensor-map cache are shared), so concurrent calls on one model run one
 *     after another on the model's CUDA stream and give the same bytes as
 *     the same calls made in sequence.  For calls that run at the same time
 *     on the GPU, use one model object per host thread: each has its own
 *     stream and workspace.  boa_free_model must not race with other calls
 *     on the same model.
 *   - Per-stream byte format: out[0] = the stream's first byte (raw), then
 *     the range coder's bytes including its 4-byte flush.  A stream of
 *     length 0 compresses to 0 bytes and a stream of length 1 to 1 byte.
 */
#ifndef BOA_H
#define BOA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BOA_OK = 0,
    BOA_ERR_ARG = 1,                /* invalid argument (null pointer, bad size) */
    BOA_ERR_IO = 2,                 /* weight file could not be read */
    BOA_ERR_FORMAT = 3,             /* weight file malformed or unsupported shape */
    BOA_ERR_CUDA = 4,               /* CUDA runtime error or no usable GPU */
    BOA_ERR_OOM = 5,                /* device allocation failed */
    BOA_ERR_OUTPUT_TOO_SMALL = 6,   /* an output capacity is below boa_max_compressed_size */
    BOA_ERR_CORRUPT = 7,            /* a coded stream did not decode cleanly */
    BOA_ERR_FINGERPRINT = 8         /* data was produced by a different model */
} boa_status;

typedef enum {
    BOA_PREC_FP32 = 0,              /* all projections in FP32 on the CUDA cores */
    BOA_PREC_BF16 = 1,              /* projections in BF16 on the tensor cores (tcgen05), FP32
                                       accumulation; norms, conv, scan, softmax and CDF stay FP32 */
    BOA_PREC_TF32X3 = 2,            /* FP32-accurate projections on the tensor cores: operands split
                                       into TF32 hi + lo parts, three products accumulated in FP32 */
    BOA_PREC_FP8 = 3                /* projections in FP8 E4M3 on the tensor cores, FP32 accumulation;
                                       weights scaled per output channel, activations per row */
} boa_precision;

typedef struct {
    int device;                     /* CUDA device ordinal */
    int precision;                  /* boa_precision */
    void* cuda_stream;              /* cudaStream_t to run on; NULL = library-owned stream */
    size_t max_rows;                /* compression workspace: rows (slot x step) per
                                       chunk; 0 = 262144 (about 3 GB at d_model 256) */
    size_t max_slots;               /* streams in flight at once; 0 = 8192.  Longer inputs are
                                       queued: a slot takes its next stream when one finishes */
} boa_opts;

typedef struct boa_model boa_model; /* opaque; owned by the library */

/* Load a weight file and upload it to the GPU.
 * Paper: the predictor Q is an embedding, n_l Mamba blocks and a linear head
 * (Alg. 1 "Forward Pass"; section "Range coding", paragraph "Alphabet,
 * sequence, and model").  The file is a 40-byte header (magic "BOAW",
 * version 1, then u32 vocab=256, d_model, n_layer, d_state, d_conv, expand,
 * dt_rank, ffn_mult) followed by little-endian float32 tensors in the fixed
 * order embed, per layer {ln_a.w, ln_a.b, in_proj.w[2E][d], conv.w[E][K],
 * conv.b, x_proj.w[r+2N][E], dt_proj.w[E][r], dt_proj.b, A_log[E][N], D,
 * out_proj.w[d][E], (ffn.w1[F][d], ffn.b1, ffn.w2[d][F], ffn.b2 when
 * ffn_mult > 0), ln_b.w, ln_b.b}, head.w[256][d], head.b.
 * opts may be NULL (device 0, FP32, library stream).  Errors: BOA_ERR_IO,
 * BOA_ERR_FORMAT, BOA_ERR_CUDA, BOA_ERR_OOM.  *out is set only on success. */
boa_status boa_load_model(const char* path, const boa_opts* opts, boa_model** out);

/* Release the model, its device weights and workspace.  NULL is a no-op. */
void boa_free_model(boa_model* model);

/* 64-bit FNV-1a hash of the weight file bytes: the model fingerprint that
 * the paper's container records (section "Coders & Parallelisation"). */
uint64_t boa_model_fingerprint(const boa_model* model);

/* Worst-case compressed size of a stream of len bytes: 1 raw byte plus at
 * most 5 coder bytes per coded symbol plus the 4-byte flush
 * (0 -> 0, 1 -> 1, n -> 1 + 5 (n - 1) + 4). */
size_t boa_max_compressed_size(size_t len);

/* Compress n_streams independent streams (host memory in and out).
 * Paper: section "Range coding" (softmax, integer CDF, encoder update and
 * renormalisation) driven by the step function of paragraph "Alphabet,
 * sequence, and model", all streams stepped together (section "Coders &
 * Parallelisation").  streams[i] holds lens[i] bytes; out[i] has room for
 * out_caps[i] bytes; out_sizes[i] receives the bytes written.  Errors:
 * BOA_ERR_ARG, BOA_ERR_OUTPUT_TOO_SMALL (checked before any work, against
 * boa_max_compressed_size), BOA_ERR_CUDA, BOA_ERR_OOM. */
boa_status boa_compress(boa_model* model, size_t n_streams, const uint8_t* const* streams,
                        const size_t* lens, uint8_t* const* out, const size_t* out_caps,
                        size_t* out_sizes);

/* Decompress streams produced by boa_compress with the same model.
 * Paper: section "Range coding", paragraph "Decoder" (target value x,
 * symbol search, identical update, code-value shift-in), streams that have
 * finished are masked out of each step (section "Coders & Parallelisation").
 * bitstreams[i] holds sizes[i] bytes and decodes to lens[i] bytes in out[i]
 * (caller-sized to lens[i]).  Errors: BOA_ERR_ARG, BOA_ERR_CORRUPT (a stream
 * read past its end or left bytes unread; its output is then unreliable),
 * BOA_ERR_CUDA, BOA_ERR_OOM. */
boa_status boa_decompress(boa_model* model, size_t n_streams, const uint8_t* const* bitstreams,
                          const size_t* sizes, const size_t* lens, uint8_t* const* out);

/* Device-resident forms of the two calls above: each batch lives in one
 * device buffer cut into slots.
 * d_in: device; stream i occupies slot [in_offsets[i], in_offsets[i+1]).
 * d_out: device; stream i may write slot [out_offsets[i], out_offsets[i+1]).
 * in_offsets, out_offsets: host arrays of n_streams + 1 non-decreasing
 * offsets.  Compression: slot i of d_in is the whole stream; out_sizes (host)
 * receives each stream's byte count.  Decompression: in_sizes (host, may be
 * NULL = whole slot) gives the coded bytes at the start of each input slot,
 * so the compressor's output buffer can be decoded in place; lens (host)
 * gives each stream's decoded length and output slot i must hold lens[i]
 * bytes.  Same errors as the host forms. */
boa_status boa_compress_device(boa_model* model, size_t n_streams, const uint8_t* d_in,
                               const uint64_t* in_offsets, uint8_t* d_out,
                               const uint64_t* out_offsets, uint64_t* out_sizes);
boa_status boa_decompress_device(boa_model* model, size_t n_streams, const uint8_t* d_in,
                                 const uint64_t* in_offsets, const uint64_t* in_sizes,
                                 const uint64_t* lens, uint8_t* d_out, const uint64_t* out_offsets);

/* Number of kernel launches the last compress / decompress call issued
 * (counted by the host as it enqueues them). */
uint64_t boa_last_launch_count(const boa_model* model);

/* Per-stream status of the last compress / decompress call on this model
 * (host out, its first n streams): 0 for a stream that was coded cleanly,
 * else bits 1 = encoder output capacity exceeded, 2 = the decoder met an
 * impossible state or its stream's coded length did not match (corrupt or
 * truncated input), 4 = renormalisation exceeded its proven bound.  A call
 * that failed with BOA_ERR_CORRUPT names the first such stream; this lists
 * all of them.  Errors: BOA_ERR_ARG (n above the last call's stream count). */
boa_status boa_last_stream_status(const boa_model* model, size_t n, uint32_t* status);

/* Kernel classes for boa_profile_read. */
typedef enum {
    BOA_KC_EMBED_LN = 0,    /* byte embedding + first LayerNorm */
    BOA_KC_GEMM_IN = 1,     /* in_proj */
    BOA_KC_CONV = 2,        /* causal depthwise conv + SiLU */
    BOA_KC_GEMM_X = 3,      /* x_proj */
    BOA_KC_SCAN = 4,        /* dt_proj + softplus + selective scan + gate */
    BOA_KC_GEMM_OUT = 5,    /* out_proj + residual */
    BOA_KC_GEMM_FFN = 6,    /* FFN projections (paper-shape blocks) */
    BOA_KC_LN = 7,          /* block-output LayerNorm (+ next block's input norm) */
    BOA_KC_GEMM_HEAD = 8,   /* head */
    BOA_KC_ENCODE = 9,      /* softmax -> CDF -> range encoder */
    BOA_KC_DECODE = 10,     /* softmax -> CDF -> range decoder */
    BOA_KC_OTHER = 11,      /* set-up, flush, compaction */
    BOA_KC_COUNT = 12
} boa_kernel_class;

/* Benchmark hook: when on, kernel launches of timed steps are bracketed by a
 * pair of CUDA events on the model's stream, and per-(phase, class) totals
 * accumulate: launches timed, summed device milliseconds, and the
 * algorithmic FLOPs and DRAM bytes those launches must at least perform.
 * phase: 0 = compression (every chunk is timed), 1 = decompression: where
 * the decode step loop runs as CUDA graphs of 32 steps, the eager step
 * before each graph launch (and the first step) is timed; otherwise every
 * decode_step_stride-th step.  A timed decode step runs its lanes one after
 * another on the model's stream.  Reset clears totals and step counts. */
boa_status boa_profile_enable(boa_model* model, int on, int decode_step_stride);
boa_status boa_profile_reset(boa_model* model);
boa_status boa_profile_read(const boa_model* model, int phase, int kernel_class, uint64_t* launches,
                            double* total_ms, double* flops, double* bytes);

/* Steps (compression chunks, decode steps) of a phase since the last reset:
 * how many were timed and how many ran in all (host out, may be NULL). */
boa_status boa_profile_steps(const boa_model* model, int phase, uint64_t* timed, uint64_t* total);

/* Launch configuration chosen by boa_autotune. */
typedef struct {
    size_t max_rows;        /* compression rows (slot x step) per chunk */
    int scan_variant;       /* decompression scan kernel: 0 = persistent, bulk-copy fed;
                               1 = four channels per thread, one stream per CTA;
                               2 = one channel per thread, one stream per CTA;
                               3 = one channel per thread, eight streams per CTA */
    int decode_lanes;       /* decompression: slots split into this many independent
                               groups whose steps run on separate CUDA streams
                               (0 = automatic: 2 from 2048 slots, else 1) */
    double compress_ms;     /* estimated time for the whole workload */
    double decompress_ms;
    int decoder;            /* decompression: 0 = one launch sequence per step, model state
                               in HBM (every form); 1 = the on-chip persistent decoder
                               (FP32 form; models of at most 3 blocks without FFN,
                               d_state 16, d_inner <= 512): one launch, one CTA per SM
                               decoding two streams at a time from first to last byte,
                               their SSM state and conv windows in the SM's tensor memory
                               across layers and steps (Alg. 1; App. B: O(1) state per
                               stream).  Both give the same bytes. */
} boa_tuning;

/* Time candidate launch configurations on a synthetic batch shaped like the
 * caller's workload (n_streams streams of stream_len bytes; a 512-byte sample
 * of each is run) and keep the fastest in the model: the compression chunk
 * size (max_rows in 2^16 .. 2^19), the decode scan kernel (scan_variant),
 * the decode lanes (1, 2 or 4) and, where it runs, the on-chip decoder.  No knob changes any result: rows are
 * computed the same way whatever the chunking, kernel or lane split.  out (host, may be NULL) receives
 * the choice and the extrapolated times.  Allocates and frees a scratch
 * batch on the device.  Errors: BOA_ERR_ARG, BOA_ERR_CUDA, BOA_ERR_OOM. */
boa_status boa_autotune(boa_model* model, size_t n_streams, size_t stream_len, boa_tuning* out);

/* Apply a launch configuration (for instance one saved from an earlier
 * boa_autotune): max_rows in 1 .. 2^24, scan_variant in 0 .. 3,
 * decode_lanes in 0 .. 16, decoder 0 or 1 (1 only where the model and form
 * allow it); the _ms fields are ignored.  Results do not depend on it.
 * Errors: BOA_ERR_ARG (out of range, or decoder 1 on a model or form it
 * does not run; boa_last_error says why). */
boa_status boa_set_tuning(boa_model* model, const boa_tuning* tuning);

/* The configuration in use (host out; the _ms fields are zero). */
boa_status boa_get_tuning(const boa_model* model, boa_tuning* out);

/* ------------------------------------------------------------ container
 * The .boa container of the paper (section "Coders & Parallelisation"): the
 * input cut into chunks of chunk_len bytes (the last one shorter), each
 * compressed as one stream (its first byte raw), plus the total length, the
 * nominal and last chunk lengths, the model fingerprint and a CRC-32
 * protected index of per-chunk payload offsets and sizes.  Byte layout:
 * 56-byte header ("BOA1", u32 version 1, u64 fingerprint, u64 total length,
 * u64 chunk length, u64 chunk count n, u64 last chunk length, u32 CRC-32 of
 * header bytes 0..47, u32 CRC-32 of the index), n x (u64 offset, u64 size),
 * payload.  All buffers are host memory owned by the caller. */

/* Capacity boa_pack needs for len bytes in chunks of chunk_len (0 if chunk_len is 0). */
size_t boa_pack_bound(size_t len, size_t chunk_len);

/* Compress data into a container.  Errors: BOA_ERR_ARG, BOA_ERR_OUTPUT_TOO_SMALL
 * (cap < boa_pack_bound), and those of boa_compress. */
boa_status boa_pack(boa_model* model, const uint8_t* data, size_t len, size_t chunk_len, uint8_t* out,
                    size_t cap, size_t* out_size);

/* Read a container header (no model needed): total length and fingerprint.
 * Errors: BOA_ERR_FORMAT (not a container), BOA_ERR_CORRUPT (short or header CRC). */
boa_status boa_unpack_info(const uint8_t* container, size_t size, uint64_t* total_len, uint64_t* fingerprint);

/* Decompress a container into out (cap >= its total length); *out_len gets the
 * length.  Errors: BOA_ERR_FINGERPRINT (written with another model),
 * BOA_ERR_CORRUPT (header or index CRC, inconsistent layout, a chunk that does
 * not decode cleanly), BOA_ERR_OUTPUT_TOO_SMALL, and those of boa_decompress. */
boa_status boa_unpack(boa_model* model, const uint8_t* container, size_t size, uint8_t* out, size_t cap,
                      size_t* out_len);

/* CRC-32, IEEE 802.3 polynomial (the container's checksum). */
uint32_t boa_crc32(const uint8_t* data, size_t n);

/* Decompress a concatenation of containers (the shards boa_stream_* writes,
 * or any containers written with this model, laid end to end) into out, one
 * after another; *out_len gets the total length.  All their chunks are
 * decoded in one batch.  out = NULL with cap = 0 only validates the
 * containers and returns the total length.  Errors: those of boa_unpack,
 * for the first container that fails. */
boa_status boa_unpack_shards(boa_model* model, const uint8_t* data, size_t size, uint8_t* out, size_t cap,
                             size_t* out_len);

/* ------------------------------------------------------------ streaming
 * The streaming pipeline of the paper (section "Streaming", Fig. 2): chunks
 * are buffered while the previous set compresses, and the next set is
 * pre-loaded.  Bytes the caller pushes are cut into chunks of chunk_len
 * bytes and gathered, in pinned host memory, into sets of set_chunks
 * chunks.  A full set is copied to the device on the pipeline's own copy
 * stream and compressed, as one batch of set_chunks streams, by the
 * pipeline's worker thread.  Meanwhile the caller fills the other set buffer
 * and its copy pre-loads the device.  Each set becomes one shard, a complete
 * container (format above) of that set's bytes, appended to the pipeline's
 * output in input order; boa_unpack decodes one shard, boa_unpack_shards a
 * concatenation.  Two set buffers exist, so a push waits while both are in
 * use.  While a pipeline is open its worker thread owns the model: make no
 * other call on that model until boa_stream_close.  A worker error (those
 * of boa_compress, BOA_ERR_CUDA) is returned by the next push or finish;
 * the pipeline then accepts no more data. */
typedef struct boa_stream boa_stream;

/* Open a pipeline on model.  Allocates 2 x chunk_len x set_chunks bytes of
 * pinned host and of device memory.  Errors: BOA_ERR_ARG (zero or oversized
 * set), BOA_ERR_OOM, BOA_ERR_CUDA. */
boa_status boa_stream_open(boa_model* model, size_t chunk_len, size_t set_chunks, boa_stream** out);

/* Append len bytes (caller-owned, read before the call returns).  Every set
 * that fills is handed to the worker.  Errors: BOA_ERR_ARG (after finish),
 * a worker error. */
boa_status boa_stream_push(boa_stream* stream, const uint8_t* data, size_t len);

/* Hand over the partial last set, if any, and wait until every shard is
 * written.  Later pushes fail; reads continue. */
boa_status boa_stream_finish(boa_stream* stream);

/* Bytes of finished shards not yet read. */
size_t boa_stream_available(const boa_stream* stream);

/* Copy up to cap bytes of finished shards, in order, into out (host);
 * *out_size gets the count. */
boa_status boa_stream_read(boa_stream* stream, uint8_t* out, size_t cap, size_t* out_size);

/* Bytes handed to the worker, shards written, and how many of those sets
 * were already on the device when the worker took them (pre-loaded while the
 * previous set compressed).  Any pointer may be NULL. */
boa_status boa_stream_stats(const boa_stream* stream, uint64_t* bytes_in, uint64_t* sets, uint64_t* preloaded);

/* Stop the pipeline (sets already handed over are still compressed) and free
 * it.  NULL is ignored. */
void boa_stream_close(boa_stream* stream);

/* ------------------------------------------------------------ training
 * The selective scan for training the predictor (paper App. A recurrence
 * h_t = exp(delta_t A) h_{t-1} + delta_t B_t u_t, y_t = C_t . h_t + D u_t,
 * h_0 = 0, and its reverse-mode gradient), on whole sequences with states
 * recomputed per chunk instead of stored.  All pointers are device memory
 * (float32) owned by the caller; work is queued on cuda_stream (NULL =
 * legacy default stream) and the calls return without waiting.  d_state N
 * must be 16.  Layouts: u, delta, y, dy, du, ddelta [Bsz][T][E]; Bm, Cm
 * [Bsz][T][N]; A [E][N]; D [E]; hin [Bsz][ceil(T/chunk)][N][E] (states
 * entering each chunk, written by the forward, read by the backward);
 * scratch [Bsz][chunk][N][E]; dA_part [Bsz][E][N] and dD_part [Bsz][E]
 * (sum over Bsz for dA, dD); dB_part, dC_part [Bsz][T][ceil(E/128)][N]
 * (sum over the third axis for dB, dC).  Errors: BOA_ERR_ARG, BOA_ERR_CUDA. */
boa_status boa_scan_train_fwd(size_t Bsz, size_t T, size_t E, size_t N, size_t chunk, const float* u,
                              const float* delta, const float* A, const float* Bm, const float* Cm,
                              const float* D, float* y, float* hin, void* cuda_stream);
boa_status boa_scan_train_bwd(size_t Bsz, size_t T, size_t E, size_t N, size_t chunk, const float* u,
                              const float* delta, const float* A, const float* Bm, const float* Cm,
                              const float* D, const float* dy, const float* hin, float* scratch,
                              float* du, float* ddelta, float* dA_part, float* dD_part, float* dB_part,
                              float* dC_part, void* cuda_stream);

/* One training step of the predictor (paper, "Entropy-Based Compression and
 * Cross-Entropy Loss": minimising the base-256 cross-entropy minimises the
 * code length), entirely in the library's kernels: the forward over
 * n_seq x (seqlen - 1) rows, the reverse-mode gradient of the mean
 * cross-entropy in bytes per byte, -log_256 Q(y_t | y_<t) averaged over
 * every predicted position, and one AdamW step (betas 0.9 / 0.999, eps 1e-8,
 * decoupled weight decay 0.01 on every tensor, bias-corrected) of the weight
 * file's tensor array with learning rate lr.  The model then uses the
 * updated weights (its device copies in every precision form are rebuilt)
 * and its fingerprint becomes that of the file boa_save_model would write.
 * Arithmetic follows the model's precision form.  FP32 (and the other
 * forms except BF16): FP32 on the CUDA cores.  BF16 (BOA_PREC_BF16): the
 * projections, the input gradients of in_proj, out_proj and the head, and
 * the weight gradients of in_proj, x_proj, out_proj and the head run on the
 * tensor cores with BF16 operands and FP32 accumulation (weight gradients in
 * fixed 4096-row parts added in order); everything else, the FP32 master
 * weights and AdamW stay FP32.  Either way sums run in a fixed order (the
 * same batch gives the same update bit for bit); the Adam moments live in
 * the model.
 * batch: host, n_seq x seqlen bytes, row-major; sequence b predicts its
 * bytes 1..seqlen-1 from their prefixes.  loss_out (host, may be NULL): the
 * loss before the update.  Blocks with an FFN (ffn_mult > 0) are not
 * supported; at most 2^22 predicted positions per batch.  Memory: about
 * 80 bytes x E per predicted position on the device.
 * Errors: BOA_ERR_ARG, BOA_ERR_CUDA, BOA_ERR_OOM. */
boa_status boa_train_step(boa_model* model, const uint8_t* batch, size_t n_seq, size_t seqlen, float lr,
                          float* loss_out);

/* Write the model's current weights as a weight file (header of the file it
 * was loaded from, then its tensor array).  Errors: BOA_ERR_ARG, BOA_ERR_IO. */
boa_status boa_save_model(const boa_model* model, const char* path);

/* Number of floats in the model's tensor array (the weight file's layout). */
size_t boa_model_param_count(const boa_model* model);

/* Thread-local message describing the last error on this thread. */
const char* boa_last_error(void);

/* ----------------------------------------------------------- test hooks
 * Exposed for parity tests; not part of the compression API. */

/* The loss and gradient boa_train_step would use for this batch, without
 * updating anything: grad_out (host, boa_model_param_count floats, may be
 * NULL) in the weight file's layout, the gradient of the mean base-256
 * cross-entropy; loss_out (host, may be NULL).  Errors as boa_train_step. */
boa_status boa_debug_train_grad(boa_model* model, const uint8_t* batch, size_t n_seq, size_t seqlen,
                                float* grad_out, float* loss_out);

/* Range-code given integer CDFs on the GPU (section "Range coding",
 * paragraphs "Encoder" and "Decoder").  n_seq independent sequences; sequence
 * i has n_syms[i] symbols, its CDF rows start at row sum_{j<i} n_syms[j] of
 * cdfs ([rows][257] u32, cdf[0] = 0, cdf[256] = 65536, strictly increasing)
 * and its symbols at the same offset of syms.  Encoder output for sequence i
 * goes to out + i * out_stride (capacity out_stride >= 5 n + 4), its size to
 * sizes[i].  The decoder reads in + i * in_stride (in_sizes[i] bytes) and
 * writes n_syms[i] symbols.  All pointers are host memory.  Errors:
 * BOA_ERR_ARG, BOA_ERR_CORRUPT (decoder), BOA_ERR_CUDA. */
boa_status boa_debug_encode_cdfs(size_t n_seq, const size_t* n_syms, const uint32_t* cdfs,
                                 const uint8_t* syms, uint8_t* out, size_t out_stride,
                                 size_t* sizes);
boa_status boa_debug_decode_cdfs(size_t n_seq, const size_t* n_syms, const uint32_t* cdfs,
                                 const uint8_t* in, size_t in_stride, const size_t* in_sizes,
                                 uint8_t* syms);

/* Integer histogram from float32 probabilities with the kernel's quantiser
 * (paper "Probabilities and integer CDF": f >= 1, sum f = 2^16):
 * f_a = 1 + floor(p_a * 65280) in float32, remainder to the most probable
 * symbol (lowest index on ties).  p: host [n_rows][256]; f: host [n_rows][256]. */
boa_status boa_debug_quantise(size_t n_rows, const float* p, uint32_t* f);

/* Teacher-forced log2 next-byte probabilities of one stream from the
 * compression path: out (host) [(len-1)][256], row t predicting byte t+1. */
boa_status boa_debug_logprobs(boa_model* model, const uint8_t* stream, size_t len, float* out);

/* One projection GEMM on the GPU, for kernel tests:
 * C_out[M][N] = epi(A[M][K] . W[N][K]^T) with the library's FP32 CUDA-core
 * kernel (precision BOA_PREC_FP32), its tcgen05 tensor-core kernel with
 * A and W rounded to BF16 (BOA_PREC_BF16), or its 3xTF32 tensor-core kernel
 * (BOA_PREC_TF32X3), or its E4M3 kernel with W scaled per row of W and
 * A per row of A (BOA_PREC_FP8).  epilogue: 0 store, 1 + bias[n],
 * 2 C_in + acc, 3 GELU(acc + bias[n]), 4 C_in + (acc + bias[n]).  All pointers
 * host memory; N % 4 == 0; K % 8 == 0 (FP32), K % 64 == 0 (BF16),
 * K % 32 == 0 (TF32X3) or K % 16 == 0 (FP8; K is zero-padded to a multiple
 * of 128 inside).  Device 0. */
boa_status boa_debug_gemm(int precision, size_t M, size_t N, size_t K, const float* A, const float* W,
                          const float* bias, int epilogue, const float* C_in, float* C_out);

/* When on, the next compress / decompress calls record a 64-bit hash of the
 * integer CDF used at every coded step; boa_debug_read_cdf_trace copies the
 * hashes of the last call, stream-major ([stream][step], sum(len-1) values). */
boa_status boa_debug_enable_cdf_trace(boa_model* model, int on);
boa_status boa_debug_read_cdf_trace(boa_model* model, uint64_t* out, size_t n);

/* Microbenchmarks of the units the hot path's rooflines are quoted
 * against (the paper gives no such figures; its throughput discussion names
 * GPU matrix multiplications as the bottleneck).  Each runs a fixed stream of
 * independent operations on every SM of `device` and is timed with CUDA
 * events; *rate receives the whole GPU's rate:
 *   BOA_MB_EX2    ex2.approx.ftz.f32 results per second (the MUFU unit that
 *                 computes the scan's exp(Delta A))
 *   BOA_MB_FFMA   FP32 FLOP/s of scalar FMAs on the CUDA cores
 *   BOA_MB_FFMA2  FP32 FLOP/s of packed fma.rn.f32x2 (two FMAs each)
 *   BOA_MB_L2     bytes/s read (16-byte loads, L2 only) from a 32 MiB buffer
 *   BOA_MB_MMA    tcgen05.mma FLOP/s (2 per multiply-add) with kind 0 TF32,
 *                 1 BF16 (kind::f16) or 2 E4M3 (kind::f8f6f4); M 128 or 64;
 *                 N a multiple of 16 (M 128) or 8 (M 64), at most 256; flags
 *                 bit 0 A operand from TMEM (TF32, M 128), bit 1 alternate
 *                 two accumulators (N <= 128), bit 2 descriptors computed
 *                 once and instructions issued in straight-line code (not
 *                 with bit 1), bit 3 k-blocks cycling through four operand
 *                 stages issued by one thread, bit 4 the same issued by a
 *                 whole warp through one elected lane (bits 2-4 exclusive,
 *                 3 and 4 without bits 0 and 1).  32 bytes of K per
 *                 instruction, one CTA per SM issuing back to back.
 * cycles_per_op (may be NULL): BOA_MB_MMA: SM clock cycles per instruction
 * in steady state (from %clock64); EX2 / FFMA: warp instructions per SM per
 * nominal clock cycle; L2: 0.  kind, M, N, flags are ignored except for
 * BOA_MB_MMA.  The call allocates and frees its own buffers and takes well
 * under a second.  Errors: BOA_ERR_ARG (unknown test or shape), BOA_ERR_CUDA. */
enum { BOA_MB_EX2 = 0, BOA_MB_FFMA = 1, BOA_MB_FFMA2 = 2, BOA_MB_L2 = 3, BOA_MB_MMA = 4 };
boa_status boa_microbench(int device, int test, int kind, int M, int N, int flags, double* rate,
                          double* cycles_per_op);

/* Allocation-free range decoder.  The paper has no counterpart: this entry
 * exists for callers that must not allocate device memory while running --
 * e.g. a data-acquisition process whose GPU memory budget is fixed at
 * start-up, or a host framework whose own pool owns all device memory.
 * It decodes like boa_debug_decode_cdfs, but every pointer except n_syms and
 * in_sizes is DEVICE memory the caller owns: d_cdfs ([sum n_syms][257] u32,
 * sequence i's rows first), d_in (sequence i's coded bytes at d_in + i *
 * in_stride, in_sizes[i] of them), d_syms (sum n_syms symbols out).  n_syms
 * and in_sizes are host arrays.  cuda_stream: cudaStream_t or NULL (legacy
 * default stream); it must belong to the current device (BOA_ERR_ARG
 * otherwise).  The call synchronises that stream before it returns (it reads
 * back a status word), so it can never be recorded into a CUDA graph: do not
 * call it while that stream is being captured.
 * Scratch (per-sequence offsets, sizes and status words) lives in one
 * statically sized device array of about 1.8 MB that every GPU loading this
 * library holds until the process exits; the call allocates nothing.
 * Limit: at most 65536 sequences per call (BOA_ERR_ARG beyond it).  The first
 * call on each device looks up the array's device address (once, under a
 * lock) and keeps it for the life of the process, so the entry point must
 * not be used on a device after cudaDeviceReset.  All calls share the one
 * array, so calls whose work overlaps on the GPU (different streams or host
 * threads) race and must be serialised by the caller.  Errors: BOA_ERR_ARG,
 * BOA_ERR_CORRUPT (some sequence did not decode cleanly), BOA_ERR_CUDA. */
boa_status boa_decode_cdfs_static(size_t n_seq, const size_t* n_syms, const uint32_t* d_cdfs,
                                  const uint8_t* d_in, size_t in_stride, const size_t* in_sizes,
                                  uint8_t* d_syms, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* BOA_H */
