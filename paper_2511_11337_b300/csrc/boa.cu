// libboa.so: C-ABI of the B300 BOA Constrictor library (declared in include/boa.h).
//
// Host side: weight loading, device workspace, and the two step loops.
//   compress   -- teacher-forced: the predictor runs over (streams x time
//                 chunk) rows at once, then one warp per stream range-codes
//                 the chunk's steps in order.
//   decompress -- one step of every stream per pass (each byte feeds the next
//                 step); same kernels with a chunk of one step.
// Both sides evaluate every row with the same kernels, so the integer CDFs
// agree bit for bit (paper, "Determinism and synchronisation").
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include <cudaTypedefs.h>
#include <cuda_fp8.h>

#include "boa.h"
#include "common.cuh"
#include "gemm_fp32.cuh"
#include "gemm_tc.cuh"
#include "kernels.cuh"
#include "scan_step.cuh"
#include "decode_onchip.cuh"
#include "scan_train.cuh"
#include "peaks.cuh"
#include "train_step.cuh"

using namespace boa;

// ------------------------------------------------------------------ errors

static thread_local std::string g_err;

static boa_status fail(boa_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define CU(call)                                                                               \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(e_ == cudaErrorMemoryAllocation ? BOA_ERR_OOM : BOA_ERR_CUDA,          \
                        "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

#define TRY(call)                         \
    do {                                  \
        boa_status s_ = (call);           \
        if (s_ != BOA_OK) return s_;      \
    } while (0)

// ------------------------------------------------------------------ model

struct DevLayer {
    float *ln_a_w, *ln_a_b, *in_wt, *conv_w, *conv_b, *x_wt, *dt_w, *dt_b, *A2, *D, *out_wt;
    float *w1t, *b1, *w2t, *b2, *ln_b_w, *ln_b_b;
};

template <typename T>
struct DevBuf {
    T* p = nullptr;
    size_t n = 0;
    boa_status ensure(size_t want) {
        if (want <= n) return BOA_OK;
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
        cudaError_t e = cudaMalloc(&p, std::max<size_t>(want, 1) * sizeof(T));
        if (e != cudaSuccess) {
            p = nullptr;
            return fail(BOA_ERR_OOM, "cudaMalloc(%zu bytes): %s", want * sizeof(T), cudaGetErrorString(e));
        }
        n = want;
        return BOA_OK;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
};

template <typename T>
struct HostBuf {
    T* p = nullptr;
    size_t n = 0;
    boa_status ensure(size_t want) {
        if (want <= n) return BOA_OK;
        if (p) cudaFreeHost(p);
        p = nullptr;
        n = 0;
        cudaError_t e = cudaMallocHost(&p, std::max<size_t>(want, 1) * sizeof(T));
        if (e != cudaSuccess) {
            p = nullptr;
            return fail(BOA_ERR_OOM, "cudaMallocHost(%zu bytes): %s", want * sizeof(T), cudaGetErrorString(e));
        }
        n = want;
        return BOA_OK;
    }
    void release() {
        if (p) cudaFreeHost(p);
        p = nullptr;
        n = 0;
    }
};

// The slice of the workspace that one sequence of launches works on: slots
// [s0, s0 + n) of the schedule, their rows (slot-major, Tc rows per slot),
// their SSM and conv state, and the stream the kernels go to.  Without
// decode lanes one view covers every slot on the model's stream.
struct View {
    float *x = nullptr, *xn = nullptr, *xz = nullptr, *u = nullptr, *dbc = nullptr, *yg = nullptr;
    float *logits = nullptr, *hid = nullptr, *h = nullptr, *conv = nullptr, *a8s = nullptr;
    __nv_bfloat16 *xn_b = nullptr, *u_b = nullptr, *yg_b = nullptr, *x_b = nullptr, *hid_b = nullptr;
    uint8_t* a8 = nullptr;
    SlotState* slots = nullptr;
    CoderState* st = nullptr;
    const int* slot_beg = nullptr;
    size_t S_all = 0;              // slots in the state arrays (their layer stride)
    cudaStream_t stream = nullptr;
};

struct TrainState;                 // native training step (boa_train_step)

struct boa_model {
    int device = 0;
    int precision = BOA_PREC_FP32;
    int d = 0, nl = 0, N = 0, K = 0, E = 0, r = 0, ffn_mult = 0, F = 0, R2 = 0;
    uint64_t fingerprint = 0;
    size_t n_params = 0;            // floats in the weight file's tensor array
    int num_sms = 148;
    cudaStream_t stream = nullptr;
    bool own_stream = false;

    float* weights = nullptr;   // one device allocation
    float *embed = nullptr, *head_wt = nullptr, *head_b = nullptr;
    std::vector<DevLayer> layers;

    // BF16 tensor-core path: weight copies in nn.Linear layout [out][in]
    __nv_bfloat16* wb = nullptr;
    struct BLayer { __nv_bfloat16 *in_w, *x_w, *out_w, *w1, *w2; };
    std::vector<BLayer> blayers;
    __nv_bfloat16* head_wb = nullptr;
    // 3xTF32 path: pre-split weights (hi, lo), [out][in]
    float* w3 = nullptr;
    struct TLayer { float *in_hi, *in_lo, *x_hi, *x_lo, *out_hi, *out_lo, *w1_hi, *w1_lo, *w2_hi, *w2_lo; };
    std::vector<TLayer> tlayers;
    float *head_hi = nullptr, *head_lo = nullptr;
    // FP8 path: E4M3 weights [out][in] and per-output-channel scales
    uint8_t* w8 = nullptr;
    float* w8s = nullptr;
    struct QLayer { const __nv_fp8_e4m3 *in_w, *x_w, *out_w, *w1, *w2; const float *in_s, *x_s, *out_s, *w1_s, *w2_s; };
    std::vector<QLayer> qlayers;
    const __nv_fp8_e4m3* head_w8 = nullptr;
    const float* head_s = nullptr;
    struct MapEnt { const void* p; uint64_t rows, cols; uint32_t box; int esz; CUtensorMap map; };
    std::vector<MapEnt> maps;

    // workspace
    DevBuf<float> x, xn, xz, u, dbc, yg, logits, hid, h, conv;
    DevBuf<__nv_bfloat16> xn_b, u_b, yg_b, x_b, hid_b;
    DevBuf<uint8_t> a8;          // FP8 activations of the current GEMM
    DevBuf<float> a8s;           // their per-row scales
    DevBuf<int> err;
    DevBuf<CoderState> st;
    DevBuf<SlotState> slots;
    DevBuf<int> sched, slot_beg;
    DevBuf<uint8_t> tokens, d_in, d_out, d_pack;
    DevBuf<uint32_t> flags;
    DevBuf<uint64_t> in_off, out_off, lens, sizes, trace_off, trace, pack_off;
    HostBuf<uint8_t> h_in, h_out;
    HostBuf<uint64_t> h_u64, h_pack;
    HostBuf<int> h_sched;
    HostBuf<uint32_t> h_u32;

    bool trace_on = false;
    size_t trace_n = 0;
    uint64_t launches = 0;

    // Kernel-class timing with CUDA events on the model's stream (bench only).
    bool prof_on = false;
    int prof_stride = 1;            // time every prof_stride-th step of the decode loop
    bool prof_step = true;          // is the current step timed?
    int prof_phase = 0;             // 0 compression, 1 decompression
    struct ProfRec { int phase, cls; cudaEvent_t a, b; double flops, bytes; };
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<ProfRec> prof_pending;
    uint64_t prof_launches[2][BOA_KC_COUNT] = {};
    double prof_ms[2][BOA_KC_COUNT] = {}, prof_flops[2][BOA_KC_COUNT] = {}, prof_bytes[2][BOA_KC_COUNT] = {};
    size_t max_rows = 1u << 18;
    size_t max_slots = 8192;        // streams in flight
    bool use_graphs = true;         // decode step loop as CUDA graphs (when not profiling)
    int scan_variant = 0;           // decode-step scan kernel (see scan())
    int decode_lanes = 0;           // independent slot groups per decode step (0 = automatic)
    int decoder = 0;                // 0: step kernels, state in HBM; 1: on-chip persistent decoder
    DevBuf<int> oc_next;            // the on-chip decoder's queue head
    bool pdl = true;                // chain kernels with programmatic dependent launch
    size_t kp8 = 0;                 // row stride of the FP8 activation scratch

    View v;                         // what the launchers work on
    std::vector<cudaStream_t> lane_streams;
    std::vector<cudaEvent_t> lane_events;   // [0] fork, [1 + p] lane p done
    uint32_t header[9] = {};        // the weight file's header words after the magic
    std::vector<float> params;      // the weight file's tensor array (host copy)
    TrainState* tr = nullptr;
    std::vector<uint32_t> last_status;   // per-stream flags of the last compress / decompress call
    uint64_t prof_steps[2][2] = {};         // [phase][timed, all] steps of the step loops
    // Held for the whole of every call that reads or writes the model's
    // workspace, tuning, profiling counters or tensor-map cache: calls on
    // one model from several host threads run one after another.
    // Recursive because container calls go through boa_compress /
    // boa_decompress.
    mutable std::recursive_mutex mu;
};

#define MODEL_LOCK(m) std::lock_guard<std::recursive_mutex> model_lock_((m)->mu)

static uint64_t fnv1a64_update(uint64_t h, const uint8_t* p, size_t n) {
    for (size_t i = 0; i < n; i++) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

static uint64_t fnv1a64(const uint8_t* p, size_t n) { return fnv1a64_update(1469598103934665603ull, p, n); }

// ---- kernel-class profiling: an event pair around each timed launch.
static const size_t kMaxProfEvents = 1u << 17;

static cudaEvent_t prof_event(boa_model* m) {
    if (m->ev_used == m->ev_pool.size()) {
        if (m->ev_pool.size() >= kMaxProfEvents) return nullptr;
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        m->ev_pool.push_back(e);
    }
    return m->ev_pool[m->ev_used++];
}

struct ProfScope {
    boa_model* m;
    int cls;
    double flops, bytes;
    cudaEvent_t a = nullptr;
    ProfScope(boa_model* m_, int cls_, double flops_, double bytes_) : m(m_), cls(cls_), flops(flops_), bytes(bytes_) {
        if (m->prof_on && m->prof_step) {
            a = prof_event(m);
            if (a) cudaEventRecord(a, m->v.stream);
        }
    }
    ~ProfScope() {
        if (!a) return;
        cudaEvent_t b = prof_event(m);
        if (!b) return;
        cudaEventRecord(b, m->v.stream);
        m->prof_pending.push_back({m->prof_phase, cls, a, b, flops, bytes});
    }
};

// Called after the stream is synchronised: fold the pending pairs into totals.
static void prof_collect(boa_model* m) {
    for (auto& r : m->prof_pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            m->prof_launches[r.phase][r.cls]++;
            m->prof_ms[r.phase][r.cls] += ms;
            m->prof_flops[r.phase][r.cls] += r.flops;
            m->prof_bytes[r.phase][r.cls] += r.bytes;
        }
    }
    m->prof_pending.clear();
    m->ev_used = 0;
}

static bool supported_scan(int N, int r) { return N == 16 && (r == 4 || r == 8 || r == 16); }

static bool supported_d(int d) { return d == 64 || d == 128 || d == 256; }

extern "C" size_t boa_max_compressed_size(size_t len) {
    if (len == 0) return 0;
    if (len == 1) return 1;
    return 1 + 5 * (len - 1) + 4;
}

extern "C" const char* boa_last_error(void) { return g_err.c_str(); }

extern "C" uint64_t boa_model_fingerprint(const boa_model* m) {
    if (!m) return 0;
    MODEL_LOCK(m);                  // a training step replaces it
    return m->fingerprint;
}

extern "C" uint64_t boa_last_launch_count(const boa_model* m) {
    if (!m) return 0;
    MODEL_LOCK(m);
    return m->launches;
}

extern "C" boa_status boa_last_stream_status(const boa_model* m, size_t n, uint32_t* status) {
    if (!m || (n && !status)) return fail(BOA_ERR_ARG, "null argument");
    MODEL_LOCK(m);
    if (n > m->last_status.size()) return fail(BOA_ERR_ARG, "the last call had %zu streams", m->last_status.size());
    if (n) memcpy(status, m->last_status.data(), n * 4);
    return BOA_OK;
}

static void free_train_state(boa_model* m);

static void free_workspace(boa_model* m) {
    m->x.release(); m->xn.release(); m->xz.release(); m->u.release(); m->dbc.release();
    m->yg.release(); m->logits.release(); m->hid.release(); m->h.release(); m->conv.release();
    m->st.release(); m->slots.release(); m->sched.release(); m->slot_beg.release(); m->tokens.release(); m->d_in.release(); m->d_out.release(); m->flags.release();
    m->in_off.release(); m->out_off.release(); m->lens.release(); m->sizes.release();
    m->trace_off.release(); m->trace.release(); m->d_pack.release(); m->pack_off.release();
    m->xn_b.release(); m->u_b.release(); m->yg_b.release(); m->x_b.release(); m->hid_b.release(); m->err.release();
    m->a8.release(); m->a8s.release();
    m->h_in.release(); m->h_out.release(); m->h_u64.release(); m->h_pack.release(); m->h_u32.release(); m->h_sched.release();
}

extern "C" void boa_free_model(boa_model* m) {
    if (!m) return;
    cudaSetDevice(m->device);
    if (m->stream) cudaStreamSynchronize(m->stream);
    free_workspace(m);
    for (auto e : m->ev_pool) cudaEventDestroy(e);
    for (auto e : m->lane_events) cudaEventDestroy(e);
    for (auto ls : m->lane_streams) cudaStreamDestroy(ls);
    if (m->weights) cudaFree(m->weights);
    if (m->wb) cudaFree(m->wb);
    if (m->w3) cudaFree(m->w3);
    if (m->w8) cudaFree(m->w8);
    if (m->w8s) cudaFree(m->w8s);
    free_train_state(m);
    if (m->own_stream && m->stream) cudaStreamDestroy(m->stream);
    delete m;
}

// Transpose a row-major [rows][cols] matrix into [cols][rows].
static void transpose(const float* src, int rows, int cols, float* dst) {
    for (int i = 0; i < rows; i++)
        for (int j = 0; j < cols; j++) dst[(size_t)j * rows + i] = src[(size_t)i * cols + j];
}

// (Re)build every device copy of the weights from the file-layout array src:
// the FP32 arrays (projection matrices K-major, A scaled by log2(e)) and the
// precision form's copies.  Allocations happen on the first call and are
// reused afterwards (training refreshes the copies after each step).
static boa_status upload_weights(boa_model* m, const float* src) {
    const int d = m->d, nl = m->nl, N = m->N, K = m->K, E = m->E, r = m->r, F = m->F, R2 = m->R2;
    const size_t total = m->n_params;
    if (d <= 0 || nl <= 0 || N <= 0 || K <= 0 || E <= 0 || r <= 0 || F < 0 || R2 <= 0)
        return fail(BOA_ERR_ARG, "model shapes not set");
    // Host-side rearrangement: weight matrices K-major, A pre-scaled by log2(e).
    std::vector<float> dev(total);
    size_t so = 0, dof = 0;
    auto copy = [&](size_t n) { size_t at = dof; memcpy(&dev[dof], src + so, n * 4); so += n; dof += n; return at; };
    auto copy_t = [&](int rows, int cols) { size_t at = dof; transpose(src + so, rows, cols, &dev[dof]); so += (size_t)rows * cols; dof += (size_t)rows * cols; return at; };
    struct Off { size_t ln_a_w, ln_a_b, in_wt, conv_w, conv_b, x_wt, dt_w, dt_b, A2, D, out_wt, w1t, b1, w2t, b2, ln_b_w, ln_b_b; };
    std::vector<Off> lo(nl);
    struct SrcOff { size_t in_w, x_w, out_w, w1, w2; };   // file offsets of the GEMM weights
    std::vector<SrcOff> sro(nl);
    size_t head_src = 0;
    size_t embed_o = copy(256 * (size_t)d);
    for (int l = 0; l < nl; l++) {
        Off& q = lo[l];
        q.ln_a_w = copy(d); q.ln_a_b = copy(d);
        sro[l].in_w = so;
        q.in_wt = copy_t(2 * E, d);
        q.conv_w = copy_t(E, K); q.conv_b = copy(E);                   // taps stored [K][E]
        sro[l].x_w = so;
        q.x_wt = copy_t(R2, E);
        q.dt_w = copy_t(E, r); q.dt_b = copy(E);                       // W_dt stored [r][E]
        q.A2 = dof;                                                     // A log2(e) stored [N][E]
        for (size_t c = 0; c < (size_t)E; c++)
            for (size_t n = 0; n < (size_t)N; n++)
                dev[dof + n * E + c] = (float)(-std::exp((double)src[so + c * N + n]) * 1.4426950408889634);
        so += (size_t)E * N; dof += (size_t)E * N;
        q.D = copy(E);
        sro[l].out_w = so;
        q.out_wt = copy_t(d, E);
        q.w1t = q.b1 = q.w2t = q.b2 = 0;
        sro[l].w1 = sro[l].w2 = 0;
        if (F) {
            sro[l].w1 = so;
            q.w1t = copy_t(F, d);
            q.b1 = copy(F);
            sro[l].w2 = so;
            q.w2t = copy_t(d, F);
            q.b2 = copy(d);
        }
        q.ln_b_w = copy(d); q.ln_b_b = copy(d);
    }
    head_src = so;
    size_t head_o = copy_t(256, d);
    size_t head_b_o = copy(256);

    if (!m->weights) CU(cudaMalloc(&m->weights, total * 4));
    CU(cudaMemcpy(m->weights, dev.data(), total * 4, cudaMemcpyHostToDevice));
    float* w = m->weights;
    m->embed = w + embed_o;
    m->head_wt = w + head_o;
    m->head_b = w + head_b_o;
    m->layers.resize(nl);
    for (int l = 0; l < nl; l++) {
        const Off& q = lo[l];
        DevLayer& L = m->layers[l];
        L.ln_a_w = w + q.ln_a_w; L.ln_a_b = w + q.ln_a_b; L.in_wt = w + q.in_wt;
        L.conv_w = w + q.conv_w; L.conv_b = w + q.conv_b; L.x_wt = w + q.x_wt;
        L.dt_w = w + q.dt_w; L.dt_b = w + q.dt_b; L.A2 = w + q.A2; L.D = w + q.D; L.out_wt = w + q.out_wt;
        L.w1t = F ? w + q.w1t : nullptr; L.b1 = F ? w + q.b1 : nullptr;
        L.w2t = F ? w + q.w2t : nullptr; L.b2 = F ? w + q.b2 : nullptr;
        L.ln_b_w = w + q.ln_b_w; L.ln_b_b = w + q.ln_b_b;
    }
    if (m->precision == BOA_PREC_BF16) {
        // BF16 copies of the projection weights, kept in the file's [out][in]
        // layout (K-major, as the tensor-core B operand wants it).
        std::vector<std::pair<size_t, size_t>> mats;   // (source offset, elements)
        for (int l = 0; l < nl; l++) {
            mats.push_back({sro[l].in_w, (size_t)2 * E * d});
            mats.push_back({sro[l].x_w, (size_t)R2 * E});
            mats.push_back({sro[l].out_w, (size_t)d * E});
            if (F) { mats.push_back({sro[l].w1, (size_t)F * d}); mats.push_back({sro[l].w2, (size_t)d * F}); }
        }
        mats.push_back({head_src, (size_t)256 * d});
        size_t tot = 0;
        std::vector<size_t> at;
        for (auto& mt : mats) { at.push_back(tot); tot += (mt.second + 63) / 64 * 64; }
        std::vector<__nv_bfloat16> hb(tot, __float2bfloat16_rn(0.f));
        for (size_t i = 0; i < mats.size(); i++)
            for (size_t j = 0; j < mats[i].second; j++) hb[at[i] + j] = __float2bfloat16_rn(src[mats[i].first + j]);
        if (!m->wb) CU(cudaMalloc(&m->wb, tot * 2));
        CU(cudaMemcpy(m->wb, hb.data(), tot * 2, cudaMemcpyHostToDevice));
        size_t k = 0;
        m->blayers.resize(nl);
        for (int l = 0; l < nl; l++) {
            auto& B = m->blayers[l];
            B.in_w = m->wb + at[k++];
            B.x_w = m->wb + at[k++];
            B.out_w = m->wb + at[k++];
            B.w1 = F ? m->wb + at[k++] : nullptr;
            B.w2 = F ? m->wb + at[k++] : nullptr;
        }
        m->head_wb = m->wb + at[k++];
    }
    if (m->precision == BOA_PREC_TF32X3) {
        // x = hi + lo with hi = x rounded to TF32 (nearest, ties away), lo = x - hi
        std::vector<std::pair<size_t, size_t>> mats;
        for (int l = 0; l < nl; l++) {
            mats.push_back({sro[l].in_w, (size_t)2 * E * d});
            mats.push_back({sro[l].x_w, (size_t)R2 * E});
            mats.push_back({sro[l].out_w, (size_t)d * E});
            if (F) { mats.push_back({sro[l].w1, (size_t)F * d}); mats.push_back({sro[l].w2, (size_t)d * F}); }
        }
        mats.push_back({head_src, (size_t)256 * d});
        size_t tot = 0;
        std::vector<size_t> at;
        for (auto& mt : mats) { at.push_back(tot); tot += 2 * ((mt.second + 31) / 32 * 32); }
        std::vector<float> hb(tot, 0.f);
        for (size_t i = 0; i < mats.size(); i++) {
            const size_t n = mats[i].second, half = (n + 31) / 32 * 32;
            for (size_t j = 0; j < n; j++) {
                const float x = src[mats[i].first + j];
                uint32_t u;
                memcpy(&u, &x, 4);
                u = (u + 0x1000u) & ~0x1FFFu;
                float hi;
                memcpy(&hi, &u, 4);
                hb[at[i] + j] = hi;
                hb[at[i] + half + j] = x - hi;
            }
        }
        if (!m->w3) CU(cudaMalloc(&m->w3, tot * 4));
        CU(cudaMemcpy(m->w3, hb.data(), tot * 4, cudaMemcpyHostToDevice));
        size_t k = 0;
        auto pair = [&](float*& hi, float*& lo) {
            const size_t half = (mats[k].second + 31) / 32 * 32;
            hi = m->w3 + at[k];
            lo = m->w3 + at[k] + half;
            k++;
        };
        m->tlayers.resize(nl);
        for (int l = 0; l < nl; l++) {
            auto& T = m->tlayers[l];
            pair(T.in_hi, T.in_lo);
            pair(T.x_hi, T.x_lo);
            pair(T.out_hi, T.out_lo);
            T.w1_hi = T.w1_lo = T.w2_hi = T.w2_lo = nullptr;
            if (F) { pair(T.w1_hi, T.w1_lo); pair(T.w2_hi, T.w2_lo); }
        }
        pair(m->head_hi, m->head_lo);
    }
    if (m->precision == BOA_PREC_FP8) {
        // w8[n][k] = e4m3(W[n][k] * 448 / max_k |W[n][k]|), scale[n] = max / 448
        struct Mat { size_t src, rows, cols; };
        std::vector<Mat> mats;
        for (int l = 0; l < nl; l++) {
            mats.push_back({sro[l].in_w, (size_t)2 * E, (size_t)d});
            mats.push_back({sro[l].x_w, (size_t)R2, (size_t)E});
            mats.push_back({sro[l].out_w, (size_t)d, (size_t)E});
            if (F) { mats.push_back({sro[l].w1, (size_t)F, (size_t)d}); mats.push_back({sro[l].w2, (size_t)d, (size_t)F}); }
        }
        mats.push_back({head_src, (size_t)256, (size_t)d});
        size_t tb = 0, ts = 0;
        std::vector<size_t> atb, ats;
        auto kpad = [](size_t k) { return (k + 127) / 128 * 128; };
        for (auto& mt : mats) {
            atb.push_back(tb); ats.push_back(ts);
            tb += (mt.rows * kpad(mt.cols) + 255) / 256 * 256;
            ts += (mt.rows + 63) / 64 * 64;
        }
        std::vector<uint8_t> hq(tb, 0);
        std::vector<float> hs(ts, 1.f);
        for (size_t i = 0; i < mats.size(); i++) {
            const size_t R = mats[i].rows, Cc = mats[i].cols;
            for (size_t rr = 0; rr < R; rr++) {
                const float* w = src + mats[i].src + rr * Cc;
                float amax = 0.f;
                for (size_t k = 0; k < Cc; k++) amax = std::max(amax, std::fabs(w[k]));
                const float inv = amax > 0.f ? 448.0f / amax : 1.0f;
                hs[ats[i] + rr] = amax > 0.f ? amax / 448.0f : 1.0f;
                for (size_t k = 0; k < Cc; k++)
                    hq[atb[i] + rr * kpad(Cc) + k] = (uint8_t)__nv_cvt_float_to_fp8(w[k] * inv, __NV_SATFINITE, __NV_E4M3);
            }
        }
        if (!m->w8) CU(cudaMalloc(&m->w8, tb));
        if (!m->w8s) CU(cudaMalloc(&m->w8s, ts * 4));
        CU(cudaMemcpy(m->w8, hq.data(), tb, cudaMemcpyHostToDevice));
        CU(cudaMemcpy(m->w8s, hs.data(), ts * 4, cudaMemcpyHostToDevice));
        size_t k = 0;
        auto q = [&](const __nv_fp8_e4m3*& w, const float*& sc) {
            w = reinterpret_cast<const __nv_fp8_e4m3*>(m->w8 + atb[k]);
            sc = m->w8s + ats[k];
            k++;
        };
        m->qlayers.resize(nl);
        for (int l = 0; l < nl; l++) {
            auto& Q = m->qlayers[l];
            q(Q.in_w, Q.in_s);
            q(Q.x_w, Q.x_s);
            q(Q.out_w, Q.out_s);
            Q.w1 = Q.w2 = nullptr;
            Q.w1_s = Q.w2_s = nullptr;
            if (F) { q(Q.w1, Q.w1_s); q(Q.w2, Q.w2_s); }
        }
        q(m->head_w8, m->head_s);
    }
    return BOA_OK;
}

extern "C" boa_status boa_load_model(const char* path, const boa_opts* opts, boa_model** out) {
    if (!path || !out) return fail(BOA_ERR_ARG, "boa_load_model: null argument");
    FILE* fp = fopen(path, "rb");
    if (!fp) return fail(BOA_ERR_IO, "cannot open weight file %s", path);
    std::vector<uint8_t> buf;
    {
        fseek(fp, 0, SEEK_END);
        long sz = ftell(fp);
        fseek(fp, 0, SEEK_SET);
        if (sz < 40) { fclose(fp); return fail(BOA_ERR_FORMAT, "weight file too short"); }
        buf.resize((size_t)sz);
        size_t got = fread(buf.data(), 1, buf.size(), fp);
        fclose(fp);
        if (got != buf.size()) return fail(BOA_ERR_IO, "short read on %s", path);
    }
    if (memcmp(buf.data(), "BOAW", 4) != 0) return fail(BOA_ERR_FORMAT, "bad magic");
    uint32_t hdr[9];
    memcpy(hdr, buf.data() + 4, sizeof hdr);
    if (hdr[0] != 1) return fail(BOA_ERR_FORMAT, "unsupported version %u", hdr[0]);
    const int vocab = (int)hdr[1], d = (int)hdr[2], nl = (int)hdr[3], N = (int)hdr[4], K = (int)hdr[5];
    const int expand = (int)hdr[6], r = (int)hdr[7], ffn = (int)hdr[8];
    const int E = expand * d, F = ffn * d, R2 = r + 2 * N;
    if (vocab != 256 || nl < 1 || nl > 64 || expand < 1 || expand > 4 || r != (d + 15) / 16)
        return fail(BOA_ERR_FORMAT, "unsupported header (vocab %d, layers %d, expand %d, dt_rank %d)", vocab, nl, expand, r);
    if (!supported_d(d) || !supported_scan(N, r) || K < 2 || K > 4 || (ffn != 0 && ffn != 2 && ffn != 4))
        return fail(BOA_ERR_FORMAT, "unsupported shape d=%d N=%d r=%d K=%d ffn=%d", d, N, r, K, ffn);

    const size_t per_layer = 2 * (size_t)d + 2 * (size_t)E * d + (size_t)E * K + E + (size_t)R2 * E +
                             (size_t)E * r + E + (size_t)E * N + E + (size_t)d * E +
                             (F ? (size_t)F * d + F + (size_t)d * F + d : 0) + 2 * (size_t)d;
    const size_t total = 256 * (size_t)d + nl * per_layer + 256 * (size_t)d + 256;
    if (buf.size() != 40 + total * 4) return fail(BOA_ERR_FORMAT, "weight file size %zu, expected %zu", buf.size(), 40 + total * 4);

    boa_opts o = {0, BOA_PREC_FP32, nullptr, 0, 0};
    if (opts) o = *opts;
    if (o.precision < BOA_PREC_FP32 || o.precision > BOA_PREC_FP8)
        return fail(BOA_ERR_ARG, "precision %d not supported", o.precision);
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return fail(BOA_ERR_CUDA, "no CUDA device available");
    if (o.device < 0 || o.device >= ndev) return fail(BOA_ERR_ARG, "bad device %d", o.device);
    CU(cudaSetDevice(o.device));

    boa_model* m = new boa_model();
    m->device = o.device;
    m->precision = o.precision;
    if (o.max_rows) m->max_rows = std::max<size_t>(o.max_rows, 1);
    if (o.max_slots) m->max_slots = std::max<size_t>(o.max_slots, 1);
    m->d = d; m->nl = nl; m->N = N; m->K = K; m->E = E; m->r = r; m->ffn_mult = ffn; m->F = F; m->R2 = R2;
    m->fingerprint = fnv1a64(buf.data(), buf.size());
    memcpy(m->header, hdr, sizeof hdr);
    cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, o.device);
    if (o.cuda_stream) {
        m->stream = (cudaStream_t)o.cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete m;
            return fail(BOA_ERR_CUDA, "cudaStreamCreate failed");
        }
        m->own_stream = true;
    }
    const float* src = reinterpret_cast<const float*>(buf.data() + 40);
    m->n_params = total;
    m->params.assign(src, src + total);
    const boa_status ws = upload_weights(m, src);
    if (ws != BOA_OK) {
        boa_free_model(m);
        return ws;
    }
    *out = m;
    return BOA_OK;
}

// ------------------------------------------------------------ launchers

static boa_status check_launch(boa_model* m, const char* what) {
    m->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(BOA_ERR_CUDA, "launch of %s failed: %s", what, cudaGetErrorString(e));
    return BOA_OK;
}

// Launch a kernel of the predictor / coder chain on the view's stream with
// programmatic stream serialization (the kernel overlaps its set-up with
// its predecessor and waits in pdl_wait_prev); splits > 1 launches clusters
// of (1, 1, splits) along z.
template <typename... P, typename... A>
static void launch_k(boa_model* m, void (*kern)(P...), dim3 grid, dim3 block, size_t smem, int splits, A&&... args) {
    cudaLaunchConfig_t cfg{};
    if (splits > 1) grid.z = (unsigned)splits;
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = m->v.stream;
    cudaLaunchAttribute at[2];
    unsigned na = 0;
    if (splits > 1) {
        at[na].id = cudaLaunchAttributeClusterDimension;
        at[na].val.clusterDim.x = 1;
        at[na].val.clusterDim.y = 1;
        at[na].val.clusterDim.z = (unsigned)splits;
        na++;
    }
    if (m->pdl) {
        at[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[na].val.programmaticStreamSerializationAllowed = 1;
        na++;
    }
    cfg.attrs = at;
    cfg.numAttrs = na;
    cudaLaunchKernelEx(&cfg, kern, std::forward<A>(args)...);
}

// Opt-in to more than 48 KB of dynamic shared memory for one kernel.  The
// attribute belongs to a device's context, so it is set once per (kernel,
// device ordinal), with that device current (every caller runs after
// cudaSetDevice(m->device)); a failure is reported, not ignored.
struct SmemOptIn {
    std::atomic<uint64_t> done[4] = {};     // bit per device ordinal 0..255
    std::mutex mu;
};

// bytes < 0: the most the device allows this kernel beside its static
// shared memory.
template <typename Kern>
static boa_status smem_opt_in(SmemOptIn& o, Kern kern, int bytes, int dev, const char* what) {
    if (dev < 0 || dev >= 256) return fail(BOA_ERR_CUDA, "device ordinal %d out of range", dev);
    const uint64_t bit = 1ull << (dev & 63);
    std::atomic<uint64_t>& word = o.done[dev >> 6];
    if (word.load(std::memory_order_acquire) & bit) return BOA_OK;
    std::lock_guard<std::mutex> lock(o.mu);
    if (word.load(std::memory_order_acquire) & bit) return BOA_OK;
    cudaError_t e = cudaSuccess;
    if (bytes < 0) {
        cudaFuncAttributes fa{};
        int optin = 0;
        e = cudaFuncGetAttributes(&fa, kern);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        bytes = optin - (int)fa.sharedSizeBytes;
    }
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess)
        return fail(BOA_ERR_CUDA, "%s: dynamic shared memory opt-in (%d bytes) on device %d failed: %s", what, bytes,
                    dev, cudaGetErrorString(e));
    word.fetch_or(bit, std::memory_order_acq_rel);
    return BOA_OK;
}

template <int EPI>
static boa_status gemm(boa_model* m, int cls, const float* A, const float* Wt, const float* bias, float* C, long long M,
                       int N, int K) {
    if (M <= 0) return BOA_OK;
    const bool resid = EPI == kEpiResid || EPI == kEpiBiasResid;
    ProfScope ps(m, cls, 2.0 * M * N * K, 4.0 * ((double)M * K + (double)K * N + (double)M * N * (resid ? 2 : 1)));
    if (N % 4 != 0 || K % kGemmBK != 0) return fail(BOA_ERR_FORMAT, "gemm shape N=%d K=%d unsupported", N, K);
    const long long t128 = ((M + 127) / 128) * ((N + 127) / 128);
    const long long t12864 = ((M + 127) / 128) * ((N + 63) / 64);
    const long long waves = 2LL * m->num_sms;
    if (N >= 128 && t128 >= waves) {
        dim3 grid((N + 127) / 128, (unsigned)((M + 127) / 128));
        launch_k(m, k_gemm_fp32<128, 128, EPI>, grid, kGemmThreads, 0, 1, A, Wt, bias, C, (int)M, N, K);
    } else if (t12864 >= waves) {
        dim3 grid((N + 63) / 64, (unsigned)((M + 127) / 128));
        launch_k(m, k_gemm_fp32<128, 64, EPI>, grid, kGemmThreads, 0, 1, A, Wt, bias, C, (int)M, N, K);
    } else {
        dim3 grid((N + 63) / 64, (unsigned)((M + 63) / 64));
        launch_k(m, k_gemm_fp32<64, 64, EPI>, grid, kGemmThreads, 0, 1, A, Wt, bias, C, (int)M, N, K);
    }
    return check_launch(m, "gemm");
}

// ---- tensor-core GEMM (BF16 operands, FP32 accumulation)

static PFN_cuTensorMapEncodeTiled_v12000 g_encode_tiled = nullptr;
static std::mutex g_encode_mu;

// 2-D BF16 tensor map over a row-major [rows][cols] matrix, boxes of
// 64 columns (128 bytes, 128-byte swizzle) by box_rows rows.
// esz: element size in bytes (1 E4M3, 2 BF16, 4 FP32).
static boa_status tmap_2d(boa_model* m, const void* ptr, uint64_t rows, uint64_t cols, uint32_t box_rows, int esz,
                          CUtensorMap* out) {
    for (auto& e : m->maps)
        if (e.p == ptr && e.rows == rows && e.cols == cols && e.box == box_rows && e.esz == esz) {
            *out = e.map;
            return BOA_OK;
        }
    {
        std::lock_guard<std::mutex> lock(g_encode_mu);
        if (!g_encode_tiled) {
            cudaDriverEntryPointQueryResult q;
            void* fn = nullptr;
            cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
            if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
                return fail(BOA_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
            g_encode_tiled = (PFN_cuTensorMapEncodeTiled_v12000)fn;
        }
    }
    if (((uintptr_t)ptr & 15) || (cols * esz) % 16) return fail(BOA_ERR_ARG, "tensor map needs 16-byte aligned rows");
    boa_model::MapEnt e;
    e.p = ptr; e.rows = rows; e.cols = cols; e.box = box_rows; e.esz = esz;
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {cols * esz};
    cuuint32_t box[2] = {(cuuint32_t)(128 / esz), box_rows};   // 128-byte rows: one swizzle atom
    cuuint32_t es[2] = {1, 1};
    const CUtensorMapDataType dt = esz == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : esz == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8;
    CUresult r = g_encode_tiled(&e.map, dt, 2,
                                const_cast<void*>(ptr), dims, strides, box, es,
                                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(BOA_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    if (m->maps.size() >= 256) m->maps.clear();
    m->maps.push_back(e);
    *out = e.map;
    return BOA_OK;
}

// Tile width.  An output element's value does not depend on the MMA's N
// (its K sums run through the same instructions whatever the tile width:
// tested bit for bit across widths), so the width may follow the batch.
// Decode-size batches keep several CTAs per output column block (128 for
// N >= 512, 64, or 48 for x_proj); compression-size batches (more than
// kWideRows rows) take 128-wide tiles.  The tensor pipe spends max(46, N/2)
// cycles on an instruction, so a 128-wide tile does as much work per cycle
// as a 256-wide one, and its smaller stages let two CTAs share an SM (one's
// epilogue overlapping the other's main loop): measured per 64 MiB against
// 256-wide tiles, 3xTF32 in_proj 610 -> 505 ms, out_proj 334 -> 264 ms.
// x_proj (N <= 64) keeps its 48-wide tile, since its split K depends on N
// alone.
static const long long kWideRows = 8192;
static int tc_bn(int N, long long M) {
    if (M > kWideRows && N > 64) return 128;
    return N >= 512 ? 128 : N > 48 ? 64 : 48;
}

// Split K across a cluster of CTAs (deterministic reduction in the
// epilogue) for x_proj (N <= 64), whose grid is otherwise a few dozen long
// K loops at decode sizes.  Chosen by (N, K) only, like the tile width, each
// CTA keeping at least two K blocks of k_elems.  (Splitting out_proj and the
// head 2 ways as well, with 128-wide decode tiles, left decompression as
// fast as before: measured, and dropped.)
static int tc_splits(int N, int K, int k_elems) {
    int s = N <= 64 ? 4 : 1;
    while (s > 1 && (K % (s * k_elems) != 0 || K / (s * k_elems) < 2)) s /= 2;
    return s;
}


template <int BN, int EPI, int KIND, bool DEEP>
static boa_status launch_tc_cfg(boa_model* m, dim3 grid, int splits, int chunks, const CUtensorMap& ta,
                                const CUtensorMap& tb, const float* bias, float* C, __nv_bfloat16* outb, long long M,
                                int N, int K, const float* rs, const float* cs, int zpart = 0) {
    using L = TcSmem<BN, DEEP>;
    static SmemOptIn optin;
    TRY((smem_opt_in(optin, k_gemm_tc_bf16<BN, EPI, KIND, DEEP>, (int)L::kBytes, m->device, "tensor-core gemm")));
    launch_k(m, k_gemm_tc_bf16<BN, EPI, KIND, DEEP>, grid, kTcThreads, L::kBytes, splits, ta, tb, bias, C, outb,
             (int)M, N, K, m->err.p, rs, cs, chunks, zpart);
    return BOA_OK;
}

// Compression-size BF16 / E4M3 projections with 128-wide tiles, no split
// K and no residual read: one persistent CTA per SM (the epilogue of one
// tile beside the next tile's main loop; the same bits as k_gemm_tc_bf16).
// Measured per 64 MiB: BF16 in_proj 263 -> 169 ms, E4M3 in_proj 251 ->
// 241 ms.  With a residual epilogue (out_proj) the short main loop of these
// forms leaves the four epilogue warps exposed (BF16 134 -> 140 ms, E4M3
// 118 -> 138 ms), so out_proj keeps the one-tile CTAs, two per SM.
template <int EPI, int KIND>
static boa_status launch_tc_persist(boa_model* m, const CUtensorMap& ta, const CUtensorMap& tb, const float* bias,
                                   float* C, __nv_bfloat16* outb, long long M, int N, int K, const float* rs,
                                   const float* cs, long long tiles) {
    static SmemOptIn optin;
    TRY((smem_opt_in(optin, k_gemm_tc_persist<EPI, KIND>, (int)TcP::kBytes, m->device, "persistent tensor-core gemm")));
    const dim3 grid((unsigned)std::min<long long>(tiles, m->num_sms));
    launch_k(m, k_gemm_tc_persist<EPI, KIND>, grid, TcP::kThreads, TcP::kBytes, 1, ta, tb, bias, C, outb, (int)M,
             N, K, m->err.p, rs, cs);
    return BOA_OK;
}

// Grids smaller than the SM count take the deep-pipeline variant.  Split K
// runs across a cluster on small grids and in one CTA's TMEM on grids that
// fill the GPU (the same additions in the same order; see launch_t3).
template <int BN, int EPI, int KIND>
static boa_status launch_tc(boa_model* m, const CUtensorMap& ta, const CUtensorMap& tb, const float* bias, float* C,
                            __nv_bfloat16* outb, long long M, int N, int K, const float* rs, const float* cs) {
    dim3 grid((N + BN - 1) / BN, (unsigned)((M + kTcBM - 1) / kTcBM));
    const int split = tc_splits(N, K, KIND == kKindE4M3 ? 128 : kTcBK);
    constexpr bool kResid = EPI == kEpiResid || EPI == kEpiBiasResid;
    if (!kResid && BN == TcP::BN && split == 1 && (long long)grid.x * grid.y >= 2LL * m->num_sms)
        return launch_tc_persist<EPI, KIND>(m, ta, tb, bias, C, outb, M, N, K, rs, cs, (long long)grid.x * grid.y);
    const bool in_cta = (long long)grid.x * grid.y >= m->num_sms;
    const int chunks = in_cta && split * TcSmem<BN>::kTmemCols <= 512 ? split : 1;
    const int peers = split / chunks;
    if ((long long)grid.x * grid.y * peers < m->num_sms)
        return launch_tc_cfg<BN, EPI, KIND, true>(m, grid, peers, chunks, ta, tb, bias, C, outb, M, N, K, rs, cs);
    return launch_tc_cfg<BN, EPI, KIND, false>(m, grid, peers, chunks, ta, tb, bias, C, outb, M, N, K, rs, cs);
}

template <int EPI>
static boa_status gemm_tc(boa_model* m, int cls, const __nv_bfloat16* A, const __nv_bfloat16* W, const float* bias,
                          float* C, __nv_bfloat16* outb, long long M, int N, int K) {
    if (M <= 0) return BOA_OK;
    if (N % 4 != 0 || K % kTcBK != 0) return fail(BOA_ERR_FORMAT, "tensor-core gemm shape N=%d K=%d unsupported", N, K);
    const bool resid = EPI == kEpiResid || EPI == kEpiBiasResid;
    ProfScope ps(m, cls, 2.0 * M * N * K,
                 2.0 * ((double)M * K + (double)K * N) + 4.0 * (double)M * N * (resid ? 2 : 1) + (outb ? 2.0 * M * N : 0));
    const int BN = tc_bn(N, M);
    CUtensorMap ta, tb;
    TRY(tmap_2d(m, A, (uint64_t)M, (uint64_t)K, kTcBM, 2, &ta));
    TRY(tmap_2d(m, W, (uint64_t)N, (uint64_t)K, (uint32_t)BN, 2, &tb));
    switch (BN) {
        case 48: TRY((launch_tc<48, EPI, kKindBF16>(m, ta, tb, bias, C, outb, M, N, K, nullptr, nullptr))); break;
        case 64: TRY((launch_tc<64, EPI, kKindBF16>(m, ta, tb, bias, C, outb, M, N, K, nullptr, nullptr))); break;
        default: TRY((launch_tc<128, EPI, kKindBF16>(m, ta, tb, bias, C, outb, M, N, K, nullptr, nullptr))); break;
    }
    return check_launch(m, "gemm_tc");
}

// Weight gradients of a BF16 model's training step on the tensor cores:
// out[z][M][N] = sum over k in part z of A[m][k] B[n][k] (A [M][K], B [N][K]
// BF16 rows, K = parts x the part length, a multiple of 64), every part's K
// blocks accumulated in order by one CTA per output tile.  The caller adds
// the parts in order (k_tr_reduce), so the result does not depend on the
// grid.
static boa_status gemm_tc_parts(boa_model* m, const __nv_bfloat16* A, const __nv_bfloat16* B, float* out, int M,
                                int N, long long K, int parts) {
    if (N % 4 != 0 || K % ((long long)parts * kTcBK) != 0)
        return fail(BOA_ERR_FORMAT, "tensor-core gradient shape N=%d K=%lld parts=%d unsupported", N, K, parts);
    const int BN = N >= 128 ? 128 : N > 48 ? 64 : 48;
    CUtensorMap ta, tb;
    TRY(tmap_2d(m, A, (uint64_t)M, (uint64_t)K, kTcBM, 2, &ta));
    TRY(tmap_2d(m, B, (uint64_t)N, (uint64_t)K, (uint32_t)BN, 2, &tb));
    const dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + kTcBM - 1) / kTcBM), (unsigned)parts);
    switch (BN) {
        case 48: TRY((launch_tc_cfg<48, kEpiStore, kKindBF16, false>(m, grid, 1, 1, ta, tb, nullptr, out, nullptr, M, N,
                                                                     (int)K, nullptr, nullptr, 1))); break;
        case 64: TRY((launch_tc_cfg<64, kEpiStore, kKindBF16, false>(m, grid, 1, 1, ta, tb, nullptr, out, nullptr, M, N,
                                                                     (int)K, nullptr, nullptr, 1))); break;
        default: TRY((launch_tc_cfg<128, kEpiStore, kKindBF16, false>(m, grid, 1, 1, ta, tb, nullptr, out, nullptr, M,
                                                                      N, (int)K, nullptr, nullptr, 1))); break;
    }
    return check_launch(m, "gemm_tc_parts");
}

// FP8 projection: quantise the FP32 activation rows (one warp per row), then
// the E4M3 tensor-core kernel with the row and weight scales in its epilogue.
// prequant: the kernel that produced A already wrote its E4M3 copy and row
// scales into the view's FP8 scratch (f8_out), so no quantisation launch.
template <int EPI>
static boa_status gemm_f8(boa_model* m, int cls, const float* A, const __nv_fp8_e4m3* W, const float* wscale,
                          const float* bias, float* C, long long M, int N, int K, bool prequant = false) {
    if (M <= 0) return BOA_OK;
    if (N % 4 != 0 || K % 16 != 0 || K > 1024) return fail(BOA_ERR_FORMAT, "fp8 gemm shape N=%d K=%d unsupported", N, K);
    const int Kp = (K + 127) / 128 * 128;     // W is stored with the same zero padding
    if (!m->v.a8 || (size_t)Kp > m->kp8) return fail(BOA_ERR_ARG, "FP8 activation scratch not sized for K=%d", K);
    if (!prequant) {
        ProfScope pq(m, BOA_KC_OTHER, 3.0 * M * K, 5.0 * M * K + 4.0 * M);
        launch_k(m, k_quant_rows_e4m3, dim3((unsigned)((M + 7) / 8)), 256, 0, 1, A,
                 reinterpret_cast<__nv_fp8_e4m3*>(m->v.a8), m->v.a8s, M, K, Kp);
        TRY(check_launch(m, "quant_rows"));
    }
    const bool resid = EPI == kEpiResid || EPI == kEpiBiasResid;
    ProfScope ps(m, cls, 2.0 * M * N * K, ((double)M * K + (double)K * N) + 4.0 * (double)M * N * (resid ? 2 : 1));
    const int BN = tc_bn(N, M);
    CUtensorMap ta, tb;
    TRY(tmap_2d(m, m->v.a8, (uint64_t)M, (uint64_t)Kp, kTcBM, 1, &ta));
    TRY(tmap_2d(m, W, (uint64_t)N, (uint64_t)Kp, (uint32_t)BN, 1, &tb));
    switch (BN) {
        case 48: TRY((launch_tc<48, EPI, kKindE4M3>(m, ta, tb, bias, C, nullptr, M, N, Kp, m->v.a8s, wscale))); break;
        case 64: TRY((launch_tc<64, EPI, kKindE4M3>(m, ta, tb, bias, C, nullptr, M, N, Kp, m->v.a8s, wscale))); break;
        default: TRY((launch_tc<128, EPI, kKindE4M3>(m, ta, tb, bias, C, nullptr, M, N, Kp, m->v.a8s, wscale))); break;
    }
    return check_launch(m, "gemm_f8");
}

// 3xTF32 split K follows tc_splits (x_proj: 4).  The partial sums are added
// in chunk order whether the chunks run on the CTAs of a cluster (small
// grids: decode steps) or sit in one CTA's TMEM (grids that fill the GPU:
// compression, where a cluster's epilogue exchange costs more than it
// hides), so both give the same bits.
// TMEM is never oversubscribed: the 3xTF32 CTAs that shared memory lets
// onto one SM (228 KB, 1 KB reserved per CTA) allocate at most its 512
// columns between them (one K chunk each; in-CTA chunks are checked in
// launch_t3).
template <int BN, bool DEEP>
constexpr bool t3_tmem_fits() {
    using L = T3Smem<BN, DEEP>;
    return L::pow2_cols((uint32_t)(L::kTmemCols + L::kStages * L::kACols)) *
               (uint32_t)((228 * 1024) / (L::kBytes + 1024)) <= 512u;
}
static_assert(t3_tmem_fits<48, false>() && t3_tmem_fits<48, true>() && t3_tmem_fits<64, false>() &&
                  t3_tmem_fits<64, true>() && t3_tmem_fits<128, false>() && t3_tmem_fits<128, true>() &&
                  t3_tmem_fits<256, false>() && t3_tmem_fits<256, true>(),
              "3xTF32 CTAs sharing an SM would need more than 512 TMEM columns");

template <int BN, int EPI, bool DEEP>
static boa_status launch_t3_cfg(boa_model* m, dim3 grid, int splits, int chunks, const CUtensorMap& ta,
                                const CUtensorMap& th, const CUtensorMap& tl, const float* bias, float* C,
                                long long M, int N, int K) {
    using L = T3Smem<BN, DEEP>;
    static SmemOptIn optin;
    TRY((smem_opt_in(optin, k_gemm_tc_tf32x3<BN, EPI, DEEP>, (int)L::kBytes, m->device, "3xTF32 gemm")));
    launch_k(m, k_gemm_tc_tf32x3<BN, EPI, DEEP>, grid, t3_threads(DEEP), L::kBytes, splits, ta, th, tl, bias, C,
             (int)M, N, K, m->err.p, chunks);
    return BOA_OK;
}

// Compression-size projections with 128-wide tiles and no split K (in_proj,
// out_proj, the head at more than two tiles per SM): one persistent CTA per
// SM, whose epilogue of one tile overlaps the main loop of the next (same
// MMAs and epilogue per tile, so the same bits as k_gemm_tc_tf32x3).
template <int EPI>
static boa_status launch_t3_persist(boa_model* m, const CUtensorMap& ta, const CUtensorMap& th,
                                    const CUtensorMap& tl, const float* bias, float* C, long long M, int N, int K,
                                    long long tiles) {
    static SmemOptIn optin;
    TRY((smem_opt_in(optin, k_gemm_t3_persist<EPI>, (int)T3P::kBytes, m->device, "persistent 3xTF32 gemm")));
    const dim3 grid((unsigned)std::min<long long>(tiles, m->num_sms));
    launch_k(m, k_gemm_t3_persist<EPI>, grid, T3P::kThreads, T3P::kBytes, 1, ta, th, tl, bias, C, (int)M, N, K,
             m->err.p);
    return BOA_OK;
}

template <int BN, int EPI>
static boa_status launch_t3(boa_model* m, const CUtensorMap& ta, const CUtensorMap& th, const CUtensorMap& tl,
                            const float* bias, float* C, long long M, int N, int K) {
    dim3 grid((N + BN - 1) / BN, (unsigned)((M + kTcBM - 1) / kTcBM));
    const int split = tc_splits(N, K, kT3BK);
    if (BN == T3P::BN && split == 1 && (long long)grid.x * grid.y >= 2LL * m->num_sms)
        return launch_t3_persist<EPI>(m, ta, th, tl, bias, C, M, N, K, (long long)grid.x * grid.y);
    const bool in_cta = (long long)grid.x * grid.y >= m->num_sms;
    // in-CTA chunks while the CTA's TMEM (accumulators + A stages) still
    // leaves room for the second CTA an SM holds
    using L = T3Smem<BN>;
    const uint32_t room = L::kOnePerSm ? 512u : 256u;
    const int chunks = in_cta && L::pow2_cols((uint32_t)(split * L::kTmemCols + L::kStages * L::kACols)) <= room
                           ? split : 1;
    const int peers = split / chunks;
    if ((long long)grid.x * grid.y * peers < m->num_sms)
        return launch_t3_cfg<BN, EPI, true>(m, grid, peers, chunks, ta, th, tl, bias, C, M, N, K);
    return launch_t3_cfg<BN, EPI, false>(m, grid, peers, chunks, ta, th, tl, bias, C, M, N, K);
}

// FP32-accurate tensor-core GEMM (3xTF32); A is FP32, W pre-split.
template <int EPI>
static boa_status gemm_t3(boa_model* m, int cls, const float* A, const float* Whi, const float* Wlo, const float* bias,
                          float* C, long long M, int N, int K) {
    if (M <= 0) return BOA_OK;
    if (N % 4 != 0 || K % kT3BK != 0) return fail(BOA_ERR_FORMAT, "3xTF32 gemm shape N=%d K=%d unsupported", N, K);
    const bool resid = EPI == kEpiResid || EPI == kEpiBiasResid;
    ProfScope ps(m, cls, 2.0 * M * N * K,
                 4.0 * ((double)M * K + 2.0 * K * N) + 4.0 * (double)M * N * (resid ? 2 : 1));
    const int BN = tc_bn(N, M);
    CUtensorMap ta, th, tl;
    TRY(tmap_2d(m, A, (uint64_t)M, (uint64_t)K, kTcBM, 4, &ta));
    TRY(tmap_2d(m, Whi, (uint64_t)N, (uint64_t)K, (uint32_t)BN, 4, &th));
    TRY(tmap_2d(m, Wlo, (uint64_t)N, (uint64_t)K, (uint32_t)BN, 4, &tl));
    switch (BN) {
        case 48: TRY((launch_t3<48, EPI>(m, ta, th, tl, bias, C, M, N, K))); break;
        case 64: TRY((launch_t3<64, EPI>(m, ta, th, tl, bias, C, M, N, K))); break;
        default: TRY((launch_t3<128, EPI>(m, ta, th, tl, bias, C, M, N, K))); break;
    }
    return check_launch(m, "gemm_t3");
}

// FP8 form: the E4M3 copy (and per-row scales) of a projection's A operand
// with K inputs, in the view's FP8 scratch, which the producing kernel
// writes itself (gemm_f8 with prequant then skips its quantisation launch).
static F8Out f8_out(const boa_model* m, int K) {
    if (m->precision != BOA_PREC_FP8) return F8Out{nullptr, nullptr, 0};
    return F8Out{reinterpret_cast<__nv_fp8_e4m3*>(m->v.a8), m->v.a8s, (K + 127) / 128 * 128};
}

// The conv kernel writes the FP8 copy of u when one CTA holds a whole row.
static bool conv_writes_f8(const boa_model* m) { return m->precision == BOA_PREC_FP8 && m->E <= 512; }
// The decode-step scan writes the FP8 copy of its output rows (variant 0).
static bool scan_writes_f8(const boa_model* m, int Tc) {
    return m->precision == BOA_PREC_FP8 && Tc == 1 && m->scan_variant == 0;
}

template <int VPT>
static void launch_embed_ln(boa_model* m, const TokenSrc& ts, int S, int Tc, const DevLayer& L0) {
    const long long rows = (long long)S * Tc;
    const bool tc = m->precision == BOA_PREC_BF16;
    launch_k(m, k_embed_ln<VPT>, dim3((unsigned)((rows + 7) / 8)), 256, 0, 1, ts, S, Tc, m->embed, L0.ln_a_w,
             L0.ln_a_b, m->v.x, m->v.xn, tc ? m->v.xn_b : nullptr, f8_out(m, m->d));
}

template <int VPT>
static void launch_ln_ln(boa_model* m, long long rows, const DevLayer& L, const DevLayer* next) {
    const bool tc = m->precision == BOA_PREC_BF16;
    // the BF16 copy of x feeds the head (last block) or the next block's FFN
    __nv_bfloat16* xb = (tc && (!next || m->F)) ? m->v.x_b : nullptr;
    // FP8: the next block's in_proj input xn, or the head's input x (both K = d)
    launch_k(m, k_ln_ln<VPT>, dim3((unsigned)((rows + 7) / 8)), 256, 0, 1, rows, m->v.x, L.ln_b_w, L.ln_b_b,
             next ? next->ln_a_w : nullptr, next ? next->ln_a_b : nullptr, m->v.xn, xb, tc ? m->v.xn_b : nullptr,
             f8_out(m, m->d));
}

static boa_status embed_ln(boa_model* m, const TokenSrc& ts, int S, int Tc) {
    const double rows = (double)S * Tc;
    ProfScope ps(m, BOA_KC_EMBED_LN, rows * m->d * 8.0, rows * (1.0 + 8.0 * m->d));
    switch (m->d) {
        case 64: launch_embed_ln<2>(m, ts, S, Tc, m->layers[0]); break;
        case 128: launch_embed_ln<4>(m, ts, S, Tc, m->layers[0]); break;
        case 256: launch_embed_ln<8>(m, ts, S, Tc, m->layers[0]); break;
    }
    return check_launch(m, "embed_ln");
}

static boa_status ln_ln(boa_model* m, long long rows, int l) {
    const DevLayer& L = m->layers[l];
    const DevLayer* next = (l + 1 < m->nl) ? &m->layers[l + 1] : nullptr;
    ProfScope ps(m, BOA_KC_LN, (double)rows * m->d * (next ? 16.0 : 8.0), (double)rows * m->d * 4.0 * (next ? 3 : 2));
    switch (m->d) {
        case 64: launch_ln_ln<2>(m, rows, L, next); break;
        case 128: launch_ln_ln<4>(m, rows, L, next); break;
        case 256: launch_ln_ln<8>(m, rows, L, next); break;
    }
    return check_launch(m, "ln_ln");
}

static boa_status conv(boa_model* m, int l, int S, int Tc) {
    const DevLayer& L = m->layers[l];
    const int G = 1;                                  // one stream per thread: more loads in flight
    dim3 grid((m->E + 511) / 512, (S + G - 1) / G);   // 4 channels per thread
    float* win = m->v.conv + (size_t)l * m->v.S_all * (m->K - 1) * m->E;
    const double rows = (double)S * Tc;
    ProfScope ps(m, BOA_KC_CONV, rows * m->E * (2.0 * m->K + 4),
                 4.0 * (2 * rows * m->E + (double)S * ((m->K - 1) + std::min(Tc, m->K - 1)) * m->E));
    __nv_bfloat16* ub = m->precision == BOA_PREC_BF16 ? m->v.u_b : nullptr;
    const F8Out f8 = conv_writes_f8(m) ? f8_out(m, m->E) : F8Out{nullptr, nullptr, 0};
#define CONV_CASE(KK, GG) \
    launch_k(m, k_conv_silu<KK, GG>, grid, 128, 0, 1, m->v.xz, m->E, L.conv_w, L.conv_b, win, \
             (const SlotState*)m->v.slots, m->v.u, ub, S, Tc, f8)
    if (G == 8) {
        switch (m->K) { case 2: CONV_CASE(2, 8); break; case 3: CONV_CASE(3, 8); break; default: CONV_CASE(4, 8); break; }
    } else {
        switch (m->K) { case 2: CONV_CASE(2, 1); break; case 3: CONV_CASE(3, 1); break; default: CONV_CASE(4, 1); break; }
    }
#undef CONV_CASE
    return check_launch(m, "conv");
}

// Decode-step scan kernels (scan_variant, a tuning knob of boa_autotune; none
// changes a result, every variant performs k_scan's per-channel arithmetic):
//   0  persistent, bulk-copy fed (k_scan_step_bulk)
//   1  four channels per thread, one stream per CTA (k_scan_step4)
//   2  one channel per thread, one stream per CTA (k_scan, G = 1)
//   3  one channel per thread, eight streams per CTA (k_scan, G = 8)
// Chunks of more than one step (compression) always take k_scan with G = 1.

// Ring stages and CTAs per SM for k_scan_step_bulk: about 512 threads per SM
// and at least two stages per CTA within 227 KB of shared memory.
static void step_bulk_shape(int E, int N, int r, int& cps, int& stages) {
    const size_t stage = 4 * (size_t)step_stage_floats(N, r, E);
    const int threads = E / 2;
    cps = std::max(1, std::min(8, 512 / threads));
    const size_t budget = 227 * 1024;
    while (cps > 1 && (2 * stage + 1024) * cps > budget) cps--;
    stages = (int)std::min<size_t>(kStepMaxStages, (budget / cps - 1024) / stage);
}

template <int RR>
static boa_status launch_step_bulk(boa_model* m, const DevLayer& L, float* hs, __nv_bfloat16* ygb, int S) {
    int cps = 1, stages = 2;
    step_bulk_shape(m->E, m->N, m->r, cps, stages);
    const size_t smem = (size_t)stages * 4 * step_stage_floats(m->N, RR, m->E);
    // opt in (once per device) to the largest dynamic shared memory this kernel can have
    static SmemOptIn optin;
    TRY((smem_opt_in(optin, k_scan_step_bulk<16, RR>, -1, m->device, "decode scan")));
    const int grid = (int)std::min<long long>(S, (long long)m->num_sms * cps);
    launch_k(m, k_scan_step_bulk<16, RR>, dim3((unsigned)grid), dim3((unsigned)(m->E / 2)), smem, 1, m->v.u, m->v.xz,
             m->v.dbc, L.dt_w, L.dt_b, L.A2, L.D, hs, m->v.yg, ygb, m->E, S, stages, m->err.p,
             scan_writes_f8(m, 1) ? f8_out(m, m->E) : F8Out{nullptr, nullptr, 0});
    return BOA_OK;
}

static boa_status scan(boa_model* m, int l, int S, int Tc) {
    const DevLayer& L = m->layers[l];
    float* hs = m->v.h + (size_t)l * m->v.S_all * m->N * m->E;
    const double rows = (double)S * Tc;
    ProfScope ps(m, BOA_KC_SCAN, rows * m->E * (2.0 * m->r + 5.0 * m->N + 12),
                 4.0 * (rows * (3.0 * m->E + m->R2) + 2.0 * S * m->N * m->E));
    __nv_bfloat16* ygb = m->precision == BOA_PREC_BF16 ? m->v.yg_b : nullptr;
    const int v = Tc == 1 ? m->scan_variant : 2;
    if (v == 0) {
        switch (m->r) {
            case 4: TRY(launch_step_bulk<4>(m, L, hs, ygb, S)); break;
            case 8: TRY(launch_step_bulk<8>(m, L, hs, ygb, S)); break;
            default: TRY(launch_step_bulk<16>(m, L, hs, ygb, S)); break;
        }
        return check_launch(m, "scan_step_bulk");
    }
    if (v == 1) {
        dim3 g4((m->E + 4 * kScanThreads - 1) / (4 * kScanThreads), S);
#define STEP4_CASE(RR)                                                                                       \
    launch_k(m, k_scan_step4<16, RR>, g4, kScanThreads, 0, 1, m->v.u, m->v.xz, m->v.dbc, L.dt_w, L.dt_b, L.A2, L.D, \
             hs, m->v.yg, ygb, m->E)
        switch (m->r) { case 4: STEP4_CASE(4); break; case 8: STEP4_CASE(8); break; default: STEP4_CASE(16); break; }
#undef STEP4_CASE
        return check_launch(m, "scan_step4");
    }
    const int G = v == 3 ? 8 : 1;
    dim3 grid((m->E + kScanThreads - 1) / kScanThreads, (S + G - 1) / G);
#define SCAN_CASE(RR, GG)                                                                                         \
    launch_k(m, k_scan<16, RR, GG>, grid, kScanThreads, 0, 1, m->v.u, m->v.xz, m->v.dbc, L.dt_w, L.dt_b, L.A2, L.D, \
             hs, m->v.yg, ygb, m->E, S, Tc)
#define SCAN_R(GG)                      \
    switch (m->r) {                     \
        case 4: SCAN_CASE(4, GG); break; \
        case 8: SCAN_CASE(8, GG); break; \
        default: SCAN_CASE(16, GG); break; \
    }
    if (G == 8) { SCAN_R(8) } else { SCAN_R(1) }
#undef SCAN_R
#undef SCAN_CASE
    return check_launch(m, "scan");
}

// The predictor over S x Tc rows: embedding, n_l blocks, head (Alg. 1).
// embedded: the input rows x / xn were already written (decode steps after
// the first, by the previous step's decode kernel).
static boa_status forward(boa_model* m, const TokenSrc& ts, int S, int Tc, bool embedded = false) {
    const long long rows = (long long)S * Tc;
    const int d = m->d, E = m->E;
    const bool tc = m->precision == BOA_PREC_BF16;
    if (!embedded) TRY(embed_ln(m, ts, S, Tc));
    for (int l = 0; l < m->nl; l++) {
        const DevLayer& L = m->layers[l];
        if (tc) {
            const auto& B = m->blayers[l];
            TRY(gemm_tc<kEpiStore>(m, BOA_KC_GEMM_IN, m->v.xn_b, B.in_w, nullptr, m->v.xz, nullptr, rows, 2 * E, d));
            TRY(conv(m, l, S, Tc));
            TRY(gemm_tc<kEpiStore>(m, BOA_KC_GEMM_X, m->v.u_b, B.x_w, nullptr, m->v.dbc, nullptr, rows, m->R2, E));
            TRY(scan(m, l, S, Tc));
            TRY(gemm_tc<kEpiResid>(m, BOA_KC_GEMM_OUT, m->v.yg_b, B.out_w, nullptr, m->v.x, m->F ? m->v.x_b : nullptr,
                                   rows, d, E));
            if (m->F) {
                TRY(gemm_tc<kEpiBiasGelu>(m, BOA_KC_GEMM_FFN, m->v.x_b, B.w1, L.b1, m->v.hid, m->v.hid_b, rows, m->F, d));
                TRY(gemm_tc<kEpiBiasResid>(m, BOA_KC_GEMM_FFN, m->v.hid_b, B.w2, L.b2, m->v.x, nullptr, rows, d, m->F));
            }
        } else if (m->precision == BOA_PREC_FP8) {
            // the LayerNorm kernels (and the decoder's next-step embedding)
            // write in_proj's FP8 input, conv x_proj's, the decode-step scan
            // out_proj's; the chunked scan and the FFN are quantised here
            const auto& Q = m->qlayers[l];
            TRY(gemm_f8<kEpiStore>(m, BOA_KC_GEMM_IN, m->v.xn, Q.in_w, Q.in_s, nullptr, m->v.xz, rows, 2 * E, d, true));
            TRY(conv(m, l, S, Tc));
            TRY(gemm_f8<kEpiStore>(m, BOA_KC_GEMM_X, m->v.u, Q.x_w, Q.x_s, nullptr, m->v.dbc, rows, m->R2, E,
                                   conv_writes_f8(m)));
            TRY(scan(m, l, S, Tc));
            TRY(gemm_f8<kEpiResid>(m, BOA_KC_GEMM_OUT, m->v.yg, Q.out_w, Q.out_s, nullptr, m->v.x, rows, d, E,
                                   scan_writes_f8(m, Tc)));
            if (m->F) {
                TRY(gemm_f8<kEpiBiasGelu>(m, BOA_KC_GEMM_FFN, m->v.x, Q.w1, Q.w1_s, L.b1, m->v.hid, rows, m->F, d));
                TRY(gemm_f8<kEpiBiasResid>(m, BOA_KC_GEMM_FFN, m->v.hid, Q.w2, Q.w2_s, L.b2, m->v.x, rows, d, m->F));
            }
        } else if (m->precision == BOA_PREC_TF32X3) {
            const auto& T = m->tlayers[l];
            TRY(gemm_t3<kEpiStore>(m, BOA_KC_GEMM_IN, m->v.xn, T.in_hi, T.in_lo, nullptr, m->v.xz, rows, 2 * E, d));
            TRY(conv(m, l, S, Tc));
            TRY(gemm_t3<kEpiStore>(m, BOA_KC_GEMM_X, m->v.u, T.x_hi, T.x_lo, nullptr, m->v.dbc, rows, m->R2, E));
            TRY(scan(m, l, S, Tc));
            TRY(gemm_t3<kEpiResid>(m, BOA_KC_GEMM_OUT, m->v.yg, T.out_hi, T.out_lo, nullptr, m->v.x, rows, d, E));
            if (m->F) {
                TRY(gemm_t3<kEpiBiasGelu>(m, BOA_KC_GEMM_FFN, m->v.x, T.w1_hi, T.w1_lo, L.b1, m->v.hid, rows, m->F, d));
                TRY(gemm_t3<kEpiBiasResid>(m, BOA_KC_GEMM_FFN, m->v.hid, T.w2_hi, T.w2_lo, L.b2, m->v.x, rows, d, m->F));
            }
        } else {
            TRY(gemm<kEpiStore>(m, BOA_KC_GEMM_IN, m->v.xn, L.in_wt, nullptr, m->v.xz, rows, 2 * E, d));
            TRY(conv(m, l, S, Tc));
            TRY(gemm<kEpiStore>(m, BOA_KC_GEMM_X, m->v.u, L.x_wt, nullptr, m->v.dbc, rows, m->R2, E));
            TRY(scan(m, l, S, Tc));
            TRY(gemm<kEpiResid>(m, BOA_KC_GEMM_OUT, m->v.yg, L.out_wt, nullptr, m->v.x, rows, d, E));
            if (m->F) {
                TRY(gemm<kEpiBiasGelu>(m, BOA_KC_GEMM_FFN, m->v.x, L.w1t, L.b1, m->v.hid, rows, m->F, d));
                TRY(gemm<kEpiBiasResid>(m, BOA_KC_GEMM_FFN, m->v.hid, L.w2t, L.b2, m->v.x, rows, d, m->F));
            }
        }
        TRY(ln_ln(m, rows, l));
    }
    if (tc) return gemm_tc<kEpiBias>(m, BOA_KC_GEMM_HEAD, m->v.x_b, m->head_wb, m->head_b, m->v.logits, nullptr, rows, 256, d);
    if (m->precision == BOA_PREC_TF32X3)
        return gemm_t3<kEpiBias>(m, BOA_KC_GEMM_HEAD, m->v.x, m->head_hi, m->head_lo, m->head_b, m->v.logits, rows, 256, d);
    if (m->precision == BOA_PREC_FP8)    // the last LayerNorm wrote the head's FP8 input
        return gemm_f8<kEpiBias>(m, BOA_KC_GEMM_HEAD, m->v.x, m->head_w8, m->head_s, m->head_b, m->v.logits, rows, 256,
                                 d, true);
    return gemm<kEpiBias>(m, BOA_KC_GEMM_HEAD, m->v.x, m->head_wt, m->head_b, m->v.logits, rows, 256, d);
}

// Bounded waits that timed out (tensor-core pipelines, the bulk-copy scan)
// leave a nonzero code in m->err.
static boa_status check_tc_error(boa_model* m) {
    if (!m->err.p) return BOA_OK;
    int h = 0;
    CU(cudaMemcpyAsync(&h, m->err.p, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
    CU(cudaStreamSynchronize(m->stream));
    if (h) {
        cudaMemsetAsync(m->err.p, 0, sizeof(int), m->stream);
        return fail(BOA_ERR_CUDA, "a pipeline wait on the device timed out (code %d: %s)", h,
                    h == 3 ? "decode scan bulk copy" : h == 4 ? "on-chip decoder weight stream" : "tensor-core GEMM");
    }
    return BOA_OK;
}

static boa_status ensure_workspace(boa_model* m, size_t S, size_t rows) {
    const size_t d = m->d, E = m->E;
    TRY(m->x.ensure(rows * d));
    TRY(m->xn.ensure(rows * d));
    TRY(m->xz.ensure(rows * 2 * E));
    TRY(m->u.ensure(rows * E));
    TRY(m->dbc.ensure(rows * m->R2));
    TRY(m->yg.ensure(rows * E));
    TRY(m->logits.ensure(rows * 256));
    if (m->F) TRY(m->hid.ensure(rows * m->F));
    if (!m->err.p) {
        TRY(m->err.ensure(1));
        CU(cudaMemset(m->err.p, 0, sizeof(int)));
    }
    if (m->precision == BOA_PREC_BF16) {
        TRY(m->xn_b.ensure(rows * d));
        TRY(m->u_b.ensure(rows * E));
        TRY(m->yg_b.ensure(rows * E));
        TRY(m->x_b.ensure(rows * d));
        if (m->F) TRY(m->hid_b.ensure(rows * m->F));
    }
    if (m->precision == BOA_PREC_FP8) {
        // E4M3 copies of a GEMM's activation rows, K padded to 128
        m->kp8 = (std::max<size_t>({d, E, (size_t)m->F}) + 127) / 128 * 128;
        TRY(m->a8.ensure(rows * m->kp8));
        TRY(m->a8s.ensure(rows));
    }
    TRY(m->h.ensure((size_t)m->nl * S * m->N * E));
    TRY(m->conv.ensure((size_t)m->nl * S * (m->K - 1) * E));
    TRY(m->st.ensure(S));
    TRY(m->slots.ensure(S));
    TRY(m->slot_beg.ensure(S + 1));
    return BOA_OK;
}

// Point the launchers at slots [s0, ...) of an S_all-slot batch with Tc rows
// per slot, launching on stream st.  The FP8 scratch (a8, a8s) of a view
// starts at row s0 Tc with room for kp8 bytes per row, but its rows are laid
// out with the stride of the projection that reads them (its K padded to
// 128), so a writer and the projection reading its rows use the same view.
static void bind_view(boa_model* m, size_t s0, size_t Tc, size_t S_all, cudaStream_t st) {
    View& v = m->v;
    const size_t r0 = s0 * Tc;
    auto at = [r0](auto* p, size_t per) { return p ? p + r0 * per : p; };
    v.x = at(m->x.p, m->d);
    v.xn = at(m->xn.p, m->d);
    v.xz = at(m->xz.p, 2 * (size_t)m->E);
    v.u = at(m->u.p, m->E);
    v.dbc = at(m->dbc.p, m->R2);
    v.yg = at(m->yg.p, m->E);
    v.logits = at(m->logits.p, 256);
    v.hid = at(m->hid.p, m->F);
    v.xn_b = at(m->xn_b.p, m->d);
    v.u_b = at(m->u_b.p, m->E);
    v.yg_b = at(m->yg_b.p, m->E);
    v.x_b = at(m->x_b.p, m->d);
    v.hid_b = at(m->hid_b.p, m->F);
    v.a8 = at(m->a8.p, m->kp8);
    v.a8s = at(m->a8s.p, 1);
    v.h = m->h.p ? m->h.p + s0 * m->N * m->E : nullptr;
    v.conv = m->conv.p ? m->conv.p + s0 * (m->K - 1) * m->E : nullptr;
    v.slots = m->slots.p ? m->slots.p + s0 : nullptr;
    v.st = m->st.p ? m->st.p + s0 : nullptr;
    v.slot_beg = m->slot_beg.p ? m->slot_beg.p + s0 : nullptr;
    v.S_all = S_all;
    v.stream = st;
}

// Streams and events for P decode lanes (created once, outside any capture).
static boa_status ensure_lanes(boa_model* m, int P) {
    while ((int)m->lane_streams.size() < P) {
        cudaStream_t ls;
        CU(cudaStreamCreateWithFlags(&ls, cudaStreamNonBlocking));
        m->lane_streams.push_back(ls);
    }
    while ((int)m->lane_events.size() < P + 1) {
        cudaEvent_t e;
        CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        m->lane_events.push_back(e);
    }
    return BOA_OK;
}

// Decode lanes: the slots split into P contiguous groups whose step loops
// are independent (a slot's rows, state and coder touch no other slot), so
// each group's launches can go to its own stream and overlap the others'.
static int decode_lanes(const boa_model* m, int S) {
    const int P = m->decode_lanes > 0 ? m->decode_lanes : (S >= 2048 ? 2 : 1);
    return std::max(1, std::min(P, S));
}

static boa_status ensure_streams(boa_model* m, size_t n) {
    TRY(m->flags.ensure(n));
    TRY(m->in_off.ensure(n + 1));
    TRY(m->out_off.ensure(n + 1));
    TRY(m->lens.ensure(n));
    TRY(m->sizes.ensure(n));
    TRY(m->trace_off.ensure(n));
    TRY(m->sched.ensure(n));
    return BOA_OK;
}

// Stage the per-stream index arrays on the device and size the CDF trace.
// Each array gets its own region of the pinned staging buffer: the copies are
// asynchronous and read the host memory only when they execute.
static boa_status upload_index(boa_model* m, size_t S, const uint64_t* in_off, const uint64_t* out_off,
                               const uint64_t* lens, const uint64_t* coded_sizes = nullptr) {
    TRY(m->h_u64.ensure(5 * (S + 1)));
    uint64_t* hb = m->h_u64.p;
    memcpy(hb, in_off, (S + 1) * 8);
    memcpy(hb + (S + 1), out_off, (S + 1) * 8);
    memcpy(hb + 2 * (S + 1), lens, S * 8);
    uint64_t* toff = hb + 3 * (S + 1);
    uint64_t acc = 0;
    for (size_t i = 0; i < S; i++) {
        toff[i] = acc;
        acc += lens[i] >= 2 ? lens[i] - 1 : 0;
    }
    CU(cudaMemcpyAsync(m->in_off.p, hb, (S + 1) * 8, cudaMemcpyHostToDevice, m->stream));
    CU(cudaMemcpyAsync(m->out_off.p, hb + (S + 1), (S + 1) * 8, cudaMemcpyHostToDevice, m->stream));
    CU(cudaMemcpyAsync(m->lens.p, hb + 2 * (S + 1), S * 8, cudaMemcpyHostToDevice, m->stream));
    CU(cudaMemcpyAsync(m->trace_off.p, toff, S * 8, cudaMemcpyHostToDevice, m->stream));
    if (coded_sizes) {
        uint64_t* cs = hb + 4 * (S + 1);
        memcpy(cs, coded_sizes, S * 8);
        CU(cudaMemcpyAsync(m->sizes.p, cs, S * 8, cudaMemcpyHostToDevice, m->stream));
    }
    m->trace_n = 0;
    if (m->trace_on) {
        TRY(m->trace.ensure(std::max<uint64_t>(acc, 1)));
        m->trace_n = acc;
    }
    return BOA_OK;
}

// Slot schedule: streams of length >= 2 go, longest first, to the slot with
// the least work so far (ties to the lower slot); each slot runs its list in
// order.  The assignment only balances work: a stream's bytes do not depend
// on its slot.
struct Schedule {
    int S = 0;
    std::vector<int> sched, beg;
    std::vector<std::vector<int>> lists;
};

static void build_schedule(const uint64_t* lens, size_t n, size_t max_slots, Schedule& out) {
    std::vector<int> order;
    for (size_t i = 0; i < n; i++)
        if (lens[i] >= 2) order.push_back((int)i);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return lens[a] > lens[b]; });
    const int S = (int)std::min(order.size(), max_slots);
    out.S = S;
    out.lists.assign(S, {});
    std::vector<std::pair<uint64_t, int>> heap;   // (load, slot), min-heap
    for (int s = 0; s < S; s++) heap.push_back({0, s});
    auto cmp = [](const std::pair<uint64_t, int>& a, const std::pair<uint64_t, int>& b) { return a > b; };
    std::make_heap(heap.begin(), heap.end(), cmp);
    for (int i : order) {
        std::pop_heap(heap.begin(), heap.end(), cmp);
        auto top = heap.back();
        heap.pop_back();
        out.lists[top.second].push_back(i);
        top.first += lens[i] - 1;
        heap.push_back(top);
        std::push_heap(heap.begin(), heap.end(), cmp);
    }
    out.sched.clear();
    out.beg.assign(S + 1, 0);
    for (int s = 0; s < S; s++) {
        out.beg[s] = (int)out.sched.size();
        out.sched.insert(out.sched.end(), out.lists[s].begin(), out.lists[s].end());
    }
    out.beg[S] = (int)out.sched.size();
}

static boa_status upload_schedule(boa_model* m, const Schedule& sc) {
    TRY(m->h_sched.ensure(sc.sched.size() + sc.beg.size() + 1));
    int* hp = m->h_sched.p;
    memcpy(hp, sc.sched.data(), sc.sched.size() * 4);
    memcpy(hp + sc.sched.size(), sc.beg.data(), sc.beg.size() * 4);
    if (!sc.sched.empty())
        CU(cudaMemcpyAsync(m->sched.p, hp, sc.sched.size() * 4, cudaMemcpyHostToDevice, m->stream));
    CU(cudaMemcpyAsync(m->slot_beg.p, hp + sc.sched.size(), sc.beg.size() * 4, cudaMemcpyHostToDevice, m->stream));
    return BOA_OK;
}

static boa_status zero_state(boa_model* m, size_t S) {
    CU(cudaMemsetAsync(m->h.p, 0, (size_t)m->nl * S * m->N * m->E * 4, m->stream));
    CU(cudaMemsetAsync(m->conv.p, 0, (size_t)m->nl * S * (m->K - 1) * m->E * 4, m->stream));
    return BOA_OK;
}

static StreamTable stream_table(boa_model* m, bool decoding) {
    StreamTable tb;
    tb.in_off = m->in_off.p;
    tb.in_size = decoding ? m->sizes.p : nullptr;
    tb.lens = m->lens.p;
    tb.out_off = m->out_off.p;
    tb.sizes = m->sizes.p;
    tb.flags = m->flags.p;
    tb.trace = m->trace_on ? m->trace.p : nullptr;
    tb.trace_off = m->trace_off.p;
    return tb;
}

// The bound view's per-slot model state, for kernels that reset a slot.
static SlotMem slot_mem(const boa_model* m) {
    SlotMem sm;
    sm.h = m->v.h;
    sm.conv = m->v.conv;
    sm.layers = m->nl;
    sm.S = (int)m->v.S_all;
    sm.h_per = m->N * m->E;
    sm.conv_per = (m->K - 1) * m->E;
    return sm;
}

static boa_status compress_impl(boa_model* m, size_t n, const uint8_t* d_in, const uint64_t* in_off,
                                uint8_t* d_out, const uint64_t* out_off, uint64_t* out_sizes) {
    if (n == 0) return BOA_OK;
    if (n > (1u << 30)) return fail(BOA_ERR_ARG, "too many streams");
    std::vector<uint64_t> lens(n);
    uint64_t maxlen = 0;
    for (size_t i = 0; i < n; i++) {
        if (in_off[i + 1] < in_off[i] || out_off[i + 1] < out_off[i]) return fail(BOA_ERR_ARG, "offsets must be non-decreasing");
        lens[i] = in_off[i + 1] - in_off[i];
        if (out_off[i + 1] - out_off[i] < boa_max_compressed_size(lens[i]))
            return fail(BOA_ERR_OUTPUT_TOO_SMALL, "stream %zu: output slot %llu < %zu", i,
                        (unsigned long long)(out_off[i + 1] - out_off[i]), boa_max_compressed_size(lens[i]));
        maxlen = std::max(maxlen, lens[i]);
    }
    m->launches = 0;
    m->prof_step = true;
    m->prof_phase = 0;
    Schedule sc;
    build_schedule(lens.data(), n, m->max_slots, sc);
    const int S = std::max(sc.S, 1);
    const int Tc = (int)std::max<uint64_t>(1, std::min<uint64_t>(maxlen > 1 ? maxlen - 1 : 1, m->max_rows / S));
    uint64_t chunks = 0;
    for (auto& lst : sc.lists) {
        uint64_t c = 0;
        for (int i : lst) c += (lens[i] - 1 + Tc - 1) / Tc;
        chunks = std::max(chunks, c);
    }
    TRY(ensure_workspace(m, S, (size_t)S * Tc));
    TRY(ensure_streams(m, n));
    TRY(upload_index(m, n, in_off, out_off, lens.data()));
    TRY(upload_schedule(m, sc));
    TRY(zero_state(m, S));
    bind_view(m, 0, Tc, S, m->stream);
    StreamTable tb = stream_table(m, false);
    SlotMem mem = slot_mem(m);
    const int tb128 = 128;
    k_enc_trivial<<<(unsigned)((n + tb128 - 1) / tb128), tb128, 0, m->stream>>>((int)n, d_in, tb, d_out);
    TRY(check_launch(m, "enc_trivial"));
    if (sc.S > 0) {
        const unsigned wgrid = (unsigned)((S + 3) / 4);
        launch_k(m, k_enc_slots, dim3(wgrid), 128, 0, 1, S, 1, 0LL, (const int*)m->sched.p, (const int*)m->slot_beg.p,
                 m->slots.p, m->st.p, d_in, tb, d_out, mem);
        TRY(check_launch(m, "enc_slots"));
        TokenSrc ts{d_in, m->in_off.p, m->lens.p, m->slots.p};
        for (uint64_t c = 0; c < chunks; c++) {
            m->prof_steps[0][0] += m->prof_on ? 1 : 0;
            m->prof_steps[0][1]++;
            TRY(forward(m, ts, S, Tc));
            {
                ProfScope ps(m, BOA_KC_ENCODE, (double)S * Tc * 256 * 8, (double)S * Tc * (256 * 4 + 2));
                launch_k(m, k_encode, dim3(wgrid), 128, 0, 1, (const float*)m->v.logits, S, Tc,
                         (const SlotState*)m->v.slots, m->v.st, d_in, tb, d_out);
            }
            TRY(check_launch(m, "encode"));
            launch_k(m, k_enc_slots, dim3(wgrid), 128, 0, 1, S, 0, (long long)Tc, (const int*)m->sched.p,
                     (const int*)m->slot_beg.p, m->slots.p, m->st.p, d_in, tb, d_out, mem);
            TRY(check_launch(m, "enc_slots"));
        }
    }
    TRY(m->h_u32.ensure(n));
    CU(cudaMemcpyAsync(out_sizes, m->sizes.p, n * 8, cudaMemcpyDeviceToHost, m->stream));
    CU(cudaMemcpyAsync(m->h_u32.p, m->flags.p, n * 4, cudaMemcpyDeviceToHost, m->stream));
    CU(cudaStreamSynchronize(m->stream));
    prof_collect(m);
    m->last_status.assign(m->h_u32.p, m->h_u32.p + n);
    for (size_t i = 0; i < n; i++)
        if (lens[i] < 2) m->last_status[i] = 0;
    TRY(check_tc_error(m));
    for (size_t i = 0; i < n; i++)
        if (lens[i] >= 2 && m->h_u32.p[i])
            return fail(BOA_ERR_CUDA, "stream %zu: encoder status %u", i, m->h_u32.p[i]);
    return BOA_OK;
}

template <int VPT>
static void launch_dec_init(boa_model* m, int S, const uint8_t* cin, const StreamTable& tb, uint8_t* out,
                            const NextEmbed& ne) {
    launch_k(m, k_dec_slots_init<VPT>, dim3((unsigned)((S + 3) / 4)), 128, 0, 1, S, (const int*)m->sched.p,
             m->v.slot_beg, m->v.slots, m->v.st, cin, tb, out, ne);
}

template <int VPT>
static void launch_decode(boa_model* m, int S, const uint8_t* cin, const StreamTable& tb, uint8_t* out,
                          const NextEmbed& ne, const SlotMem& mem) {
    launch_k(m, k_decode<VPT>, dim3((unsigned)((S + 3) / 4)), 128, 0, 1, (const float*)m->v.logits, S,
             (const int*)m->sched.p, m->v.slot_beg, m->v.slots, m->v.st, cin, tb, out, ne, mem);
}

// After a decompression's launches: per-stream status back to the host,
// profiling totals folded in, device-side wait failures and streams that did
// not decode cleanly reported.
static boa_status finish_decode(boa_model* m, size_t n) {
    TRY(m->h_u32.ensure(n));
    CU(cudaMemcpyAsync(m->h_u32.p, m->flags.p, n * 4, cudaMemcpyDeviceToHost, m->stream));
    CU(cudaStreamSynchronize(m->stream));
    prof_collect(m);
    m->last_status.assign(m->h_u32.p, m->h_u32.p + n);
    TRY(check_tc_error(m));
    for (size_t i = 0; i < n; i++)
        if (m->h_u32.p[i]) return fail(BOA_ERR_CORRUPT, "stream %zu did not decode cleanly (flags %u)", i, m->h_u32.p[i]);
    return BOA_OK;
}

// Why the on-chip decoder cannot run this model (nullptr: it can).  Its
// state layout holds kOcSlots streams' SSM state and conv windows for up to
// kOcMaxLayers blocks in TMEM, and its weight stream covers the Mamba blocks
// without an FFN.
static const char* onchip_unsupported(const boa_model* m) {
    if (m->precision != BOA_PREC_FP32) return "it runs the FP32 form only";
    if (m->N != kOcNS) return "d_state must be 16";
    if (m->E > kOcMaxE || m->E % 4) return "d_inner must be a multiple of 4, at most 512";
    if (m->nl > kOcMaxLayers) return "at most 3 blocks";
    if (m->F) return "blocks with an FFN are not supported";
    if (m->K < 2 || m->K > 4) return "conv width must be 2 .. 4";
    if (m->r != 4 && m->r != 8 && m->r != 16) return "dt_rank must be 4, 8 or 16";
    if (!supported_d(m->d)) return "d_model must be 64, 128 or 256";
    if (oc_smem_bytes(m->d, m->E) > 227 * 1024) return "activations do not fit shared memory";
    auto al = [](const void* p) { return ((uintptr_t)p & 15) == 0; };
    if (!al(m->head_wt)) return "weight matrices must be 16-byte aligned";
    for (const DevLayer& L : m->layers)
        if (!al(L.in_wt) || !al(L.x_wt) || !al(L.out_wt)) return "weight matrices must be 16-byte aligned";
    return nullptr;
}

template <int VPT, int R>
static boa_status launch_onchip(boa_model* m, const OcModel& M, const OcWork& W, int grid) {
    static SmemOptIn optin;
    const size_t smem = oc_smem_bytes(m->d, m->E);
    TRY((smem_opt_in(optin, k_decode_onchip<VPT, R>, (int)smem, m->device, "on-chip decoder")));
    launch_k(m, k_decode_onchip<VPT, R>, dim3((unsigned)grid), dim3(kOcBlock), smem, 1, M, W);
    return BOA_OK;
}

// Decompression by the on-chip persistent decoder: one launch decodes every
// stream of two bytes or more (longest first from a device-side queue, one
// CTA per SM with kOcSlots streams at a time); streams of 0 or 1 bytes as in
// decompress_impl.
static boa_status decompress_onchip(boa_model* m, size_t n, const uint8_t* d_in, const uint64_t* in_off,
                                    const uint64_t* csz, const uint64_t* lens, uint8_t* d_out,
                                    const uint64_t* out_off) {
    if (const char* why = onchip_unsupported(m)) return fail(BOA_ERR_ARG, "on-chip decoder: %s", why);
    m->launches = 0;
    m->prof_phase = 1;
    TRY(ensure_workspace(m, 1, 1));
    TRY(ensure_streams(m, n));
    TRY(upload_index(m, n, in_off, out_off, lens, csz));
    bind_view(m, 0, 1, 1, m->stream);
    StreamTable tb = stream_table(m, true);
    const int tb128 = 128;
    k_dec_trivial<<<(unsigned)((n + tb128 - 1) / tb128), tb128, 0, m->stream>>>((int)n, d_in, tb, d_out);
    TRY(check_launch(m, "dec_trivial"));
    std::vector<int> order;
    uint64_t steps = 0;
    for (size_t i = 0; i < n; i++)
        if (lens[i] >= 2) {
            order.push_back((int)i);
            steps += lens[i] - 1;
        }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return lens[a] > lens[b]; });
    if (!order.empty()) {
        TRY(m->h_sched.ensure(order.size()));
        memcpy(m->h_sched.p, order.data(), order.size() * sizeof(int));
        CU(cudaMemcpyAsync(m->sched.p, m->h_sched.p, order.size() * sizeof(int), cudaMemcpyHostToDevice, m->stream));
        TRY(m->oc_next.ensure(1));
        CU(cudaMemsetAsync(m->oc_next.p, 0, sizeof(int), m->stream));
        OcModel M{};
        for (int l = 0; l < m->nl; l++) {
            const DevLayer& L = m->layers[l];
            M.L[l] = OcLayer{L.in_wt, L.x_wt, L.out_wt, L.conv_w, L.conv_b, L.dt_w, L.dt_b, L.A2, L.D,
                             L.ln_a_w, L.ln_a_b, L.ln_b_w, L.ln_b_b};
        }
        M.embed = m->embed;
        M.head_wt = m->head_wt;
        M.head_b = m->head_b;
        M.nl = m->nl;
        M.E = m->E;
        M.K = m->K;
        const OcWork W{m->sched.p, (int)order.size(), m->oc_next.p, d_in, tb, d_out, m->err.p};
        const int grid = (int)std::min<size_t>((size_t)m->num_sms, (order.size() + kOcSlots - 1) / kOcSlots);
        m->prof_step = true;
        m->prof_steps[1][0] += steps;
        m->prof_steps[1][1] += steps;
        {
            // per decoded byte: the projections (2 flops per weight) and the
            // weight bytes one CTA streams per step, shared by its slots
            const double wfloats = (double)m->nl * (2.0 * m->E * m->d + (double)m->E * m->R2 + (double)m->E * m->d) +
                                   256.0 * m->d;
            ProfScope ps(m, BOA_KC_DECODE, 2.0 * wfloats * (double)steps, 4.0 * wfloats * (double)steps / kOcSlots);
            boa_status st = BOA_OK;
            switch (m->d * 100 + m->r) {
                case 6404: st = launch_onchip<2, 4>(m, M, W, grid); break;
                case 6408: st = launch_onchip<2, 8>(m, M, W, grid); break;
                case 6416: st = launch_onchip<2, 16>(m, M, W, grid); break;
                case 12804: st = launch_onchip<4, 4>(m, M, W, grid); break;
                case 12808: st = launch_onchip<4, 8>(m, M, W, grid); break;
                case 12816: st = launch_onchip<4, 16>(m, M, W, grid); break;
                case 25604: st = launch_onchip<8, 4>(m, M, W, grid); break;
                case 25608: st = launch_onchip<8, 8>(m, M, W, grid); break;
                default: st = launch_onchip<8, 16>(m, M, W, grid); break;
            }
            TRY(st);
        }
        TRY(check_launch(m, "decode_onchip"));
    }
    return finish_decode(m, n);
}

static boa_status decompress_impl(boa_model* m, size_t n, const uint8_t* d_in, const uint64_t* in_off,
                                  const uint64_t* in_sizes, const uint64_t* lens, uint8_t* d_out,
                                  const uint64_t* out_off) {
    if (n == 0) return BOA_OK;
    if (n > (1u << 30)) return fail(BOA_ERR_ARG, "too many streams");
    std::vector<uint64_t> csz(n);
    for (size_t i = 0; i < n; i++) {
        if (in_off[i + 1] < in_off[i] || out_off[i + 1] < out_off[i]) return fail(BOA_ERR_ARG, "offsets must be non-decreasing");
        csz[i] = in_sizes ? in_sizes[i] : in_off[i + 1] - in_off[i];
        if (csz[i] > in_off[i + 1] - in_off[i]) return fail(BOA_ERR_ARG, "stream %zu: in_sizes exceeds its slot", i);
        if (out_off[i + 1] - out_off[i] < lens[i]) return fail(BOA_ERR_OUTPUT_TOO_SMALL, "stream %zu: output slot too small", i);
        if (lens[i] >= 2 && csz[i] < 1) return fail(BOA_ERR_CORRUPT, "stream %zu: empty coded stream", i);
    }
    if (m->decoder == 1) return decompress_onchip(m, n, d_in, in_off, csz.data(), lens, d_out, out_off);
    m->launches = 0;
    m->prof_phase = 1;
    Schedule sc;
    build_schedule(lens, n, m->max_slots, sc);
    const int S = std::max(sc.S, 1);
    uint64_t steps = 0;
    for (auto& lst : sc.lists) {
        uint64_t c = 0;
        for (int i : lst) c += lens[i] - 1;
        steps = std::max(steps, c);
    }
    TRY(ensure_workspace(m, S, S));
    TRY(ensure_streams(m, n));
    TRY(upload_index(m, n, in_off, out_off, lens, csz.data()));
    TRY(upload_schedule(m, sc));
    TRY(zero_state(m, S));
    const int P = decode_lanes(m, S);
    TRY(ensure_lanes(m, P));
    bind_view(m, 0, 1, S, m->stream);
    StreamTable tb = stream_table(m, true);
    const DevLayer& L0 = m->layers[0];
    // the next step's input rows of the bound view's slots
    auto next_embed = [&] {
        return NextEmbed{m->embed, L0.ln_a_w, L0.ln_a_b, m->v.x, m->v.xn,
                         m->precision == BOA_PREC_BF16 ? m->v.xn_b : nullptr, f8_out(m, m->d)};
    };
    const int tb128 = 128;
    k_dec_trivial<<<(unsigned)((n + tb128 - 1) / tb128), tb128, 0, m->stream>>>((int)n, d_in, tb, d_out);
    TRY(check_launch(m, "dec_trivial"));
    if (sc.S > 0) {
        // Each lane's slots start through that lane's view, like its steps:
        // the FP8 form's input rows sit in the view's FP8 scratch with the
        // consuming projection's row stride, so a lane's rows are valid only
        // when written through the same view that reads them.
        for (int p = 0; p < P; p++) {
            const int s0 = (int)((long long)S * p / P), n_p = (int)((long long)S * (p + 1) / P) - s0;
            bind_view(m, s0, 1, S, m->stream);
            const NextEmbed ne0 = next_embed();
            switch (m->d) {
                case 64: launch_dec_init<2>(m, n_p, d_in, tb, d_out, ne0); break;
                case 128: launch_dec_init<4>(m, n_p, d_in, tb, d_out, ne0); break;
                default: launch_dec_init<8>(m, n_p, d_in, tb, d_out, ne0); break;
            }
            TRY(check_launch(m, "dec_init"));
        }
        bind_view(m, 0, 1, S, m->stream);
        // One decode step of lane p (slots [S p / P, S (p + 1) / P)) on stream ls.
        auto lane_step = [&](int p, cudaStream_t ls) -> boa_status {
            const int s0 = (int)((long long)S * p / P), n_p = (int)((long long)S * (p + 1) / P) - s0;
            bind_view(m, s0, 1, S, ls);
            TokenSrc ts{nullptr, m->in_off.p, m->lens.p, m->v.slots};
            TRY(forward(m, ts, n_p, 1, /*embedded=*/true));
            const NextEmbed ne = next_embed();
            const SlotMem mem = slot_mem(m);
            {
                ProfScope ps(m, BOA_KC_DECODE, (double)n_p * 256 * 8, (double)n_p * (256 * 4 + 2 + 8.0 * m->d));
                switch (m->d) {
                    case 64: launch_decode<2>(m, n_p, d_in, tb, d_out, ne, mem); break;
                    case 128: launch_decode<4>(m, n_p, d_in, tb, d_out, ne, mem); break;
                    default: launch_decode<8>(m, n_p, d_in, tb, d_out, ne, mem); break;
                }
            }
            return check_launch(m, "decode");
        };
        // `count` steps.  Timed steps run the lanes one after another on the
        // model's stream (one event pair per launch); otherwise each lane's
        // steps go to its own stream between a fork and a join, so one lane's
        // memory-bound scan overlaps another's projections.
        auto steps_block = [&](uint64_t count, bool timed) -> boa_status {
            m->prof_step = timed;
            m->prof_steps[1][0] += timed ? count : 0;
            m->prof_steps[1][1] += count;
            if (P == 1 || timed) {
                for (uint64_t k = 0; k < count; k++)
                    for (int p = 0; p < P; p++) TRY(lane_step(p, m->stream));
                return BOA_OK;
            }
            CU(cudaEventRecord(m->lane_events[0], m->stream));
            for (int p = 0; p < P; p++) {
                CU(cudaStreamWaitEvent(m->lane_streams[p], m->lane_events[0], 0));
                for (uint64_t k = 0; k < count; k++) TRY(lane_step(p, m->lane_streams[p]));
                CU(cudaEventRecord(m->lane_events[1 + p], m->lane_streams[p]));
                CU(cudaStreamWaitEvent(m->stream, m->lane_events[1 + p], 0));
            }
            return BOA_OK;
        };
        // Without profiling every step is eager or in a CUDA graph of
        // kGraphSteps steps (all its arguments are fixed for the call: slot
        // positions live in device memory).  With profiling, graphs still
        // run and one eager timed step precedes each graph launch; without
        // graphs every prof_stride-th step is timed.
        const uint64_t kGraphSteps = 32;
        uint64_t t = 0;
        if (m->use_graphs && steps >= 2 * kGraphSteps) {
            // one eager step first: lazily created resources (workspace
            // growth, kernel attributes, tensor maps) must not be created
            // under capture
            TRY(steps_block(1, m->prof_on));
            t++;
            cudaGraph_t g = nullptr;
            cudaGraphExec_t ge = nullptr;
            const uint64_t before = m->launches;
            const uint64_t all_before = m->prof_steps[1][1];
            CU(cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal));
            boa_status cs = steps_block(kGraphSteps, false);
            cudaError_t ce = cudaStreamEndCapture(m->stream, &g);
            bind_view(m, 0, 1, S, m->stream);
            if (cs != BOA_OK) { if (g) cudaGraphDestroy(g); return cs; }
            if (ce != cudaSuccess) return fail(BOA_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ce));
            ce = cudaGraphInstantiate(&ge, g, 0);
            cudaGraphDestroy(g);
            if (ce != cudaSuccess) return fail(BOA_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ce));
            const uint64_t per_graph = m->launches - before;
            m->launches = before;
            m->prof_steps[1][1] = all_before;
            while (t + kGraphSteps <= steps) {
                if (m->prof_on) {
                    boa_status st = steps_block(1, true);
                    if (st != BOA_OK) { cudaGraphExecDestroy(ge); return st; }
                    if (++t + kGraphSteps > steps) break;
                }
                ce = cudaGraphLaunch(ge, m->stream);
                if (ce != cudaSuccess) { cudaGraphExecDestroy(ge); return fail(BOA_ERR_CUDA, "graph launch: %s", cudaGetErrorString(ce)); }
                m->launches += per_graph;
                m->prof_steps[1][1] += kGraphSteps;
                t += kGraphSteps;
            }
            CU(cudaStreamSynchronize(m->stream));
            cudaGraphExecDestroy(ge);
        }
        for (; t < steps; t++) TRY(steps_block(1, m->prof_on && (t % (uint64_t)m->prof_stride) == 0));
        m->prof_step = true;
    }
    bind_view(m, 0, 1, S, m->stream);
    return finish_decode(m, n);
}

// ------------------------------------------------------------ public API

extern "C" boa_status boa_compress_device(boa_model* m, size_t n, const uint8_t* d_in, const uint64_t* in_off,
                                          uint8_t* d_out, const uint64_t* out_off, uint64_t* out_sizes) {
    if (!m || (n && (!d_in || !in_off || !d_out || !out_off || !out_sizes))) return fail(BOA_ERR_ARG, "null argument");
    MODEL_LOCK(m);
    CU(cudaSetDevice(m->device));
    return compress_impl(m, n, d_in, in_off, d_out, out_off, out_sizes);
}

extern "C" boa_status boa_decompress_device(boa_model* m, size_t n, const uint8_t* d_in, const uint64_t* in_off,
                                            const uint64_t* in_sizes, const uint64_t* lens, uint8_t* d_out,
                                            const uint64_t* out_off) {
    if (!m || (n && (!d_in || !in_off || !lens || !d_out || !out_off))) return fail(BOA_ERR_ARG, "null argument");
    MODEL_LOCK(m);
    CU(cudaSetDevice(m->device));
    return decompress_impl(m, n, d_in, in_off, in_sizes, lens, d_out, out_off);
}

// After compress_impl into m->d_out: the used part of every output slot
// packed on the device, then one copy back; stream i's bytes land at
// m->h_out.p + pk[i] (m->h_out holds at least the slots' total capacity).
static boa_status fetch_compressed(boa_model* m, size_t n, const uint64_t* sizes, std::vector<uint64_t>& pk) {
    pk.assign(n + 1, 0);
    for (size_t i = 0; i < n; i++) pk[i + 1] = pk[i] + sizes[i];
    TRY(m->pack_off.ensure(n + 1));
    TRY(m->d_pack.ensure(pk[n]));
    TRY(m->h_pack.ensure(n + 1));
    memcpy(m->h_pack.p, pk.data(), (n + 1) * 8);
    CU(cudaMemcpyAsync(m->pack_off.p, m->h_pack.p, (n + 1) * 8, cudaMemcpyHostToDevice, m->stream));
    k_compact<<<(unsigned)n, 256, 0, m->stream>>>(m->d_out.p, m->out_off.p, m->pack_off.p, m->d_pack.p, (int)n);
    TRY(check_launch(m, "compact"));
    CU(cudaMemcpyAsync(m->h_out.p, m->d_pack.p, pk[n], cudaMemcpyDeviceToHost, m->stream));
    CU(cudaStreamSynchronize(m->stream));
    return BOA_OK;
}

extern "C" boa_status boa_compress(boa_model* m, size_t n, const uint8_t* const* streams, const size_t* lens,
                                   uint8_t* const* out, const size_t* out_caps, size_t* out_sizes) {
    if (!m || (n && (!streams || !lens || !out || !out_caps || !out_sizes))) return fail(BOA_ERR_ARG, "null argument");
    MODEL_LOCK(m);
    if (n == 0) return BOA_OK;
    CU(cudaSetDevice(m->device));
    std::vector<uint64_t> in_off(n + 1), out_off(n + 1), sizes(n);
    in_off[0] = out_off[0] = 0;
    for (size_t i = 0; i < n; i++) {
        if (lens[i] && !streams[i]) return fail(BOA_ERR_ARG, "stream %zu is null", i);
        if (out_caps[i] < boa_max_compressed_size(lens[i]))
            return fail(BOA_ERR_OUTPUT_TOO_SMALL, "stream %zu: capacity %zu < %zu", i, out_caps[i], boa_max_compressed_size(lens[i]));
        in_off[i + 1] = in_off[i] + lens[i];
        out_off[i + 1] = out_off[i] + boa_max_compressed_size(lens[i]);
    }
    TRY(m->h_in.ensure(in_off[n]));
    TRY(m->h_out.ensure(out_off[n]));
    TRY(m->d_in.ensure(in_off[n]));
    TRY(m->d_out.ensure(out_off[n]));
    for (size_t i = 0; i < n; i++)
        if (lens[i]) memcpy(m->h_in.p + in_off[i], streams[i], lens[i]);
    CU(cudaMemcpyAsync(m->d_in.p, m->h_in.p, in_off[n], cudaMemcpyHostToDevice, m->stream));
    TRY(compress_impl(m, n, m->d_in.p, in_off.data(), m->d_out.p, out_off.data(), sizes.data()));
    std::vector<uint64_t> pk;
    TRY(fetch_compressed(m, n, sizes.data(), pk));
    for (size_t i = 0; i < n; i++) {
        out_sizes[i] = sizes[i];
        if (sizes[i]) memcpy(out[i], m->h_out.p + pk[i], sizes[i]);
    }
    return BOA_OK;
}

extern "C" boa_status boa_decompress(boa_model* m, size_t n, const uint8_t* const* bitstreams, const size_t* sizes,
                                     const size_t* lens, uint8_t* const* out) {
    if (!m || (n && (!bitstreams || !sizes || !lens || !out))) return fail(BOA_ERR_ARG, "null argument");
    MODEL_LOCK(m);
    if (n == 0) return BOA_OK;
    CU(cudaSetDevice(m->device));
    std::vector<uint64_t> in_off(n + 1), out_off(n + 1), l64(n);
    in_off[0] = out_off[0] = 0;
    for (size_t i = 0; i < n; i++) {
        if (sizes[i] && !bitstreams[i]) return fail(BOA_ERR_ARG, "bitstream %zu is null", i);
        in_off[i + 1] = in_off[i] + sizes[i];
        out_off[i + 1] = out_off[i] + lens[i];
        l64[i] = lens[i];
    }
    TRY(m->h_in.ensure(in_off[n]));
    TRY(m->h_out.ensure(out_off[n]));
    TRY(m->d_in.ensure(in_off[n]));
    TRY(m->d_out.ensure(out_off[n]));
    for (size_t i = 0; i < n; i++)
        if (sizes[i]) memcpy(m->h_in.p + in_off[i], bitstreams[i], sizes[i]);
    CU(cudaMemcpyAsync(m->d_in.p, m->h_in.p, in_off[n], cudaMemcpyHostToDevice, m->stream));
    boa_status st = decompress_impl(m, n, m->d_in.p, in_off.data(), nullptr, l64.data(), m->d_out.p, out_off.data());
    if (st != BOA_OK && st != BOA_ERR_CORRUPT) return st;
    std::string msg = g_err;
    CU(cudaMemcpyAsync(m->h_out.p, m->d_out.p, out_off[n], cudaMemcpyDeviceToHost, m->stream));
    CU(cudaStreamSynchronize(m->stream));
    for (size_t i = 0; i < n; i++)
        if (lens[i]) memcpy(out[i], m->h_out.p + out_off[i], lens[i]);
    if (st != BOA_OK) g_err = msg;
    return st;
}

extern "C" boa_status boa_profile_enable(boa_model* m, int on, int stride) {
    if (!m) return fail(BOA_ERR_ARG, "null model");
    MODEL_LOCK(m);
    m->prof_on = on != 0;
    m->prof_stride = stride > 0 ? stride : 1;
    return BOA_OK;
}

extern "C" boa_status boa_profile_reset(boa_model* m) {
    if (!m) return fail(BOA_ERR_ARG, "null model");
    MODEL_LOCK(m);
    for (int ph = 0; ph < 2; ph++)
        for (int i = 0; i < BOA_KC_COUNT; i++) {
            m->prof_launches[ph][i] = 0;
            m->prof_ms[ph][i] = m->prof_flops[ph][i] = m->prof_bytes[ph][i] = 0.0;
        }
    for (int ph = 0; ph < 2; ph++) m->prof_steps[ph][0] = m->prof_steps[ph][1] = 0;
    return BOA_OK;
}

extern "C" boa_status boa_profile_steps(const boa_model* m, int phase, uint64_t* timed, uint64_t* total) {
    if (!m || phase < 0 || phase > 1) return fail(BOA_ERR_ARG, "bad argument");
    MODEL_LOCK(m);
    if (timed) *timed = m->prof_steps[phase][0];
    if (total) *total = m->prof_steps[phase][1];
    return BOA_OK;
}

extern "C" boa_status boa_profile_read(const boa_model* m, int phase, int cls, uint64_t* launches,
                                       double* total_ms, double* flops, double* bytes) {
    if (!m || cls < 0 || cls >= BOA_KC_COUNT || phase < 0 || phase > 1) return fail(BOA_ERR_ARG, "bad argument");
    MODEL_LOCK(m);
    if (launches) *launches = m->prof_launches[phase][cls];
    if (total_ms) *total_ms = m->prof_ms[phase][cls];
    if (flops) *flops = m->prof_flops[phase][cls];
    if (bytes) *bytes = m->prof_bytes[phase][cls];
    return BOA_OK;
}

// ------------------------------------------------------------ microbenchmarks

extern "C" boa_status boa_microbench(int device, int test, int kind, int M, int N, int flags, double* rate,
                                     double* cycles_per_op) {
    if (!rate) return fail(BOA_ERR_ARG, "null argument");
    CU(cudaSetDevice(device));
    int sms = 0;
    CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    DevBuf<float> out, buf;
    DevBuf<unsigned long long> cyc;
    DevBuf<int> err;
    boa_status s = BOA_OK;
    auto body = [&]() -> boa_status {
        CU(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        CU(cudaEventCreate(&e0));
        CU(cudaEventCreate(&e1));
        float ms = 0.f;
        if (test == BOA_MB_EX2 || test == BOA_MB_FFMA || test == BOA_MB_FFMA2) {
            const int blocks = sms * 8, threads = 256, iters = 4096;
            TRY(out.ensure((size_t)blocks * threads));
            auto run = [&]() {
                if (test == BOA_MB_EX2) k_mb_ex2<<<blocks, threads, 0, st>>>(iters, out.p);
                else if (test == BOA_MB_FFMA) k_mb_ffma<<<blocks, threads, 0, st>>>(iters, out.p);
                else k_mb_ffma2<<<blocks, threads, 0, st>>>(iters, out.p);
            };
            run();                                    // warm-up
            CU(cudaEventRecord(e0, st));
            run();
            CU(cudaEventRecord(e1, st));
            CU(cudaEventSynchronize(e1));
            CU(cudaGetLastError());
            CU(cudaEventElapsedTime(&ms, e0, e1));
            const double ops = (double)blocks * threads * iters * 8;
            // results per second (ex2) or FLOP per second (2 per FMA, 4 per packed FMA)
            *rate = test == BOA_MB_EX2 ? ops / (ms * 1e-3) : ops * (test == BOA_MB_FFMA2 ? 4.0 : 2.0) / (ms * 1e-3);
            if (cycles_per_op) {
                int khz = 0;
                CU(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, device));
                // warp instructions per SM per cycle at the nominal clock
                *cycles_per_op = (ops / 32.0) / ((double)sms * ms * 1e-3 * khz * 1e3);
            }
            return BOA_OK;
        }
        if (test == BOA_MB_L2) {
            const size_t bytes = (size_t)32 << 20;
            const int passes = 20, blocks = sms * 4, threads = 512;
            TRY(buf.ensure(bytes / 4));
            TRY(out.ensure((size_t)blocks * threads));
            CU(cudaMemsetAsync(buf.p, 0, bytes, st));
            k_mb_l2<<<blocks, threads, 0, st>>>(reinterpret_cast<const float4*>(buf.p), bytes / 16, 1, out.p);
            CU(cudaEventRecord(e0, st));
            k_mb_l2<<<blocks, threads, 0, st>>>(reinterpret_cast<const float4*>(buf.p), bytes / 16, passes, out.p);
            CU(cudaEventRecord(e1, st));
            CU(cudaEventSynchronize(e1));
            CU(cudaGetLastError());
            CU(cudaEventElapsedTime(&ms, e0, e1));
            *rate = (double)bytes * passes / (ms * 1e-3);
            if (cycles_per_op) *cycles_per_op = 0.0;
            return BOA_OK;
        }
        if (test == BOA_MB_MMA) {
            const bool m_ok = M == 128 || M == 64;
            const bool n_ok = N >= (M == 64 ? 8 : 16) && N <= 256 && N % (M == 64 ? 8 : 16) == 0;
            const int modes = ((flags & kMbFlagFastIssue) ? 1 : 0) + ((flags & kMbFlagStages) ? 1 : 0) +
                              ((flags & kMbFlagStagesWarp) ? 1 : 0);
            if (kind < 0 || kind > 2 || !m_ok || !n_ok || (flags & ~31) || modes > 1 || (modes && (flags & 2)) ||
                ((flags & (kMbFlagStages | kMbFlagStagesWarp)) && (flags & kMbFlagATmem)) ||
                ((flags & kMbFlagATmem) && (kind != 0 || M != 128)) || ((flags & kMbFlagTwoAcc) && N > 128))
                return fail(BOA_ERR_ARG, "unsupported MMA microbenchmark shape (kind %d, M %d, N %d, flags %d)", kind,
                            M, N, flags);
            const bool fast = (flags & kMbFlagFastIssue) != 0;
            const int reps = 2048;
            TRY(cyc.ensure((size_t)sms));
            TRY(err.ensure(1));
            CU(cudaMemsetAsync(err.p, 0, 4, st));
            double instr = 4.0 * reps;
            const bool staged = (flags & (kMbFlagStages | kMbFlagStagesWarp)) != 0;
            if (staged) {
                const bool w = (flags & kMbFlagStagesWarp) != 0;
                void (*kern)(int, int, int, unsigned long long*, int*) =
                    kind == 0 ? (w ? k_mb_mma_stages<0, true> : k_mb_mma_stages<0, false>)
                    : kind == 1 ? (w ? k_mb_mma_stages<1, true> : k_mb_mma_stages<1, false>)
                                : (w ? k_mb_mma_stages<2, true> : k_mb_mma_stages<2, false>);
                static SmemOptIn opt_st[6];
                TRY(smem_opt_in(opt_st[2 * kind + (w ? 1 : 0)], kern, kMbStagesSmemBytes, device,
                                "MMA microbenchmark"));
                kern<<<sms, 128, kMbStagesSmemBytes, st>>>(M, N, 4, cyc.p, err.p);             // warm-up
                CU(cudaEventRecord(e0, st));
                kern<<<sms, 128, kMbStagesSmemBytes, st>>>(M, N, reps, cyc.p, err.p);
                CU(cudaEventRecord(e1, st));
            } else if (!fast) {
                static SmemOptIn optin;
                TRY(smem_opt_in(optin, k_mb_mma, kMbSmemBytes, device, "MMA microbenchmark"));
                k_mb_mma<<<sms, 128, kMbSmemBytes, st>>>(kind, M, N, flags, 16, cyc.p, err.p);   // warm-up
                CU(cudaEventRecord(e0, st));
                k_mb_mma<<<sms, 128, kMbSmemBytes, st>>>(kind, M, N, flags, reps, cyc.p, err.p);
                CU(cudaEventRecord(e1, st));
            } else {
                // straight-line issue: 16 instructions per iteration plus the first
                const int freps = reps / 4;
                instr = 16.0 * freps + 1.0;
                void (*kern)(int, int, int, unsigned long long*, int*) =
                    kind == 0 ? ((flags & kMbFlagATmem) ? k_mb_mma_fast<0, true> : k_mb_mma_fast<0, false>)
                              : kind == 1 ? k_mb_mma_fast<1, false> : k_mb_mma_fast<2, false>;
                static SmemOptIn opt_fast[4];
                const int slot = kind == 0 ? ((flags & kMbFlagATmem) ? 1 : 0) : kind + 1;
                TRY(smem_opt_in(opt_fast[slot], kern, kMbSmemBytes, device, "MMA microbenchmark"));
                kern<<<sms, 128, kMbSmemBytes, st>>>(M, N, 4, cyc.p, err.p);                 // warm-up
                CU(cudaEventRecord(e0, st));
                kern<<<sms, 128, kMbSmemBytes, st>>>(M, N, freps, cyc.p, err.p);
                CU(cudaEventRecord(e1, st));
            }
            CU(cudaEventSynchronize(e1));
            CU(cudaGetLastError());
            CU(cudaEventElapsedTime(&ms, e0, e1));
            int h_err = 0;
            CU(cudaMemcpy(&h_err, err.p, 4, cudaMemcpyDeviceToHost));
            if (h_err) return fail(BOA_ERR_CUDA, "MMA microbenchmark: a wait timed out");
            std::vector<unsigned long long> h((size_t)sms);
            CU(cudaMemcpy(h.data(), cyc.p, (size_t)sms * 8, cudaMemcpyDeviceToHost));
            const int kelems = kind == 0 ? 8 : kind == 1 ? 16 : 32;     // 32 bytes of K per instruction
            *rate = (double)sms * instr * 2.0 * M * N * kelems / (ms * 1e-3);
            if (cycles_per_op) {
                double c = 0.0;
                for (auto v : h) c += (double)v;
                *cycles_per_op = c / sms / instr;
            }
            return BOA_OK;
        }
        return fail(BOA_ERR_ARG, "unknown microbenchmark %d", test);
    };
    s = body();
    if (st) cudaStreamSynchronize(st);
    out.release(); buf.release(); cyc.release(); err.release();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    return s;
}

// ------------------------------------------------------------ training scan

extern "C" boa_status boa_scan_train_fwd(size_t Bsz, size_t T, size_t E, size_t N, size_t chunk, const float* u,
                                         const float* delta, const float* A, const float* Bm, const float* Cm,
                                         const float* D, float* y, float* hin, void* stream) {
    if (N != 16 || chunk == 0 || !u || !delta || !A || !Bm || !Cm || !D || !y || !hin)
        return fail(BOA_ERR_ARG, "boa_scan_train_fwd: bad argument (d_state must be 16)");
    if (Bsz == 0 || T == 0 || E == 0) return BOA_OK;
    dim3 grid((unsigned)((E + kTrainThreads - 1) / kTrainThreads), (unsigned)Bsz);
    k_scan_train_fwd<16><<<grid, kTrainThreads, 0, (cudaStream_t)stream>>>((int)T, (int)E, (int)chunk, u, delta, A, Bm,
                                                                          Cm, D, y, hin);
    CU(cudaGetLastError());
    return BOA_OK;
}

extern "C" boa_status boa_scan_train_bwd(size_t Bsz, size_t T, size_t E, size_t N, size_t chunk, const float* u,
                                         const float* delta, const float* A, const float* Bm, const float* Cm,
                                         const float* D, const float* dy, const float* hin, float* scratch,
                                         float* du, float* ddelta, float* dA_part, float* dD_part, float* dB_part,
                                         float* dC_part, void* stream) {
    if (N != 16 || chunk == 0 || !u || !delta || !A || !Bm || !Cm || !D || !dy || !hin || !scratch || !du ||
        !ddelta || !dA_part || !dD_part || !dB_part || !dC_part)
        return fail(BOA_ERR_ARG, "boa_scan_train_bwd: bad argument (d_state must be 16)");
    if (Bsz == 0 || T == 0 || E == 0) return BOA_OK;
    dim3 grid((unsigned)((E + kTrainThreads - 1) / kTrainThreads), (unsigned)Bsz);
    k_scan_train_bwd<16><<<grid, kTrainThreads, 0, (cudaStream_t)stream>>>((int)T, (int)E, (int)chunk, u, delta, A, Bm,
                                                                          Cm, D, dy, hin, scratch, du, ddelta,
                                                                          dA_part, dD_part, dB_part, dC_part);
    CU(cudaGetLastError());
    return BOA_OK;
}

// ------------------------------------------------------------ autotuner

extern "C" boa_status boa_set_tuning(boa_model* m, const boa_tuning* t) {
    if (!m || !t) return fail(BOA_ERR_ARG, "null argument");
    MODEL_LOCK(m);
    if (t->max_rows < 1 || t->max_rows > (1u << 24)) return fail(BOA_ERR_ARG, "max_rows %zu out of range", t->max_rows);
    if (t->scan_variant < 0 || t->scan_variant > 3) return fail(BOA_ERR_ARG, "scan_variant %d out of range", t->scan_variant);
    if (t->decode_lanes < 0 || t->decode_lanes > 16) return fail(BOA_ERR_ARG, "decode_lanes %d out of range", t->decode_lanes);
    if (t->decoder < 0 || t->decoder > 1) return fail(BOA_ERR_ARG, "decoder %d out of range", t->decoder);
    if (t->decoder == 1)
        if (const char* why = onchip_unsupported(m)) return fail(BOA_ERR_ARG, "on-chip decoder: %s", why);
    m->max_rows = t->max_rows;
    m->scan_variant = t->scan_variant;
    m->decode_lanes = t->decode_lanes;
    m->decoder = t->decoder;
    return BOA_OK;
}

extern "C" boa_status boa_get_tuning(const boa_model* m, boa_tuning* out) {
    if (!m || !out) return fail(BOA_ERR_ARG, "null argument");
    MODEL_LOCK(m);
    *out = boa_tuning{m->max_rows, m->scan_variant, m->decode_lanes, 0.0, 0.0, m->decoder};
    return BOA_OK;
}

extern "C" boa_status boa_autotune(boa_model* m, size_t n_streams, size_t stream_len, boa_tuning* out) {
    if (!m || n_streams == 0 || stream_len < 2) return fail(BOA_ERR_ARG, "bad argument");
    MODEL_LOCK(m);
    CU(cudaSetDevice(m->device));
    const size_t len = std::min<size_t>(stream_len, 512);   // a short sample of every stream
    const size_t n = std::min(n_streams, m->max_slots);
    std::vector<uint64_t> in_off(n + 1), out_off(n + 1), lens(n, len), sizes(n);
    for (size_t i = 0; i <= n; i++) {
        in_off[i] = i * len;
        out_off[i] = i * boa_max_compressed_size(len);
    }
    DevBuf<uint8_t> din, dout, ddec;
    TRY(din.ensure(n * len));
    TRY(dout.ensure(out_off[n]));
    TRY(ddec.ensure(n * len));
    {
        std::vector<uint8_t> h(n * len);
        uint64_t x = 0x9E3779B97F4A7C15ull;
        for (auto& b : h) { x = x * 6364136223846793005ull + 1442695040888963407ull; b = (uint8_t)(x >> 56); }
        CU(cudaMemcpy(din.p, h.data(), h.size(), cudaMemcpyHostToDevice));
    }
    const bool prof = m->prof_on;
    m->prof_on = false;
    cudaEvent_t a, b;
    CU(cudaEventCreate(&a));
    CU(cudaEventCreate(&b));
    auto timed = [&](auto&& fn, double& ms) -> boa_status {
        TRY(fn());   // warm
        CU(cudaEventRecord(a, m->stream));
        TRY(fn());
        CU(cudaEventRecord(b, m->stream));
        CU(cudaEventSynchronize(b));
        float f = 0.f;
        CU(cudaEventElapsedTime(&f, a, b));
        ms = f;
        return BOA_OK;
    };
    boa_status st = BOA_OK;
    boa_tuning best{m->max_rows, m->scan_variant, m->decode_lanes, 1e30, 1e30, 0};
    m->decoder = 0;
    const size_t rows_cand[] = {1u << 16, 1u << 17, 1u << 18, 1u << 19};
    for (size_t r : rows_cand) {
        if (st != BOA_OK) break;
        m->max_rows = r;
        double ms = 0;
        st = timed([&] { return compress_impl(m, n, din.p, in_off.data(), dout.p, out_off.data(), sizes.data()); }, ms);
        if (st == BOA_OK && ms < best.compress_ms) { best.compress_ms = ms; best.max_rows = r; }
    }
    m->max_rows = best.max_rows;
    auto time_decode = [&](double& ms) {
        return timed([&] { return decompress_impl(m, n, dout.p, out_off.data(), sizes.data(), lens.data(), ddec.p,
                                                  in_off.data()); }, ms);
    };
    // Scan variants under the automatic lane count (decode_lanes 0: two
    // lanes from 2048 slots), then other lane counts, which replace it only
    // when they win clearly on the short sample: a few hundred steps cannot
    // resolve a difference of a few per cent, and the automatic rule is the
    // one measured best at full length on the 64 MiB jet table (decoding 2
    // lanes 4779 ms, 3 lanes 4822 ms, 4 lanes 4930 ms, 1 lane about 20 %
    // slower).
    m->decode_lanes = 0;
    best.decode_lanes = 0;
    for (int g = 0; g < 4; g++) {
        if (st != BOA_OK) break;
        m->scan_variant = g;
        double ms = 0;
        st = time_decode(ms);
        if (st == BOA_OK && ms < best.decompress_ms) { best.decompress_ms = ms; best.scan_variant = g; }
    }
    m->scan_variant = best.scan_variant;
    for (int p : {1, 2, 4}) {
        if (st != BOA_OK || (size_t)p > n || p == decode_lanes(m, (int)n)) continue;
        m->decode_lanes = p;
        double ms = 0;
        st = time_decode(ms);
        if (st == BOA_OK && ms < 0.95 * best.decompress_ms) { best.decompress_ms = ms; best.decode_lanes = p; }
        m->decode_lanes = 0;
    }
    m->decode_lanes = best.decode_lanes;
    // the on-chip persistent decoder, where the model and form allow it,
    // under the same rule
    if (st == BOA_OK && !onchip_unsupported(m)) {
        m->decoder = 1;
        double ms = 0;
        st = time_decode(ms);
        if (st == BOA_OK && ms < 0.95 * best.decompress_ms) { best.decompress_ms = ms; best.decoder = 1; }
    }
    m->decoder = best.decoder;
    m->prof_on = prof;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    din.release(); dout.release(); ddec.release();
    if (st != BOA_OK) return st;
    best.compress_ms *= (double)n_streams / n * (double)(stream_len - 1) / (len - 1);
    best.decompress_ms *= (double)n_streams / n * (double)(stream_len - 1) / (len - 1);
    if (out) *out = best;
    return BOA_OK;
}

// ------------------------------------------------------------ test hooks

extern "C" boa_status boa_debug_encode_cdfs(size_t n_seq, const size_t* n_syms, const uint32_t* cdfs,
                                            const uint8_t* syms, uint8_t* out, size_t out_stride, size_t* sizes) {
    if (n_seq == 0) return BOA_OK;
    if (!n_syms || !cdfs || !syms || !out || !sizes) return fail(BOA_ERR_ARG, "null argument");
    std::vector<uint64_t> off(n_seq + 1, 0);
    for (size_t i = 0; i < n_seq; i++) {
        off[i + 1] = off[i] + n_syms[i];
        if (out_stride < 5 * n_syms[i] + 4) return fail(BOA_ERR_OUTPUT_TOO_SMALL, "out_stride too small");
    }
    const size_t rows = off[n_seq];
    uint64_t *d_off = nullptr, *d_sizes = nullptr;
    uint32_t *d_cdf = nullptr, *d_flags = nullptr;
    uint8_t *d_syms = nullptr, *d_out = nullptr;
    boa_status st = BOA_OK;
    std::vector<uint64_t> hs(n_seq);
    std::vector<uint32_t> hf(n_seq);
    cudaError_t e = cudaSuccess;
    if ((e = cudaMalloc(&d_off, (n_seq + 1) * 8)) || (e = cudaMalloc(&d_sizes, n_seq * 8)) ||
        (e = cudaMalloc(&d_cdf, std::max<size_t>(rows, 1) * 257 * 4)) || (e = cudaMalloc(&d_flags, n_seq * 4)) ||
        (e = cudaMalloc(&d_syms, std::max<size_t>(rows, 1))) || (e = cudaMalloc(&d_out, n_seq * out_stride)) ||
        (e = cudaMemcpy(d_off, off.data(), (n_seq + 1) * 8, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(d_cdf, cdfs, rows * 257 * 4, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(d_syms, syms, rows, cudaMemcpyHostToDevice))) {
        st = fail(BOA_ERR_CUDA, "debug encode setup: %s", cudaGetErrorString(e));
    } else {
        k_debug_encode_cdfs<<<(unsigned)((n_seq + 63) / 64), 64>>>((int)n_seq, d_off, d_cdf, d_syms, d_out, out_stride,
                                                                  d_sizes, d_flags);
        if ((e = cudaGetLastError()) || (e = cudaDeviceSynchronize()) ||
            (e = cudaMemcpy(out, d_out, n_seq * out_stride, cudaMemcpyDeviceToHost)) ||
            (e = cudaMemcpy(hs.data(), d_sizes, n_seq * 8, cudaMemcpyDeviceToHost)) ||
            (e = cudaMemcpy(hf.data(), d_flags, n_seq * 4, cudaMemcpyDeviceToHost))) {
            st = fail(BOA_ERR_CUDA, "debug encode: %s", cudaGetErrorString(e));
        } else {
            for (size_t i = 0; i < n_seq; i++) {
                sizes[i] = hs[i];
                if (hf[i]) st = fail(BOA_ERR_OUTPUT_TOO_SMALL, "sequence %zu flags %u", i, hf[i]);
            }
        }
    }
    cudaFree(d_off); cudaFree(d_sizes); cudaFree(d_cdf); cudaFree(d_flags); cudaFree(d_syms); cudaFree(d_out);
    return st;
}

extern "C" boa_status boa_debug_decode_cdfs(size_t n_seq, const size_t* n_syms, const uint32_t* cdfs,
                                            const uint8_t* in, size_t in_stride, const size_t* in_sizes,
                                            uint8_t* syms) {
    if (n_seq == 0) return BOA_OK;
    if (!n_syms || !cdfs || !in || !in_sizes || !syms) return fail(BOA_ERR_ARG, "null argument");
    std::vector<uint64_t> off(n_seq + 1, 0), isz(n_seq);
    for (size_t i = 0; i < n_seq; i++) {
        off[i + 1] = off[i] + n_syms[i];
        isz[i] = in_sizes[i];
        if (in_sizes[i] > in_stride) return fail(BOA_ERR_ARG, "in_sizes[%zu] > in_stride", i);
    }
    const size_t rows = off[n_seq];
    uint64_t *d_off = nullptr, *d_isz = nullptr;
    uint32_t *d_cdf = nullptr, *d_flags = nullptr;
    uint8_t *d_syms = nullptr, *d_in = nullptr;
    boa_status st = BOA_OK;
    std::vector<uint32_t> hf(n_seq);
    cudaError_t e = cudaSuccess;
    if ((e = cudaMalloc(&d_off, (n_seq + 1) * 8)) || (e = cudaMalloc(&d_isz, n_seq * 8)) ||
        (e = cudaMalloc(&d_cdf, std::max<size_t>(rows, 1) * 257 * 4)) || (e = cudaMalloc(&d_flags, n_seq * 4)) ||
        (e = cudaMalloc(&d_syms, std::max<size_t>(rows, 1))) || (e = cudaMalloc(&d_in, std::max<size_t>(n_seq * in_stride, 1))) ||
        (e = cudaMemcpy(d_off, off.data(), (n_seq + 1) * 8, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(d_isz, isz.data(), n_seq * 8, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(d_cdf, cdfs, rows * 257 * 4, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(d_in, in, n_seq * in_stride, cudaMemcpyHostToDevice))) {
        st = fail(BOA_ERR_CUDA, "debug decode setup: %s", cudaGetErrorString(e));
    } else {
        k_debug_decode_cdfs<<<(unsigned)((n_seq + 3) / 4), 128>>>((int)n_seq, d_off, d_cdf, d_in, in_stride, d_isz,
                                                                  d_syms, d_flags);
        if ((e = cudaGetLastError()) || (e = cudaDeviceSynchronize()) ||
            (e = cudaMemcpy(syms, d_syms, rows, cudaMemcpyDeviceToHost)) ||
            (e = cudaMemcpy(hf.data(), d_flags, n_seq * 4, cudaMemcpyDeviceToHost))) {
            st = fail(BOA_ERR_CUDA, "debug decode: %s", cudaGetErrorString(e));
        } else {
            for (size_t i = 0; i < n_seq; i++)
                if (hf[i]) st = fail(BOA_ERR_CORRUPT, "sequence %zu flags %u", i, hf[i]);
        }
    }
    cudaFree(d_off); cudaFree(d_isz); cudaFree(d_cdf); cudaFree(d_flags); cudaFree(d_syms); cudaFree(d_in);
    return st;
}

extern "C" boa_status boa_debug_quantise(size_t n_rows, const float* p, uint32_t* f) {
    if (n_rows == 0) return BOA_OK;
    if (!p || !f) return fail(BOA_ERR_ARG, "null argument");
    float* d_p = nullptr;
    uint32_t* d_f = nullptr;
    boa_status st = BOA_OK;
    cudaError_t e = cudaSuccess;
    if ((e = cudaMalloc(&d_p, n_rows * 1024)) || (e = cudaMalloc(&d_f, n_rows * 1024)) ||
        (e = cudaMemcpy(d_p, p, n_rows * 1024, cudaMemcpyHostToDevice))) {
        st = fail(BOA_ERR_CUDA, "debug quantise setup: %s", cudaGetErrorString(e));
    } else {
        k_debug_quantise<<<(unsigned)((n_rows + 7) / 8), 256>>>(d_p, d_f, (long long)n_rows);
        if ((e = cudaGetLastError()) || (e = cudaDeviceSynchronize()) ||
            (e = cudaMemcpy(f, d_f, n_rows * 1024, cudaMemcpyDeviceToHost)))
            st = fail(BOA_ERR_CUDA, "debug quantise: %s", cudaGetErrorString(e));
    }
    cudaFree(d_p); cudaFree(d_f);
    return st;
}

extern "C" boa_status boa_debug_logprobs(boa_model* m, const uint8_t* stream, size_t len, float* out) {
    if (!m || (len && (!stream || !out))) return fail(BOA_ERR_ARG, "null argument");
    MODEL_LOCK(m);
    if (len < 2) return BOA_OK;
    CU(cudaSetDevice(m->device));
    const size_t T = len - 1;
    const int Tc = (int)std::min<size_t>(T, m->max_rows);
    TRY(ensure_workspace(m, 1, Tc));
    TRY(ensure_streams(m, 1));
    TRY(m->d_in.ensure(len));
    DevBuf<float> lp;
    TRY(lp.ensure(T * 256));
    uint64_t off[2] = {0, len}, lens1[1] = {len};
    TRY(upload_index(m, 1, off, off, lens1));
    TRY(zero_state(m, 1));
    bind_view(m, 0, Tc, 1, m->stream);
    boa_status st = BOA_OK;
    cudaError_t e = cudaMemcpyAsync(m->d_in.p, stream, len, cudaMemcpyHostToDevice, m->stream);
    if (e != cudaSuccess) st = fail(BOA_ERR_CUDA, "%s", cudaGetErrorString(e));
    TokenSrc ts{m->d_in.p, m->in_off.p, m->lens.p, m->slots.p};
    for (size_t t0 = 0; st == BOA_OK && t0 < T; t0 += Tc) {
        const int tc = (int)std::min<size_t>(Tc, T - t0);
        k_set_slot<<<1, 1, 0, m->stream>>>(m->slots.p, 0, (long long)t0);
        st = check_launch(m, "set_slot");
        if (st == BOA_OK) st = forward(m, ts, 1, tc);
        if (st == BOA_OK) {
            k_log2_softmax<<<(unsigned)((tc + 7) / 8), 256, 0, m->stream>>>(m->logits.p, lp.p + t0 * 256, tc);
            st = check_launch(m, "log2_softmax");
        }
    }
    if (st == BOA_OK) {
        e = cudaMemcpyAsync(out, lp.p, T * 256 * 4, cudaMemcpyDeviceToHost, m->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
        if (e != cudaSuccess) st = fail(BOA_ERR_CUDA, "%s", cudaGetErrorString(e));
    }
    cudaStreamSynchronize(m->stream);
    lp.release();
    if (st == BOA_OK) st = check_tc_error(m);
    return st;
}

extern "C" boa_status boa_debug_gemm(int precision, size_t M, size_t N, size_t K, const float* A, const float* W,
                                     const float* bias, int epilogue, const float* C_in, float* C_out) {
    if (!A || !W || !C_out || M == 0 || N == 0 || K == 0) return fail(BOA_ERR_ARG, "bad argument");
    if (epilogue < 0 || epilogue > kEpiBiasResid) return fail(BOA_ERR_ARG, "bad epilogue %d", epilogue);
    if ((epilogue == kEpiBias || epilogue == kEpiBiasGelu || epilogue == kEpiBiasResid) && !bias)
        return fail(BOA_ERR_ARG, "epilogue needs a bias");
    if ((epilogue == kEpiResid || epilogue == kEpiBiasResid) && !C_in) return fail(BOA_ERR_ARG, "epilogue needs C_in");
    if (precision < BOA_PREC_FP32 || precision > BOA_PREC_FP8) return fail(BOA_ERR_ARG, "bad precision");
    CU(cudaSetDevice(0));
    boa_model t;
    t.precision = precision;
    cudaDeviceGetAttribute(&t.num_sms, cudaDevAttrMultiProcessorCount, 0);
    DevBuf<float> dA, dW, dB, dC;
    DevBuf<__nv_bfloat16> bA, bW;
    boa_status st = BOA_OK;
    auto body = [&]() -> boa_status {
        TRY(dA.ensure(M * K)); TRY(dC.ensure(M * N)); TRY(dB.ensure(N)); TRY(dW.ensure(N * K));
        CU(cudaMemcpy(dA.p, A, M * K * 4, cudaMemcpyHostToDevice));
        CU(cudaMemset(dB.p, 0, N * 4));
        if (bias) CU(cudaMemcpy(dB.p, bias, N * 4, cudaMemcpyHostToDevice));
        CU(cudaMemset(dC.p, 0, M * N * 4));
        if (C_in) CU(cudaMemcpy(dC.p, C_in, M * N * 4, cudaMemcpyHostToDevice));
        if (precision == BOA_PREC_BF16) {
            TRY(t.err.ensure(1));
            CU(cudaMemset(t.err.p, 0, 4));
            TRY(bA.ensure(M * K)); TRY(bW.ensure(N * K));
            CU(cudaMemcpy(dW.p, W, N * K * 4, cudaMemcpyHostToDevice));
            k_to_bf16<<<256, 256>>>(dA.p, bA.p, M * K);
            k_to_bf16<<<256, 256>>>(dW.p, bW.p, N * K);
            switch (epilogue) {
                case kEpiStore: TRY(gemm_tc<kEpiStore>(&t, BOA_KC_OTHER, bA.p, bW.p, dB.p, dC.p, nullptr, M, N, K)); break;
                case kEpiBias: TRY(gemm_tc<kEpiBias>(&t, BOA_KC_OTHER, bA.p, bW.p, dB.p, dC.p, nullptr, M, N, K)); break;
                case kEpiResid: TRY(gemm_tc<kEpiResid>(&t, BOA_KC_OTHER, bA.p, bW.p, dB.p, dC.p, nullptr, M, N, K)); break;
                case kEpiBiasGelu: TRY(gemm_tc<kEpiBiasGelu>(&t, BOA_KC_OTHER, bA.p, bW.p, dB.p, dC.p, nullptr, M, N, K)); break;
                default: TRY(gemm_tc<kEpiBiasResid>(&t, BOA_KC_OTHER, bA.p, bW.p, dB.p, dC.p, nullptr, M, N, K)); break;
            }
        } else if (precision == BOA_PREC_FP8) {
            TRY(t.err.ensure(1));
            CU(cudaMemset(t.err.p, 0, 4));
            const size_t Kp = (K + 127) / 128 * 128;
            std::vector<uint8_t> q(N * Kp, 0);
            std::vector<float> sc(N);
            for (size_t n = 0; n < N; n++) {
                float amax = 0.f;
                for (size_t k = 0; k < K; k++) amax = std::max(amax, std::fabs(W[n * K + k]));
                const float inv = amax > 0.f ? 448.0f / amax : 1.0f;
                sc[n] = amax > 0.f ? amax / 448.0f : 1.0f;
                for (size_t k = 0; k < K; k++)
                    q[n * Kp + k] = (uint8_t)__nv_cvt_float_to_fp8(W[n * K + k] * inv, __NV_SATFINITE, __NV_E4M3);
            }
            DevBuf<uint8_t> dq;
            DevBuf<float> ds;
            TRY(dq.ensure(N * Kp));
            TRY(ds.ensure(N));
            CU(cudaMemcpy(dq.p, q.data(), N * Kp, cudaMemcpyHostToDevice));
            CU(cudaMemcpy(ds.p, sc.data(), N * 4, cudaMemcpyHostToDevice));
            const __nv_fp8_e4m3* w8 = reinterpret_cast<const __nv_fp8_e4m3*>(dq.p);
            t.kp8 = Kp;
            TRY(t.a8.ensure(M * Kp));
            TRY(t.a8s.ensure(M));
            t.v.a8 = t.a8.p;
            t.v.a8s = t.a8s.p;
            boa_status r = BOA_OK;
            switch (epilogue) {
                case kEpiStore: r = gemm_f8<kEpiStore>(&t, BOA_KC_OTHER, dA.p, w8, ds.p, dB.p, dC.p, M, N, K); break;
                case kEpiBias: r = gemm_f8<kEpiBias>(&t, BOA_KC_OTHER, dA.p, w8, ds.p, dB.p, dC.p, M, N, K); break;
                case kEpiResid: r = gemm_f8<kEpiResid>(&t, BOA_KC_OTHER, dA.p, w8, ds.p, dB.p, dC.p, M, N, K); break;
                case kEpiBiasGelu: r = gemm_f8<kEpiBiasGelu>(&t, BOA_KC_OTHER, dA.p, w8, ds.p, dB.p, dC.p, M, N, K); break;
                default: r = gemm_f8<kEpiBiasResid>(&t, BOA_KC_OTHER, dA.p, w8, ds.p, dB.p, dC.p, M, N, K); break;
            }
            cudaDeviceSynchronize();
            dq.release();
            ds.release();
            t.a8.release();
            t.a8s.release();
            TRY(r);
        } else if (precision == BOA_PREC_TF32X3) {
            TRY(t.err.ensure(1));
            CU(cudaMemset(t.err.p, 0, 4));
            std::vector<float> hl(2 * N * K);
            for (size_t i = 0; i < N * K; i++) {
                uint32_t u;
                memcpy(&u, &W[i], 4);
                u = (u + 0x1000u) & ~0x1FFFu;
                float hi;
                memcpy(&hi, &u, 4);
                hl[i] = hi;
                hl[N * K + i] = W[i] - hi;
            }
            DevBuf<float> dW2;
            TRY(dW2.ensure(2 * N * K));
            CU(cudaMemcpy(dW2.p, hl.data(), 2 * N * K * 4, cudaMemcpyHostToDevice));
            const float* hi = dW2.p;
            const float* lo = dW2.p + N * K;
            boa_status r = BOA_OK;
            switch (epilogue) {
                case kEpiStore: r = gemm_t3<kEpiStore>(&t, BOA_KC_OTHER, dA.p, hi, lo, dB.p, dC.p, M, N, K); break;
                case kEpiBias: r = gemm_t3<kEpiBias>(&t, BOA_KC_OTHER, dA.p, hi, lo, dB.p, dC.p, M, N, K); break;
                case kEpiResid: r = gemm_t3<kEpiResid>(&t, BOA_KC_OTHER, dA.p, hi, lo, dB.p, dC.p, M, N, K); break;
                case kEpiBiasGelu: r = gemm_t3<kEpiBiasGelu>(&t, BOA_KC_OTHER, dA.p, hi, lo, dB.p, dC.p, M, N, K); break;
                default: r = gemm_t3<kEpiBiasResid>(&t, BOA_KC_OTHER, dA.p, hi, lo, dB.p, dC.p, M, N, K); break;
            }
            cudaDeviceSynchronize();
            dW2.release();
            TRY(r);
        } else {
            std::vector<float> wt(N * K);
            transpose(W, (int)N, (int)K, wt.data());
            CU(cudaMemcpy(dW.p, wt.data(), N * K * 4, cudaMemcpyHostToDevice));
            switch (epilogue) {
                case kEpiStore: TRY(gemm<kEpiStore>(&t, BOA_KC_OTHER, dA.p, dW.p, dB.p, dC.p, M, N, K)); break;
                case kEpiBias: TRY(gemm<kEpiBias>(&t, BOA_KC_OTHER, dA.p, dW.p, dB.p, dC.p, M, N, K)); break;
                case kEpiResid: TRY(gemm<kEpiResid>(&t, BOA_KC_OTHER, dA.p, dW.p, dB.p, dC.p, M, N, K)); break;
                case kEpiBiasGelu: TRY(gemm<kEpiBiasGelu>(&t, BOA_KC_OTHER, dA.p, dW.p, dB.p, dC.p, M, N, K)); break;
                default: TRY(gemm<kEpiBiasResid>(&t, BOA_KC_OTHER, dA.p, dW.p, dB.p, dC.p, M, N, K)); break;
            }
        }
        CU(cudaDeviceSynchronize());
        if (precision != BOA_PREC_FP32) {
            int h = 0;
            CU(cudaMemcpy(&h, t.err.p, 4, cudaMemcpyDeviceToHost));
            if (h) return fail(BOA_ERR_CUDA, "tensor-core GEMM wait timed out");
        }
        CU(cudaMemcpy(C_out, dC.p, M * N * 4, cudaMemcpyDeviceToHost));
        return BOA_OK;
    };
    st = body();
    dA.release(); dW.release(); dB.release(); dC.release(); bA.release(); bW.release(); t.err.release();
    return st;
}

extern "C" boa_status boa_debug_enable_cdf_trace(boa_model* m, int on) {
    if (!m) return fail(BOA_ERR_ARG, "null model");
    MODEL_LOCK(m);
    m->trace_on = on != 0;
    return BOA_OK;
}

extern "C" boa_status boa_debug_read_cdf_trace(boa_model* m, uint64_t* out, size_t n) {
    if (!m || (n && !out)) return fail(BOA_ERR_ARG, "null argument");
    MODEL_LOCK(m);
    if (n > m->trace_n) return fail(BOA_ERR_ARG, "trace holds %zu entries, asked for %zu", m->trace_n, n);
    if (n == 0) return BOA_OK;
    CU(cudaSetDevice(m->device));
    CU(cudaMemcpyAsync(out, m->trace.p, n * 8, cudaMemcpyDeviceToHost, m->stream));
    CU(cudaStreamSynchronize(m->stream));
    return BOA_OK;
}

// ------------------------------------------------- allocation-free decoder
//
// boa_decode_cdfs_static: the CDF-driven range decoder for callers that may
// not allocate device memory once they are running -- for example a
// data-acquisition process whose device memory budget is fixed at start-up,
// or a host framework whose own memory pool owns the GPU and forbids other
// allocations.  The caller passes device inputs and outputs; the decoder's
// scratch (per-sequence symbol offsets, coded sizes, status words) lives in
// the file-scope array below, which every GPU that loads this library holds
// until the process exits.

static constexpr size_t kStaticMaxSeq = 65536;
static constexpr size_t kStaticCountsOff = 0;                                  // u64[kStaticMaxSeq]
static constexpr size_t kStaticSymOffOff = kStaticCountsOff + 8 * kStaticMaxSeq;   // u64[kStaticMaxSeq + 1]
static constexpr size_t kStaticSizesOff = kStaticSymOffOff + 8 * (kStaticMaxSeq + 256);  // u64[kStaticMaxSeq]
static constexpr size_t kStaticFlagsOff = kStaticSizesOff + 8 * kStaticMaxSeq;     // u32[kStaticMaxSeq]
static constexpr size_t kStaticOrOff = kStaticFlagsOff + 4 * kStaticMaxSeq;        // u32 (OR of all flags)
static constexpr size_t kStaticScratchBytes = kStaticOrOff + 256;
static_assert(sizeof(size_t) == sizeof(uint64_t), "size_t arrays are copied as u64");

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Exclusive prefix sum of n counts in one block of 1024 threads.
__global__ void k_static_prefix(const uint64_t* __restrict__ counts, uint64_t* __restrict__ off, int n) {
    __shared__ uint64_t part[1024];
    const int tid = threadIdx.x;
    const int per = (n + 1023) / 1024;
    const int b = tid * per, e = min(n, b + per);
    uint64_t s = 0;
    for (int i = b; i < e; i++) s += counts[i];
    part[tid] = s;
    __syncthreads();
    if (tid == 0) {
        uint64_t acc = 0;
        for (int i = 0; i < 1024; i++) { uint64_t v = part[i]; part[i] = acc; acc += v; }
    }
    __syncthreads();
    uint64_t acc = part[tid];
    for (int i = b; i < e; i++) { off[i] = acc; acc += counts[i]; }
    if (e == n && b < e) off[n] = acc;
    if (n == 0 && tid == 0) off[0] = 0;
}

__global__ void k_static_flags_or(const uint32_t* __restrict__ flags, int n, uint32_t* __restrict__ out) {
    uint32_t v = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v |= flags[i];
    if (v) atomicOr(out, v);
}

static std::mutex g_static_mu;
static unsigned char* g_static_ptr[256];   // per device ordinal, set once

// Once per device, with that device current: the device address of the
// scratch array (host code cannot use the symbol itself as an address).
// The stream must belong to the current device, whose array the call uses.
// The address is kept for the life of the process, so the entry point is
// not for use after cudaDeviceReset on that device.
static boa_status static_scratch(cudaStream_t st, unsigned char** out) {
    int dev = -1, sdev = -1;
    CU(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) return fail(BOA_ERR_CUDA, "device ordinal %d out of range", dev);
    CU(cudaStreamGetDevice(st, &sdev));
    if (sdev != dev)
        return fail(BOA_ERR_ARG, "boa_decode_cdfs_static: the stream belongs to device %d, the current device is %d",
                    sdev, dev);
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) return fail(BOA_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
        g_static_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_static_ptr[dev];
    return BOA_OK;
}

extern "C" boa_status boa_decode_cdfs_static(size_t n_seq, const size_t* n_syms, const uint32_t* d_cdfs,
                                             const uint8_t* d_in, size_t in_stride, const size_t* in_sizes,
                                             uint8_t* d_syms, void* cuda_stream) {
    if (n_seq == 0) return BOA_OK;
    if (n_seq > kStaticMaxSeq)
        return fail(BOA_ERR_ARG, "boa_decode_cdfs_static: %zu sequences exceed the static scratch limit of %zu",
                    n_seq, kStaticMaxSeq);
    if (!n_syms || !d_cdfs || !d_in || !in_sizes || !d_syms) return fail(BOA_ERR_ARG, "null argument");
    for (size_t i = 0; i < n_seq; i++)
        if (in_sizes[i] > in_stride) return fail(BOA_ERR_ARG, "in_sizes[%zu] > in_stride", i);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    unsigned char* base = nullptr;
    TRY(static_scratch(st, &base));
    uint64_t* counts = reinterpret_cast<uint64_t*>(base + kStaticCountsOff);
    uint64_t* sym_off = reinterpret_cast<uint64_t*>(base + kStaticSymOffOff);
    uint64_t* sizes = reinterpret_cast<uint64_t*>(base + kStaticSizesOff);
    uint32_t* flags = reinterpret_cast<uint32_t*>(base + kStaticFlagsOff);
    uint32_t* flag_or = reinterpret_cast<uint32_t*>(base + kStaticOrOff);
    CU(cudaMemcpyAsync(counts, n_syms, n_seq * 8, cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(sizes, in_sizes, n_seq * 8, cudaMemcpyHostToDevice, st));
    CU(cudaMemsetAsync(flag_or, 0, 4, st));   // the array keeps the previous call's contents
    k_static_prefix<<<1, 1024, 0, st>>>(counts, sym_off, (int)n_seq);
    k_debug_decode_cdfs<<<(unsigned)((n_seq + 3) / 4), 128, 0, st>>>((int)n_seq, sym_off, d_cdfs, d_in, in_stride,
                                                                    sizes, d_syms, flags);
    k_static_flags_or<<<(unsigned)std::min<size_t>((n_seq + 255) / 256, 64), 256, 0, st>>>(flags, (int)n_seq, flag_or);
    CU(cudaGetLastError());
    uint32_t h_or = 0;
    CU(cudaMemcpyAsync(&h_or, flag_or, 4, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (h_or) return fail(BOA_ERR_CORRUPT, "a sequence did not decode cleanly (flags %u)", h_or);
    return BOA_OK;
}

// ------------------------------------------------------------ .boa container
//
// Layout (little-endian), after the paper's container description (section
// "Coders & Parallelisation"):
//   0  "BOA1"                      magic
//   4  u32 version (1)
//   8  u64 model fingerprint
//  16  u64 total uncompressed length
//  24  u64 nominal chunk length
//  32  u64 number of chunks n
//  40  u64 length of the last chunk
//  48  u32 CRC-32 of bytes 0..47
//  52  u32 CRC-32 of the index
//  56  index: n x (u64 payload offset, u64 compressed size)
//  56 + 16 n  payload: each chunk's bytes (raw first byte + coded bytes)

static const uint32_t kBoaVersion = 1;
static const size_t kHeaderBytes = 56;

// CRC-32 with the IEEE 802.3 polynomial (reflected 0xEDB88320, initial and
// final XOR 0xFFFFFFFF), bitwise.
extern "C" uint32_t boa_crc32(const uint8_t* p, size_t n) {
    uint32_t c = 0xFFFFFFFFu;
    for (size_t i = 0; i < n; i++) {
        c ^= p[i];
        for (int k = 0; k < 8; k++) c = (c >> 1) ^ (0xEDB88320u & (0u - (c & 1u)));
    }
    return c ^ 0xFFFFFFFFu;
}

static void put64(uint8_t* p, uint64_t v) { for (int i = 0; i < 8; i++) p[i] = (uint8_t)(v >> (8 * i)); }
static void put32(uint8_t* p, uint32_t v) { for (int i = 0; i < 4; i++) p[i] = (uint8_t)(v >> (8 * i)); }
static uint64_t get64(const uint8_t* p) { uint64_t v = 0; for (int i = 7; i >= 0; i--) v = (v << 8) | p[i]; return v; }
static uint32_t get32(const uint8_t* p) { uint32_t v = 0; for (int i = 3; i >= 0; i--) v = (v << 8) | p[i]; return v; }

// Header of a container whose n index entries already sit at out + 56.
static void write_container_header(uint8_t* out, uint64_t fingerprint, uint64_t total, uint64_t chunk, uint64_t n,
                                   uint64_t last) {
    memcpy(out, "BOA1", 4);
    put32(out + 4, kBoaVersion);
    put64(out + 8, fingerprint);
    put64(out + 16, total);
    put64(out + 24, chunk);
    put64(out + 32, n);
    put64(out + 40, last);
    put32(out + 48, boa_crc32(out, 48));
    put32(out + 52, boa_crc32(out + kHeaderBytes, 16 * n));
}

// One validated container at the start of c (size bytes, possibly followed
// by more containers): its layout, chunk extents and its own byte length.
struct ContainerView {
    uint64_t total = 0, chunk = 0, n = 0, last = 0;
    const uint8_t* idx = nullptr;
    const uint8_t* pay = nullptr;
    size_t bytes = 0;                  // header + index + payload up to the farthest chunk end
};

static boa_status parse_container(const boa_model* m, const uint8_t* c, size_t size, ContainerView* v) {
    uint64_t total = 0, fp = 0;
    TRY(boa_unpack_info(c, size, &total, &fp));
    if (fp != m->fingerprint) return fail(BOA_ERR_FINGERPRINT, "container was written with a different model");
    const uint64_t chunk = get64(c + 24), n = get64(c + 32), last = get64(c + 40);
    if (chunk == 0 || n != (total + chunk - 1) / chunk || (n && last != total - (n - 1) * chunk))
        return fail(BOA_ERR_CORRUPT, "inconsistent chunk layout");
    if (n > (size - kHeaderBytes) / 16) return fail(BOA_ERR_CORRUPT, "index runs past the container");
    const uint8_t* idx = c + kHeaderBytes;
    if (get32(c + 52) != boa_crc32(idx, 16 * n)) return fail(BOA_ERR_CORRUPT, "index CRC mismatch");
    const size_t pay_size = size - kHeaderBytes - 16 * n;
    size_t end = 0;
    for (uint64_t i = 0; i < n; i++) {
        const uint64_t o = get64(idx + 16 * i), z = get64(idx + 16 * i + 8);
        if (o > pay_size || z > pay_size - o) return fail(BOA_ERR_CORRUPT, "chunk %llu lies outside the payload", (unsigned long long)i);
        end = std::max<size_t>(end, o + z);
    }
    v->total = total;
    v->chunk = chunk;
    v->n = n;
    v->last = last;
    v->idx = idx;
    v->pay = idx + 16 * n;
    v->bytes = kHeaderBytes + 16 * n + end;
    return BOA_OK;
}

extern "C" size_t boa_pack_bound(size_t len, size_t chunk_len) {
    if (chunk_len == 0) return 0;
    const size_t n = (len + chunk_len - 1) / chunk_len;
    size_t b = kHeaderBytes + 16 * n;
    for (size_t i = 0; i < n; i++) b += boa_max_compressed_size(std::min(chunk_len, len - i * chunk_len));
    return b;
}

extern "C" boa_status boa_pack(boa_model* m, const uint8_t* data, size_t len, size_t chunk_len, uint8_t* out,
                               size_t cap, size_t* out_size) {
    if (!m || (len && !data) || !out || !out_size || chunk_len == 0) return fail(BOA_ERR_ARG, "bad argument");
    MODEL_LOCK(m);
    if (cap < boa_pack_bound(len, chunk_len)) return fail(BOA_ERR_OUTPUT_TOO_SMALL, "capacity below boa_pack_bound");
    const size_t n = (len + chunk_len - 1) / chunk_len;
    std::vector<const uint8_t*> ptrs(n);
    std::vector<size_t> lens(n), caps(n), sizes(n);
    std::vector<uint8_t*> outs(n);
    // chunks are compressed straight into the payload area at worst-case
    // offsets, then packed down
    size_t at = kHeaderBytes + 16 * n;
    std::vector<size_t> slot(n);
    for (size_t i = 0; i < n; i++) {
        ptrs[i] = data + i * chunk_len;
        lens[i] = std::min(chunk_len, len - i * chunk_len);
        caps[i] = boa_max_compressed_size(lens[i]);
        slot[i] = at;
        outs[i] = out + at;
        at += caps[i];
    }
    if (n) TRY(boa_compress(m, n, ptrs.data(), lens.data(), outs.data(), caps.data(), sizes.data()));
    uint8_t* idx = out + kHeaderBytes;
    size_t pay = 0, w = kHeaderBytes + 16 * n;
    for (size_t i = 0; i < n; i++) {
        if (w != slot[i]) memmove(out + w, out + slot[i], sizes[i]);
        put64(idx + 16 * i, pay);
        put64(idx + 16 * i + 8, sizes[i]);
        w += sizes[i];
        pay += sizes[i];
    }
    write_container_header(out, m->fingerprint, len, chunk_len, n, n ? lens[n - 1] : 0);
    *out_size = w;
    return BOA_OK;
}

extern "C" boa_status boa_unpack_info(const uint8_t* c, size_t size, uint64_t* total_len, uint64_t* fingerprint) {
    if (!c || size < kHeaderBytes) return fail(BOA_ERR_CORRUPT, "container shorter than its header");
    if (memcmp(c, "BOA1", 4) != 0 || get32(c + 4) != kBoaVersion) return fail(BOA_ERR_FORMAT, "not a .boa container");
    if (get32(c + 48) != boa_crc32(c, 48)) return fail(BOA_ERR_CORRUPT, "header CRC mismatch");
    if (total_len) *total_len = get64(c + 16);
    if (fingerprint) *fingerprint = get64(c + 8);
    return BOA_OK;
}

extern "C" boa_status boa_unpack(boa_model* m, const uint8_t* c, size_t size, uint8_t* out, size_t cap,
                                 size_t* out_len) {
    if (!m || !out_len || (cap && !out)) return fail(BOA_ERR_ARG, "bad argument");
    MODEL_LOCK(m);
    ContainerView v;
    TRY(parse_container(m, c, size, &v));
    if (cap < v.total) return fail(BOA_ERR_OUTPUT_TOO_SMALL, "output needs %llu bytes", (unsigned long long)v.total);
    const size_t n = v.n;
    std::vector<const uint8_t*> ptrs(n);
    std::vector<size_t> sizes(n), lens(n);
    std::vector<uint8_t*> outs(n);
    for (size_t i = 0; i < n; i++) {
        ptrs[i] = v.pay + get64(v.idx + 16 * i);
        sizes[i] = get64(v.idx + 16 * i + 8);
        lens[i] = i + 1 < n ? v.chunk : v.last;
        outs[i] = out + i * v.chunk;
    }
    if (n) TRY(boa_decompress(m, n, ptrs.data(), sizes.data(), lens.data(), outs.data()));
    *out_len = v.total;
    return BOA_OK;
}

// Every container in data[0, size), one after another, decoded with one
// batched decompression of all their chunks.
extern "C" boa_status boa_unpack_shards(boa_model* m, const uint8_t* data, size_t size, uint8_t* out, size_t cap,
                                        size_t* out_len) {
    if (!m || !out_len || (size && !data) || (cap && !out)) return fail(BOA_ERR_ARG, "bad argument");
    MODEL_LOCK(m);
    if (!out) {                                  // size query: validate and sum the lengths
        size_t at = 0, total = 0;
        while (at < size) {
            ContainerView v;
            TRY(parse_container(m, data + at, size - at, &v));
            total += v.total;
            at += v.bytes;
        }
        *out_len = total;
        return BOA_OK;
    }
    std::vector<const uint8_t*> ptrs;
    std::vector<size_t> sizes, lens;
    std::vector<uint8_t*> outs;
    size_t at = 0, total = 0;
    while (at < size) {
        ContainerView v;
        TRY(parse_container(m, data + at, size - at, &v));
        if (cap < total || cap - total < v.total)
            return fail(BOA_ERR_OUTPUT_TOO_SMALL, "output needs more than %zu bytes", cap);
        for (uint64_t i = 0; i < v.n; i++) {
            ptrs.push_back(v.pay + get64(v.idx + 16 * i));
            sizes.push_back(get64(v.idx + 16 * i + 8));
            lens.push_back(i + 1 < v.n ? v.chunk : v.last);
            outs.push_back(out + total + i * v.chunk);
        }
        total += v.total;
        at += v.bytes;
    }
    if (!ptrs.empty()) TRY(boa_decompress(m, ptrs.size(), ptrs.data(), sizes.data(), lens.data(), outs.data()));
    *out_len = total;
    return BOA_OK;
}

// ------------------------------------------------------------ streaming pipeline
//
// The caller's thread cuts pushed bytes into sets (set_chunks chunks of
// chunk_len bytes) in two pinned buffers; a full set is copied to its device
// buffer on the pipeline's copy stream and queued.  The worker thread takes
// sets in order, waits for the copy, compresses the set as one batch of
// streams (compress_impl on the device copy), fetches the coded bytes and
// appends the set's container to the output.  A set buffer is reused only
// after the worker has finished with it, so at most two sets are in flight:
// one compressing, one filling / preloading.

struct boa_stream {
    boa_model* m = nullptr;
    size_t chunk = 0, per_set = 0, set_bytes = 0;
    HostBuf<uint8_t> host[2];
    DevBuf<uint8_t> dev[2];
    cudaStream_t copy = nullptr;
    cudaEvent_t loaded[2] = {nullptr, nullptr};
    int cur = 0;                  // set buffer being filled (caller's thread)
    size_t fill = 0;
    bool finished = false;
    std::thread worker;
    mutable std::mutex mu;
    std::condition_variable cv;
    std::deque<std::pair<int, size_t>> jobs;   // (set buffer, bytes)
    bool busy[2] = {false, false};
    bool running = false;         // worker is compressing a set
    bool stop = false;
    boa_status err = BOA_OK;
    std::string err_msg;
    std::vector<uint8_t> shards;  // finished containers, in input order
    size_t read_at = 0;
    uint64_t sets = 0, preloaded = 0, bytes_in = 0;
};

// One set (device buffer b, bytes long) into a container appended to shards.
static boa_status stream_compress_set(boa_stream* s, int b, size_t bytes, std::vector<uint8_t>& shard) {
    boa_model* m = s->m;
    MODEL_LOCK(m);
    const size_t n = (bytes + s->chunk - 1) / s->chunk;
    std::vector<uint64_t> in_off(n + 1), out_off(n + 1), sizes(n);
    in_off[0] = out_off[0] = 0;
    for (size_t i = 0; i < n; i++) {
        in_off[i + 1] = std::min(bytes, (i + 1) * s->chunk);
        out_off[i + 1] = out_off[i] + boa_max_compressed_size(in_off[i + 1] - in_off[i]);
    }
    TRY(m->d_out.ensure(out_off[n]));
    TRY(m->h_out.ensure(out_off[n]));
    TRY(compress_impl(m, n, s->dev[b].p, in_off.data(), m->d_out.p, out_off.data(), sizes.data()));
    std::vector<uint64_t> pk;
    TRY(fetch_compressed(m, n, sizes.data(), pk));
    shard.resize(kHeaderBytes + 16 * n + pk[n]);
    for (size_t i = 0; i < n; i++) {
        put64(shard.data() + kHeaderBytes + 16 * i, pk[i]);
        put64(shard.data() + kHeaderBytes + 16 * i + 8, sizes[i]);
    }
    if (pk[n]) memcpy(shard.data() + kHeaderBytes + 16 * n, m->h_out.p, pk[n]);
    write_container_header(shard.data(), m->fingerprint, bytes, s->chunk, n, in_off[n] - in_off[n - 1]);
    return BOA_OK;
}

static void stream_worker(boa_stream* s) {
    cudaSetDevice(s->m->device);
    for (;;) {
        std::pair<int, size_t> job;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait(lk, [&] { return s->stop || !s->jobs.empty(); });
            if (s->jobs.empty()) return;
            job = s->jobs.front();
            s->jobs.pop_front();
            s->running = true;
        }
        const int b = job.first;
        // the set's copy finished while the previous set was compressing
        const bool early = cudaEventQuery(s->loaded[b]) == cudaSuccess;
        boa_status st = BOA_OK;
        std::vector<uint8_t> shard;
        if (cudaEventSynchronize(s->loaded[b]) != cudaSuccess)
            st = fail(BOA_ERR_CUDA, "set copy failed: %s", cudaGetErrorString(cudaGetLastError()));
        bool skip;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            skip = s->err != BOA_OK;
        }
        if (st == BOA_OK && !skip) st = stream_compress_set(s, b, job.second, shard);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (st != BOA_OK && s->err == BOA_OK) {
                s->err = st;
                s->err_msg = boa_last_error();
            }
            if (st == BOA_OK && !skip) {
                s->shards.insert(s->shards.end(), shard.begin(), shard.end());
                s->sets++;
                s->preloaded += early ? 1 : 0;
            }
            s->busy[b] = false;
            s->running = false;
        }
        s->cv.notify_all();
    }
}

// The worker's first error, re-raised on the caller's thread.
static boa_status stream_error(boa_stream* s) {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->err == BOA_OK) return BOA_OK;
    return fail(s->err, "streaming pipeline: %s", s->err_msg.c_str());
}

// Hands the filled set buffer to the worker and switches to the other one.
static boa_status stream_submit(boa_stream* s) {
    const int b = s->cur;
    CU(cudaMemcpyAsync(s->dev[b].p, s->host[b].p, s->fill, cudaMemcpyHostToDevice, s->copy));
    CU(cudaEventRecord(s->loaded[b], s->copy));
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->busy[b] = true;
        s->jobs.emplace_back(b, s->fill);
        s->bytes_in += s->fill;
    }
    s->cv.notify_all();
    s->cur ^= 1;
    s->fill = 0;
    return BOA_OK;
}

extern "C" boa_status boa_stream_open(boa_model* m, size_t chunk_len, size_t set_chunks, boa_stream** out) {
    if (!m || !out || chunk_len == 0 || set_chunks == 0) return fail(BOA_ERR_ARG, "bad argument");
    if (set_chunks > (1u << 30) || chunk_len > ((size_t)1 << 40) / set_chunks)
        return fail(BOA_ERR_ARG, "set of %zu x %zu bytes is too large", set_chunks, chunk_len);
    *out = nullptr;
    CU(cudaSetDevice(m->device));
    auto* s = new boa_stream();
    s->m = m;
    s->chunk = chunk_len;
    s->per_set = set_chunks;
    s->set_bytes = chunk_len * set_chunks;
    boa_status st = BOA_OK;
    for (int b = 0; b < 2 && st == BOA_OK; b++) {
        st = s->host[b].ensure(s->set_bytes);
        if (st == BOA_OK) st = s->dev[b].ensure(s->set_bytes);
        if (st == BOA_OK && cudaEventCreateWithFlags(&s->loaded[b], cudaEventDisableTiming) != cudaSuccess)
            st = fail(BOA_ERR_CUDA, "cudaEventCreate failed");
    }
    if (st == BOA_OK && cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking) != cudaSuccess)
        st = fail(BOA_ERR_CUDA, "cudaStreamCreate failed");
    if (st != BOA_OK) {
        boa_stream_close(s);
        return st;
    }
    s->worker = std::thread(stream_worker, s);
    *out = s;
    return BOA_OK;
}

extern "C" boa_status boa_stream_push(boa_stream* s, const uint8_t* data, size_t len) {
    if (!s || (len && !data)) return fail(BOA_ERR_ARG, "bad argument");
    if (s->finished) return fail(BOA_ERR_ARG, "pipeline already finished");
    TRY(stream_error(s));
    CU(cudaSetDevice(s->m->device));
    while (len) {
        if (s->fill == 0) {
            // wait until the worker is done with this set buffer
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait(lk, [&] { return !s->busy[s->cur] || s->err != BOA_OK; });
        }
        TRY(stream_error(s));
        const size_t take = std::min(len, s->set_bytes - s->fill);
        memcpy(s->host[s->cur].p + s->fill, data, take);
        s->fill += take;
        data += take;
        len -= take;
        if (s->fill == s->set_bytes) TRY(stream_submit(s));
    }
    return BOA_OK;
}

extern "C" boa_status boa_stream_finish(boa_stream* s) {
    if (!s) return fail(BOA_ERR_ARG, "bad argument");
    if (!s->finished) {
        s->finished = true;
        if (s->fill) {
            {
                std::unique_lock<std::mutex> lk(s->mu);
                s->cv.wait(lk, [&] { return !s->busy[s->cur] || s->err != BOA_OK; });
            }
            TRY(stream_error(s));
            CU(cudaSetDevice(s->m->device));
            TRY(stream_submit(s));
        }
    }
    {
        std::unique_lock<std::mutex> lk(s->mu);
        s->cv.wait(lk, [&] { return s->jobs.empty() && !s->running; });
    }
    return stream_error(s);
}

extern "C" size_t boa_stream_available(const boa_stream* s) {
    if (!s) return 0;
    std::lock_guard<std::mutex> lk(s->mu);
    return s->shards.size() - s->read_at;
}

extern "C" boa_status boa_stream_read(boa_stream* s, uint8_t* out, size_t cap, size_t* out_size) {
    if (!s || !out_size || (cap && !out)) return fail(BOA_ERR_ARG, "bad argument");
    std::lock_guard<std::mutex> lk(s->mu);
    const size_t k = std::min(cap, s->shards.size() - s->read_at);
    if (k) memcpy(out, s->shards.data() + s->read_at, k);
    s->read_at += k;
    if (s->read_at == s->shards.size()) {
        s->shards.clear();
        s->read_at = 0;
    }
    *out_size = k;
    return BOA_OK;
}

extern "C" boa_status boa_stream_stats(const boa_stream* s, uint64_t* bytes_in, uint64_t* sets,
                                       uint64_t* preloaded) {
    if (!s) return fail(BOA_ERR_ARG, "bad argument");
    std::lock_guard<std::mutex> lk(s->mu);
    if (bytes_in) *bytes_in = s->bytes_in;
    if (sets) *sets = s->sets;
    if (preloaded) *preloaded = s->preloaded;
    return BOA_OK;
}

extern "C" void boa_stream_close(boa_stream* s) {
    if (!s) return;
    if (s->worker.joinable()) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stop = true;
        }
        s->cv.notify_all();
        s->worker.join();           // the worker drains the queued sets first
    }
    cudaSetDevice(s->m->device);
    if (s->copy) {
        cudaStreamSynchronize(s->copy);
        cudaStreamDestroy(s->copy);
    }
    for (int b = 0; b < 2; b++) {
        if (s->loaded[b]) cudaEventDestroy(s->loaded[b]);
        s->host[b].release();
        s->dev[b].release();
    }
    delete s;
}

// ------------------------------------------------------------ training step
//
// boa_train_step: the predictor's forward over n_seq x (seqlen - 1) rows
// keeping its intermediates, the gradient of the mean base-256
// cross-entropy, and one AdamW step of the weight file's tensor array; the
// device copies of the weights are then rebuilt from the updated array.
// FP32 throughout, fixed reduction order (kernels in train_step.cuh).

// Offsets of every tensor in the weight file's array.
struct FileOffsets {
    struct Layer { size_t ln_a_w, ln_a_b, in_w, conv_w, conv_b, x_w, dt_w, dt_b, A_log, D, out_w, ln_b_w, ln_b_b; };
    size_t embed = 0, head_w = 0, head_b = 0;
    std::vector<Layer> layers;
};

static FileOffsets file_offsets(const boa_model* m) {
    const size_t d = m->d, E = m->E, N = m->N, K = m->K, r = m->r, R2 = m->R2, F = m->F;
    FileOffsets fo;
    size_t o = 0;
    auto take = [&](size_t n) { size_t at = o; o += n; return at; };
    fo.embed = take(256 * d);
    fo.layers.resize(m->nl);
    for (auto& L : fo.layers) {
        L.ln_a_w = take(d); L.ln_a_b = take(d);
        L.in_w = take(2 * E * d);
        L.conv_w = take(E * K); L.conv_b = take(E);
        L.x_w = take(R2 * E);
        L.dt_w = take(E * r); L.dt_b = take(E);
        L.A_log = take(E * N); L.D = take(E);
        L.out_w = take(d * E);
        if (F) take(F * d + F + d * F + d);
        L.ln_b_w = take(d); L.ln_b_b = take(d);
    }
    fo.head_w = take(256 * d);
    fo.head_b = take(256);
    return fo;
}

struct TrainState {
    size_t rows = 0;                 // capacity of the row buffers
    int bsz = 0, T = 0;
    DevBuf<float> master, grad, m1, m2;
    DevBuf<uint8_t> tok;
    // per layer
    std::vector<DevBuf<float>> X, XN, mA, rA, XZ, CPRE, U, DBC, DPRE, DELTA, AN, BM, CM, YS, HIN, YG, URES, mB, rB;
    // shared by the backward
    DevBuf<float> logits, dlogits, loss_rows, loss, dX, dXin, dU, dCPRE, dXZ, dYG, dYS, dDELTA, dDPRE, dDBC, dDL,
        dXN, dyxh, dURES, hs, dA_part, dD_part, dB_part, dC_part, part;
    // BF16 model: tensor-core operands (A rows, transposed A / B for the
    // weight gradients, a transposed weight for the input gradients)
    DevBuf<__nv_bfloat16> ab, tA, tB, wT;
    size_t rows_pad = 0;             // row count of tA / tB, a multiple of kTrRowsPerPart
    uint64_t step = 0;
    ~TrainState() {
        for (auto* v : {&X, &XN, &mA, &rA, &XZ, &CPRE, &U, &DBC, &DPRE, &DELTA, &AN, &BM, &CM, &YS, &HIN, &YG, &URES,
                        &mB, &rB})
            for (auto& b : *v) b.release();
        for (auto* b : {&master, &grad, &m1, &m2, &logits, &dlogits, &loss_rows, &loss, &dX, &dXin, &dU, &dCPRE, &dXZ,
                        &dYG, &dYS, &dDELTA, &dDPRE, &dDBC, &dDL, &dXN, &dyxh, &dURES, &hs, &dA_part, &dD_part,
                        &dB_part, &dC_part, &part})
            b->release();
        tok.release();
        ab.release(); tA.release(); tB.release(); wT.release();
    }
};

static void free_train_state(boa_model* m) {
    delete m->tr;
    m->tr = nullptr;
}

static const int kTrainChunk = 256;        // scan backward recomputation chunk
static const long long kTrRowsPerPart = 4096;

// Train on n_seq sequences of seqlen bytes (device copy of the batch in
// tr->tok); fills tr->grad and tr->loss.
static boa_status train_forward_backward(boa_model* m, int bsz, int T, int seqlen) {
    TrainState& t = *m->tr;
    const long long rows = (long long)bsz * T;
    const int d = m->d, E = m->E, N = m->N, K = m->K, r = m->r, R2 = m->R2, nl = m->nl;
    const FileOffsets fo = file_offsets(m);
    const float* P = t.master.p;
    float* G = t.grad.p;
    cudaStream_t st = m->stream;
    const uint8_t* tok = t.tok.p;
    auto blocks = [](long long n, int b) { return (unsigned)((n + b - 1) / b); };
    auto nn = [&](int M, int Nn, int Kk, const float* A, int lda, const float* B, int ldb, float* C, int ldc,
                  const float* bias, int acc) {
        dim3 g(blocks(Nn, kTrTile), blocks(M, kTrTile));
        k_tr_gemm_nn<<<g, 256, 0, st>>>(M, Nn, Kk, A, lda, B, ldb, C, ldc, bias, acc);
    };
    const int nparts = (int)((rows + kTrRowsPerPart - 1) / kTrRowsPerPart);
    // out[Nn][Kk] = A^T B over all rows (A rows x Nn, B rows x Kk)
    auto tn = [&](int Nn, int Kk, const float* A, int lda, const float* B, int ldb, float* out) {
        dim3 g(blocks(Kk, kTrTile), blocks(Nn, kTrTile), nparts);
        k_tr_gemm_tn<<<g, 256, 0, st>>>(rows, Nn, Kk, A, lda, B, ldb, t.part.p, kTrRowsPerPart);
        const size_t cnt = (size_t)Nn * Kk;
        k_tr_reduce<<<blocks((long long)cnt, 256), 256, 0, st>>>(t.part.p, nparts, cnt, out, 0, nullptr);
    };
    auto colsum = [&](const float* A, int n, int lda, float* out) {
        dim3 g(blocks(n, 128), nparts);
        k_tr_colsum<<<g, 128, 0, st>>>(A, rows, n, lda, t.part.p, kTrRowsPerPart);
        k_tr_reduce<<<blocks(n, 256), 256, 0, st>>>(t.part.p, nparts, (size_t)n, out, 0, nullptr);
    };
    const unsigned warps_grid = blocks(rows, 8);   // one warp per row, 8 per CTA
    // BF16 model: the projections (forward), the input gradients of in_proj,
    // out_proj and the head, and the weight gradients of those three and
    // x_proj run on the tensor cores with BF16 operands and FP32
    // accumulation; dt_proj (K = r) and x_proj's input gradient (K = r + 2N)
    // stay on the CUDA cores.  Their operands are written by the kernel just
    // before them, so these launches go without programmatic dependent
    // launch (each starts after its predecessor has finished).
    const bool tc = m->precision == BOA_PREC_BF16;
    const bool pdl_saved = m->pdl;
    m->pdl = false;
    m->v.stream = st;
    struct PdlRestore { boa_model* m; bool v; ~PdlRestore() { m->pdl = v; } } pdl_restore{m, pdl_saved};
    auto bf16 = [&](const float* src, size_t n) -> const __nv_bfloat16* {
        k_tr_bf16<<<blocks((long long)n, 256), 256, 0, st>>>(src, t.ab.p, n);
        return t.ab.p;
    };
    // dst [C][rows_pad] = bf16(src[rows][C])^T (src leading dimension lds)
    auto bf16_t = [&](const float* src, int lds, int C, __nv_bfloat16* dst) {
        k_tr_bf16_t<<<dim3((unsigned)(t.rows_pad / 32), blocks(C, 32)), dim3(32, 8), 0, st>>>(src, lds, rows, C,
                                                                                                (long long)t.rows_pad, dst);
    };
    // BF16 W^T ([in][out]) of a master weight stored [out][in]
    auto weight_t = [&](const float* w, int out, int in) -> const __nv_bfloat16* {
        k_tr_bf16_t<<<dim3(blocks(out, 32), blocks(in, 32)), dim3(32, 8), 0, st>>>(w, in, out, in, out, t.wT.p);
        return t.wT.p;
    };
    // G[Nn][Kk] = A^T B over all rows (A rows x Nn, B rows x Kk), by parts
    auto tn_tc = [&](int Nn, int Kk, const float* A, int lda, const float* B, int ldb, float* out) -> boa_status {
        bf16_t(A, lda, Nn, t.tA.p);
        bf16_t(B, ldb, Kk, t.tB.p);
        const int parts = (int)(t.rows_pad / kTrRowsPerPart);
        TRY(gemm_tc_parts(m, t.tA.p, t.tB.p, t.part.p, Nn, Kk, (long long)t.rows_pad, parts));
        const size_t cnt = (size_t)Nn * Kk;
        k_tr_reduce<<<blocks((long long)cnt, 256), 256, 0, st>>>(t.part.p, parts, cnt, out, 0, nullptr);
        return BOA_OK;
    };

    // ---- forward
    k_tr_embed<<<blocks(rows * d, 256), 256, 0, st>>>(tok, T, seqlen, P + fo.embed, t.X[0].p, rows, d);
    for (int l = 0; l < nl; l++) {
        const auto& o = fo.layers[l];
        const DevLayer& L = m->layers[l];
        k_tr_ln_fwd<<<warps_grid, 256, 0, st>>>(t.X[l].p, P + o.ln_a_w, P + o.ln_a_b, t.XN[l].p, t.mA[l].p, t.rA[l].p,
                                                rows, d);
        if (tc) TRY(gemm_tc<kEpiStore>(m, BOA_KC_GEMM_IN, bf16(t.XN[l].p, (size_t)rows * d), m->blayers[l].in_w,
                                       nullptr, t.XZ[l].p, nullptr, rows, 2 * E, d));
        else nn((int)rows, 2 * E, d, t.XN[l].p, d, L.in_wt, 2 * E, t.XZ[l].p, 2 * E, nullptr, 0);
        k_tr_conv_fwd<<<dim3(blocks(E, 128), bsz), 128, 0, st>>>(t.XZ[l].p, E, P + o.conv_w, P + o.conv_b,
                                                                  t.CPRE[l].p, t.U[l].p, T, K);
        if (tc) TRY(gemm_tc<kEpiStore>(m, BOA_KC_GEMM_X, bf16(t.U[l].p, (size_t)rows * E), m->blayers[l].x_w, nullptr,
                                       t.DBC[l].p, nullptr, rows, R2, E));
        else nn((int)rows, R2, E, t.U[l].p, E, L.x_wt, R2, t.DBC[l].p, R2, nullptr, 0);
        nn((int)rows, E, r, t.DBC[l].p, R2, L.dt_w, E, t.DPRE[l].p, E, P + o.dt_b, 0);
        k_tr_softplus<<<blocks(rows * E, 256), 256, 0, st>>>(t.DPRE[l].p, t.DELTA[l].p, (size_t)rows * E);
        k_tr_neg_exp<<<blocks((long long)E * N, 256), 256, 0, st>>>(P + o.A_log, t.AN[l].p, (size_t)E * N);
        k_tr_split_bc<<<blocks(rows * N, 256), 256, 0, st>>>(t.DBC[l].p, r, N, t.BM[l].p, t.CM[l].p, rows);
        k_scan_train_fwd<16><<<dim3(blocks(E, kTrainThreads), bsz), kTrainThreads, 0, st>>>(
            T, E, kTrainChunk, t.U[l].p, t.DELTA[l].p, t.AN[l].p, t.BM[l].p, t.CM[l].p, P + o.D, t.YS[l].p, t.HIN[l].p);
        k_tr_gate_fwd<<<blocks(rows * E, 256), 256, 0, st>>>(t.YS[l].p, t.XZ[l].p, E, t.YG[l].p, rows);
        CU(cudaMemcpyAsync(t.URES[l].p, t.X[l].p, (size_t)rows * d * 4, cudaMemcpyDeviceToDevice, st));
        if (tc) TRY(gemm_tc<kEpiResid>(m, BOA_KC_GEMM_OUT, bf16(t.YG[l].p, (size_t)rows * E), m->blayers[l].out_w,
                                       nullptr, t.URES[l].p, nullptr, rows, d, E));
        else nn((int)rows, d, E, t.YG[l].p, E, L.out_wt, d, t.URES[l].p, d, nullptr, 1);
        k_tr_ln_fwd<<<warps_grid, 256, 0, st>>>(t.URES[l].p, P + o.ln_b_w, P + o.ln_b_b, t.X[l + 1].p, t.mB[l].p,
                                                t.rB[l].p, rows, d);
    }
    if (tc) TRY(gemm_tc<kEpiBias>(m, BOA_KC_GEMM_HEAD, bf16(t.X[nl].p, (size_t)rows * d), m->head_wb, P + fo.head_b,
                                  t.logits.p, nullptr, rows, 256, d));
    else nn((int)rows, 256, d, t.X[nl].p, d, m->head_wt, 256, t.logits.p, 256, P + fo.head_b, 0);
    const float scale = (float)(1.0 / ((double)rows * std::log(256.0)));
    k_tr_xent<<<warps_grid, 256, 0, st>>>(t.logits.p, tok, T, seqlen, t.dlogits.p, t.loss_rows.p, rows, scale);
    k_tr_sum<<<1, kTrBlock, 0, st>>>(t.loss_rows.p, rows, t.loss.p);

    // ---- backward
    if (tc) TRY(tn_tc(256, d, t.dlogits.p, 256, t.X[nl].p, d, G + fo.head_w));
    else tn(256, d, t.dlogits.p, 256, t.X[nl].p, d, G + fo.head_w);
    colsum(t.dlogits.p, 256, 256, G + fo.head_b);
    if (tc) {
        const __nv_bfloat16* w = weight_t(P + fo.head_w, 256, d);
        TRY(gemm_tc<kEpiStore>(m, BOA_KC_OTHER, bf16(t.dlogits.p, (size_t)rows * 256), w, nullptr, t.dX.p, nullptr,
                               rows, d, 256));
    } else {
        nn((int)rows, d, 256, t.dlogits.p, 256, P + fo.head_w, d, t.dX.p, d, nullptr, 0);
    }
    const int nblk = (E + kTrainThreads - 1) / kTrainThreads;
    for (int l = nl - 1; l >= 0; l--) {
        const auto& o = fo.layers[l];
        // LN_b
        k_tr_ln_bwd<<<warps_grid, 256, 0, st>>>(t.dX.p, t.URES[l].p, t.mB[l].p, t.rB[l].p, P + o.ln_b_w, t.dURES.p,
                                                t.dyxh.p, rows, d, 0);
        colsum(t.dyxh.p, d, d, G + o.ln_b_w);
        colsum(t.dX.p, d, d, G + o.ln_b_b);
        // residual: the block input receives dURES directly
        CU(cudaMemcpyAsync(t.dXin.p, t.dURES.p, (size_t)rows * d * 4, cudaMemcpyDeviceToDevice, st));
        // out_proj
        if (tc) {
            TRY(tn_tc(d, E, t.dURES.p, d, t.YG[l].p, E, G + o.out_w));
            const __nv_bfloat16* w = weight_t(P + o.out_w, d, E);
            TRY(gemm_tc<kEpiStore>(m, BOA_KC_OTHER, bf16(t.dURES.p, (size_t)rows * d), w, nullptr, t.dYG.p, nullptr,
                                   rows, E, d));
        } else {
            tn(d, E, t.dURES.p, d, t.YG[l].p, E, G + o.out_w);
            nn((int)rows, E, d, t.dURES.p, d, P + o.out_w, E, t.dYG.p, E, nullptr, 0);
        }
        // gate
        k_tr_gate_bwd<<<blocks(rows * E, 256), 256, 0, st>>>(t.dYG.p, t.YS[l].p, t.XZ[l].p, E, t.dYS.p, t.dXZ.p, rows);
        // scan
        k_scan_train_bwd<16><<<dim3(blocks(E, kTrainThreads), bsz), kTrainThreads, 0, st>>>(
            T, E, kTrainChunk, t.U[l].p, t.DELTA[l].p, t.AN[l].p, t.BM[l].p, t.CM[l].p, P + o.D, t.dYS.p, t.HIN[l].p,
            t.hs.p, t.dU.p, t.dDELTA.p, t.dA_part.p, t.dD_part.p, t.dB_part.p, t.dC_part.p);
        k_tr_reduce<<<blocks(E, 256), 256, 0, st>>>(t.dD_part.p, bsz, (size_t)E, G + o.D, 0, nullptr);
        k_tr_reduce<<<blocks((long long)E * N, 256), 256, 0, st>>>(t.dA_part.p, bsz, (size_t)E * N, G + o.A_log, 0,
                                                                    t.AN[l].p);   // dA/dA_log = A
        // softplus, dt_proj
        k_tr_softplus_bwd<<<blocks(rows * E, 256), 256, 0, st>>>(t.dDELTA.p, t.DPRE[l].p, t.dDPRE.p, (size_t)rows * E);
        tn(E, r, t.dDPRE.p, E, t.DBC[l].p, R2, G + o.dt_w);
        colsum(t.dDPRE.p, E, E, G + o.dt_b);
        nn((int)rows, r, E, t.dDPRE.p, E, P + o.dt_w, r, t.dDL.p, r, nullptr, 0);
        // x_proj
        k_tr_assemble_ddbc<<<blocks(rows * R2, 256), 256, 0, st>>>(t.dDL.p, t.dB_part.p, t.dC_part.p, nblk, r, N,
                                                                    t.dDBC.p, rows);
        if (tc) TRY(tn_tc(R2, E, t.dDBC.p, R2, t.U[l].p, E, G + o.x_w));
        else tn(R2, E, t.dDBC.p, R2, t.U[l].p, E, G + o.x_w);
        nn((int)rows, E, R2, t.dDBC.p, R2, P + o.x_w, E, t.dU.p, E, nullptr, 1);
        // SiLU, conv
        k_tr_silu_bwd<<<blocks(rows * E, 256), 256, 0, st>>>(t.dU.p, t.CPRE[l].p, t.dCPRE.p, (size_t)rows * E);
        k_tr_conv_bwd<<<dim3(blocks(E, 128), bsz), 128, 0, st>>>(t.dCPRE.p, P + o.conv_w, t.dXZ.p, T, E, K);
        {
            dim3 g(blocks(E, 128), nparts);
            k_tr_conv_wgrad<<<g, 128, 0, st>>>(t.dCPRE.p, t.XZ[l].p, t.part.p, T, E, K, rows, kTrRowsPerPart);
            // parts are [z][c][K+1]: weights [c][k] and bias c
            const size_t cnt = (size_t)E * (K + 1);
            k_tr_reduce<<<blocks((long long)cnt, 256), 256, 0, st>>>(t.part.p, nparts, cnt, t.dDL.p, 0, nullptr);
            // scatter: weight grads [E][K] and bias [E] from the [E][K+1] sums
            CU(cudaMemcpy2DAsync(G + o.conv_w, (size_t)K * 4, t.dDL.p, (size_t)(K + 1) * 4, (size_t)K * 4, E,
                                 cudaMemcpyDeviceToDevice, st));
            CU(cudaMemcpy2DAsync(G + o.conv_b, 4, t.dDL.p + K, (size_t)(K + 1) * 4, 4, E, cudaMemcpyDeviceToDevice, st));
        }
        // in_proj
        if (tc) {
            TRY(tn_tc(2 * E, d, t.dXZ.p, 2 * E, t.XN[l].p, d, G + o.in_w));
            const __nv_bfloat16* w = weight_t(P + o.in_w, 2 * E, d);
            TRY(gemm_tc<kEpiStore>(m, BOA_KC_OTHER, bf16(t.dXZ.p, (size_t)rows * 2 * E), w, nullptr, t.dXN.p, nullptr,
                                   rows, d, 2 * E));
        } else {
            tn(2 * E, d, t.dXZ.p, 2 * E, t.XN[l].p, d, G + o.in_w);
            nn((int)rows, d, 2 * E, t.dXZ.p, 2 * E, P + o.in_w, d, t.dXN.p, d, nullptr, 0);
        }
        // LN_a (adds into the residual gradient of the block input)
        k_tr_ln_bwd<<<warps_grid, 256, 0, st>>>(t.dXN.p, t.X[l].p, t.mA[l].p, t.rA[l].p, P + o.ln_a_w, t.dXin.p,
                                                t.dyxh.p, rows, d, 1);
        colsum(t.dyxh.p, d, d, G + o.ln_a_w);
        colsum(t.dXN.p, d, d, G + o.ln_a_b);
        std::swap(t.dX.p, t.dXin.p);
        std::swap(t.dX.n, t.dXin.n);
    }
    k_tr_embed_bwd<<<256, d, 0, st>>>(t.dX.p, tok, T, seqlen, rows, d, G + fo.embed);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(BOA_ERR_CUDA, "training kernels: %s", cudaGetErrorString(e));
    return BOA_OK;
}

// Buffers for bsz x T rows (kept and grown across calls).
static boa_status ensure_train_state(boa_model* m, int bsz, int T, int seqlen) {
    if (m->F) return fail(BOA_ERR_ARG, "boa_train_step supports blocks without FFN (ffn_mult 0)");
    if (!m->tr) m->tr = new TrainState();
    TrainState& t = *m->tr;
    const size_t rows = (size_t)bsz * T;
    const size_t d = m->d, E = m->E, N = m->N, R2 = m->R2, nl = m->nl, r = m->r, K = m->K;
    if (!t.master.p) {
        TRY(t.master.ensure(m->n_params));
        TRY(t.grad.ensure(m->n_params));
        TRY(t.m1.ensure(m->n_params));
        TRY(t.m2.ensure(m->n_params));
        CU(cudaMemcpy(t.master.p, m->params.data(), m->n_params * 4, cudaMemcpyHostToDevice));
        CU(cudaMemset(t.m1.p, 0, m->n_params * 4));
        CU(cudaMemset(t.m2.p, 0, m->n_params * 4));
    }
    TRY(t.tok.ensure((size_t)bsz * seqlen));
    auto per_layer = [&](std::vector<DevBuf<float>>& v, size_t count, size_t layers) -> boa_status {
        if (v.size() < layers) v.resize(layers);
        for (size_t i = 0; i < layers; i++) TRY(v[i].ensure(std::max<size_t>(count, 1)));
        return BOA_OK;
    };
    const size_t nck = (T + kTrainChunk - 1) / kTrainChunk, nblk = (E + kTrainThreads - 1) / kTrainThreads;
    TRY(per_layer(t.X, rows * d, nl + 1));
    TRY(per_layer(t.XN, rows * d, nl));
    TRY(per_layer(t.mA, rows, nl));
    TRY(per_layer(t.rA, rows, nl));
    TRY(per_layer(t.XZ, rows * 2 * E, nl));
    TRY(per_layer(t.CPRE, rows * E, nl));
    TRY(per_layer(t.U, rows * E, nl));
    TRY(per_layer(t.DBC, rows * R2, nl));
    TRY(per_layer(t.DPRE, rows * E, nl));
    TRY(per_layer(t.DELTA, rows * E, nl));
    TRY(per_layer(t.AN, E * N, nl));
    TRY(per_layer(t.BM, rows * N, nl));
    TRY(per_layer(t.CM, rows * N, nl));
    TRY(per_layer(t.YS, rows * E, nl));
    TRY(per_layer(t.HIN, (size_t)bsz * nck * N * E, nl));
    TRY(per_layer(t.YG, rows * E, nl));
    TRY(per_layer(t.URES, rows * d, nl));
    TRY(per_layer(t.mB, rows, nl));
    TRY(per_layer(t.rB, rows, nl));
    TRY(t.logits.ensure(rows * 256));
    TRY(t.dlogits.ensure(rows * 256));
    TRY(t.loss_rows.ensure(rows));
    TRY(t.loss.ensure(1));
    TRY(t.dX.ensure(rows * d));
    TRY(t.dXin.ensure(rows * d));
    TRY(t.dU.ensure(rows * E));
    TRY(t.dCPRE.ensure(rows * E));
    TRY(t.dXZ.ensure(rows * 2 * E));
    TRY(t.dYG.ensure(rows * E));
    TRY(t.dYS.ensure(rows * E));
    TRY(t.dDELTA.ensure(rows * E));
    TRY(t.dDPRE.ensure(rows * E));
    TRY(t.dDBC.ensure(rows * R2));
    TRY(t.dDL.ensure(std::max(rows * r, E * (K + 1))));
    TRY(t.dXN.ensure(rows * d));
    TRY(t.dyxh.ensure(rows * d));
    TRY(t.dURES.ensure(rows * d));
    TRY(t.hs.ensure((size_t)bsz * kTrainChunk * N * E));
    TRY(t.dA_part.ensure((size_t)bsz * E * N));
    TRY(t.dD_part.ensure((size_t)bsz * E));
    TRY(t.dB_part.ensure(rows * nblk * N));
    TRY(t.dC_part.ensure(rows * nblk * N));
    const size_t nparts = (rows + kTrRowsPerPart - 1) / kTrRowsPerPart;
    const size_t widest = std::max({2 * E * d, d * E, R2 * E, E * r, (size_t)256 * d, E * (K + 1), 2 * E, (size_t)256});
    TRY(t.part.ensure(nparts * widest));
    if (!m->err.p) {                 // pipeline-timeout code of the tensor-core kernels
        TRY(m->err.ensure(1));
        CU(cudaMemset(m->err.p, 0, sizeof(int)));
    }
    if (m->precision == BOA_PREC_BF16) {
        t.rows_pad = nparts * kTrRowsPerPart;
        TRY(t.ab.ensure(rows * std::max<size_t>(2 * E, 256)));
        TRY(t.tA.ensure(t.rows_pad * std::max<size_t>(2 * E, 256)));
        TRY(t.tB.ensure(t.rows_pad * std::max(E, d)));
        TRY(t.wT.ensure(std::max<size_t>(2 * E * d, (size_t)256 * d)));
    }
    t.rows = std::max(t.rows, rows);
    return BOA_OK;
}

static boa_status train_batch(boa_model* m, const uint8_t* batch, size_t n_seq, size_t seqlen) {
    if (!m || !batch || n_seq == 0 || seqlen < 2) return fail(BOA_ERR_ARG, "bad argument");
    if (n_seq > 65535 || seqlen > (1u << 24) || n_seq * (seqlen - 1) > (1ull << 22))
        return fail(BOA_ERR_ARG, "batch too large (at most 2^22 predicted positions)");
    CU(cudaSetDevice(m->device));
    const int bsz = (int)n_seq, T = (int)seqlen - 1;
    TRY(ensure_train_state(m, bsz, T, (int)seqlen));
    CU(cudaMemcpyAsync(m->tr->tok.p, batch, n_seq * seqlen, cudaMemcpyHostToDevice, m->stream));
    TRY(train_forward_backward(m, bsz, T, (int)seqlen));
    return m->precision == BOA_PREC_BF16 ? check_tc_error(m) : BOA_OK;
}

static boa_status read_loss(boa_model* m, size_t rows, float* loss_out) {
    float s = 0.f;
    CU(cudaMemcpyAsync(&s, m->tr->loss.p, 4, cudaMemcpyDeviceToHost, m->stream));
    CU(cudaStreamSynchronize(m->stream));
    if (loss_out) *loss_out = (float)(s / (rows * std::log(256.0)));
    return BOA_OK;
}

extern "C" boa_status boa_train_step(boa_model* m, const uint8_t* batch, size_t n_seq, size_t seqlen, float lr,
                                     float* loss_out) {
    if (!m) return fail(BOA_ERR_ARG, "null model");
    MODEL_LOCK(m);
    TRY(train_batch(m, batch, n_seq, seqlen));
    TrainState& t = *m->tr;
    t.step++;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f, wd = 0.01f;
    const float bc1 = (float)(1.0 - std::pow((double)b1, (double)t.step));
    const float bc2 = (float)(1.0 - std::pow((double)b2, (double)t.step));
    k_tr_adamw<<<(unsigned)((m->n_params + 255) / 256), 256, 0, m->stream>>>(t.master.p, t.grad.p, t.m1.p, t.m2.p,
                                                                           m->n_params, lr, b1, b2, eps, wd, bc1, bc2);
    CU(cudaGetLastError());
    TRY(read_loss(m, n_seq * (seqlen - 1), loss_out));
    // the updated array becomes the model: host copy, device copies, fingerprint
    CU(cudaMemcpyAsync(m->params.data(), t.master.p, m->n_params * 4, cudaMemcpyDeviceToHost, m->stream));
    CU(cudaStreamSynchronize(m->stream));
    TRY(upload_weights(m, m->params.data()));
    // FNV-1a of the file boa_save_model would write, as boa_load_model takes it
    uint64_t h = fnv1a64_update(1469598103934665603ull, reinterpret_cast<const uint8_t*>("BOAW"), 4);
    h = fnv1a64_update(h, reinterpret_cast<const uint8_t*>(m->header), sizeof m->header);
    m->fingerprint = fnv1a64_update(h, reinterpret_cast<const uint8_t*>(m->params.data()), m->n_params * 4);
    return BOA_OK;
}

extern "C" boa_status boa_debug_train_grad(boa_model* m, const uint8_t* batch, size_t n_seq, size_t seqlen,
                                           float* grad_out, float* loss_out) {
    if (!m) return fail(BOA_ERR_ARG, "null model");
    MODEL_LOCK(m);
    TRY(train_batch(m, batch, n_seq, seqlen));
    TRY(read_loss(m, n_seq * (seqlen - 1), loss_out));
    if (grad_out) {
        CU(cudaMemcpyAsync(grad_out, m->tr->grad.p, m->n_params * 4, cudaMemcpyDeviceToHost, m->stream));
        CU(cudaStreamSynchronize(m->stream));
    }
    return BOA_OK;
}

extern "C" size_t boa_model_param_count(const boa_model* m) { return m ? m->n_params : 0; }

extern "C" boa_status boa_save_model(const boa_model* m, const char* path) {
    if (!m || !path) return fail(BOA_ERR_ARG, "null argument");
    MODEL_LOCK(m);
    FILE* fp = fopen(path, "wb");
    if (!fp) return fail(BOA_ERR_IO, "cannot open %s for writing", path);
    bool ok = fwrite("BOAW", 1, 4, fp) == 4 && fwrite(m->header, 4, 9, fp) == 9 &&
              fwrite(m->params.data(), 4, m->n_params, fp) == m->n_params;
    ok = (fclose(fp) == 0) && ok;
    if (!ok) return fail(BOA_ERR_IO, "short write on %s", path);
    return BOA_OK;
}
