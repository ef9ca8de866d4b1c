// Persistent decoder with on-chip model state (the FP32 form).
//
// One CTA per SM decodes kOcSlots streams side by side, each from its first
// byte to its last, and then takes the next stream from a queue (longest
// first).  The whole of a decode step runs inside the kernel: embedding and
// LayerNorm, per block in_proj, causal conv + SiLU, x_proj, dt_proj +
// softplus + selective scan + gate, out_proj + residual, the LayerNorm pair,
// then the head, softmax, quantiser and range decoder (Alg. 1 and the
// paper's "Decoder" paragraph), so a stream's model state never leaves the
// SM: its SSM state (N x E per block) and conv window ((K - 1) x E per block)
// sit in the SM's tensor memory (TMEM, used here as a 256 KB scratchpad by
// SIMT code), its activations in shared memory.
//
// Per step every weight of the model is needed once per CTA.  A producer
// warp streams the projection matrices (in_proj, x_proj, out_proj of every
// block, then the head), stored K-major, through a ring of shared-memory
// stages with cp.async.bulk in that fixed order, step after step; the
// compute warps consume the stages in the same order and release each one
// through an mbarrier.  The small per-channel parameters (conv taps, W_dt,
// A, D, biases, LayerNorm weights) are read from global memory (L2).
//
// Every value is computed with the operations, in the order, of the FP32
// form's step kernels: each projection output is the chain acc = fma(a[k],
// W[k][n], acc) over k = 0 .. K-1 from zero followed by the same epilogue
// (k_gemm_fp32), the conv, scan, LayerNorm, softmax and quantiser are those
// of k_conv_silu, k_scan, k_ln_ln, warp_logits_to_hist and warp_quantise_p.
// A stream encoded in the FP32 form therefore decodes here with the same
// CDFs at every step.
//
// Compute threads: 256 (8 warps).  Thread t owns channels 2t and 2t + 1
// (E <= 512) in the conv and the scan, and its TMEM lane 32 (w % 4) + lane
// of warp w, columns 256 (w / 4) .. + 255:
//   SSM state of (slot p, block l, channel j): 16 columns at
//     ((p * kOcMaxLayers + l) * 2 + j) * 16
//   conv window (oldest first, K - 1 <= 3 values and one pad): 4 columns at
//     kOcConvCol0 + ((p * kOcMaxLayers + l) * 2 + j) * 4
// Waits are bounded (about 2 s of globaltimer each): on expiry the CTA
// records code 4 in *err, lets its copies in flight land, frees TMEM and
// returns.
#pragma once
#include "scan_step.cuh"

namespace boa {

constexpr int kOcSlots = 2;                        // streams per CTA
constexpr int kOcThreads = 256;                    // compute threads
constexpr int kOcBlock = kOcThreads + 32;          // + the weight-streaming warp
// Ring: three 64 KB stages.  Each stage costs every compute warp a wait and
// a release, so fewer, larger stages are cheaper: measured per decode step
// of 2 x 148 streams, 6 x 32 KB 75.8 us, 3 x 64 KB 64.9 us (sixteen compute
// warps with one channel each: 83.9 / 72.6 us).  Sharing one weight stream
// across a cluster by multicast copies was slower still (2 CTAs 102 us,
// 4 CTAs 118 us): each chunk then waits for every CTA's release.
constexpr int kOcStage = 65536;                    // bytes per ring stage
constexpr int kOcStages = 3;
constexpr int kOcMaxLayers = 3;
constexpr int kOcNS = 16;                          // d_state
constexpr int kOcMaxE = 2 * kOcThreads;
constexpr int kOcConvCol0 = kOcSlots * kOcMaxLayers * 2 * kOcNS;
static_assert(kOcConvCol0 + kOcSlots * kOcMaxLayers * 2 * 4 <= 256, "a compute thread's state fits its TMEM columns");

// Activation floats per slot in shared memory: x, xn (d each), xz (2E), u
// (E), [delta|B|C] (48), the gated scan output (E), logits (256).
__host__ __device__ constexpr int oc_act_floats(int d, int E) { return 2 * d + 4 * E + 48 + 256; }
__host__ __device__ constexpr size_t oc_smem_bytes(int d, int E) {
    return (size_t)kOcStages * kOcStage + (size_t)kOcSlots * oc_act_floats(d, E) * 4;
}

struct OcLayer {
    const float *in_wt, *x_wt, *out_wt;           // [d][2E], [E][R2], [E][d]
    const float *conv_w, *conv_b;                 // [K][E], [E]
    const float *dt_w, *dt_b, *A2, *D;            // [R][E], [E], [N][E] (A log2 e), [E]
    const float *ln_a_w, *ln_a_b, *ln_b_w, *ln_b_b;
};

struct OcModel {
    OcLayer L[kOcMaxLayers];
    const float *embed, *head_wt, *head_b;        // [256][d], [d][256], [256]
    int nl, E, K;                                 // blocks, channels, conv width
};

struct OcWork {
    const int* order;        // streams of >= 2 bytes, longest first
    int n;
    int* next;               // queue head, zero at launch
    const uint8_t* cin;      // coded streams
    StreamTable tb;
    uint8_t* out;
    int* err;
};

// Component q (compile-time after unrolling) of a float4.
__device__ __forceinline__ float f4_at(const float4& v, int q) {
    return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w;
}

// Rows of a K-major matrix with `cols` columns that one stage holds (a
// multiple of 4; every matrix has a multiple of 4 rows, so every stage
// does).
__host__ __device__ inline int oc_rpc(int rows, int cols) {
    const int r = (kOcStage / 4 / cols) & ~3;
    return r < rows ? r : rows;
}

// Matrix i of a step's weight stream: 3 l + 0/1/2 = block l's in_proj,
// x_proj, out_proj; 3 nl = the head.
template <int VPT, int R>
__device__ __forceinline__ void oc_matrix(const OcModel& M, int i, const float*& W, int& rows, int& cols) {
    constexpr int d = VPT * 32;
    if (i == 3 * M.nl) {
        W = M.head_wt; rows = d; cols = 256;
        return;
    }
    const OcLayer& L = M.L[i / 3];
    switch (i % 3) {
        case 0: W = L.in_wt; rows = d; cols = 2 * M.E; break;
        case 1: W = L.x_wt; rows = M.E; cols = R + 2 * kOcNS; break;
        default: W = L.out_wt; rows = M.E; cols = d; break;
    }
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; i++) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float (&v)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
                 ::"r"(taddr), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                   "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                   "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
                 : "memory");
}

// Wait for a ring stage, giving up when another thread of the CTA has
// already given up (abort flag) or after the bounded wait.
__device__ __forceinline__ bool oc_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    while (!mbar_try(bar, parity)) {
        if (*abort_flag) return false;
        if (globaltimer() - t0 > kWaitNs) {
            *abort_flag = 1;
            return false;
        }
    }
    return true;
}

// Barrier of the 256 compute threads (the streaming warp never joins it),
// with an OR of their votes.
__device__ __forceinline__ void oc_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

__device__ __forceinline__ bool oc_sync_or(bool v) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n"
        " setp.ne.u32 p, %1, 0;\n"
        " bar.red.or.pred q, 1, 256, p;\n"
        " selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)v)
        : "memory");
    return r != 0;
}

// Consume the ring stages of one matrix (rows of `cols` floats, in the
// order the streaming warp sends them): body(stage, k0, nr) sees rows
// k0 .. k0 + nr - 1.  The wait is warp-uniform; lane 0 releases the stage
// once the whole warp is done with it.  False: the wait gave up.
template <typename F>
__device__ __forceinline__ bool oc_consume(int rows, int cols, int& gc, uint64_t* full, uint64_t* empty,
                                           const float* ring, volatile int* abort_flag, int lane, F&& body) {
    const int rpc = oc_rpc(rows, cols);
    for (int k0 = 0; k0 < rows; k0 += rpc, gc++) {
        const int s = gc % kOcStages;
        if (!__all_sync(0xffffffffu, oc_wait(&full[s], (uint32_t)((gc / kOcStages) & 1), abort_flag))) return false;
        body(ring + (size_t)s * (kOcStage / 4), k0, min(rpc, rows - k0));
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty[s])) : "memory");
    }
    return true;
}

// x = embed[tok], xn = LN_a(x) of the first block (warp_embed_ln's
// arithmetic) into a slot's shared-memory rows.
template <int VPT>
__device__ __forceinline__ void oc_embed(const OcModel& M, int tok, float* x, float* xn, int lane) {
    constexpr int d = VPT * 32;
    float v[VPT], y[VPT];
#pragma unroll
    for (int i = 0; i < VPT; i++) v[i] = M.embed[(size_t)tok * d + lane + 32 * i];
    warp_layernorm<VPT>(v, M.L[0].ln_a_w, M.L[0].ln_a_b, lane, y);
#pragma unroll
    for (int i = 0; i < VPT; i++) {
        x[lane + 32 * i] = v[i];
        xn[lane + 32 * i] = y[i];
    }
}

// A slot takes the next stream of the queue (one warp): raw first byte to
// the output, coder from the next 4 coded bytes, the first step's input
// rows.  Returns the stream, -1 once the queue is empty.
template <int VPT>
__device__ __forceinline__ int oc_take(const OcModel& M, const OcWork& W, CoderState& cs, float* x, float* xn,
                                       int lane) {
    int take = 0;
    if (lane == 0) take = atomicAdd(W.next, 1);
    take = __shfl_sync(0xffffffffu, take, 0);
    if (take >= W.n) return -1;
    const int stream = W.order[take];
    const uint64_t size = W.tb.in_size[stream];               // >= 1 (checked on the host)
    const uint8_t first = W.cin[W.tb.in_off[stream]];
    if (lane == 0) {
        rc_decoder_init(cs, W.cin + W.tb.in_off[stream] + 1, size - 1);
        W.out[W.tb.out_off[stream]] = first;
    }
    oc_embed<VPT>(M, first, x, xn, lane);
    return stream;
}

template <int VPT, int R>
__global__ void __launch_bounds__(kOcBlock, 1) k_decode_onchip(const OcModel M, const OcWork W) {
    constexpr int d = VPT * 32;
    constexpr int P = kOcSlots;
    constexpr int S = kOcStages;
    constexpr int R2 = R + 2 * kOcNS;
    static_assert(R2 % 4 == 0 && R2 <= 48, "[delta|B|C] rows are read as float4");
    extern __shared__ __align__(128) uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[S];
    __shared__ __align__(8) uint64_t empty[S];
    __shared__ CoderState cs[P];
    __shared__ long long spos[P];
    __shared__ int sstream[P], fresh[P];
    __shared__ int stop_flag, abort_flag;
    __shared__ uint32_t tmem_slot;

    float* ring = reinterpret_cast<float*>(smem_raw);
    float* act = ring + (size_t)S * (kOcStage / 4);
    const int E = M.E, nl = M.nl;
    const int APS = oc_act_floats(d, E);
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    volatile int* vabort = &abort_flag;
    volatile int* vstop = &stop_flag;

    if (tid == 0) {
        for (int i = 0; i < S; i++) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], kOcThreads / 32);
        }
        stop_flag = 0;
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&tmem_slot)), "r"(512u));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    pdl_wait_prev();

    if (warp == kOcThreads / 32) {
        // ---- weight stream: every matrix of a step, step after step, until
        // the compute warps stop (or give up)
        if (lane == 0) {
            int g = 0;
            bool stopped = false;
            const int n_mats = 3 * nl + 1;
            while (!stopped) {
                for (int i = 0; i < n_mats && !stopped; i++) {
                    const float* Wm;
                    int rows, cols;
                    oc_matrix<VPT, R>(M, i, Wm, rows, cols);
                    const int rpc = oc_rpc(rows, cols);
                    for (int k0 = 0; k0 < rows; k0 += rpc, g++) {
                        const int s = g % S;
                        if (g >= S) {
                            const uint32_t par = (uint32_t)(((g / S) - 1) & 1);
                            const uint64_t t0 = globaltimer();
                            while (!mbar_try(&empty[s], par)) {
                                if (*vstop || *vabort) { stopped = true; break; }
                                if (globaltimer() - t0 > kWaitNs) { *vabort = 1; stopped = true; break; }
                            }
                            if (stopped) break;
                        }
                        const int nr = min(rpc, rows - k0);
                        const uint32_t bytes = (uint32_t)(nr * cols * 4);
                        mbar_expect_tx(&full[s], bytes);
                        bulk_g2s(ring + (size_t)s * (kOcStage / 4), Wm + (size_t)k0 * cols, bytes, &full[s]);
                    }
                }
            }
            // the copies no compute warp will wait for land before the CTA
            // leaves: the last issue of every stage
            for (int j = g - 1; j >= 0 && j >= g - S; j--) mbar_wait(&full[j % S], (uint32_t)((j / S) & 1));
        }
    } else {
        // ---- compute warps
        const uint32_t trow = tmem + ((uint32_t)(32 * (warp % 4)) << 16) + (uint32_t)(256 * (warp / 4));
        const int c0 = 2 * tid;                  // this thread's channels c0, c0 + 1
        const bool live = c0 < E;
        int gc = 0;
        bool ok = true;
        for (int i = tid; i < P * APS; i += kOcThreads) act[i] = 0.f;
        oc_sync();
        if (warp < P) {
            const int st = oc_take<VPT>(M, W, cs[warp], act + warp * APS, act + warp * APS + d, lane);
            if (lane == 0) {
                sstream[warp] = st;
                spos[warp] = 0;
                fresh[warp] = st >= 0;
            }
        }
        oc_sync();
        // activation rows of slot p: x at 0, xn d, xz 2d, u 2d + 2E,
        // [delta|B|C] 2d + 3E, gated scan output 2d + 3E + 48, logits 2d + 4E + 48
        const int oXZ = 2 * d, oU = 2 * d + 2 * E, oDBC = 2 * d + 3 * E, oYG = oDBC + 48, oLG = 2 * d + 4 * E + 48;
        while (true) {
            // a slot that took a new stream starts from zero state
#pragma unroll
            for (int p = 0; p < P; p++) {
                if (!fresh[p]) continue;
                const uint32_t z16[16] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
                const float z8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                for (int l = 0; l < nl; l++) {
                    const uint32_t sa = trow + (uint32_t)((p * kOcMaxLayers + l) * 2 * kOcNS);
                    tmem_st16(sa, z16);
                    tmem_st16(sa + kOcNS, z16);
                    tmem_st8(trow + (uint32_t)(kOcConvCol0 + (p * kOcMaxLayers + l) * 8), z8);
                }
            }
            tmem_wait_st();
            bool any = false;
#pragma unroll
            for (int p = 0; p < P; p++) any |= sstream[p] >= 0;
            oc_sync();
            if (tid == 0)
                for (int p = 0; p < P; p++) fresh[p] = 0;
            if (!any) break;

            for (int l = 0; l < nl; l++) {
                const OcLayer& L = M.L[l];
                // in_proj: xz = xn . W_in; this thread's columns 4 tid .. 4 tid + 3
                {
                    const int cols = 2 * E;
                    const bool on = 4 * tid < cols;
                    float acc[P][4];
#pragma unroll
                    for (int p = 0; p < P; p++) acc[p][0] = acc[p][1] = acc[p][2] = acc[p][3] = 0.f;
                    ok = oc_consume(d, cols, gc, full, empty, ring, vabort, lane, [&](const float* st, int k0, int nr) {
                        if (!on) return;
                        // four rows at a time: each slot's four inputs in one load
#pragma unroll 2
                        for (int r = 0; r < nr; r += 4) {
                            float4 xa[P], w[4];
#pragma unroll
                            for (int p = 0; p < P; p++)
                                xa[p] = *reinterpret_cast<const float4*>(act + p * APS + d + k0 + r);
#pragma unroll
                            for (int q = 0; q < 4; q++)
                                w[q] = *reinterpret_cast<const float4*>(st + (size_t)(r + q) * cols + 4 * tid);
#pragma unroll
                            for (int q = 0; q < 4; q++)
#pragma unroll
                                for (int p = 0; p < P; p++) {
                                    const float a = f4_at(xa[p], q);
                                    acc[p][0] = __fmaf_rn(a, w[q].x, acc[p][0]);
                                    acc[p][1] = __fmaf_rn(a, w[q].y, acc[p][1]);
                                    acc[p][2] = __fmaf_rn(a, w[q].z, acc[p][2]);
                                    acc[p][3] = __fmaf_rn(a, w[q].w, acc[p][3]);
                                }
                        }
                    });
                    if (on)
#pragma unroll
                        for (int p = 0; p < P; p++)
                            *reinterpret_cast<float4*>(act + p * APS + oXZ + 4 * tid) =
                                make_float4(acc[p][0], acc[p][1], acc[p][2], acc[p][3]);
                }
                if (oc_sync_or(!ok)) { ok = false; break; }

                // causal conv + SiLU over the window held in TMEM (k_conv_silu's arithmetic)
                {
                    const int Kc = M.K;
                    float wv[2][4], bc[2];
#pragma unroll
                    for (int j = 0; j < 2; j++) {
#pragma unroll
                        for (int k = 0; k < 4; k++) wv[j][k] = (live && k < Kc) ? L.conv_w[(size_t)k * E + c0 + j] : 0.f;
                        bc[j] = live ? L.conv_b[c0 + j] : 0.f;
                    }
#pragma unroll
                    for (int p = 0; p < P; p++) {
                        float win[8];
                        const uint32_t ca = trow + (uint32_t)(kOcConvCol0 + (p * kOcMaxLayers + l) * 8);
                        tmem_ld8(ca, win);
                        if (live) {
                            const float* xzp = act + p * APS + oXZ;
                            float* up = act + p * APS + oU;
#pragma unroll
                            for (int j = 0; j < 2; j++) {
                                float* h = win + 4 * j;
                                const float xi = xzp[c0 + j];
                                float acc = bc[j];
#pragma unroll
                                for (int k = 0; k < 3; k++)
                                    if (k < Kc - 1) acc = __fmaf_rn(wv[j][k], h[k], acc);
                                const float wl = Kc == 4 ? wv[j][3] : Kc == 3 ? wv[j][2] : wv[j][1];
                                acc = __fmaf_rn(wl, xi, acc);
                                up[c0 + j] = silu_f(acc);
#pragma unroll
                                for (int k = 0; k < 2; k++)
                                    if (k + 1 < Kc - 1) h[k] = h[k + 1];
#pragma unroll
                                for (int k = 0; k < 3; k++)
                                    if (k == Kc - 2) h[k] = xi;
                            }
                        }
                        tmem_st8(ca, win);
                    }
                    tmem_wait_st();
                }
                oc_sync();

                // x_proj: [delta|B|C] = u . W_x, one chain per (slot, column)
                {
                    const bool on = tid < R2 * P;
                    const int p = on ? tid / R2 : 0, n = on ? tid % R2 : 0;
                    const float* up = act + p * APS + oU;
                    float acc = 0.f;
                    ok = oc_consume(E, R2, gc, full, empty, ring, vabort, lane, [&](const float* st, int k0, int nr) {
                        if (!on) return;
#pragma unroll 4
                        for (int r = 0; r < nr; r += 4) {
                            const float4 ua = *reinterpret_cast<const float4*>(up + k0 + r);
                            float w[4];
#pragma unroll
                            for (int q = 0; q < 4; q++) w[q] = st[(size_t)(r + q) * R2 + n];
#pragma unroll
                            for (int q = 0; q < 4; q++) acc = __fmaf_rn(f4_at(ua, q), w[q], acc);
                        }
                    });
                    if (on) act[p * APS + oDBC + n] = acc;
                }
                if (oc_sync_or(!ok)) { ok = false; break; }

                // dt_proj + softplus + selective scan + gate (k_scan's arithmetic),
                // the SSM state in TMEM
                {
                    float a2[kOcNS][2], wdt[R][2];
                    float2 bdt = make_float2(0.f, 0.f), dv = make_float2(0.f, 0.f);
#pragma unroll
                    for (int n = 0; n < kOcNS; n++) {
                        const float2 v = live ? *reinterpret_cast<const float2*>(L.A2 + (size_t)n * E + c0)
                                              : make_float2(0.f, 0.f);
                        a2[n][0] = v.x;
                        a2[n][1] = v.y;
                    }
#pragma unroll
                    for (int k = 0; k < R; k++) {
                        const float2 v = live ? *reinterpret_cast<const float2*>(L.dt_w + (size_t)k * E + c0)
                                              : make_float2(0.f, 0.f);
                        wdt[k][0] = v.x;
                        wdt[k][1] = v.y;
                    }
                    if (live) {
                        bdt = *reinterpret_cast<const float2*>(L.dt_b + c0);
                        dv = *reinterpret_cast<const float2*>(L.D + c0);
                    }
#pragma unroll
                    for (int p = 0; p < P; p++) {
                        uint32_t hs[2][16];
                        const uint32_t sa = trow + (uint32_t)((p * kOcMaxLayers + l) * 2 * kOcNS);
                        tmem_ld16_nowait(sa, hs[0]);
                        tmem_ld16_nowait(sa + kOcNS, hs[1]);
                        tmem_wait_ld();
                        if (live) {
                            const float* base = act + p * APS;
                            const float* db = base + oDBC;
                            const float2 u2 = *reinterpret_cast<const float2*>(base + oU + c0);
                            const float2 z2 = *reinterpret_cast<const float2*>(base + oXZ + E + c0);
                            const float uu[2] = {u2.x, u2.y}, zz[2] = {z2.x, z2.y};
                            const float bb[2] = {bdt.x, bdt.y}, dd[2] = {dv.x, dv.y};
                            float o[2];
#pragma unroll
                            for (int j = 0; j < 2; j++) {
                                float pre = 0.f;
#pragma unroll
                                for (int k = 0; k < R; k++) pre = __fmaf_rn(wdt[k][j], db[k], pre);
                                const float delta = softplus_f(__fadd_rn(pre, bb[j]));
                                const float du = __fmul_rn(delta, uu[j]);
                                float y = 0.f;
#pragma unroll
                                for (int n = 0; n < kOcNS; n++) {
                                    const float da = ex2_approx(__fmul_rn(delta, a2[n][j]));
                                    const float h = __fmaf_rn(da, __uint_as_float(hs[j][n]), __fmul_rn(du, db[R + n]));
                                    hs[j][n] = __float_as_uint(h);
                                    y = __fmaf_rn(db[R + kOcNS + n], h, y);
                                }
                                y = __fmaf_rn(dd[j], uu[j], y);
                                o[j] = __fmul_rn(y, silu_f(zz[j]));
                            }
                            *reinterpret_cast<float2*>(act + p * APS + oYG + c0) = make_float2(o[0], o[1]);
                        }
                        tmem_st16(sa, hs[0]);
                        tmem_st16(sa + kOcNS, hs[1]);
                    }
                    tmem_wait_st();
                }
                oc_sync();

                // out_proj + residual: x = x + yg . W_out (k_gemm_fp32's kEpiResid)
                {
                    const bool on = tid < d;
                    float acc[P];
#pragma unroll
                    for (int p = 0; p < P; p++) acc[p] = 0.f;
                    ok = oc_consume(E, d, gc, full, empty, ring, vabort, lane, [&](const float* st, int k0, int nr) {
                        if (!on) return;
#pragma unroll 2
                        for (int r = 0; r < nr; r += 4) {
                            float4 ya[P];
                            float w[4];
#pragma unroll
                            for (int p = 0; p < P; p++)
                                ya[p] = *reinterpret_cast<const float4*>(act + p * APS + oYG + k0 + r);
#pragma unroll
                            for (int q = 0; q < 4; q++) w[q] = st[(size_t)(r + q) * d + tid];
#pragma unroll
                            for (int q = 0; q < 4; q++)
#pragma unroll
                                for (int p = 0; p < P; p++) acc[p] = __fmaf_rn(f4_at(ya[p], q), w[q], acc[p]);
                        }
                    });
                    if (on)
#pragma unroll
                        for (int p = 0; p < P; p++) act[p * APS + tid] = __fadd_rn(act[p * APS + tid], acc[p]);
                }
                if (oc_sync_or(!ok)) { ok = false; break; }

                // x = LN_b(x); xn = LN_a'(x) when a block follows (k_ln_ln)
                if (warp < P) {
                    float* xp = act + warp * APS;
                    float v[VPT], y[VPT];
#pragma unroll
                    for (int i = 0; i < VPT; i++) v[i] = xp[lane + 32 * i];
                    warp_layernorm<VPT>(v, L.ln_b_w, L.ln_b_b, lane, y);
#pragma unroll
                    for (int i = 0; i < VPT; i++) xp[lane + 32 * i] = y[i];
                    if (l + 1 < nl) {
                        float z[VPT];
                        warp_layernorm<VPT>(y, M.L[l + 1].ln_a_w, M.L[l + 1].ln_a_b, lane, z);
#pragma unroll
                        for (int i = 0; i < VPT; i++) xp[d + lane + 32 * i] = z[i];
                    }
                }
                oc_sync();
            }
            if (!ok) break;

            // head: logits = x . W_head + b (column tid)
            {
                float acc[P];
#pragma unroll
                for (int p = 0; p < P; p++) acc[p] = 0.f;
                ok = oc_consume(d, 256, gc, full, empty, ring, vabort, lane, [&](const float* st, int k0, int nr) {
#pragma unroll 2
                    for (int r = 0; r < nr; r += 4) {
                        float4 xa[P];
                        float w[4];
#pragma unroll
                        for (int p = 0; p < P; p++) xa[p] = *reinterpret_cast<const float4*>(act + p * APS + k0 + r);
#pragma unroll
                        for (int q = 0; q < 4; q++) w[q] = st[(size_t)(r + q) * 256 + tid];
#pragma unroll
                        for (int q = 0; q < 4; q++)
#pragma unroll
                            for (int p = 0; p < P; p++) acc[p] = __fmaf_rn(f4_at(xa[p], q), w[q], acc[p]);
                    }
                });
                const float hb = M.head_b[tid];
#pragma unroll
                for (int p = 0; p < P; p++) act[p * APS + oLG + tid] = __fadd_rn(acc[p], hb);
            }
            if (oc_sync_or(!ok)) { ok = false; break; }

            // softmax -> histogram -> decode byte t + 1 (k_decode), one warp per slot
            if (warp < P && sstream[warp] >= 0) {
                const int p = warp;
                const int stream = sstream[p];
                const long long t = spos[p];
                float* xp = act + p * APS;
                uint32_t f[8], cbase;
                warp_logits_to_hist(xp + oLG, lane, f, cbase);
                if (W.tb.trace) {
                    const uint64_t hsh = warp_hist_hash(f, lane);
                    if (lane == 0) W.tb.trace[W.tb.trace_off[stream] + t] = hsh;
                }
                const uint8_t* in = W.cin + W.tb.in_off[stream] + 1;
                const uint64_t size = W.tb.in_size[stream] - 1;
                uint32_t x = 0;
                if (lane == 0) x = rc_target(cs[p]);
                x = __shfl_sync(0xffffffffu, x, 0);
                int sym;
                uint32_t c_lo, freq;
                warp_find_symbol(f, cbase, x, lane, sym, c_lo, freq);
                if (lane == 0) {
                    rc_decode_update(cs[p], c_lo, freq, in, size);
                    W.out[W.tb.out_off[stream] + t + 1] = (uint8_t)sym;
                }
                if (t + 2 < (long long)W.tb.lens[stream]) {
                    oc_embed<VPT>(M, sym, xp, xp + d, lane);
                    if (lane == 0) spos[p] = t + 1;
                } else {
                    if (lane == 0)
                        W.tb.flags[stream] = cs[p].flags | (cs[p].pos != size ? (uint32_t)kFlagCorrupt : 0u);
                    __syncwarp();
                    const int ns = oc_take<VPT>(M, W, cs[p], xp, xp + d, lane);
                    if (lane == 0) {
                        sstream[p] = ns;
                        spos[p] = 0;
                        fresh[p] = ns >= 0;
                    }
                }
            }
            oc_sync();
        }
        if (tid == 0) {
            if (!ok) {
                atomicExch(W.err, 4);
                *vabort = 1;
            }
            __threadfence_block();
            *vstop = 1;
        }
    }

    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u));
}

}  // namespace boa
