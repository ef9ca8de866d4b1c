// Per-row and per-stream kernels of the BOA hot path (everything but the GEMMs).
//
// Row layout: a batch of rows is S streams x Tc consecutive steps, row index
// s * Tc + tau.  Compression runs Tc > 1 (teacher forcing over a time
// chunk); decompression runs Tc = 1 (one step of every stream).  Kernels that
// carry state along time (conv window, SSM state, coder) loop over tau inside
// one thread or warp, so results never depend on Tc.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "common.cuh"

namespace boa {

// ---------------------------------------------------------------- LayerNorm

// (x - mean) / sqrt(var + 1e-5) * g + b over d features, one warp per row,
// fixed butterfly reductions (identical in every lane and every launch).
template <int VPT>
__device__ __forceinline__ void warp_layernorm(const float (&x)[VPT], const float* __restrict__ g,
                                               const float* __restrict__ b, int lane, float (&y)[VPT]) {
    constexpr int d = VPT * 32;
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < VPT; i++) s = __fadd_rn(s, x[i]);
    const float mean = __fdiv_rn(warp_sum(s), (float)d);
    float v = 0.f;
#pragma unroll
    for (int i = 0; i < VPT; i++) {
        float c = __fsub_rn(x[i], mean);
        v = __fmaf_rn(c, c, v);
    }
    const float var = __fdiv_rn(warp_sum(v), (float)d);
    const float inv = __fdiv_rn(1.0f, __fsqrt_rn(__fadd_rn(var, 1e-5f)));
#pragma unroll
    for (int i = 0; i < VPT; i++) {
        int k = lane + 32 * i;
        y[i] = __fadd_rn(__fmul_rn(__fmul_rn(__fsub_rn(x[i], mean), inv), g[k]), b[k]);
    }
}

// ------------------------------------------------------ FP8 activation rows
//
// The E4M3 projections' A operand: per row, scale = amax / 448 and
// q[k] = e4m3(a[k] * (448 / amax)), rounded to nearest and saturated, with
// amax = max_k |a[k]| (scale 1 for an all-zero row); rows of Kp >= K bytes
// (the consumer GEMM's K rounded up to its 128-wide K blocks), the padding
// zero.  k_quant_rows_e4m3 writes it from any FP32 matrix; a kernel that
// holds whole rows (LayerNorm, conv + SiLU, the decode-step scan) writes it
// itself through the same functions.  The maximum does not depend on the
// order it is taken in, so both give the same bytes and scales.
struct F8Out {
    __nv_fp8_e4m3* q;     // [rows][Kp]; nullptr: no FP8 copy
    float* scale;         // [rows]
    int Kp;
};

__device__ __forceinline__ float e4m3_row_inv(float amax) { return amax > 0.f ? __fdiv_rn(448.0f, amax) : 1.0f; }
__device__ __forceinline__ float e4m3_row_scale(float amax) { return amax > 0.f ? __fdiv_rn(amax, 448.0f) : 1.0f; }
__device__ __forceinline__ __nv_fp8_e4m3 e4m3_of(float v, float inv) { return __nv_fp8_e4m3(__fmul_rn(v, inv)); }

// One warp's row of d = 32 VPT values, lane holding columns lane + 32 i.
template <int VPT>
__device__ __forceinline__ void warp_write_f8(const F8Out& f8, size_t row, const float (&y)[VPT], int lane) {
    constexpr int d = VPT * 32;
    float amax = 0.f;
#pragma unroll
    for (int i = 0; i < VPT; i++) amax = fmaxf(amax, fabsf(y[i]));
    amax = warp_max(amax);
    const float inv = e4m3_row_inv(amax);
    if (lane == 0) f8.scale[row] = e4m3_row_scale(amax);
    __nv_fp8_e4m3* o = f8.q + row * (size_t)f8.Kp;
#pragma unroll
    for (int i = 0; i < VPT; i++) o[lane + 32 * i] = e4m3_of(y[i], inv);
    for (int k = d + lane; k < f8.Kp; k += 32) o[k] = __nv_fp8_e4m3(0.0f);
}

// Streams run in a fixed pool of slots (row block s of every launch belongs
// to slot s).  A slot works through its own list of streams, one after the
// other; t is the position in the current stream: the first step of the
// current chunk when compressing, the step being decoded when decompressing.
struct SlotState {
    int idx;        // index into the schedule (the slot's current list entry)
    int stream;     // current stream, -1 once the slot's list is exhausted
    long long t;
};

// Token source for a compression row (slot s, step tau of the chunk).
struct TokenSrc {
    const uint8_t* data;        // packed stream bytes
    const uint64_t* offsets;    // [n+1]
    const uint64_t* lens;       // [n]
    const SlotState* slots;     // [S]
};

__device__ __forceinline__ int row_token(const TokenSrc& ts, int s, int tau) {
    const SlotState ss = ts.slots[s];
    if (ss.stream < 0) return 0;
    const long long t = ss.t + tau;
    return (t + 1 < (long long)ts.lens[ss.stream]) ? ts.data[ts.offsets[ss.stream] + t] : 0;
}

// x = embed[token]; xn = LN_a(x)   (Alg. 1: ByteEmbed, then the first block's norm)
template <int VPT>
__global__ void k_embed_ln(TokenSrc ts, int S, int Tc, const float* __restrict__ embed,
                           const float* __restrict__ g, const float* __restrict__ b,
                           float* __restrict__ x, float* __restrict__ xn, __nv_bfloat16* __restrict__ xn_b,
                           F8Out f8) {
    pdl_launch_next();
    pdl_wait_prev();
    constexpr int d = VPT * 32;
    const int lane = threadIdx.x & 31;
    const long long row = (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    if (row >= (long long)S * Tc) return;
    const int s = (int)(row / Tc), tau = (int)(row % Tc);
    const int tok = row_token(ts, s, tau);
    float v[VPT], y[VPT];
#pragma unroll
    for (int i = 0; i < VPT; i++) v[i] = embed[(size_t)tok * d + lane + 32 * i];
    warp_layernorm<VPT>(v, g, b, lane, y);
#pragma unroll
    for (int i = 0; i < VPT; i++) {
        x[(size_t)row * d + lane + 32 * i] = v[i];
        if (xn_b) xn_b[(size_t)row * d + lane + 32 * i] = __float2bfloat16_rn(y[i]);
        else if (!f8.q) xn[(size_t)row * d + lane + 32 * i] = y[i];
    }
    if (f8.q) warp_write_f8<VPT>(f8, (size_t)row, y, lane);
}

// x = LN_b(x); then, when another block follows, xn = LN_a'(x).
// Optional BF16 copies for the tensor-core path: x_b (input of the head or the
// FFN) and xn_b (input of the next in_proj, replacing xn).
// f8: the FP8 copy of the next projection's input: xn when another block
// follows (its in_proj), else x (the head).
template <int VPT>
__global__ void k_ln_ln(long long rows, float* __restrict__ x, const float* __restrict__ gb,
                        const float* __restrict__ bb, const float* __restrict__ ga,
                        const float* __restrict__ ba, float* __restrict__ xn,
                        __nv_bfloat16* __restrict__ x_b, __nv_bfloat16* __restrict__ xn_b, F8Out f8) {
    pdl_launch_next();
    pdl_wait_prev();
    constexpr int d = VPT * 32;
    const int lane = threadIdx.x & 31;
    const long long row = (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    if (row >= rows) return;
    float v[VPT], y[VPT];
#pragma unroll
    for (int i = 0; i < VPT; i++) v[i] = x[(size_t)row * d + lane + 32 * i];
    warp_layernorm<VPT>(v, gb, bb, lane, y);
#pragma unroll
    for (int i = 0; i < VPT; i++) {
        x[(size_t)row * d + lane + 32 * i] = y[i];
        if (x_b) x_b[(size_t)row * d + lane + 32 * i] = __float2bfloat16_rn(y[i]);
    }
    if (ga) {
        float z[VPT];
        warp_layernorm<VPT>(y, ga, ba, lane, z);
#pragma unroll
        for (int i = 0; i < VPT; i++) {
            if (xn_b) xn_b[(size_t)row * d + lane + 32 * i] = __float2bfloat16_rn(z[i]);
            else if (!f8.q) xn[(size_t)row * d + lane + 32 * i] = z[i];
        }
        if (f8.q) warp_write_f8<VPT>(f8, (size_t)row, z, lane);
    } else if (f8.q) {
        warp_write_f8<VPT>(f8, (size_t)row, y, lane);
    }
}

// ---------------------------------------------------- causal conv1d + SiLU

// The per-channel conv + SiLU of k_conv_silu (same operations in the same
// order) for one stream per CTA that covers the whole row (the FP8 form):
// after each row the CTA takes the row's maximum and writes its E4M3 copy
// (f8) besides u.  Threads past the row's end take part in the barriers.
template <int K>
__device__ __forceinline__ void conv_silu_rows_f8(const float* __restrict__ xz, int E, const float* __restrict__ wt,
                                                  const float* __restrict__ bconv, float* __restrict__ win,
                                                  const SlotState* __restrict__ slots, float* __restrict__ u, int S,
                                                  int Tc, const F8Out& f8, int c) {
    __shared__ float red[2][4];
    const int s = blockIdx.y;
    const bool live = c < E && s < S;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    float4 wv[K], bc = make_float4(0.f, 0.f, 0.f, 0.f), h[K];
    long long t0 = 0;
    float* ring = nullptr;
    if (live) {
#pragma unroll
        for (int k = 0; k < K; k++) wv[k] = *reinterpret_cast<const float4*>(wt + (size_t)k * E + c);
        bc = *reinterpret_cast<const float4*>(bconv + c);
        t0 = slots[s].t;
        ring = win + (size_t)s * (K - 1) * E + c;
#pragma unroll
        for (int k = 0; k < K - 1; k++) h[k] = *reinterpret_cast<const float4*>(ring + (size_t)((t0 + k) % (K - 1)) * E);
    }
    size_t row = (size_t)s * Tc;
    for (int tau = 0; tau < Tc; tau++, row++) {
        float o[4] = {0.f, 0.f, 0.f, 0.f};
        if (live) {
            const float4 xi = *reinterpret_cast<const float4*>(xz + row * 2 * E + c);
#pragma unroll
            for (int j = 0; j < 4; j++) {
                float acc = reinterpret_cast<const float*>(&bc)[j];
#pragma unroll
                for (int k = 0; k < K - 1; k++)
                    acc = __fmaf_rn(reinterpret_cast<const float*>(&wv[k])[j], reinterpret_cast<const float*>(&h[k])[j], acc);
                acc = __fmaf_rn(reinterpret_cast<const float*>(&wv[K - 1])[j], reinterpret_cast<const float*>(&xi)[j], acc);
                o[j] = silu_f(acc);
            }
#pragma unroll
            for (int k = 0; k + 1 < K - 1; k++) h[k] = h[k + 1];
            h[K - 2] = xi;
            *reinterpret_cast<float4*>(u + row * E + c) = make_float4(o[0], o[1], o[2], o[3]);
        }
        float a = fmaxf(fmaxf(fabsf(o[0]), fabsf(o[1])), fmaxf(fabsf(o[2]), fabsf(o[3])));
        a = warp_max(a);
        if (lane == 0) red[tau & 1][warp] = a;
        __syncthreads();
        const float amax = fmaxf(fmaxf(red[tau & 1][0], red[tau & 1][1]), fmaxf(red[tau & 1][2], red[tau & 1][3]));
        if (live) {
            const float inv = e4m3_row_inv(amax);
            if (c == 0) f8.scale[row] = e4m3_row_scale(amax);
            __nv_fp8_e4m3* q = f8.q + row * (size_t)f8.Kp + c;
#pragma unroll
            for (int j = 0; j < 4; j++) q[j] = e4m3_of(o[j], inv);
        }
    }
    if (live) {
        const long long t1 = t0 + Tc;
#pragma unroll
        for (int k = 0; k < K - 1; k++) {
            const long long pos = t1 - (K - 1) + k;
            if (pos >= t0) *reinterpret_cast<float4*>(ring + (size_t)(pos % (K - 1)) * E) = h[k];
        }
    }
}

// u[s, t, c] = SiLU(b_c + sum_k w[c][k] xi[s, t-K+1+k, c]); the last K-1
// inputs of every (stream, channel) persist in win[S][K-1][E] across calls
// as a ring: the input of stream position t sits in row t mod (K-1), so a
// decode step rewrites one row (its own input over the oldest) instead of
// shifting all K-1.  slots[s].t is the position of the slot's first row in
// this call.  wt is the tap matrix stored [K][E] (channel innermost).  A
// thread owns four adjacent channels (16-byte loads and stores) of G
// consecutive streams.
// f8 (FP8 form, one CTA per row: E <= 4 x 128): the row's E4M3 copy for
// x_proj, its scale from a CTA-wide maximum per row.
template <int K, int G>
__global__ void __launch_bounds__(128)
k_conv_silu(const float* __restrict__ xz, int E, const float* __restrict__ wt,
            const float* __restrict__ bconv, float* __restrict__ win, const SlotState* __restrict__ slots,
            float* __restrict__ u, __nv_bfloat16* __restrict__ u_b, int S, int Tc, F8Out f8) {
    pdl_launch_next();
    pdl_wait_prev();
    const int c = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (f8.q) {
        conv_silu_rows_f8<K>(xz, E, wt, bconv, win, slots, u, S, Tc, f8, c);
        return;
    }
    if (c >= E) return;
    float4 wv[K];
#pragma unroll
    for (int k = 0; k < K; k++) wv[k] = *reinterpret_cast<const float4*>(wt + (size_t)k * E + c);
    const float4 bc = *reinterpret_cast<const float4*>(bconv + c);
    for (int g = 0; g < G; g++) {
        const int s = blockIdx.y * G + g;
        if (s >= S) break;
        const long long t0 = slots[s].t;
        float* ring = win + (size_t)s * (K - 1) * E + c;
        float4 h[K];                             // oldest first: positions t0 - K + 1 .. t0 - 1
#pragma unroll
        for (int k = 0; k < K - 1; k++) h[k] = *reinterpret_cast<const float4*>(ring + (size_t)((t0 + k) % (K - 1)) * E);
        size_t row = (size_t)s * Tc;
        float4 xi = *reinterpret_cast<const float4*>(xz + row * 2 * E + c);
        for (int tau = 0; tau < Tc; tau++, row++) {
            float4 xnext = make_float4(0.f, 0.f, 0.f, 0.f);
            if (tau + 1 < Tc) xnext = *reinterpret_cast<const float4*>(xz + (row + 1) * 2 * E + c);
            float o[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                float acc = reinterpret_cast<const float*>(&bc)[j];
#pragma unroll
                for (int k = 0; k < K - 1; k++)
                    acc = __fmaf_rn(reinterpret_cast<const float*>(&wv[k])[j], reinterpret_cast<const float*>(&h[k])[j], acc);
                acc = __fmaf_rn(reinterpret_cast<const float*>(&wv[K - 1])[j], reinterpret_cast<const float*>(&xi)[j], acc);
                o[j] = silu_f(acc);
            }
#pragma unroll
            for (int k = 0; k + 1 < K - 1; k++) h[k] = h[k + 1];
            h[K - 2] = xi;
            *reinterpret_cast<float4*>(u + row * E + c) = make_float4(o[0], o[1], o[2], o[3]);
            if (u_b) {
                __nv_bfloat162* bp = reinterpret_cast<__nv_bfloat162*>(u_b + row * E + c);
                bp[0] = __floats2bfloat162_rn(o[0], o[1]);
                bp[1] = __floats2bfloat162_rn(o[2], o[3]);
            }
            xi = xnext;
        }
        // the inputs of this call's rows that are still in the window
        const long long t1 = t0 + Tc;
#pragma unroll
        for (int k = 0; k < K - 1; k++) {
            const long long pos = t1 - (K - 1) + k;
            if (pos >= t0) *reinterpret_cast<float4*>(ring + (size_t)(pos % (K - 1)) * E) = h[k];
        }
    }
}

// --------------------------------------- dt_proj + softplus + selective scan

// One thread per (stream, channel) walks the chunk's steps (App. A):
//   Delta = softplus(W_dt . delta + b_dt)
//   h[n]  = exp(Delta A[n]) h[n] + (Delta u) B[n]
//   y     = sum_n C[n] h[n] + D u ;   out = y * SiLU(z)
// h lives in registers for the chunk and in hstate[S][N][E] between chunks.
// A2t = (A * log2 e) stored [N][E] and dtwt = W_dt stored [R][E] (channel
// innermost, so the per-channel loads coalesce); exp(Delta A) = 2^(Delta A2).
// A CTA covers 128 channels of G consecutive streams and loads the weights
// once (before waiting for the previous kernel: they are not its outputs).
// Six CTAs per SM (80 registers).
//
// Chunks of more than one step (compression) stage the rows a CTA visits
// (stream-major) through shared memory in batches of kScanRB rows: the
// batch's u and z values of the CTA's channels and its [delta|B|C] rows,
// double buffered with cp.async, so the next batch is in flight while the
// current one is computed.  The per-channel arithmetic is the same sequence
// of operations in every path (and in the decode-step kernels).
constexpr int kScanThreads = 128;
constexpr int kScanRowsSmem = 32;          // single-step path: up to 32 streams' [delta|B|C] rows
constexpr int kScanRB = 8;                 // chunked path: rows per staged batch

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int NS, int R, int G>
__global__ void __launch_bounds__(kScanThreads, 6)
k_scan(const float* __restrict__ u, const float* __restrict__ xz, const float* __restrict__ dbc,
       const float* __restrict__ dtwt, const float* __restrict__ dt_b, const float* __restrict__ A2t,
       const float* __restrict__ Dv, float* __restrict__ hstate, float* __restrict__ yg,
       __nv_bfloat16* __restrict__ yg_b, int E, int S, int Tc) {
    constexpr int W = R + 2 * NS;   // dbc row width
    static_assert(R % 4 == 0 && NS % 4 == 0, "rows are read as float4");
    // staging: [2][kScanRB][128] u, the same for z, [2][kScanRB][W] dbc
    // (chunked path); [kScanRowsSmem][W] dbc (single-step path)
    constexpr int kStageF = 2 * kScanRB * (2 * kScanThreads + W);
    constexpr int kSmemF = kStageF > kScanRowsSmem * W ? kStageF : kScanRowsSmem * W;
    __shared__ __align__(16) float sbuf[kSmemF];
    const int tid = threadIdx.x;
    const int c0 = blockIdx.x * blockDim.x;
    const int c = c0 + tid;
    const int s_first = blockIdx.y * G;
    const bool live = c < E;
    float a2[NS], wdt[R];
    float bdt = 0.f, dv = 0.f;
    if (live) {
#pragma unroll
        for (int n = 0; n < NS; n++) a2[n] = A2t[(size_t)n * E + c];
#pragma unroll
        for (int j = 0; j < R; j++) wdt[j] = dtwt[(size_t)j * E + c];
        bdt = dt_b[c];
        dv = Dv[c];
    }
    pdl_launch_next();
    pdl_wait_prev();                             // u, z, dbc and the state come from earlier kernels
    const int n_streams = min(G, S - s_first);
    const int total = n_streams * Tc;       // rows this CTA visits, stream-major
    const size_t row0 = (size_t)s_first * Tc;
    float h[NS];
    if (Tc == 1) {
        // One step per stream (decompression): the next stream's state is
        // fetched before the current one is computed, so state loads stay in
        // flight during the arithmetic.
        float (*sm)[W] = reinterpret_cast<float (*)[W]>(sbuf);
        for (int i = tid; i < total * W; i += blockDim.x) sm[i / W][i % W] = dbc[(row0 + i / W) * W + i % W];
        __syncthreads();
        if (!live) return;
        float hn[NS];
#pragma unroll
        for (int n = 0; n < NS; n++) hn[n] = hstate[((size_t)s_first * NS + n) * E + c];
        for (int rr = 0; rr < total; rr++) {
            const int s = s_first + rr;
            const size_t row = row0 + rr;
#pragma unroll
            for (int n = 0; n < NS; n++) h[n] = hn[n];
            if (rr + 1 < total) {
#pragma unroll
                for (int n = 0; n < NS; n++) hn[n] = hstate[((size_t)(s + 1) * NS + n) * E + c];
            }
            const float uc = u[row * E + c];
            const float z = xz[row * 2 * E + E + c];
            float pre = 0.f;
#pragma unroll
            for (int j = 0; j < R; j++) pre = __fmaf_rn(wdt[j], sm[rr][j], pre);
            const float delta = softplus_f(__fadd_rn(pre, bdt));
            const float du = __fmul_rn(delta, uc);
            float y = 0.f;
#pragma unroll
            for (int n = 0; n < NS; n++) {
                const float da = ex2_approx(__fmul_rn(delta, a2[n]));
                h[n] = __fmaf_rn(da, h[n], __fmul_rn(du, sm[rr][R + n]));
                y = __fmaf_rn(sm[rr][R + NS + n], h[n], y);
            }
            y = __fmaf_rn(dv, uc, y);
            const float o = __fmul_rn(y, silu_f(z));
            if (yg_b) yg_b[row * E + c] = __float2bfloat16_rn(o);
            else yg[row * E + c] = o;
#pragma unroll
            for (int n = 0; n < NS; n++) hstate[((size_t)s * NS + n) * E + c] = h[n];
        }
        return;
    }
    // chunked path: every thread takes part in the copies (the 128 channels
    // of a CTA are 512 contiguous bytes of a row: 32 16-byte pieces)
    float* su = sbuf;                                    // [2][kScanRB][128]
    float* sz = su + 2 * kScanRB * kScanThreads;         // [2][kScanRB][128]
    float* sd = sz + 2 * kScanRB * kScanThreads;         // [2][kScanRB][W]
    const int n_batches = (total + kScanRB - 1) / kScanRB;
    const int cw = E - c0 < kScanThreads ? E - c0 : kScanThreads;   // channels of this CTA (multiple of 4)
    auto issue = [&](int b) {
        const int r_beg = b * kScanRB;
        const int nr = min(kScanRB, total - r_beg);
        const int buf = b & 1;
        for (int i = tid; i < nr * 32; i += kScanThreads) {
            const int rr = i / 32, q = 4 * (i % 32);
            if (q < cw) {
                const size_t row = row0 + r_beg + rr;
                cp_async16(su + (buf * kScanRB + rr) * kScanThreads + q, u + row * E + c0 + q);
                cp_async16(sz + (buf * kScanRB + rr) * kScanThreads + q, xz + row * 2 * E + E + c0 + q);
            }
        }
        for (int i = tid; i < nr * (W / 4); i += kScanThreads) {
            const int rr = i / (W / 4), q = 4 * (i % (W / 4));
            cp_async16(sd + (buf * kScanRB + rr) * W + q, dbc + (row0 + r_beg + rr) * W + q);
        }
        cp_async_commit();
    };
    issue(0);
    int tau = 0, s = s_first;                            // step within the stream, stream of the current row
    for (int b = 0; b < n_batches; b++) {
        if (b + 1 < n_batches) {
            issue(b + 1);
            cp_async_wait<1>();                          // this thread's copies of batch b have landed
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();                                 // ... and every thread's
        const int buf = b & 1;
        const int nr = min(kScanRB, total - b * kScanRB);
        if (live) {
            for (int rr = 0; rr < nr; rr++) {
                const size_t row = row0 + (size_t)b * kScanRB + rr;
                if (tau == 0) {
#pragma unroll
                    for (int n = 0; n < NS; n++) h[n] = hstate[((size_t)s * NS + n) * E + c];
                }
                const float* d = sd + (buf * kScanRB + rr) * W;
                const float uc = su[(buf * kScanRB + rr) * kScanThreads + tid];
                const float z = sz[(buf * kScanRB + rr) * kScanThreads + tid];
                float pre = 0.f;
#pragma unroll
                for (int j = 0; j < R; j++) pre = __fmaf_rn(wdt[j], d[j], pre);
                const float delta = softplus_f(__fadd_rn(pre, bdt));
                const float du = __fmul_rn(delta, uc);
                float y = 0.f;
#pragma unroll
                for (int n = 0; n < NS; n++) {
                    const float da = ex2_approx(__fmul_rn(delta, a2[n]));
                    h[n] = __fmaf_rn(da, h[n], __fmul_rn(du, d[R + n]));
                    y = __fmaf_rn(d[R + NS + n], h[n], y);
                }
                y = __fmaf_rn(dv, uc, y);
                const float o = __fmul_rn(y, silu_f(z));
                if (yg_b) yg_b[row * E + c] = __float2bfloat16_rn(o);
                else yg[row * E + c] = o;
                if (tau == Tc - 1) {
#pragma unroll
                    for (int n = 0; n < NS; n++) hstate[((size_t)s * NS + n) * E + c] = h[n];
                    tau = 0;
                    s++;
                } else {
                    tau++;
                }
            }
        }
        __syncthreads();                                 // batch b's buffer is free for batch b + 2
    }
}

// One decode step of the scan with four adjacent channels per thread (one
// stream per CTA): every SSM-state access is a 16-byte load or store, all 16
// state loads are issued before the arithmetic, and the per-channel weights
// (A2t [N][E], dtwt [R][E]) come through L1.  Per channel it performs exactly
// the operations of k_scan, in the same order.
template <int NS, int R>
__global__ void __launch_bounds__(kScanThreads)
k_scan_step4(const float* __restrict__ u, const float* __restrict__ xz, const float* __restrict__ dbc,
             const float* __restrict__ dtwt, const float* __restrict__ dt_b, const float* __restrict__ A2t,
             const float* __restrict__ Dv, float* __restrict__ hstate, float* __restrict__ yg,
             __nv_bfloat16* __restrict__ yg_b, int E) {
    pdl_launch_next();
    pdl_wait_prev();
    constexpr int W = R + 2 * NS;
    __shared__ float sm[W];
    const int s = blockIdx.y;
    const int c = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    for (int i = threadIdx.x; i < W; i += blockDim.x) sm[i] = dbc[(size_t)s * W + i];
    __syncthreads();
    if (c >= E) return;
    float4 h[NS];
#pragma unroll
    for (int n = 0; n < NS; n++) h[n] = *reinterpret_cast<const float4*>(hstate + ((size_t)s * NS + n) * E + c);
    const float4 u4 = *reinterpret_cast<const float4*>(u + (size_t)s * E + c);
    const float4 z4 = *reinterpret_cast<const float4*>(xz + (size_t)s * 2 * E + E + c);
    const float4 b4 = *reinterpret_cast<const float4*>(dt_b + c);
    const float4 d4 = *reinterpret_cast<const float4*>(Dv + c);
    float pre[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int j = 0; j < R; j++) {
        const float4 w = *reinterpret_cast<const float4*>(dtwt + (size_t)j * E + c);
        pre[0] = __fmaf_rn(w.x, sm[j], pre[0]);
        pre[1] = __fmaf_rn(w.y, sm[j], pre[1]);
        pre[2] = __fmaf_rn(w.z, sm[j], pre[2]);
        pre[3] = __fmaf_rn(w.w, sm[j], pre[3]);
    }
    const float uv[4] = {u4.x, u4.y, u4.z, u4.w};
    const float bv[4] = {b4.x, b4.y, b4.z, b4.w};
    float delta[4], du[4], y[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
        delta[q] = softplus_f(__fadd_rn(pre[q], bv[q]));
        du[q] = __fmul_rn(delta[q], uv[q]);
        y[q] = 0.f;
    }
#pragma unroll
    for (int n = 0; n < NS; n++) {
        const float4 a = *reinterpret_cast<const float4*>(A2t + (size_t)n * E + c);
        const float av[4] = {a.x, a.y, a.z, a.w};
        float hv[4] = {h[n].x, h[n].y, h[n].z, h[n].w};
        const float Bn = sm[R + n], Cn = sm[R + NS + n];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const float da = ex2_approx(__fmul_rn(delta[q], av[q]));
            hv[q] = __fmaf_rn(da, hv[q], __fmul_rn(du[q], Bn));
            y[q] = __fmaf_rn(Cn, hv[q], y[q]);
        }
        h[n] = make_float4(hv[0], hv[1], hv[2], hv[3]);
    }
    const float dvv[4] = {d4.x, d4.y, d4.z, d4.w};
    const float zv[4] = {z4.x, z4.y, z4.z, z4.w};
    float o[4];
#pragma unroll
    for (int q = 0; q < 4; q++) o[q] = __fmul_rn(__fmaf_rn(dvv[q], uv[q], y[q]), silu_f(zv[q]));
    if (yg_b) {
        __nv_bfloat162* bp = reinterpret_cast<__nv_bfloat162*>(yg_b + (size_t)s * E + c);
        bp[0] = __floats2bfloat162_rn(o[0], o[1]);
        bp[1] = __floats2bfloat162_rn(o[2], o[3]);
    } else {
        *reinterpret_cast<float4*>(yg + (size_t)s * E + c) = make_float4(o[0], o[1], o[2], o[3]);
    }
#pragma unroll
    for (int n = 0; n < NS; n++) *reinterpret_cast<float4*>(hstate + ((size_t)s * NS + n) * E + c) = h[n];
}

// ------------------------------------ softmax -> integer histogram -> CDF

// Lane l owns symbols 8l .. 8l+7.  Result: f[8] (the lane's frequencies) and
// cbase = C(8l), the exclusive prefix of the histogram at the lane's first
// symbol.  Paper "Probabilities and integer CDF": f_a >= 1, sum f = 2^16.
__device__ __forceinline__ void warp_quantise_p(float (&p)[8], int lane, uint32_t (&f)[8], uint32_t& cbase) {
    float best = -1.0f;
    int best_idx = 0;
    uint32_t lsum = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        float q = p[j];
        if (!(q >= 0.0f)) q = 0.0f;     // NaN or negative -> 0
        if (q > 1.0f) q = 1.0f;
        p[j] = q;
        if (q > best) { best = q; best_idx = lane * 8 + j; }
        uint32_t fj = 1u + (uint32_t)floorf(__fmul_rn(q, (float)kQuantScale));
        f[j] = fj;
        lsum += fj;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float ob = __shfl_xor_sync(0xffffffffu, best, o);
        int oi = __shfl_xor_sync(0xffffffffu, best_idx, o);
        if (ob > best || (ob == best && oi < best_idx)) { best = ob; best_idx = oi; }
    }
    const uint32_t total = warp_sum_u32(lsum);
    const int rem = (int)kM - (int)total;            // signed remainder to the argmax
    uint32_t mine = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        if (best_idx == lane * 8 + j) f[j] = (uint32_t)((int)f[j] + rem);
        mine += f[j];
    }
    uint32_t incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    cbase = incl - mine;
}

// Softmax of one 256-logit row (paper, "Probabilities and integer CDF"),
// then the quantiser above.
__device__ __forceinline__ void warp_logits_to_hist(const float* __restrict__ lrow, int lane, uint32_t (&f)[8],
                                                    uint32_t& cbase) {
    const float4 v0 = reinterpret_cast<const float4*>(lrow)[lane * 2];
    const float4 v1 = reinterpret_cast<const float4*>(lrow)[lane * 2 + 1];
    float l[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
    float m = l[0];
#pragma unroll
    for (int j = 1; j < 8; j++) m = fmaxf(m, l[j]);
    m = warp_max(m);
    float e[8];
#pragma unroll
    for (int j = 0; j < 8; j++) e[j] = expf(__fsub_rn(l[j], m));
    float s = __fadd_rn(__fadd_rn(__fadd_rn(e[0], e[1]), __fadd_rn(e[2], e[3])),
                        __fadd_rn(__fadd_rn(e[4], e[5]), __fadd_rn(e[6], e[7])));
    s = warp_sum(s);
    float p[8];
#pragma unroll
    for (int j = 0; j < 8; j++) p[j] = __fdiv_rn(e[j], s);
    warp_quantise_p(p, lane, f, cbase);
}

// 64-bit hash of the 256 frequencies (test trace of the CDF each step used).
__device__ __forceinline__ uint64_t warp_hist_hash(const uint32_t (&f)[8], int lane) {
    uint64_t h = 1469598103934665603ull;
#pragma unroll
    for (int j = 0; j < 8; j++) { h ^= f[j]; h *= 1099511628211ull; }
    uint64_t w = 0x9E3779B97F4A7C15ull;
    uint64_t pw = 1;
    for (int i = 0; i <= lane; i++) pw *= w;
    return warp_sum_u64(h * pw);
}

// C(sym) and f(sym) for a symbol owned by lane sym/8, broadcast to all lanes.
__device__ __forceinline__ void warp_sym_range(const uint32_t (&f)[8], uint32_t cbase, int sym, int lane,
                                               uint32_t& c_lo, uint32_t& freq) {
    uint32_t cl = cbase, fr = 0;
    const int j0 = sym & 7;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        if (j < j0) cl += f[j];
        if (j == j0) fr = f[j];
    }
    c_lo = __shfl_sync(0xffffffffu, cl, sym >> 3);
    freq = __shfl_sync(0xffffffffu, fr, sym >> 3);
}

// ------------------------------------------------------------ range coder

// Encoder update and renormalisation (paper, paragraph "Encoder"), with the
// straddle rule for R < 2^16 and no modulo on R.
__device__ __forceinline__ void rc_encode(CoderState& st, uint32_t c_lo, uint32_t freq, uint8_t* out,
                                          uint64_t cap) {
    uint64_t L = st.L, R = st.R, pos = st.pos;
    L = L + ((R * c_lo) >> kProbBits);
    R = (R * freq) >> kProbBits;
    int it = 0;
    for (; it < 16; it++) {
        if ((L >> 24) == ((L + R - 1) >> 24)) {
            if (pos < cap) out[pos] = (uint8_t)(L >> 24); else st.flags |= kFlagOverflow;
            pos++;
            L = (L << 8) & kMask32;
            R = R << 8;
        } else if (R < kBot) {
            R = kBot - (L & (kBot - 1));
        } else {
            break;
        }
    }
    if (it == 16) st.flags |= kFlagLoop;
    st.L = L; st.R = R; st.pos = pos;
}

__device__ __forceinline__ void rc_flush(CoderState& st, uint8_t* out, uint64_t cap) {
    for (int i = 3; i >= 0; i--) {
        if (st.pos < cap) out[st.pos] = (uint8_t)(st.L >> (8 * i)); else st.flags |= kFlagOverflow;
        st.pos++;
    }
}

__device__ __forceinline__ uint8_t rc_read(CoderState& st, const uint8_t* in, uint64_t size) {
    uint8_t b = 0;
    if (st.pos < size) b = in[st.pos]; else st.flags |= kFlagCorrupt;
    st.pos++;
    return b;
}

__device__ __forceinline__ void rc_decoder_init(CoderState& st, const uint8_t* in, uint64_t size) {
    st.L = 0; st.R = 1ull << 32; st.C = 0; st.pos = 0; st.flags = 0;
    for (int i = 0; i < 4; i++) st.C = (st.C << 8) | rc_read(st, in, size);
}

// Decoder target x = floor(((C - L + 1) M - 1) / R)  (paragraph "Decoder").
__device__ __forceinline__ uint32_t rc_target(CoderState& st) {
    if (st.C < st.L || st.C - st.L >= st.R) {   // impossible on a valid stream
        st.flags |= kFlagCorrupt;
        st.C = st.L;
    }
    return (uint32_t)((((st.C - st.L + 1) << kProbBits) - 1) / st.R);
}

__device__ __forceinline__ void rc_decode_update(CoderState& st, uint32_t c_lo, uint32_t freq, const uint8_t* in,
                                                 uint64_t size) {
    uint64_t L = st.L, R = st.R;
    L = L + ((R * c_lo) >> kProbBits);
    R = (R * freq) >> kProbBits;
    int it = 0;
    for (; it < 16; it++) {
        if ((L >> 24) == ((L + R - 1) >> 24)) {
            L = (L << 8) & kMask32;
            R = R << 8;
            st.C = ((st.C << 8) | rc_read(st, in, size)) & kMask32;
        } else if (R < kBot) {
            R = kBot - (L & (kBot - 1));
        } else {
            break;
        }
    }
    if (it == 16) st.flags |= kFlagLoop;
    st.L = L; st.R = R;
}

// Symbol search: the lane whose range [C(8l), C(8l+8)) holds x is found by a
// ballot, then a rank search over its 8 cumulative counts.
__device__ __forceinline__ void warp_find_symbol(const uint32_t (&f)[8], uint32_t cbase, uint32_t x, int lane,
                                                 int& sym, uint32_t& c_lo, uint32_t& freq) {
    uint32_t mine = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) mine += f[j];
    const unsigned hit = __ballot_sync(0xffffffffu, cbase <= x && x < cbase + mine);
    const int owner = hit ? __ffs(hit) - 1 : 31;
    uint32_t cum = cbase, cl = cbase, fr = f[0];
    int j_hit = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        if (cum <= x) { j_hit = j; cl = cum; fr = f[j]; }
        cum += f[j];
    }
    sym = __shfl_sync(0xffffffffu, lane * 8 + j_hit, owner);
    c_lo = __shfl_sync(0xffffffffu, cl, owner);
    freq = __shfl_sync(0xffffffffu, fr, owner);
}

// ------------------------------------------------------- coder kernels

// Per-stream bookkeeping shared by the slot kernels.
struct StreamTable {
    const uint64_t* in_off;     // [n+1] input slots (raw bytes, or coded bytes when decoding)
    const uint64_t* in_size;    // [n] coded bytes per input slot (decoding) or nullptr
    const uint64_t* lens;       // [n] uncompressed lengths
    const uint64_t* out_off;    // [n+1] output slots
    uint64_t* sizes;            // [n] compressed sizes (encoding)
    uint32_t* flags;            // [n] per-stream status bits
    uint64_t* trace;            // per-step CDF hashes or nullptr
    const uint64_t* trace_off;  // [n]
};

// Carried model state of one slot: SSM state [L][S][N][E] and conv window
// [L][S][K-1][E] (the slot's part of each layer is contiguous).
struct SlotMem {
    float* h;
    float* conv;
    int layers, S, h_per, conv_per;   // floats per (layer, slot)
};

__device__ __forceinline__ void warp_zero_slot(const SlotMem& sm, int s, int lane) {
    for (int l = 0; l < sm.layers; l++) {
        float* hp = sm.h + ((size_t)l * sm.S + s) * sm.h_per;
        for (int i = lane; i < sm.h_per; i += 32) hp[i] = 0.f;
        float* cp = sm.conv + ((size_t)l * sm.S + s) * sm.conv_per;
        for (int i = lane; i < sm.conv_per; i += 32) cp[i] = 0.f;
    }
}

// Streams of length 0 or 1 never enter a slot: 0 bytes, or the raw byte.
__global__ void k_enc_trivial(int n, const uint8_t* __restrict__ data, StreamTable tb, uint8_t* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t len = tb.lens[i];
    if (len == 0) tb.sizes[i] = 0;
    if (len == 1) {
        out[tb.out_off[i]] = data[tb.in_off[i]];
        tb.sizes[i] = 1;
    }
}

// Slot bookkeeping between compression chunks, one warp per slot.  init:
// take the first stream of the slot's list.  Otherwise advance the chunk
// start by tc; a stream whose last step is done is flushed (4 bytes of L,
// paper "Encoder"; its size recorded) and the slot moves to its next stream:
// coder reset, raw first byte written, model state zeroed.
__global__ void k_enc_slots(int S, int init, long long tc, const int* __restrict__ sched,
                            const int* __restrict__ slot_beg, SlotState* slots, CoderState* st,
                            const uint8_t* __restrict__ data, StreamTable tb, uint8_t* __restrict__ out, SlotMem mem) {
    pdl_launch_next();
    pdl_wait_prev();
    const int lane = threadIdx.x & 31;
    const int s = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    if (s >= S) return;
    SlotState ss = slots[s];
    bool start = false;
    if (init) {
        ss.idx = slot_beg[s];
        start = true;
    } else if (ss.stream >= 0) {
        ss.t += tc;
        if (ss.t + 1 >= (long long)tb.lens[ss.stream]) {
            if (lane == 0) {
                CoderState c = st[s];
                const uint64_t o = tb.out_off[ss.stream];
                const uint64_t cap = tb.out_off[ss.stream + 1] - o - 1;
                rc_flush(c, out + o + 1, cap);
                tb.sizes[ss.stream] = 1 + c.pos;
                tb.flags[ss.stream] = c.flags;
            }
            ss.idx++;
            start = true;
        }
    }
    if (start) {
        ss.stream = ss.idx < slot_beg[s + 1] ? sched[ss.idx] : -1;
        ss.t = 0;
        if (ss.stream >= 0) {
            if (lane == 0) {
                CoderState c;
                c.L = 0; c.R = 1ull << 32; c.C = 0; c.pos = 0; c.flags = 0; c.pad = 0;
                st[s] = c;
                out[tb.out_off[ss.stream]] = data[tb.in_off[ss.stream]];
            }
            if (!init) warp_zero_slot(mem, s, lane);
        }
    }
    if (lane == 0) slots[s] = ss;
}

// One warp per slot: for every step of the chunk, softmax -> histogram ->
// encode the true next byte of the slot's current stream (paper "Encoder").
__global__ void k_encode(const float* __restrict__ logits, int S, int Tc, const SlotState* __restrict__ slots,
                         CoderState* st, const uint8_t* __restrict__ data, StreamTable tb, uint8_t* __restrict__ out) {
    pdl_launch_next();
    pdl_wait_prev();
    const int lane = threadIdx.x & 31;
    const int s = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    if (s >= S) return;
    const SlotState ss = slots[s];
    if (ss.stream < 0) return;
    const long long len = (long long)tb.lens[ss.stream];
    CoderState c;
    if (lane == 0) c = st[s];
    const uint64_t o = tb.out_off[ss.stream];
    uint8_t* op = out + o + 1;
    const uint64_t cap = tb.out_off[ss.stream + 1] - o - 1;
    const uint8_t* in = data + tb.in_off[ss.stream];
    for (int tau = 0; tau < Tc; tau++) {
        const long long t = ss.t + tau;
        if (t + 1 >= len) break;
        uint32_t f[8], cbase;
        warp_logits_to_hist(logits + ((size_t)s * Tc + tau) * 256, lane, f, cbase);
        if (tb.trace) {
            const uint64_t hsh = warp_hist_hash(f, lane);
            if (lane == 0) tb.trace[tb.trace_off[ss.stream] + t] = hsh;
        }
        const int sym = in[t + 1];
        uint32_t c_lo, freq;
        warp_sym_range(f, cbase, sym, lane, c_lo, freq);
        if (lane == 0) rc_encode(c, c_lo, freq, op, cap);
    }
    if (lane == 0) st[s] = c;
}

// Embedding + first-block LayerNorm of one token by one warp (the same
// arithmetic as k_embed_ln), used to prepare the next decode step.
struct NextEmbed {
    const float* embed;
    const float* g;
    const float* b;
    float* x;
    float* xn;
    __nv_bfloat16* xn_b;
    F8Out f8;             // FP8 form: xn's E4M3 copy instead of xn
};

template <int VPT>
__device__ __forceinline__ void warp_embed_ln(const NextEmbed& ne, int tok, size_t row, int lane) {
    constexpr int d = VPT * 32;
    float v[VPT], y[VPT];
#pragma unroll
    for (int i = 0; i < VPT; i++) v[i] = ne.embed[(size_t)tok * d + lane + 32 * i];
    warp_layernorm<VPT>(v, ne.g, ne.b, lane, y);
#pragma unroll
    for (int i = 0; i < VPT; i++) {
        ne.x[row * d + lane + 32 * i] = v[i];
        if (ne.xn_b) ne.xn_b[row * d + lane + 32 * i] = __float2bfloat16_rn(y[i]);
        else if (!ne.f8.q) ne.xn[row * d + lane + 32 * i] = y[i];
    }
    if (ne.f8.q) warp_write_f8<VPT>(ne.f8, row, y, lane);
}

// Decoder start for the stream now in slot s: raw first byte to the output,
// code value from the first 4 coded bytes, next-step input rows prepared.
template <int VPT>
__device__ __forceinline__ void warp_dec_start(int s, int stream, const uint8_t* __restrict__ cin, const StreamTable& tb,
                                               uint8_t* __restrict__ out, CoderState* st, const NextEmbed& ne,
                                               int lane) {
    const uint64_t size = tb.in_size[stream];
    const uint8_t first = cin[tb.in_off[stream]];   // size >= 1 (checked on the host)
    if (lane == 0) {
        CoderState c;
        rc_decoder_init(c, cin + tb.in_off[stream] + 1, size - 1);
        st[s] = c;
        out[tb.out_off[stream]] = first;
    }
    warp_embed_ln<VPT>(ne, first, (size_t)s, lane);
}

// Point slot 0 at (stream, t): the teacher-forced log-probability pass.
__global__ void k_set_slot(SlotState* slots, int stream, long long t) {
    SlotState ss;
    ss.idx = 0; ss.stream = stream; ss.t = t;
    slots[0] = ss;
}

__global__ void k_dec_trivial(int n, const uint8_t* __restrict__ cin, StreamTable tb, uint8_t* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t len = tb.lens[i], size = tb.in_size[i];
    if (len == 0) tb.flags[i] = size == 0 ? 0u : (uint32_t)kFlagCorrupt;
    if (len == 1) {
        if (size >= 1) out[tb.out_off[i]] = cin[tb.in_off[i]];
        tb.flags[i] = size == 1 ? 0u : (uint32_t)kFlagCorrupt;
    }
}

template <int VPT>
__global__ void k_dec_slots_init(int S, const int* __restrict__ sched, const int* __restrict__ slot_beg,
                                 SlotState* slots, CoderState* st, const uint8_t* __restrict__ cin, StreamTable tb,
                                 uint8_t* __restrict__ out, NextEmbed ne) {
    pdl_launch_next();
    pdl_wait_prev();
    const int lane = threadIdx.x & 31;
    const int s = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    if (s >= S) return;
    SlotState ss;
    ss.idx = slot_beg[s];
    ss.stream = ss.idx < slot_beg[s + 1] ? sched[ss.idx] : -1;
    ss.t = 0;
    if (ss.stream >= 0) warp_dec_start<VPT>(s, ss.stream, cin, tb, out, st, ne, lane);
    if (lane == 0) slots[s] = ss;
}

// One warp per slot, one step: softmax -> histogram -> decode byte t+1 of the
// slot's stream (paper "Decoder"), then prepare the next step's input rows.
// A completed stream is checked (every coded byte consumed) and the slot
// moves to its next stream with zeroed model state; slots whose lists are
// exhausted are masked.
template <int VPT>
__global__ void k_decode(const float* __restrict__ logits, int S, const int* __restrict__ sched,
                         const int* __restrict__ slot_beg, SlotState* slots, CoderState* st,
                         const uint8_t* __restrict__ cin, StreamTable tb, uint8_t* __restrict__ out, NextEmbed ne,
                         SlotMem mem) {
    pdl_launch_next();
    pdl_wait_prev();
    const int lane = threadIdx.x & 31;
    const int s = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    if (s >= S) return;
    SlotState ss = slots[s];
    if (ss.stream < 0) return;
    const int stream = ss.stream;
    const long long len = (long long)tb.lens[stream];
    const long long t = ss.t;
    uint32_t f[8], cbase;
    warp_logits_to_hist(logits + (size_t)s * 256, lane, f, cbase);
    if (tb.trace) {
        const uint64_t hsh = warp_hist_hash(f, lane);
        if (lane == 0) tb.trace[tb.trace_off[stream] + t] = hsh;
    }
    const uint8_t* in = cin + tb.in_off[stream] + 1;
    const uint64_t size = tb.in_size[stream] - 1;
    CoderState c;
    uint32_t x = 0;
    if (lane == 0) {
        c = st[s];
        x = rc_target(c);
    }
    x = __shfl_sync(0xffffffffu, x, 0);
    int sym;
    uint32_t c_lo, freq;
    warp_find_symbol(f, cbase, x, lane, sym, c_lo, freq);
    if (lane == 0) {
        rc_decode_update(c, c_lo, freq, in, size);
        st[s] = c;
        out[tb.out_off[stream] + t + 1] = (uint8_t)sym;
    }
    if (t + 2 < len) {
        ss.t = t + 1;
        warp_embed_ln<VPT>(ne, sym, (size_t)s, lane);
    } else {
        if (lane == 0) tb.flags[stream] = c.flags | (c.pos != size ? (uint32_t)kFlagCorrupt : 0u);
        ss.idx++;
        ss.stream = ss.idx < slot_beg[s + 1] ? sched[ss.idx] : -1;
        ss.t = 0;
        if (ss.stream >= 0) {
            warp_zero_slot(mem, s, lane);
            warp_dec_start<VPT>(s, ss.stream, cin, tb, out, st, ne, lane);
        }
    }
    if (lane == 0) slots[s] = ss;
}

__global__ void k_to_bf16(const float* __restrict__ in, __nv_bfloat16* __restrict__ out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = __float2bfloat16_rn(in[i]);
}

// Per-row FP8 quantisation of an activation matrix for the E4M3 GEMM:
// scale[m] = max_k |A[m][k]| / 448 and q[m][k] = e4m3(A[m][k] * (448 / max)),
// rounded to nearest and saturated; q has Kp >= K columns, the extra ones
// zero (the GEMM's K blocks are 128 wide).  One warp per row, K <= 1024.
__global__ void k_quant_rows_e4m3(const float* __restrict__ A, __nv_fp8_e4m3* __restrict__ q,
                                  float* __restrict__ scale, long long M, int K, int Kp) {
    pdl_launch_next();
    pdl_wait_prev();
    const int lane = threadIdx.x & 31;
    const long long row = (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    if (row >= M) return;
    const float* a = A + row * K;
    float amax = 0.f;
    for (int k = 4 * lane; k < K; k += 128) {
        const float4 v = *reinterpret_cast<const float4*>(a + k);
        amax = fmaxf(amax, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
    }
    amax = warp_max(amax);
    const float inv = e4m3_row_inv(amax);
    if (lane == 0) scale[row] = e4m3_row_scale(amax);
    __nv_fp8_e4m3* o = q + row * Kp;
    for (int k = 4 * lane; k < Kp; k += 128) {
        if (k < K) {
            const float4 v = *reinterpret_cast<const float4*>(a + k);
            o[k + 0] = e4m3_of(v.x, inv);
            o[k + 1] = e4m3_of(v.y, inv);
            o[k + 2] = e4m3_of(v.z, inv);
            o[k + 3] = e4m3_of(v.w, inv);
        } else {
            o[k + 0] = o[k + 1] = o[k + 2] = o[k + 3] = __nv_fp8_e4m3(0.0f);
        }
    }
}

// Gather each stream's used bytes from its output slot into one packed buffer.
__global__ void k_compact(const uint8_t* __restrict__ src, const uint64_t* __restrict__ src_off,
                          const uint64_t* __restrict__ dst_off, uint8_t* __restrict__ dst, int S) {
    const int s = blockIdx.x;
    if (s >= S) return;
    const uint64_t n = dst_off[s + 1] - dst_off[s];
    const uint8_t* a = src + src_off[s];
    uint8_t* b = dst + dst_off[s];
    for (uint64_t i = threadIdx.x; i < n; i += blockDim.x) b[i] = a[i];
}

// log2 p rows for tests: (l - m - ln Z) / ln 2.
__global__ void k_log2_softmax(const float* __restrict__ logits, float* __restrict__ out, long long rows) {
    const int lane = threadIdx.x & 31;
    const long long row = (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    if (row >= rows) return;
    const float* l = logits + row * 256;
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; j++) v[j] = l[lane * 8 + j];
    float m = v[0];
#pragma unroll
    for (int j = 1; j < 8; j++) m = fmaxf(m, v[j]);
    m = warp_max(m);
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; j++) s = __fadd_rn(s, expf(__fsub_rn(v[j], m)));
    s = warp_sum(s);
    const float lz = logf(s);
#pragma unroll
    for (int j = 0; j < 8; j++)
        out[row * 256 + lane * 8 + j] = __fmul_rn(__fsub_rn(__fsub_rn(v[j], m), lz), 1.4426950408889634f);
}

// ------------------------------------------- CDF-driven coder test kernels

// One warp per sequence; the CDF rows come from the caller.
__global__ void k_debug_encode_cdfs(int n_seq, const uint64_t* sym_off, const uint32_t* cdfs, const uint8_t* syms,
                                    uint8_t* out, uint64_t out_stride, uint64_t* sizes, uint32_t* flags) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_seq) return;
    CoderState st;
    st.L = 0; st.R = 1ull << 32; st.C = 0; st.pos = 0; st.flags = 0; st.pad = 0;
    uint8_t* o = out + (size_t)i * out_stride;
    for (uint64_t t = sym_off[i]; t < sym_off[i + 1]; t++) {
        const uint32_t* c = cdfs + t * 257;
        const int s = syms[t];
        rc_encode(st, c[s], c[s + 1] - c[s], o, out_stride);
    }
    rc_flush(st, o, out_stride);
    sizes[i] = st.pos;
    flags[i] = st.flags;
}

__global__ void k_debug_decode_cdfs(int n_seq, const uint64_t* sym_off, const uint32_t* cdfs, const uint8_t* in,
                                    uint64_t in_stride, const uint64_t* in_sizes, uint8_t* syms, uint32_t* flags) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    if (i >= n_seq) return;
    const uint8_t* src = in + (size_t)i * in_stride;
    CoderState st;
    if (lane == 0) rc_decoder_init(st, src, in_sizes[i]);
    for (uint64_t t = sym_off[i]; t < sym_off[i + 1]; t++) {
        const uint32_t* c = cdfs + t * 257;
        uint32_t f[8];
#pragma unroll
        for (int j = 0; j < 8; j++) f[j] = c[lane * 8 + j + 1] - c[lane * 8 + j];
        const uint32_t cbase = c[lane * 8];
        uint32_t x = 0;
        if (lane == 0) x = rc_target(st);
        x = __shfl_sync(0xffffffffu, x, 0);
        int sym;
        uint32_t c_lo, freq;
        warp_find_symbol(f, cbase, x, lane, sym, c_lo, freq);
        if (lane == 0) {
            rc_decode_update(st, c_lo, freq, src, in_sizes[i]);
            syms[t] = (uint8_t)sym;
        }
    }
    if (lane == 0) {
        if (st.pos != in_sizes[i]) st.flags |= kFlagCorrupt;
        flags[i] = st.flags;
    }
}

__global__ void k_debug_quantise(const float* __restrict__ p, uint32_t* __restrict__ f_out, long long rows) {
    const int lane = threadIdx.x & 31;
    const long long row = (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    if (row >= rows) return;
    float q[8];
#pragma unroll
    for (int j = 0; j < 8; j++) q[j] = p[row * 256 + lane * 8 + j];
    uint32_t f[8], cbase;
    warp_quantise_p(q, lane, f, cbase);
#pragma unroll
    for (int j = 0; j < 8; j++) f_out[row * 256 + lane * 8 + j] = f[j];
}

}  // namespace boa
